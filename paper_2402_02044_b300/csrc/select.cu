// Query preparation, merging of per-split top-k1 lists, residual re-ranking
// (Sec. 2.2, App. C) and the ID-gather search (the frontier-scoring step of
// greedy graph search, Alg. 1).
#include "kernels.cuh"
#include "score.cuh"

namespace lvq {

namespace {

// ---- query preparation (one warp per query; one per (query, mean) pair for <q, mu_m>)
__global__ void __launch_bounds__(256) prep_kernel(DeviceStore st, const float* __restrict__ q, int64_t nq,
                                                   QueryPrep p) {
  const int lane = threadIdx.x & 31;
  const int warps = blockDim.x >> 5;
  const int d = st.d;
  const int64_t rows = p.q16 ? (p.nq_pad > nq ? p.nq_pad : nq) : nq;
  for (int64_t i = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5); i < rows; i += (int64_t)gridDim.x * warps) {
    const bool real = i < nq;
    if (p.q16) {
      __half* dst = reinterpret_cast<__half*>(p.q16) + i * p.kq;
      float hs = 0.0f;
      for (int j = lane; j < p.kq; j += 32) {
        float v = (real && j < d) ? q[i * d + j] : 0.0f;
        if (st.bits1 == 4 && (j & 2)) v *= 0.0625f;  // j % 8 in {2, 3, 6, 7}
        const __half h = __float2half_rn(v);
        dst[j] = h;
        hs += __half2float(h);
      }
      hs = warp_sum(hs);
      if (real && lane == 0) p.q16sum[i] = hs;
    }
    if (!real) continue;
    const float* qi = q + i * d;
    float s = 0.0f, s2 = 0.0f;
    for (int j = lane; j < d; j += 32) {
      const float v = qi[j];
      s += v;
      s2 = __fmaf_rn(v, v, s2);
    }
    s = warp_sum(s);
    s2 = warp_sum(s2);
    if (lane == 0) {
      p.qsum[i] = s;
      p.qnorm[i] = s2;
    }
  }
  // <q_i, mu_m>: one warp per (query, mean) pair
  const int64_t items = nq * st.n_means;
  for (int64_t it = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5); it < items; it += (int64_t)gridDim.x * warps) {
    const int64_t i = it / st.n_means;
    const int m = (int)(it - i * st.n_means);
    const float* qi = q + i * d;
    const float* mu = st.means + (int64_t)m * d;
    float c = 0.0f;
    for (int j = lane; j < d; j += 32) c = __fmaf_rn(qi[j], __ldg(mu + j), c);
    c = warp_sum(c);
    if (lane == 0) p.cm[it] = c;
  }
}

// ---- shared re-rank tail -------------------------------------------------------
// keys[0..n) hold candidate keys (sorted or not, possibly with repeats).  Each
// warp scores candidates with both levels; the block then sorts the new keys
// and writes the k best.  scratch: pow2_at_least(n) keys of shared memory.
__device__ void rerank_tail(const DeviceStore& st, const float* qsh, const uint64_t* keys, int n, int k,
                            uint64_t* scratch, int* sh_pos, int64_t* out_ids, float* out_scores) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int np2 = pow2_at_least(n < 1 ? 1 : n);
  for (int i = threadIdx.x; i < np2; i += blockDim.x) scratch[i] = kNoKey;
  __syncthreads();
  for (int i = wid; i < n; i += nw) {
    const uint64_t key = keys[i];
    if (key == kNoKey) continue;
    const uint32_t s = (uint32_t)key;
    const float sc = score2_warp(st, s, qsh);
    if (lane == 0) scratch[i] = make_key(sc, s, st.metric);
  }
  __syncthreads();
  block_sort(scratch, np2);
  write_results(scratch, np2, k, st.metric, out_ids, out_scores, sh_pos);
}

// ---- merge of per-split lists + optional re-rank (one block per query) --------
// T threads per block (128, or 512 when there are fewer queries than SMs, so
// that a lone query's re-rank has more warps); rounds of kMergeRound keys.
constexpr int kMergeRound = 1024;

template <int T>
__global__ void __launch_bounds__(T) merge_rerank_kernel(DeviceStore st, const float* __restrict__ q,
                                                         const uint64_t* __restrict__ partial,
                                                         const int* __restrict__ counts, int splits, int k1, int k,
                                                         int rerank, int64_t* out_ids, float* out_scores) {
  constexpr int kMergePer = kMergeRound / T;
  extern __shared__ __align__(16) unsigned char smem[];
  const int qi = blockIdx.x;
  const int cap = pow2_at_least(k1 + kMergeRound);
  uint64_t* buf = reinterpret_cast<uint64_t*>(smem);
  uint64_t* scratch = buf + cap;                   // pow2_at_least(k1) keys
  float* qsh = reinterpret_cast<float*>(scratch + pow2_at_least(k1));
  int* sh_pos = reinterpret_cast<int*>(qsh + st.d);
  __shared__ int cnt;
  __shared__ uint64_t thr;
  __shared__ int hist[288];
  __shared__ int len[kMaxMergeLists];  // valid keys per list (counts given)
  if (threadIdx.x == 0) {
    cnt = 0;
    thr = kNoKey;
  }
  for (int j = threadIdx.x; j < st.d; j += blockDim.x) qsh[j] = q[(int64_t)qi * st.d + j];
  if (counts)
    for (int i = threadIdx.x; i < splits; i += blockDim.x) len[i] = counts[(int64_t)qi * splits + i];
  __syncthreads();
  const uint64_t* src = partial + (int64_t)qi * splits * k1;
  const int total = splits * k1;
  const int lane = threadIdx.x & 31;
  // rounds of kMergeRound keys, kMergePer independent loads per thread; with
  // counts, positions past a list's length are not read
  for (int base = 0; base < total; base += kMergeRound) {
    uint64_t v[kMergePer];
#pragma unroll
    for (int r = 0; r < kMergePer; ++r) {
      const int i = base + r * T + threadIdx.x;
      bool in = i < total;
      if (in && counts) in = (i % k1) < len[i / k1];
      v[r] = in ? __ldg(src + i) : kNoKey;
    }
    const uint64_t t = thr;
#pragma unroll
    for (int r = 0; r < kMergePer; ++r) {
      const bool pass = v[r] < t;
      const unsigned m = __ballot_sync(0xffffffffu, pass);
      if (m) {
        int at = 0;
        if (lane == 0) at = atomicAdd(&cnt, __popc(m));
        at = __shfl_sync(0xffffffffu, at, 0);
        if (pass) buf[at + __popc(m & ((1u << lane) - 1u))] = v[r];
      }
    }
    __syncthreads();
    if (cnt > cap - kMergeRound) {
      if (threadIdx.x < 32) {
        uint64_t tk;
        const int kept = warp_select6(buf, cnt, k1, hist, &tk);
        if (threadIdx.x == 0) {
          cnt = kept;
          thr = tk;
        }
      }
      __syncthreads();
    }
  }
  if (threadIdx.x < 32) {
    uint64_t tk;
    const int kept = warp_select6(buf, cnt, k1, hist, &tk);
    if (threadIdx.x == 0) cnt = kept;
  }
  __syncthreads();
  const int n1 = cnt;
  const int np2 = pow2_at_least(k1);
  for (int i = n1 + threadIdx.x; i < np2; i += blockDim.x) buf[i] = kNoKey;
  block_sort(buf, np2);
  int64_t* oi = out_ids + (int64_t)qi * k;
  float* os = out_scores + (int64_t)qi * k;
  if (!rerank) {
    write_results(buf, n1, k, st.metric, oi, os, sh_pos);
    return;
  }
  rerank_tail(st, qsh, buf, n1, k, scratch, sh_pos, oi, os);
}

// ---- re-rank of caller-given candidates (one block per query) -----------------
__global__ void __launch_bounds__(256) rerank_kernel(DeviceStore st, const float* __restrict__ q,
                                                      const int64_t* __restrict__ ids, int k1, int k,
                                                      int64_t* out_ids, float* out_scores) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int qi = blockIdx.x;
  const int np2 = pow2_at_least(k1);
  uint64_t* keys = reinterpret_cast<uint64_t*>(smem);
  uint64_t* scratch = keys + np2;
  float* qsh = reinterpret_cast<float*>(scratch + np2);
  int* sh_pos = reinterpret_cast<int*>(qsh + st.d);
  for (int j = threadIdx.x; j < st.d; j += blockDim.x) qsh[j] = q[(int64_t)qi * st.d + j];
  for (int i = threadIdx.x; i < k1; i += blockDim.x) {
    const int64_t s = ids[(int64_t)qi * k1 + i];
    const bool ok = s >= 0 && s < st.capacity && is_live(st.live, s);
    keys[i] = ok ? (uint64_t)s : kNoKey;  // the score is filled in by rerank_tail
  }
  __syncthreads();
  rerank_tail(st, qsh, keys, k1, k, scratch, sh_pos, out_ids + (int64_t)qi * k, out_scores + (int64_t)qi * k);
}

// ---- ID-gather search (one block per query, one thread per candidate) ---------
constexpr int kGatherThreads = 256;

__global__ void __launch_bounds__(kGatherThreads, 3) gather_kernel(DeviceStore st, const float* __restrict__ q,
                                                                 QueryPrep p, const int64_t* __restrict__ cand,
                                                                 int n_cand, int k1, int k, int rerank,
                                                                 int64_t* out_ids, float* out_scores) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int qi = blockIdx.x;
  const int d = st.d;
  const int stage1 = rerank ? k1 : k;
  const int cap = pow2_at_least(stage1 + kGatherThreads);
  const int groups = (d + 7) >> 3;
  uint64_t* buf = reinterpret_cast<uint64_t*>(smem);
  uint64_t* scratch = buf + cap;
  float* qsh = reinterpret_cast<float*>(scratch + pow2_at_least(stage1));
  uint64_t* tmp = reinterpret_cast<uint64_t*>(qsh + groups * 8 * 2);  // cap keys
  float* qc = qsh + groups * 8;  // centred / shifted copy used by the first level
  int* sh_pos = reinterpret_cast<int*>(tmp + cap);
  __shared__ int cnt;
  __shared__ uint64_t thr;
  __shared__ int scan_sh[kGatherThreads / 32 + 1];
  // the round's candidates: slot id (-1: skipped) and per-row constants
  __shared__ int64_t r_id[kGatherThreads];
  __shared__ float r_lo[kGatherThreads], r_step[kGatherThreads];
  __shared__ int r_m[kGatherThreads];
  const bool ip = st.metric == LVQ_IP;
  const bool one_mean = st.n_means == 1;
  for (int j = threadIdx.x; j < groups * 8; j += blockDim.x) {
    const float v = j < d ? q[(int64_t)qi * d + j] : 0.0f;
    qsh[j] = v;
    qc[j] = (!ip && one_mean && j < d) ? __fsub_rn(v, st.means[j]) : v;
  }
  if (threadIdx.x == 0) {
    cnt = 0;
    thr = kNoKey;
  }
  __syncthreads();
  const float off = code_offset(st.bits1);
  const float qs = ip ? p.qsum[qi] : 0.0f;
  const float* cmq = ip ? p.cm + (int64_t)qi * st.n_means : nullptr;
  const int64_t* cl = cand + (int64_t)qi * n_cand;
  // Each round: the round's candidate ids and per-row constants are staged
  // in shared memory by all threads (independent loads), then S lanes score
  // one candidate (its code words spread over the lanes, so a row is read
  // with a few wide loads), kC candidates per sub-warp in flight at once.
  constexpr int kC = 4;
  const int S = groups >= 32 ? 32 : pow2_at_least(groups);
  const int per_warp = 32 / S;
  const int lane = threadIdx.x & 31, sub = lane / S, sl = lane % S;
  const int slot0 = (threadIdx.x >> 5) * per_warp + sub;
  const int nsub = (kGatherThreads / 32) * per_warp;
  for (int base = 0; base < n_cand; base += kGatherThreads) {
    {
      const int i = base + threadIdx.x;
      const int64_t s = i < n_cand ? cl[i] : -1;
      const bool ok = s >= 0 && s < st.capacity && is_live(st.live, s);
      r_id[threadIdx.x] = ok ? s : -1;
      r_lo[threadIdx.x] = ok ? __ldg(st.lower + s) : 0.0f;
      r_step[threadIdx.x] = ok ? __ldg(st.step + s) : 0.0f;
      r_m[threadIdx.x] = ok ? __ldg(st.mean_id + s) : 0;
    }
    __syncthreads();
    for (int j0 = 0; j0 < kGatherThreads; j0 += nsub * kC) {
      float acc[kC];
      // the first kGL groups of each lane for all kC candidates are loaded
      // before any is used, so their loads are in flight together
      constexpr int kGL = 4;
      uint2 w[kC][kGL];
#pragma unroll
      for (int u = 0; u < kC; ++u) {
        acc[u] = 0.0f;
        const int t = j0 + u * nsub + slot0;
        const int64_t s = t < kGatherThreads ? r_id[t] : -1;
        const uint8_t* row = st.codes1 + (s < 0 ? 0 : s) * st.row1;
#pragma unroll
        for (int gi = 0; gi < kGL; ++gi) {
          const int g = sl + gi * S;
          w[u][gi] = (s >= 0 && g < groups) ? group_words(row, st.bits1, g) : make_uint2(0u, 0u);
        }
      }
#pragma unroll
      for (int u = 0; u < kC; ++u) {
        const int t = j0 + u * nsub + slot0;
        const int64_t s = t < kGatherThreads ? r_id[t] : -1;
        if (s < 0) continue;
        const uint8_t* row = st.codes1 + s * st.row1;
        const float lo = r_lo[t], step = r_step[t];
        const float* mu = st.means + (int64_t)r_m[t] * d;
        auto add_group = [&](uint2 ww, int g) {
          float c[8];
          if (ip) {
            words_codes(ww, st.bits1, 8388608.0f + off, c);
#pragma unroll
            for (int e = 0; e < 8; ++e) acc[u] = __fmaf_rn(qc[g * 8 + e], c[e], acc[u]);
          } else {
            words_codes(ww, st.bits1, 8388608.0f, c);
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const int jj = g * 8 + e;
              if (jj < d) {
                float xh = __fmaf_rn(step, c[e], lo);
                if (!one_mean) xh = __fadd_rn(xh, __ldg(mu + jj));
                const float df = qc[jj] - xh;
                acc[u] = __fmaf_rn(df, df, acc[u]);
              }
            }
          }
        };
#pragma unroll
        for (int gi = 0; gi < kGL; ++gi)
          if (sl + gi * S < groups) add_group(w[u][gi], sl + gi * S);
        for (int g = sl + kGL * S; g < groups; g += S) add_group(group_words(row, st.bits1, g), g);
      }
#pragma unroll
      for (int u = 0; u < kC; ++u) {
        // sum over the S lanes of each candidate (every lane takes part)
        float a = acc[u];
        for (int o = S >> 1; o > 0; o >>= 1) a += __shfl_xor_sync(kFull, a, o);
        const int t = j0 + u * nsub + slot0;
        const int64_t s = t < kGatherThreads ? r_id[t] : -1;
        if (s >= 0 && sl == 0) {
          const float step = r_step[t], lo = r_lo[t];
          const float sc = ip ? __fmaf_rn(step, a, __fmaf_rn(__fmaf_rn(off, step, lo), qs, cmq[r_m[t]])) : a;
          const uint64_t key = make_key(sc, (uint32_t)s, st.metric);
          if (key < thr) buf[atomicAdd(&cnt, 1)] = key;
        }
      }
    }
    __syncthreads();
    if (cnt > cap - kGatherThreads) {
      uint64_t t;
      const int kept = block_select_dedupe(buf, tmp, cap, cnt, stage1, scan_sh, &t);
      if (threadIdx.x == 0) {
        cnt = kept;
        thr = t;
      }
      __syncthreads();
    }
  }
  {
    uint64_t t;
    const int kept = block_select_dedupe(buf, tmp, cap, cnt, stage1, scan_sh, &t);
    if (threadIdx.x == 0) cnt = kept;
    __syncthreads();
  }
  int64_t* oi = out_ids + (int64_t)qi * k;
  float* os = out_scores + (int64_t)qi * k;
  if (!rerank) {
    write_results(buf, cnt, k, st.metric, oi, os, sh_pos);
    return;
  }
  rerank_tail(st, qsh, buf, cnt, k, scratch, sh_pos, oi, os);
}

}  // namespace

cudaError_t launch_prep_queries(const DeviceStore& st, const float* q, int64_t nq, const QueryPrep& p,
                                cudaStream_t stream) {
  const int64_t rows = p.q16 ? (p.nq_pad > nq ? p.nq_pad : nq) : nq;
  if (rows <= 0) return cudaSuccess;
  const int64_t work = rows > nq * st.n_means ? rows : nq * st.n_means;
  const int blocks = (int)(ceil_div(work, 8) < 65536 ? ceil_div(work, 8) : 65536);
  prep_kernel<<<blocks, 256, 0, stream>>>(st, q, nq, p);
  return cudaGetLastError();
}

template <int T>
cudaError_t launch_merge_t(const DeviceStore& st, const float* q, int64_t nq, const uint64_t* partial,
                           const int* counts, int splits, int k1, int k, bool rerank, int64_t* out_ids,
                           float* out_scores, size_t sm, cudaStream_t stream) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(merge_rerank_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  merge_rerank_kernel<T><<<(unsigned)nq, T, sm, stream>>>(st, q, partial, counts, splits, k1, k, rerank ? 1 : 0,
                                                          out_ids, out_scores);
  return cudaGetLastError();
}

static size_t merge_smem(int d, int k1) {
  return (size_t)(pow2_at_least(k1 + kMergeRound) + pow2_at_least(k1)) * 8 + (size_t)d * 4 +
         (size_t)(k1 + 2) * 4 + 16;
}

cudaError_t launch_merge_rerank(const DeviceStore& st, const float* q, int64_t nq, const QueryPrep&,
                                const uint64_t* partial, int splits, int k1, int k, bool rerank,
                                int64_t* out_ids, float* out_scores, cudaStream_t stream, const int* counts,
                                int sm_count) {
  if (nq <= 0) return cudaSuccess;
  if (counts && splits > kMaxMergeLists) return cudaErrorInvalidValue;
  const size_t sm = merge_smem(st.d, k1 > k ? k1 : k);
  if (nq < sm_count)
    return launch_merge_t<512>(st, q, nq, partial, counts, splits, k1, k, rerank, out_ids, out_scores, sm, stream);
  return launch_merge_t<128>(st, q, nq, partial, counts, splits, k1, k, rerank, out_ids, out_scores, sm, stream);
}

cudaError_t launch_rerank(const DeviceStore& st, const float* q, int64_t nq, const QueryPrep&, const int64_t* ids,
                          int k1, int k, int64_t* out_ids, float* out_scores, cudaStream_t stream) {
  if (nq <= 0) return cudaSuccess;
  const size_t sm = (size_t)pow2_at_least(k1) * 16 + (size_t)st.d * 4 + (size_t)(k + 2) * 4 + 16;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(rerank_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  rerank_kernel<<<(unsigned)nq, 256, sm, stream>>>(st, q, ids, k1, k, out_ids, out_scores);
  return cudaGetLastError();
}

cudaError_t launch_gather(const DeviceStore& st, const float* q, int64_t nq, const QueryPrep& p,
                          const int64_t* cand, int n_cand, int k1, int k, bool rerank, int64_t* out_ids,
                          float* out_scores, cudaStream_t stream) {
  if (nq <= 0) return cudaSuccess;
  const int stage1 = rerank ? k1 : k;
  const int groups = (st.d + 7) / 8;
  const size_t sm = (size_t)(2 * pow2_at_least(stage1 + kGatherThreads) + pow2_at_least(stage1)) * 8 +
                    (size_t)groups * 8 * 4 * 2 + (size_t)(k + 2) * 4 + 16;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(gather_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  gather_kernel<<<(unsigned)nq, kGatherThreads, sm, stream>>>(st, q, p, cand, n_cand, k1, k, rerank ? 1 : 0,
                                                              out_ids, out_scores);
  return cudaGetLastError();
}

}  // namespace lvq
