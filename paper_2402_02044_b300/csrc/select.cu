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
// warp scores kRU candidates at a time with both levels, their code words for
// the first kRG groups of each lane loaded before any is used, so the loads of
// the candidates are in flight together; the block then sorts the new keys and
// writes the k best.  With a single centring mean the mean is folded into the
// query first: q - mu for L2 (qsh is overwritten), <q, mu> added once for the
// inner product.  scratch: pow2_at_least(n) keys of shared memory.
constexpr int kRU = 2;
constexpr int kRG = 3;

__device__ void rerank_tail(const DeviceStore& st, float* qsh, const uint64_t* keys, int n, int k, uint64_t* scratch,
                            int* sh_pos, int64_t* out_ids, float* out_scores) {
  __shared__ float red_sh[33];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int d = st.d;
  const int groups = (d + 7) >> 3;
  const bool ip = st.metric == LVQ_IP;
  const bool one_mean = st.n_means == 1;
  const int np2 = pow2_at_least(n < 1 ? 1 : n);
  for (int i = threadIdx.x; i < np2; i += blockDim.x) scratch[i] = kNoKey;
  float c0 = 0.0f;
  if (one_mean) {
    float part = 0.0f;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
      const float mu = st.means[j];
      if (ip)
        part = __fmaf_rn(qsh[j], mu, part);
      else
        qsh[j] = __fsub_rn(qsh[j], mu);
    }
    if (ip) {
      part = warp_sum(part);
      if (lane == 0) red_sh[wid] = part;
      __syncthreads();
      if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int i = 0; i < nw; ++i) t += red_sh[i];
        red_sh[32] = t;
      }
    }
  }
  __syncthreads();
  if (one_mean && ip) c0 = red_sh[32];
  for (int i0 = wid * kRU; i0 < n; i0 += nw * kRU) {
    uint32_t sid[kRU];
    bool ok[kRU];
#pragma unroll
    for (int u = 0; u < kRU; ++u) {
      const uint64_t key = i0 + u < n ? keys[i0 + u] : kNoKey;
      // ids past the store are skipped (only a scan that gave up leaves any)
      ok[u] = key != kNoKey && (int64_t)(uint32_t)key < st.capacity;
      sid[u] = (uint32_t)key;
    }
    // per-candidate constants, one lane each
    float lo_l = 0.0f, st_l = 0.0f;
    int m_l = 0;
    {
      const uint64_t key = (lane < kRU && i0 + lane < n) ? keys[i0 + lane] : kNoKey;
      if (key != kNoKey && (int64_t)(uint32_t)key < st.capacity) {
        const uint32_t sl = (uint32_t)key;
        lo_l = __ldg(st.lower + sl);
        st_l = __ldg(st.step + sl);
        m_l = __ldg(st.mean_id + sl);
      }
    }
    uint2 w1[kRU][kRG], w2[kRU][kRG];
#pragma unroll
    for (int u = 0; u < kRU; ++u) {
      const uint8_t* r1 = st.codes1 + (int64_t)sid[u] * st.stride1;
      const uint8_t* r2 = st.codes2 + (int64_t)sid[u] * st.row2;
#pragma unroll
      for (int gi = 0; gi < kRG; ++gi) {
        const int g = lane + 32 * gi;
        const bool in = ok[u] && g < groups;
        w1[u][gi] = in ? group_words(r1, st.bits1, g) : make_uint2(0u, 0u);
        w2[u][gi] = in ? __ldg(reinterpret_cast<const uint2*>(r2) + g) : make_uint2(0u, 0u);
      }
    }
#pragma unroll
    for (int u = 0; u < kRU; ++u) {
      const float lo = __shfl_sync(kFull, lo_l, u), step = __shfl_sync(kFull, st_l, u);
      const int m = __shfl_sync(kFull, m_l, u);
      if (!ok[u]) continue;
      const Resid R = resid_of(st, step);
      const float lo2 = R.lo2, step2 = R.step2;
      const float* mu = st.means + (int64_t)m * d;
      const uint8_t* r1 = st.codes1 + (int64_t)sid[u] * st.stride1;
      const uint8_t* r2 = st.codes2 + (int64_t)sid[u] * st.row2;
      float acc = 0.0f;
      auto add_group = [&](uint2 a, uint2 b, int g) {
        float c[8];
        words_codes(a, st.bits1, 8388608.0f, c);
        float part = 0.0f;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int j = g * 8 + e;
          if (j < d) {
            const float c2 = byte_centred((e < 4 ? b.x : b.y) ^ R.flip, e & 3, R.sub);
            float x2 = __fadd_rn(__fmaf_rn(step, c[e], lo), __fmaf_rn(step2, c2, lo2));
            if (!one_mean) x2 = __fadd_rn(x2, __ldg(mu + j));
            if (ip) {
              part = __fmaf_rn(qsh[j], x2, part);
            } else {
              const float df = qsh[j] - x2;
              part = __fmaf_rn(df, df, part);
            }
          }
        }
        acc += part;
      };
#pragma unroll
      for (int gi = 0; gi < kRG; ++gi)
        if (lane + 32 * gi < groups) add_group(w1[u][gi], w2[u][gi], lane + 32 * gi);
      for (int g = lane + 32 * kRG; g < groups; g += 32)
        add_group(group_words(r1, st.bits1, g), __ldg(reinterpret_cast<const uint2*>(r2) + g), g);
      float sc = warp_sum(acc);
      if (ip) sc = __fadd_rn(sc, c0);
      if (lane == 0) scratch[i0 + u] = make_key(sc, sid[u], st.metric);
    }
  }
  __syncthreads();
  block_sort(scratch, np2);
  write_results(scratch, np2, k, st.metric, out_ids, out_scores, sh_pos);
}

// ---- merge of per-split lists + optional re-rank (one block per query) --------
// T threads per block (128, or 512 when there are fewer queries than SMs, so
// that a lone query's re-rank has more warps); rounds of kMergeRound keys.
constexpr int kMergeRound = 1024;

// Cut buf[0..n) to its k best keys (called by all threads; the result is
// meaningful in thread 0).  A 512-thread block (few queries: the block has an
// SM to itself) sorts with every warp; a 128-thread block leaves the select
// to one warp (6-bit radix select) while its other blocks keep the SM busy.
template <int T>
__device__ __forceinline__ int cut_keys(uint64_t* buf, int cap, int n, int k, int* hist, int* scan_sh, uint64_t* thr) {
  if (T >= 512) return block_select_dedupe(buf, cap, n, k, scan_sh, thr);
  int kept = 0;
  if (threadIdx.x < 32) kept = warp_select6(buf, n, k, hist, thr);
  return kept;
}

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
  __shared__ int start[kMaxMergeLists + 1];  // first position of each list's keys (counts given)
  __shared__ int scan_sh[T / 32 + 1];
  if (threadIdx.x == 0) {
    cnt = 0;
    thr = kNoKey;
  }
  for (int j = threadIdx.x; j < st.d; j += blockDim.x) qsh[j] = q[(int64_t)qi * st.d + j];
  const uint64_t* src = partial + (int64_t)qi * splits * k1;
  // With counts only the valid keys are visited: position p of the packed
  // sequence is key p - start[l] of list l (start: exclusive prefix sums).
  int total = splits * k1;
  if (counts) {
    int run = 0;
    for (int c0 = 0; c0 < splits; c0 += T) {
      const int i = c0 + threadIdx.x;
      // a list holds at most k1 keys; the clamp keeps a scan that gave up
      // (LVQ_ETIMEOUT, lists left unwritten) from sending the merge past them
      int v = i < splits ? counts[(int64_t)qi * splits + i] : 0;
      v = v < 0 ? 0 : v > k1 ? k1 : v;
      int sum;
      const int at = run + block_exclusive_scan(v, scan_sh, sum);
      if (i < splits) start[i] = at;
      run += sum;
    }
    if (threadIdx.x == 0) start[splits] = run;
    total = run;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  // rounds of kMergeRound keys, kMergePer independent loads per thread
  for (int base = 0; base < total; base += kMergeRound) {
    uint64_t v[kMergePer];
#pragma unroll
    for (int r = 0; r < kMergePer; ++r) {
      const int i = base + r * T + threadIdx.x;
      int at = i;
      if (counts && i < total) {
        int lo = 0, hi = splits;  // the last list with start <= i
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (start[mid] <= i) lo = mid; else hi = mid;
        }
        at = lo * k1 + (i - start[lo]);
      }
      v[r] = i < total ? __ldg(src + at) : kNoKey;
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
    // every thread reads the count before any starts the next round's
    // appends, so all take the same branch
    __syncthreads();
    const int c_now = cnt;
    __syncthreads();
    if (c_now > cap - kMergeRound) {
      uint64_t tk;
      const int kept = cut_keys<T>(buf, cap, cnt, k1, hist, scan_sh, &tk);
      if (threadIdx.x == 0) {
        cnt = kept;
        thr = tk;
      }
      __syncthreads();
    }
  }
  {
    uint64_t tk;
    const int kept = cut_keys<T>(buf, cap, cnt, k1, hist, scan_sh, &tk);
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
constexpr int kRerankThreads = 128;

__global__ void __launch_bounds__(kRerankThreads, 8) rerank_kernel(DeviceStore st, const float* __restrict__ q,
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

// ---- ID-gather search (persistent blocks, one query at a time per block) ---------
// Rows: each warp streams its share of a query's candidate rows (batches of R
// rows, R = 32 / L) into its own ring of P shared-memory slots with 16-byte
// cp.async copies (one commit group per batch; the lanes of a warp copy
// consecutive chunks of a row, so every row is read with coalesced requests),
// issuing P - 1 batches ahead of the one it scores, across query boundaries
// too, so the next query's first rows load while the block selects the
// query's best keys.  A row is scored by L lanes (16-byte chunks l, l + L, ...); the
// slot stride makes the lanes of a quarter warp hit distinct banks.
// Products: <q, c> is computed exactly in integers: the query is scaled by a
// power of two, s = 2^(e - 30) with 2^e <= max|q| < 2^(e+1), and rounded once
// (Q_j = rint(q_j / s), |Q_j| < 2^31; elements within 2^7 of the largest are
// exact), Q is split into four byte planes (three unsigned, the top one
// signed) laid out in code-word order, and dp4a accumulates each plane's
// products with the code bytes in 32 bits; the planes are recombined in 64
// bits, centred by the code offset and scaled by s once per candidate.
// Rounding q moves a score by at most (s / 2) D sum_j |c_j - off|
// <= 2^-31 max|q| d D 2^(B1-1), under 4 % of the float32 tolerance even when
// every rounding error lines up with the codes (one dominant query element,
// one code far from the rest).
constexpr int kGatherThreads = 128;
constexpr int kGW = kGatherThreads / 32;
constexpr uint32_t kNoSlot = 0xFFFFFFFFu;  // an empty row of a batch

__device__ __forceinline__ uint32_t g_dp4a_uu(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("dp4a.u32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ int g_dp4a_us(uint32_t a, uint32_t b, int c) {
  int d;
  asm("dp4a.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
// Dim (within its group of 8) of byte b of the query word that meets code
// bytes in dp4a: for 4-bit codes half h = 0 pairs with (w & 0x0F0F0F0F),
// dims (0, 4, 1, 5), h = 1 with ((w >> 4) & 0x0F0F0F0F), dims (2, 6, 3, 7);
// for 8-bit codes half h is code word h, dims 4h..4h+3.
__device__ __forceinline__ int plane_dim(int bits1, int h, int b) {
  if (bits1 == 4) return (b >> 1) + 4 * (b & 1) + 2 * h;
  return 4 * h + b;
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

struct GatherAcc {
  uint32_t a0, a1, a2;
  int a3;
};
// one code group (two 32-bit words of code bytes) against the four planes
__device__ __forceinline__ void plane_step(GatherAcc& A, uint32_t x0, uint32_t x1, uint2 p0, uint2 p1, uint2 p2,
                                           uint2 p3) {
  A.a0 = g_dp4a_uu(x0, p0.x, g_dp4a_uu(x1, p0.y, A.a0));
  A.a1 = g_dp4a_uu(x0, p1.x, g_dp4a_uu(x1, p1.y, A.a1));
  A.a2 = g_dp4a_uu(x0, p2.x, g_dp4a_uu(x1, p2.y, A.a2));
  A.a3 = g_dp4a_us(x0, p3.x, g_dp4a_us(x1, p3.y, A.a3));
}
__device__ __forceinline__ void group4(GatherAcc& A, uint32_t w, uint2 p0, uint2 p1, uint2 p2, uint2 p3) {
  plane_step(A, w & 0x0F0F0F0Fu, (w >> 4) & 0x0F0F0F0Fu, p0, p1, p2, p3);
}

__global__ void __launch_bounds__(kGatherThreads, 2) gather_kernel(DeviceStore st, const float* __restrict__ q,
                                                                 int64_t nq, QueryPrep p,
                                                                 const int64_t* __restrict__ cand, int n_cand,
                                                                 int k, GatherGeom gg, int64_t* out_ids,
                                                                 float* out_scores) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int d = st.d;
  const int groups = (d + 7) >> 3, gpad = (groups + 3) & ~3;
  const int cap = pow2_at_least(k + 2 * kGatherThreads);  // cuts are rare once the bound is set
  const int R = gg.R, L = 32 / gg.R, P = gg.P;
  unsigned char* slots = smem;  // [kGW][P][slot_bytes]
  uint32_t* slot_ids = reinterpret_cast<uint32_t*>(slots + (size_t)kGW * P * gg.slot_bytes);  // [kGW][P][32]
  uint2* planes = reinterpret_cast<uint2*>(slot_ids + kGW * P * 32);                       // [4][gpad]
  uint64_t* buf = reinterpret_cast<uint64_t*>(planes + 4 * gpad);                         // [cap]
  int* sh_pos = reinterpret_cast<int*>(buf + cap);                                          // [k + 2]
  __shared__ int cnt;
  __shared__ uint64_t thr;
  __shared__ int scan_sh[kGW + 1];
  __shared__ float qmax_sh[kGW];
  __shared__ unsigned long long qsum_int;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool ip = st.metric == LVQ_IP;
  const bool b4 = st.bits1 == 4;
  const int nchunks = b4 ? gpad / 4 : (groups + 1) / 2;
  const int nb = (n_cand + R - 1) / R;  // batches of a query
  const int rounds = (nb + kGW - 1) / kGW;
  const int per_q = nb > w ? (nb - w + kGW - 1) / kGW : 0;  // this warp's batches of a query
  const int64_t my_q = nq > (int64_t)blockIdx.x ? (nq - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const int64_t items = (int64_t)per_q * my_q;
  const int r16 = st.row1 / 16;
  const uint32_t r16_magic = 0xFFFFFFFFu / (uint32_t)r16 + 1u;  // c / r16 == umulhi(c, magic) for c < 2^13
  // This warp's items in order: query blockIdx.x + qk * gridDim.x, batch
  // w + rd * kGW for rd < per_q.  Every issue commits one group (empty past
  // the last item), so waiting for all but the newest P - 1 groups completes
  // the oldest.
  int64_t i_n = 0, i_qk = 0;  // items issued; query iteration of the next one
  int i_rd = 0, i_slot = 0;
  auto issue_next = [&]() {
    if (i_n < items) {
      const int slot = i_slot;
      const int64_t qi = blockIdx.x + i_qk * gridDim.x;
      const int b = w + i_rd * kGW;
      int64_t s = -1;
      if (lane < R) {
        const int i = b * R + lane;
        if (i < n_cand) {
          s = cand[qi * n_cand + i];
          if (s < 0 || s >= st.capacity) s = -1;
        }
        slot_ids[(w * P + slot) * 32 + lane] = s < 0 ? kNoSlot : (uint32_t)s;
      }
      unsigned char* base = slots + (size_t)(w * P + slot) * gg.slot_bytes;
      // chunk c of the batch: row c / r16, column c % r16 (the same trip count
      // on every lane, so that the shuffle has all of them)
      for (int c0 = 0; c0 < R * r16; c0 += 32) {
        const int c = c0 + lane;
        const int row = (int)__umulhi((uint32_t)c, r16_magic), col = c - row * r16;
        const bool in = c < R * r16;
        const int64_t sr = __shfl_sync(kFull, s, in ? row : 0);
        if (in && sr >= 0) cp_async16(base + (size_t)row * gg.stride + 16 * col, st.codes1 + sr * st.stride1 + 16 * col);
      }
      ++i_n;
      if (++i_rd == per_q) {
        i_rd = 0;
        ++i_qk;
      }
      i_slot = i_slot + 1 == P ? 0 : i_slot + 1;
    }
    cp_async_commit();
  };
  // Per-row constants of the next item, loaded one item ahead by the first
  // lane of each row so that their latency hides behind a batch's products.
  const int r = lane / L, l = lane % L;
  bool pf_live = false;
  float pf_lo = 0.0f, pf_stp = 0.0f, pf_nrm = 0.0f;
  int pf_m = 0;
  auto load_consts = [&](int64_t t, int slot) {
    pf_live = false;
    if (t >= i_n || l != 0) return;
    const uint32_t su = slot_ids[(w * P + slot) * 32 + r];
    if (su == kNoSlot) return;
    pf_live = is_live(st.live, su);
    pf_lo = __ldg(st.lower + su);
    pf_stp = __ldg(st.step + su);
    pf_m = __ldg(st.mean_id + su);
    pf_nrm = ip ? 0.0f : __ldg(st.norm2 + su);
  };
  for (int i = 0; i < P - 1; ++i) issue_next();
  __syncwarp();
  load_consts(0, 0);
  int64_t c_n = 0;  // items consumed
  int c_slot = 0;
  const int ioff = b4 ? 8 : 128;
  const float off = code_offset(st.bits1);
  for (int64_t qk = 0; qk < my_q; ++qk) {
    const int64_t qi = blockIdx.x + qk * gridDim.x;
    // ---- the query's byte planes
    const float* qrow = q + qi * d;
    float mx = 0.0f;
    for (int j = threadIdx.x; j < groups * 8; j += blockDim.x) {
      const float v = j < d ? qrow[j] : 0.0f;
      mx = fmaxf(mx, fabsf(v));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
    if (lane == 0) qmax_sh[w] = mx;
    if (threadIdx.x == 0) {
      cnt = 0;
      thr = kNoKey;
      qsum_int = 0ull;
    }
    __syncthreads();
    mx = 0.0f;
#pragma unroll
    for (int i = 0; i < kGW; ++i) mx = fmaxf(mx, qmax_sh[i]);
    // s = 2^qe: q_j / s is exact in float32, so only its fraction is rounded
    const int qe = mx > 0.0f ? ilogbf(mx) - 30 : 0;
    const float qscale = mx > 0.0f ? ldexpf(1.0f, qe) : 0.0f;
    {
      long long part = 0;
      for (int g = threadIdx.x; g < gpad; g += blockDim.x) {
        uint32_t pw[4][2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          pw[0][h] = pw[1][h] = pw[2][h] = pw[3][h] = 0u;
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const int j = 8 * g + plane_dim(st.bits1, h, b);
            const int v = j < d ? max(-2147483647, __float2int_rn(ldexpf(qrow[j], -qe))) : 0;
            part += v;
            pw[0][h] |= (uint32_t)(v & 255) << (8 * b);
            pw[1][h] |= (uint32_t)((v >> 8) & 255) << (8 * b);
            pw[2][h] |= (uint32_t)((v >> 16) & 255) << (8 * b);
            pw[3][h] |= (uint32_t)((v >> 24) & 255) << (8 * b);
          }
        }
#pragma unroll
        for (int pl = 0; pl < 4; ++pl) planes[pl * gpad + g] = make_uint2(pw[pl][0], pw[pl][1]);
      }
      if (part != 0) atomicAdd(&qsum_int, (unsigned long long)part);
    }
    __syncthreads();
    // <Q, c - off> = <Q, c> - off * sum(Q)
    const long long qoff = (long long)qsum_int * ioff;
    const float qs = p.qsum[qi];
    const float qn = ip ? 0.0f : p.qnorm[qi];
    const float* cmq = p.cm + qi * st.n_means;
    const uint4* pl4 = reinterpret_cast<const uint4*>(planes);
    const int pstride4 = gpad / 2;  // uint4 per plane
    for (int rd = 0; rd < rounds; ++rd) {
      if (rd < per_q) {
        issue_next();
        const int slot = c_slot;
        if (P == 3)
          cp_async_wait<2>();
        else
          cp_async_wait<1>();
        __syncwarp();
        {
          const uint32_t su = slot_ids[(w * P + slot) * 32 + r];
          const bool live = pf_live;
          const float lo = pf_lo, stp = pf_stp, nrm = pf_nrm;
          const int m = pf_m;
          c_slot = c_slot + 1 == P ? 0 : c_slot + 1;
          ++c_n;
          load_consts(c_n, c_slot);
          // four accumulator sets (one per code group of a chunk, two chunks at
          // a time) keep the dp4a dependence chains short
          GatherAcc A[4] = {{0u, 0u, 0u, 0}, {0u, 0u, 0u, 0}, {0u, 0u, 0u, 0}, {0u, 0u, 0u, 0}};
          if (su != kNoSlot) {
            const uint4* row = reinterpret_cast<const uint4*>(slots + (size_t)(w * P + slot) * gg.slot_bytes +
                                                              (size_t)r * gg.stride);
            auto lo2 = [](uint4 v) { return make_uint2(v.x, v.y); };
            auto hi2 = [](uint4 v) { return make_uint2(v.z, v.w); };
            auto chunk4 = [&](const uint4 cw, int c) {
              uint4 p[4][2];
#pragma unroll
              for (int pl = 0; pl < 4; ++pl) {
                p[pl][0] = pl4[pl * pstride4 + 2 * c];
                p[pl][1] = pl4[pl * pstride4 + 2 * c + 1];
              }
              group4(A[0], cw.x, lo2(p[0][0]), lo2(p[1][0]), lo2(p[2][0]), lo2(p[3][0]));
              group4(A[1], cw.y, hi2(p[0][0]), hi2(p[1][0]), hi2(p[2][0]), hi2(p[3][0]));
              group4(A[2], cw.z, lo2(p[0][1]), lo2(p[1][1]), lo2(p[2][1]), lo2(p[3][1]));
              group4(A[3], cw.w, hi2(p[0][1]), hi2(p[1][1]), hi2(p[2][1]), hi2(p[3][1]));
            };
            auto chunk8 = [&](const uint4 cw, int c, int h) {
              uint4 p[4];
#pragma unroll
              for (int pl = 0; pl < 4; ++pl) p[pl] = pl4[pl * pstride4 + c];
              plane_step(A[2 * h], cw.x, cw.y, lo2(p[0]), lo2(p[1]), lo2(p[2]), lo2(p[3]));
              plane_step(A[2 * h + 1], cw.z, cw.w, hi2(p[0]), hi2(p[1]), hi2(p[2]), hi2(p[3]));
            };
            int c = l;
            for (; c + L < nchunks; c += 2 * L) {
              const uint4 cw0 = row[c], cw1 = row[c + L];
              if (b4) {
                chunk4(cw0, c);
                chunk4(cw1, c + L);
              } else {
                chunk8(cw0, c, 0);
                chunk8(cw1, c + L, 1);
              }
            }
            if (c < nchunks) {
              if (b4)
                chunk4(row[c], c);
              else
                chunk8(row[c], c, 0);
            }
#pragma unroll
            for (int i = 1; i < 4; ++i) {
              A[0].a0 += A[i].a0;
              A[0].a1 += A[i].a1;
              A[0].a2 += A[i].a2;
              A[0].a3 += A[i].a3;
            }
          }
          // the L lanes of a row are consecutive
          for (int o = L >> 1; o > 0; o >>= 1) {
            A[0].a0 += __shfl_xor_sync(kFull, A[0].a0, o);
            A[0].a1 += __shfl_xor_sync(kFull, A[0].a1, o);
            A[0].a2 += __shfl_xor_sync(kFull, A[0].a2, o);
            A[0].a3 += __shfl_xor_sync(kFull, A[0].a3, o);
          }
          if (l == 0 && live) {
            const long long dot = (long long)A[0].a0 + ((long long)A[0].a1 << 8) + ((long long)A[0].a2 << 16) +
                                  ((long long)A[0].a3 << 24) - qoff;
            const float a = __fmul_rn(qscale, (float)dot);
            float sc = __fmaf_rn(stp, a, __fmaf_rn(__fmaf_rn(off, stp, lo), qs, cmq[m]));
            if (!ip) sc = __fadd_rn(__fadd_rn(qn, nrm), -2.0f * sc);
            const uint64_t key = make_key(sc, su, st.metric);
            if (key < thr) buf[atomicAdd(&cnt, 1)] = key;
          }
          __syncwarp();
        }
      }
      // every thread reads the count before any starts the next round's
      // appends, so all take the same branch
      __syncthreads();
      const int c_now = cnt;
      __syncthreads();
      if (c_now > cap - kGatherThreads) {
        uint64_t t;
        const int kept = block_select_dedupe(buf, cap, cnt, k, scan_sh, &t);
        if (threadIdx.x == 0) {
          cnt = kept;
          thr = t;
        }
        __syncthreads();
      }
    }
    {
      // the last cut sorts only the keys there are (rounded up to a power of two)
      const int n_left = cnt;
      const int span = pow2_at_least(n_left > 32 ? n_left : 32);
      uint64_t t;
      const int kept = block_select_dedupe(buf, span < cap ? span : cap, n_left, k, scan_sh, &t);
      if (threadIdx.x == 0) cnt = kept;
      __syncthreads();
    }
    int64_t* oi = out_ids + qi * k;
    float* os = out_scores + qi * k;
    write_results(buf, cnt, k, st.metric, oi, os, sh_pos);
  }
  cp_async_wait<0>();
}

// ---- ID-gather search with the query in registers (short records) ----------
// One query at a time per 128-thread block (persistent blocks).  A record
// (code words, then the 16-byte trailer l, D, ||x^||^2, mean id) is read by
// L consecutive lanes (a power of two), lane l loading its 16-byte chunk l in
// one access, so a candidate costs one load instruction per lane; lanes
// below row1 / 16 hold four code words each (4-bit: four 8-dim groups,
// 8-bit: two), the lane of chunk row1 / 16 holds the trailer.  Each lane
// keeps the query's four byte planes for its code words in registers for the
// whole query, so a row costs its record read and dp4a, with no shared-memory
// traffic for the query.  Each warp keeps P steps of R = 32 / L rows in
// flight (the loads of step t + P are issued as step t is scored; the
// candidate ids a round earlier still).  The exact integer products and the
// score follow the fixed-point scheme above; the trailer's lane scores the row.
constexpr int kG2Threads = 128;
constexpr int kG2Warps = kG2Threads / 32;
constexpr int kG2Steps = 4;  // steps of R rows each warp keeps in flight

__host__ __device__ inline int pow2_ceil(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

// One 16-byte chunk of a record, asking L2 for its 64-byte half line only:
// a randomly addressed 64-byte record then costs 64 bytes of DRAM traffic,
// not a whole 128-byte line.
__device__ __forceinline__ uint4 ldg_chunk(const void* p) {
  uint4 v;
  asm("ld.global.nc.L2::64B.v4.u32 {%0, %1, %2, %3}, [%4];"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(p));
  return v;
}

template <int BITS, int L>
__global__ void __launch_bounds__(kG2Threads) gather2_kernel(DeviceStore st, const float* __restrict__ q, int64_t nq,
                                                             QueryPrep p, const int64_t* __restrict__ cand, int n_cand,
                                                             int k, int cap, int64_t* out_ids, float* out_scores) {
  constexpr int P = kG2Steps;
  constexpr int GPC = BITS == 4 ? 4 : 2;  // 8-dim code groups per 16-byte chunk
  constexpr int R = 32 / L;
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* buf = reinterpret_cast<uint64_t*>(smem);  // [cap]
  int* sh_pos = reinterpret_cast<int*>(buf + cap);    // [k + 2]
  __shared__ int cnt;
  __shared__ uint64_t thr;
  __shared__ int scan_sh[kG2Warps + 1];
  __shared__ float qmax_sh[kG2Warps];
  __shared__ long long qsum_sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int d = st.d, W = (d + 7) >> 3;  // 8-dim groups
  const int r = lane / L, l = lane % L;
  const int tchunk = st.row1 >> 4;       // the trailer's chunk
  const bool has_chunk = 16 * l < st.stride1;
  const bool scorer = l == tchunk;
  const bool ip = st.metric == LVQ_IP;
  const long long ioff = BITS == 4 ? 8 : 128;
  const float off = BITS == 4 ? 8.0f : 128.0f;
  const int per_round = kG2Warps * P * R;  // rows a round of the block scores
  const int rounds = (n_cand + per_round - 1) / per_round;
  for (int64_t qi = blockIdx.x; qi < nq; qi += gridDim.x) {
    const float* qrow = q + qi * d;
    float mx = 0.0f;
    for (int j = threadIdx.x; j < d; j += blockDim.x) mx = fmaxf(mx, fabsf(qrow[j]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
    if (lane == 0) qmax_sh[warp] = mx;
    if (threadIdx.x == 0) {
      cnt = 0;
      thr = kNoKey;
    }
    __syncthreads();
    mx = 0.0f;
#pragma unroll
    for (int i = 0; i < kG2Warps; ++i) mx = fmaxf(mx, qmax_sh[i]);
    const int qe = mx > 0.0f ? ilogbf(mx) - 30 : 0;
    const float qscale = mx > 0.0f ? ldexpf(1.0f, qe) : 0.0f;
    // this lane's planes: pw[i][plane][half] for group GPC l + i (none past
    // the code chunks)
    uint32_t pw[GPC][4][2];
    long long part = 0;
#pragma unroll
    for (int i = 0; i < GPC; ++i) {
      const int g = GPC * l + i;
      const bool mine = l < tchunk && g < W;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        pw[i][0][h] = pw[i][1][h] = pw[i][2][h] = pw[i][3][h] = 0u;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int j = 8 * g + plane_dim(BITS, h, b);
          const int v = (mine && j < d) ? max(-2147483647, __float2int_rn(ldexpf(qrow[j], -qe))) : 0;
          part += v;
          pw[i][0][h] |= (uint32_t)(v & 255) << (8 * b);
          pw[i][1][h] |= (uint32_t)((v >> 8) & 255) << (8 * b);
          pw[i][2][h] |= (uint32_t)((v >> 16) & 255) << (8 * b);
          pw[i][3][h] |= (uint32_t)((v >> 24) & 255) << (8 * b);
        }
      }
    }
    // sum of the rounded query over all dims: the lanes of row 0 of warp 0
    // hold every group once
    if (warp == 0) {
      if (r != 0) part = 0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(kFull, part, o);
      if (lane == 0) qsum_sh = part;
    }
    __syncthreads();
    const long long qoff = qsum_sh * ioff;
    const float qs = p.qsum[qi];
    const float qn = ip ? 0.0f : p.qnorm[qi];
    const float* cmq = p.cm + qi * st.n_means;
    // the candidate rows of this warp's step t: s = kG2Warps t + warp, rows s R + r
    uint4 ch[P];     // this lane's chunk of the row in flight
    uint32_t lv[P];  // its live word (trailer lane)
    int sid[P];      // slot of the row whose record is in flight
    int nid[P];      // slot of the row one round later (its id read a round ahead)
    // a step's candidate id (-1: skipped); ids are read a round before the
    // records they address, so no record load waits on an id load
    auto load_id = [&](int t) -> int {
      const int i = (kG2Warps * t + warp) * R + r;
      int id = -1;
      if (i < n_cand) {
        const int64_t c = __ldg(cand + qi * n_cand + i);
        if (c >= 0 && c < st.capacity) id = (int)c;
      }
      return id;
    };
    auto load_rec = [&](int id, uint4& chu, uint32_t& lvu) {
      const unsigned char* rec = st.codes1 + (int64_t)(id < 0 ? 0 : id) * st.stride1;
      chu = (id >= 0 && has_chunk) ? ldg_chunk(rec + 16 * l) : make_uint4(0u, 0u, 0u, 0u);
      lvu = (id >= 0 && scorer) ? __ldg(st.live + (id >> 5)) : 0u;
    };
#pragma unroll
    for (int u = 0; u < P; ++u) sid[u] = load_id(u);
#pragma unroll
    for (int u = 0; u < P; ++u) {
      load_rec(sid[u], ch[u], lv[u]);
      nid[u] = load_id(P + u);
    }
    for (int rd = 0; rd < rounds; ++rd) {
#pragma unroll
      for (int u = 0; u < P; ++u) {
        GatherAcc A = {0u, 0u, 0u, 0};
        const uint32_t cw[4] = {ch[u].x, ch[u].y, ch[u].z, ch[u].w};
#pragma unroll
        for (int i = 0; i < GPC; ++i) {
          const uint32_t x0 = BITS == 4 ? (cw[i] & 0x0F0F0F0Fu) : cw[2 * i];
          const uint32_t x1 = BITS == 4 ? ((cw[i] >> 4) & 0x0F0F0F0Fu) : cw[2 * i + 1];
          plane_step(A, x0, x1, make_uint2(pw[i][0][0], pw[i][0][1]), make_uint2(pw[i][1][0], pw[i][1][1]),
                     make_uint2(pw[i][2][0], pw[i][2][1]), make_uint2(pw[i][3][0], pw[i][3][1]));
        }
        // planes 0 + 1 and 2 + 3 in 32 bits each, exactly: with c <= 2^B1 - 1
        // and at most 28 groups of 8 dims (224 dims, 4-bit) or 14 (112,
        // 8-bit), the first pair is at most 8 W (2^B1 - 1) 255 257 < 2^32
        // (unsigned) and the second (plane 3 signed) at most
        // 8 W (2^B1 - 1) (255 + 128 256) < 2^31 in magnitude
        uint32_t lo = A.a0 + (A.a1 << 8);
        int hi = (int)A.a2 + (A.a3 << 8);
#pragma unroll
        for (int o = L >> 1; o > 0; o >>= 1) {
          lo += __shfl_xor_sync(kFull, lo, o);
          hi += __shfl_xor_sync(kFull, hi, o);
        }
        const long long dot = (long long)lo + ((long long)hi << 16);
        const uint4 t4 = ch[u];  // the trailer, in the scoring lane
        const int id = sid[u];
        const bool live = scorer && id >= 0 && ((lv[u] >> (id & 31)) & 1u);
        // refill this slot with step t + P (its id is already here) while the
        // row is scored, and read the id of step t + 2 P
        sid[u] = nid[u];
        load_rec(sid[u], ch[u], lv[u]);
        nid[u] = load_id((rd + 2) * P + u);
        if (live) {
          const float lo_r = __uint_as_float(t4.x), stp = __uint_as_float(t4.y), nrm = __uint_as_float(t4.z);
          const int m = (int)t4.w;
          const float a = __fmul_rn(qscale, (float)(dot - qoff));
          float sc = __fmaf_rn(stp, a, __fmaf_rn(__fmaf_rn(off, stp, lo_r), qs, cmq[m]));
          if (!ip) sc = __fadd_rn(__fadd_rn(qn, nrm), -2.0f * sc);
          const uint64_t key = make_key(sc, (uint32_t)id, st.metric);
          if (key < thr) buf[atomicAdd(&cnt, 1)] = key;
        }
      }
      // every thread reads the count before any starts the next round's
      // appends, so all take the same branch
      __syncthreads();
      const int c_now = cnt;
      __syncthreads();
      if (c_now > cap - per_round) {
        uint64_t t;
        const int kept = block_select_dedupe(buf, cap, cnt, k, scan_sh, &t);
        if (threadIdx.x == 0) {
          cnt = kept;
          thr = t;
        }
        __syncthreads();
      }
    }
    {
      // the last cut sorts only the keys there are (rounded up to a power of two)
      const int n_left = cnt;
      const int span = pow2_at_least(n_left > 32 ? n_left : 32);
      uint64_t t;
      const int kept = block_select_dedupe(buf, span < cap ? span : cap, n_left, k, scan_sh, &t);
      if (threadIdx.x == 0) cnt = kept;
      __syncthreads();
    }
    write_results(buf, cnt, k, st.metric, out_ids + qi * k, out_scores + qi * k, sh_pos);
    __syncthreads();
  }
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
  static std::atomic<uint64_t> attr{0};
  const cudaError_t e = max_dyn_smem_once((const void*)merge_rerank_kernel<T>, 200 * 1024, attr);
  if (e != cudaSuccess) return e;
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
  static std::atomic<uint64_t> attr{0};
  const cudaError_t e = max_dyn_smem_once((const void*)rerank_kernel, 200 * 1024, attr);
  if (e != cudaSuccess) return e;
  rerank_kernel<<<(unsigned)nq, kRerankThreads, sm, stream>>>(st, q, ids, k1, k, out_ids, out_scores);
  return cudaGetLastError();
}

GatherGeom gather_geom(int row1, int d, int k) {
  // The widest batches (fewest per-batch steps per row, at least 16 rows)
  // with three slots per warp, else two, that let three blocks share an SM,
  // else two (more warps to issue while others wait on their rings; one
  // block's select overlaps the others' streaming); failing that, the widest
  // that fit at all.  Each batch holds at most kGatherSlotBudget bytes.
  // Measured at d = 768, 4-bit, 1,024 x 2,048 ids: 3 blocks x 16-row batches
  // 0.43 ms, 2 blocks x 32 rows 0.49 ms, 4 blocks x 8 rows 0.63 ms.
  const int r16 = row1 / 16;
  const int groups = (d + 7) / 8, gpad = (groups + 3) & ~3;
  (void)groups;
  const size_t rest = (size_t)pow2_at_least(k + 2 * kGatherThreads) * 8 + (size_t)gpad * 4 * 8 + (size_t)(k + 2) * 4 + 16;
  GatherGeom g{};
  for (const size_t budget : {kGatherSmemBudget / 3 - 1024, kGatherSmemBudget / 2 - 1024, kGatherSmemBudget}) {
    for (int R = 32; R >= 1; R >>= 1) {
      if (budget < kGatherSmemBudget && R < 16) break;
      const int L = 32 / R;
      int s16 = r16;
      if (L < 8)
        while (s16 % (2 * L) != L) ++s16;  // the rows of a quarter warp start in distinct banks
      g.R = R;
      g.stride = s16 * 16;
      g.slot_bytes = R * g.stride;
      if (g.slot_bytes > kGatherSlotBudget && R > 1) continue;
      for (g.P = 3; g.P >= 2; --g.P) {
        g.smem = (size_t)kGW * g.P * (g.slot_bytes + 32 * 4) + rest;
        if (g.smem <= budget) return g;
      }
    }
  }
  return g;  // does not fit: the launcher refuses it
}

// Lanes per row of gather2_kernel: the record's 16-byte chunks rounded up to
// a power of two, 2 to 8 (records of up to 128 bytes: d <= 224 at 4 bits,
// d <= 112 at 8); 0 when the record is longer (the ring kernel takes it).
static int gather2_lanes(const DeviceStore& st) {
  if (st.bits1 != 4 && st.bits1 != 8) return 0;
  const int l = pow2_ceil((int)(st.stride1 / 16));
  return l >= 2 && l <= 8 ? l : 0;
}

template <int BITS, int L>
static cudaError_t launch_gather2_t(const DeviceStore& st, const float* q, int64_t nq, const QueryPrep& p,
                                    const int64_t* cand, int n_cand, int k, int64_t* out_ids, float* out_scores,
                                    cudaStream_t stream) {
  const int per_round = kG2Warps * kG2Steps * (32 / L);
  const int cap = pow2_at_least(k + 2 * per_round);
  const size_t smem = (size_t)cap * 8 + (size_t)(k + 2) * 4 + 16;
  static std::atomic<uint64_t> attr{0};
  {
    const cudaError_t e = max_dyn_smem_once((const void*)gather2_kernel<BITS, L>, 200 * 1024, attr);
    if (e != cudaSuccess) return e;
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gather2_kernel<BITS, L>, kG2Threads, smem);
  if (per_sm < 1) per_sm = 1;
  const int64_t grid = std::min<int64_t>(nq, (int64_t)sms * per_sm);
  gather2_kernel<BITS, L><<<(unsigned)grid, kG2Threads, smem, stream>>>(st, q, nq, p, cand, n_cand, k, cap, out_ids,
                                                                          out_scores);
  return cudaGetLastError();
}

cudaError_t launch_gather(const DeviceStore& st, const float* q, int64_t nq, const QueryPrep& p,
                          const int64_t* cand, int n_cand, int k, int64_t* out_ids, float* out_scores,
                          cudaStream_t stream) {
  if (nq <= 0) return cudaSuccess;
  const int L = gather2_lanes(st);
  if (L > 0) {
    const bool b4 = st.bits1 == 4;
#define LVQ_G2(b, l) launch_gather2_t<b, l>(st, q, nq, p, cand, n_cand, k, out_ids, out_scores, stream)
    switch (L) {
      case 2: return b4 ? LVQ_G2(4, 2) : LVQ_G2(8, 2);
      case 4: return b4 ? LVQ_G2(4, 4) : LVQ_G2(8, 4);
      default: return b4 ? LVQ_G2(4, 8) : LVQ_G2(8, 8);
    }
#undef LVQ_G2
  }
  // wider rows: the shared-memory ring kernel
  const GatherGeom g = gather_geom(st.row1, st.d, k);
  if (g.smem > kGatherSmemBudget) return cudaErrorInvalidValue;
  static std::atomic<uint64_t> attr{0};
  {
    const cudaError_t e = max_dyn_smem_once((const void*)gather_kernel, (int)kGatherSmemBudget, attr);
    if (e != cudaSuccess) return e;
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gather_kernel, kGatherThreads, g.smem);
  if (per_sm < 1) per_sm = 1;
  const int64_t grid = std::min<int64_t>(nq, (int64_t)sms * per_sm);
  gather_kernel<<<(unsigned)grid, kGatherThreads, g.smem, stream>>>(st, q, nq, p, cand, n_cand, k, g, out_ids,
                                                                   out_scores);
  return cudaGetLastError();
}

}  // namespace lvq
