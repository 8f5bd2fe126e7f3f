// Greedy beam search over a graph (Alg. 1), one CTA per query.
//
// The search list holds at most L keys sorted in shared memory: the
// first-level score in the high word and (id << 1 | expanded) in the low
// word, so that equal scores order by id whether or not a node has been
// expanded (ids are below 2^31).  The k1 best leave as plain (score, id) keys.
// Each step expands the best listed node not yet expanded: its out-
// neighbours that are live and not seen before (an open-addressing set in
// shared memory) are scored with the first level in float32, one warp per
// neighbour, appended behind the list, and the list is re-sorted and cut
// back to L.  The search ends when every listed node is expanded or after
// max_expand expansions (the seen set then still has room).  The k1 best
// keys go to out[q][0..k1); re-ranking is a separate launch.
#include "kernels.cuh"
#include "score.cuh"

namespace lvq {

namespace {

constexpr int kBeamThreads = 256;
constexpr uint32_t kExpanded = 1u;  // low bit of a list key's id word

// First-level float32 score of slot s by one warp (valid in every lane):
// x1_j = mu_mj + l + D c_j; L2: sum (q_j - x1_j)^2, IP: sum q_j x1_j.
__device__ __forceinline__ float score1_warp(const DeviceStore& st, int64_t s, const float* qsh) {
  const int lane = threadIdx.x & 31;
  const int d = st.d;
  const int groups = (d + 7) >> 3;
  const float lo = __ldg(st.lower + s), step = __ldg(st.step + s);
  const float* mu = st.means + (int64_t)__ldg(st.mean_id + s) * d;
  const uint8_t* row1 = st.codes1 + s * st.stride1;
  float acc = 0.0f;
  for (int g = lane; g < groups; g += 32) {
    float c[8];
    group_codes(row1, st.bits1, g, 8388608.0f, c);
    float part = 0.0f;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int j = g * 8 + e;
      if (j < d) {
        const float x1 = __fadd_rn(__fmaf_rn(step, c[e], lo), __ldg(mu + j));
        if (st.metric == LVQ_L2) {
          const float df = qsh[j] - x1;
          part = __fmaf_rn(df, df, part);
        } else {
          part = __fmaf_rn(qsh[j], x1, part);
        }
      }
    }
    acc += part;
  }
  return warp_sum(acc);
}

// true when id was not in the set (and is now); set: H slots of id + 1, 0 = empty
__device__ __forceinline__ bool set_insert(int* set, int H, int id) {
  uint32_t h = ((uint32_t)id * 2654435761u) & (H - 1);
  for (int probe = 0; probe < H; ++probe, h = (h + 1) & (H - 1)) {
    const int old = atomicCAS(set + h, 0, id + 1);
    if (old == 0) return true;
    if (old == id + 1) return false;
  }
  return false;  // full: treated as seen (not reached: the set has room for every insert)
}

__global__ void __launch_bounds__(kBeamThreads) beam_kernel(DeviceStore st, const float* __restrict__ q,
                                                            const int32_t* __restrict__ graph, int64_t n_graph, int R,
                                                            const int64_t* __restrict__ starts, int n_starts, int L,
                                                            int max_expand, int H, int k1, uint64_t* out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int LP = pow2_at_least(L + R);
  uint64_t* list = reinterpret_cast<uint64_t*>(smem);  // [LP]
  int* set = reinterpret_cast<int*>(list + LP);        // [H]
  float* qsh = reinterpret_cast<float*>(set + H);      // [d]
  __shared__ int cnt, nnew, sel;
  const int qi = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = threadIdx.x; j < st.d; j += blockDim.x) qsh[j] = q[(int64_t)qi * st.d + j];
  for (int i = threadIdx.x; i < H; i += blockDim.x) set[i] = 0;
  for (int i = threadIdx.x; i < LP; i += blockDim.x) list[i] = kNoKey;
  if (threadIdx.x == 0) {
    cnt = 0;
    nnew = 0;
  }
  __syncthreads();
  // the start nodes, one warp each
  for (int i = warp; i < n_starts; i += nw) {
    const int64_t s = starts[i];
    bool take = false;
    if (lane == 0) take = s >= 0 && s < n_graph && is_live(st.live, s) && set_insert(set, H, (int)s);
    take = __shfl_sync(kFull, take, 0);
    if (take) {
      const float sc = score1_warp(st, s, qsh);
      if (lane == 0) list[atomicAdd(&nnew, 1)] = make_key(sc, (uint32_t)s << 1, st.metric);
    }
  }
  __syncthreads();
  block_sort(list, LP);
  if (threadIdx.x == 0) {
    cnt = nnew < L ? nnew : L;
    nnew = 0;
  }
  __syncthreads();
  for (int step = 0; step < max_expand; ++step) {
    // the best listed node not yet expanded (the list is sorted)
    if (warp == 0) {
      int found = -1;
      for (int base = 0; base < cnt && found < 0; base += 32) {
        const int i = base + lane;
        const bool open = i < cnt && !((uint32_t)list[i] & kExpanded);
        const unsigned b = __ballot_sync(kFull, open);
        if (b) found = base + __ffs(b) - 1;
      }
      if (lane == 0) {
        sel = found;
        if (found >= 0) list[found] |= kExpanded;
      }
    }
    __syncthreads();
    if (sel < 0) break;
    const int node = (int)((uint32_t)list[sel] >> 1);
    const int32_t* nb = graph + (int64_t)node * R;
    for (int r = warp; r < R; r += nw) {
      const int u = nb[r];
      bool take = false;
      if (lane == 0) take = u >= 0 && u < n_graph && is_live(st.live, u) && set_insert(set, H, u);
      take = __shfl_sync(kFull, take, 0);
      if (take) {
        const float sc = score1_warp(st, u, qsh);
        if (lane == 0) list[L + atomicAdd(&nnew, 1)] = make_key(sc, (uint32_t)u << 1, st.metric);
      }
    }
    __syncthreads();
    if (nnew > 0) {
      // list[0, cnt) sorted, list[cnt, L) empty, new keys at [L, L + nnew)
      block_sort(list, LP);
      if (threadIdx.x == 0) {
        const int t = cnt + nnew;
        cnt = t < L ? t : L;
      }
      __syncthreads();
      for (int i = L + threadIdx.x; i < LP; i += blockDim.x) list[i] = kNoKey;
      if (threadIdx.x == 0) nnew = 0;
    }
    __syncthreads();
  }
  uint64_t* dst = out + (int64_t)qi * k1;
  for (int i = threadIdx.x; i < k1; i += blockDim.x) {
    uint64_t v = i < cnt ? list[i] : kNoKey;
    if (v != kNoKey) v = (v & 0xFFFFFFFF00000000ull) | ((uint32_t)v >> 1);
    dst[i] = v;
  }
}

// keys -> ids (the re-rank input)
__global__ void keys_to_ids(const uint64_t* keys, int64_t n, int64_t* ids) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) ids[i] = keys[i] == kNoKey ? -1 : (int64_t)(uint32_t)keys[i];
}

// the k best of each query's k1 sorted keys as (id, score), padded -1 / +-inf
__global__ void keys_to_results(const uint64_t* keys, int64_t nq, int k1, int k, int metric, int64_t* out_ids,
                                float* out_scores) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq * k) return;
  const int64_t qi = i / k;
  const int j = (int)(i % k);
  const uint64_t v = keys[qi * k1 + j];
  out_ids[i] = v == kNoKey ? -1 : (int64_t)(uint32_t)v;
  out_scores[i] = v == kNoKey ? (metric == LVQ_IP ? __int_as_float(0xff800000) : __int_as_float(0x7f800000))
                              : key_score(v, metric);
}

}  // namespace

int beam_set_slots(int n_starts, int R, int max_expand) {
  return pow2_at_least(2 * (n_starts + R * max_expand) + 1);
}

size_t beam_smem(const DeviceStore& st, int L, int R, int H) {
  return (size_t)pow2_at_least(L + R) * 8 + (size_t)H * 4 + (size_t)st.d * 4;
}

cudaError_t launch_beam(const DeviceStore& st, const float* q, int64_t nq, const int32_t* graph, int64_t n_graph,
                        int R, const int64_t* starts, int n_starts, int L, int max_expand, int k1, uint64_t* keys,
                        int64_t* ids, cudaStream_t stream) {
  if (nq <= 0) return cudaSuccess;
  const int H = beam_set_slots(n_starts, R, max_expand);
  const size_t sm = beam_smem(st, L, R, H);
  // the kernel also has a few bytes of static shared memory
  static std::atomic<uint64_t> attr{0};
  {
    const cudaError_t ea = max_dyn_smem_once((const void*)beam_kernel, 220 * 1024, attr);
    if (ea != cudaSuccess) return ea;
  }
  beam_kernel<<<(unsigned)nq, kBeamThreads, sm, stream>>>(st, q, graph, n_graph, R, starts, n_starts, L, max_expand,
                                                          H, k1, keys);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t n = nq * k1;
  keys_to_ids<<<(unsigned)ceil_div(n, 256), 256, 0, stream>>>(keys, n, ids);
  return cudaGetLastError();
}

cudaError_t launch_keys_to_results(const uint64_t* keys, int64_t nq, int k1, int k, int metric, int64_t* out_ids,
                                  float* out_scores, cudaStream_t stream) {
  const int64_t n = nq * k;
  if (n <= 0) return cudaSuccess;
  keys_to_results<<<(unsigned)ceil_div(n, 256), 256, 0, stream>>>(keys, nq, k1, k, metric, out_ids, out_scores);
  return cudaGetLastError();
}

}  // namespace lvq
