// Plain float32 first-level scan on CUDA cores (Sec. 3.2 scoring, fused with
// top-k1 selection).  A persistent CTA takes work items (a group of QB
// queries, a range of database rows); each of its 256 threads scores one
// database row per tile against the QB queries held in shared memory.
//   IP:  s = <q, mu_m> + (l + off*D) sum(q) + D * sum_j q_j (c_j - off)
//   L2:  s = sum_j (q_j - mu_mj - (l + D c_j))^2    (direct difference)
// Keys better than the query's running threshold are appended to a
// per-(CTA, query) buffer in global memory (L2-resident), compacted by one
// warp when it fills.  At the end of an item every query's k1 best keys go
// to partial[q][split].
#include "kernels.cuh"
#include "score.cuh"

namespace lvq {

namespace {

constexpr int kThreads = 256;

struct Fp32Args {
  DeviceStore st;
  const float* q;
  int64_t nq;
  QueryPrep p;
  ScanPlan plan;
  int cap;         // candidate buffer capacity per query (power of two)
  int kd;          // dims held per query in shared memory (whole 16-byte chunks)
  int chunks;      // 16-byte code chunks per row that hold real dims
  int64_t tiles_per_split;
};

template <int QB, int BITS>
__global__ void __launch_bounds__(kThreads) scan_fp32_kernel(Fp32Args a) {
  extern __shared__ __align__(16) unsigned char smem[];
  float* qs = reinterpret_cast<float*>(smem);  // [QB][kd]
  __shared__ int cnt[QB];
  __shared__ uint64_t thr[QB];
  __shared__ float qsum_s[QB];
  __shared__ int hist[kThreads / 32][288];
  const DeviceStore& st = a.st;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const bool ip = st.metric == LVQ_IP;
  const bool one_mean = st.n_means == 1;
  const float off = code_offset(BITS);
  constexpr int DPC = BITS == 4 ? 32 : 16;  // dims per 16-byte chunk
  const int64_t ntiles = ceil_div(a.plan.n_rows, kThreads);
  const int64_t ngroups = ceil_div(a.nq, QB);
  const int64_t items = ngroups * a.plan.splits;
  const int k1 = a.plan.k1;
  uint64_t* mybuf = a.plan.cand + (int64_t)blockIdx.x * QB * a.cap;

  for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
    const int64_t grp = item / a.plan.splits;
    const int split = (int)(item % a.plan.splits);
    const int64_t q0 = grp * QB;
    // queries of the group (zero rows beyond nq); L2 with one mean: q - mu
    for (int i = tid; i < QB * a.kd; i += kThreads) {
      const int b = i / a.kd, j = i % a.kd;
      float v = 0.0f;
      if (q0 + b < a.nq && j < st.d) {
        v = a.q[(q0 + b) * st.d + j];
        if (!ip && one_mean) v = __fsub_rn(v, st.means[j]);
      }
      qs[i] = v;
    }
    if (tid < QB) {
      cnt[tid] = 0;
      thr[tid] = (q0 + tid < a.nq) ? kNoKey : 0ull;  // absent queries accept nothing
      qsum_s[tid] = (ip && q0 + tid < a.nq) ? a.p.qsum[q0 + tid] : 0.0f;
    }
    __syncthreads();
    const int64_t t_begin = split * a.tiles_per_split;
    const int64_t t_end = min(ntiles, t_begin + a.tiles_per_split);
    for (int64_t tile = t_begin; tile < t_end; ++tile) {
      const int64_t row = tile * kThreads + tid;
      if (row < a.plan.n_rows && is_live(st.live, row)) {
        const uint4* codes = reinterpret_cast<const uint4*>(st.codes1 + row * st.stride1);
        const float lo = __ldg(st.lower + row), step = __ldg(st.step + row);
        const int m = __ldg(st.mean_id + row);
        const float* mu = st.means + (int64_t)m * st.d;
        float tot[QB];
#pragma unroll
        for (int b = 0; b < QB; ++b) tot[b] = 0.0f;
        for (int ch = 0; ch < a.chunks; ++ch) {
          const uint4 w4 = __ldg(codes + ch);
          const uint32_t ws[4] = {w4.x, w4.y, w4.z, w4.w};
          float c[DPC];
          const float sub = ip ? 8388608.0f + off : 8388608.0f;
#pragma unroll
          for (int wi = 0; wi < 4; ++wi) {
            if (BITS == 4) {
#pragma unroll
              for (int p = 0; p < 4; ++p) {
                const uint32_t t = nib_pair(ws[wi], p);
                c[wi * 8 + 2 * p] = lo_centred(t, sub);
                c[wi * 8 + 2 * p + 1] = hi_centred(t, sub);
              }
            } else {
#pragma unroll
              for (int i = 0; i < 4; ++i) c[wi * 4 + i] = byte_centred(ws[wi], i, sub);
            }
          }
          const int j0 = ch * DPC;
          if (!ip) {
            // reconstruction (centred for one mean, else with mu_m)
#pragma unroll
            for (int e = 0; e < DPC; ++e) {
              float xh = __fmaf_rn(step, c[e], lo);
              if (!one_mean) xh = __fadd_rn(xh, (j0 + e < st.d) ? __ldg(mu + j0 + e) : 0.0f);
              c[e] = (j0 + e < st.d) ? xh : 0.0f;
            }
          }
#pragma unroll
          for (int b = 0; b < QB; ++b) {
            const float4* qv = reinterpret_cast<const float4*>(qs + b * a.kd + j0);
            float part = 0.0f;
#pragma unroll
            for (int e4 = 0; e4 < DPC / 4; ++e4) {
              const float4 qq = qv[e4];
              const float qa[4] = {qq.x, qq.y, qq.z, qq.w};
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                if (ip) {
                  part = __fmaf_rn(qa[u], c[e4 * 4 + u], part);
                } else {
                  const float df = qa[u] - c[e4 * 4 + u];
                  part = __fmaf_rn(df, df, part);
                }
              }
            }
            tot[b] += part;
          }
        }
        const float base_ip = __fmaf_rn(off, step, lo);
#pragma unroll
        for (int b = 0; b < QB; ++b) {
          if (q0 + b < a.nq) {
            float sc = tot[b];
            if (ip) sc = __fmaf_rn(step, sc, __fmaf_rn(base_ip, qsum_s[b], a.p.cm[(q0 + b) * st.n_means + m]));
            const uint64_t key = make_key(sc, (uint32_t)row, st.metric);
            if (key < thr[b]) mybuf[b * a.cap + atomicAdd(&cnt[b], 1)] = key;
          }
        }
      }
      __syncthreads();
      // compaction of the buffers that may not take another tile
      for (int b = wid; b < QB; b += kThreads / 32) {
        if (cnt[b] > a.cap - kThreads) {
          uint64_t t;
          const int kept = warp_select(mybuf + b * a.cap, cnt[b], k1, hist[wid], &t);
          if (lane == 0) {
            cnt[b] = kept;
            thr[b] = t;
          }
        }
      }
      __syncthreads();
    }
    // final: each query's k1 best (unsorted) to partial[q][split]
    for (int b = wid; b < QB; b += kThreads / 32) {
      if (q0 + b >= a.nq) continue;
      uint64_t t;
      const int kept = warp_select(mybuf + b * a.cap, cnt[b], k1, hist[wid], &t);
      uint64_t* dst = a.plan.partial + ((q0 + b) * a.plan.splits + split) * k1;
      for (int i = lane; i < k1; i += 32) dst[i] = i < kept ? mybuf[b * a.cap + i] : kNoKey;
    }
    __syncthreads();
  }
}

template <int QB, int BITS>
cudaError_t launch_t(const Fp32Args& a, size_t smem, int grid, cudaStream_t stream) {
  static std::atomic<uint64_t> attr{0};
  const cudaError_t e = max_dyn_smem_once((const void*)scan_fp32_kernel<QB, BITS>, 160 * 1024, attr);
  if (e != cudaSuccess) return e;
  scan_fp32_kernel<QB, BITS><<<grid, kThreads, smem, stream>>>(a);
  return cudaGetLastError();
}

template <int BITS>
cudaError_t launch_bits(int qb, const Fp32Args& a, size_t smem, int grid, cudaStream_t stream) {
  switch (qb) {
    case 1: return launch_t<1, BITS>(a, smem, grid, stream);
    case 2: return launch_t<2, BITS>(a, smem, grid, stream);
    case 4: return launch_t<4, BITS>(a, smem, grid, stream);
    case 8: return launch_t<8, BITS>(a, smem, grid, stream);
    default: return launch_t<16, BITS>(a, smem, grid, stream);
  }
}

}  // namespace

int fp32_scan_grid(const DeviceStore& st, int qb, int sm_count) {
  const int code_bytes = (int)ceil_div((int64_t)st.d * st.bits1, 8);
  const int kd = (int)ceil_div(code_bytes, 16) * (st.bits1 == 4 ? 32 : 16);
  const size_t smem = (size_t)qb * kd * 4;
  int per_sm = 0;
  cudaError_t e;
  if (st.bits1 == 4) {
    switch (qb) {
      case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scan_fp32_kernel<1, 4>, kThreads, smem); break;
      case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scan_fp32_kernel<2, 4>, kThreads, smem); break;
      case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scan_fp32_kernel<4, 4>, kThreads, smem); break;
      case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scan_fp32_kernel<8, 4>, kThreads, smem); break;
      default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scan_fp32_kernel<16, 4>, kThreads, smem); break;
    }
  } else {
    switch (qb) {
      case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scan_fp32_kernel<1, 8>, kThreads, smem); break;
      case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scan_fp32_kernel<2, 8>, kThreads, smem); break;
      case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scan_fp32_kernel<4, 8>, kThreads, smem); break;
      case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scan_fp32_kernel<8, 8>, kThreads, smem); break;
      default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scan_fp32_kernel<16, 8>, kThreads, smem); break;
    }
  }
  if (e != cudaSuccess || per_sm < 1) per_sm = 1;
  return sm_count * per_sm;
}

size_t fp32_scan_cand_bytes(int grid, int qb, int k1) {
  return (size_t)grid * qb * pow2_at_least(k1 + kThreads) * 8;
}

cudaError_t launch_scan_fp32(const DeviceStore& st, const float* q, int64_t nq, const QueryPrep& p, int qb,
                             const ScanPlan& plan, cudaStream_t stream) {
  if (nq <= 0) return cudaSuccess;
  Fp32Args a;
  a.st = st;
  a.q = q;
  a.nq = nq;
  a.p = p;
  a.plan = plan;
  a.cap = pow2_at_least(plan.k1 + kThreads);
  const int code_bytes = (int)ceil_div((int64_t)st.d * st.bits1, 8);
  a.chunks = (int)ceil_div(code_bytes, 16);
  a.kd = a.chunks * (st.bits1 == 4 ? 32 : 16);
  const int64_t ntiles = ceil_div(plan.n_rows, kThreads);
  a.tiles_per_split = ceil_div(ntiles > 0 ? ntiles : 1, plan.splits);
  const size_t smem = (size_t)qb * a.kd * 4;
  return st.bits1 == 4 ? launch_bits<4>(qb, a, smem, plan.grid, stream)
                       : launch_bits<8>(qb, a, smem, plan.grid, stream);
}

}  // namespace lvq
