// LVQ encoding (Eq. 1-3, Def. 1, Sec. 2.2) and the store's slot management
// (inserts into free slots, lazy deletes, export of stored records).
#include "kernels.cuh"
#include "topk.cuh"

namespace lvq {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(FULL, v, o));
  return v;
}
__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(FULL, v, o));
  return v;
}
// Sum over the warp; every lane receives lane 0's total so that all lanes
// take the same decisions from it.
__device__ __forceinline__ float warp_sum_bcast(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(FULL, v, o));
  return __shfl_sync(FULL, v, 0);
}

// One code of the scalar quantiser Q_{B,l,u} (Eq. 2) in the reciprocal form:
// floor(fl(fl(inv * fl(v - l)) + 1/2)) clamped to [0, maxc].  Every operation
// is rounded separately (the _rn intrinsics are never contracted into FMAs).
__device__ __forceinline__ uint32_t quant_code(float v, float lo, float inv, float maxc) {
  float t = __fadd_rn(__fmul_rn(inv, __fsub_rn(v, lo)), 0.5f);
  t = fminf(fmaxf(floorf(t), 0.0f), maxc);
  return (uint32_t)t;
}

// WPL = groups of 8 dims handled by each lane (group g = lane + 32*i).
template <int WPL>
__global__ void __launch_bounds__(256) encode_kernel(DeviceStore st, const float* __restrict__ x,
                                                     int64_t n, EncodeOut out) {
  const int lane = threadIdx.x & 31;
  const int warps = blockDim.x >> 5;
  const int d = st.d;
  const int groups = (d + 7) >> 3;
  const float maxc1 = (float)st.lev1;  // 2^B1 - 1
  if (out.abort_flag && *out.abort_flag) return;

  for (int64_t v = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5); v < n;
       v += (int64_t)gridDim.x * warps) {
    float xv[WPL][8];
    const float* xr = x + v * d;
#pragma unroll
    for (int i = 0; i < WPL; ++i) {
      const int g = lane + 32 * i;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int j = g * 8 + e;
        xv[i][e] = (g < groups && j < d) ? __ldg(xr + j) : 0.0f;
      }
    }
    // Def. 1: nearest centre, lowest index on ties (or the forced one).
    int m_star = out.force_mean >= 0 ? out.force_mean : 0;
    if (st.n_means > 1 && out.force_mean < 0) {
      float best = __int_as_float(0x7f800000);
      for (int m = 0; m < st.n_means; ++m) {
        const float* mu = st.means + (int64_t)m * d;
        float part = 0.0f;
#pragma unroll
        for (int i = 0; i < WPL; ++i) {
          const int g = lane + 32 * i;
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int j = g * 8 + e;
            if (g < groups && j < d) {
              const float t = __fsub_rn(xv[i][e], __ldg(mu + j));
              part = __fmaf_rn(t, t, part);
            }
          }
        }
        const float tot = warp_sum_bcast(part);
        if (tot < best) { best = tot; m_star = m; }
      }
    }
    const float* mu = st.means + (int64_t)m_star * d;
    // Eq. 1: centred vector and its bounds (max / min are exact).
    float hi = __int_as_float(0xff800000), lo = __int_as_float(0x7f800000);
#pragma unroll
    for (int i = 0; i < WPL; ++i) {
      const int g = lane + 32 * i;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int j = g * 8 + e;
        if (g < groups && j < d) {
          xv[i][e] = __fsub_rn(xv[i][e], __ldg(mu + j));
          hi = fmaxf(hi, xv[i][e]);
          lo = fminf(lo, xv[i][e]);
        }
      }
    }
    hi = warp_max(hi);
    lo = warp_min(lo);
    // Eq. 2: step and its reciprocal (a zero step codes with a unit step).
    const float step = __fdiv_rn(__fsub_rn(hi, lo), maxc1);
    const float inv = __frcp_rn(step == 0.0f ? 1.0f : step);
    // Second level: the text's grid Q_{B2,-D/2,D/2} (Sec. 2.2) or the App. C
    // listing's signed grid (step D/2^B2, exact; no offset)
    float step2 = 0.0f, inv2 = 0.0f, lo2 = 0.0f;
    if (st.bits2) {
      if (st.grid2) {
        step2 = __fmul_rn(step, __int_as_float((127 - st.b2) << 23));
      } else {
        lo2 = __fmul_rn(-step, 0.5f);
        step2 = __fdiv_rn(step, (float)st.lev2);
      }
      inv2 = __frcp_rn(step2 == 0.0f ? 1.0f : step2);
    }
    const float half2 = (float)(1 << (st.b2 > 0 ? st.b2 - 1 : 0));
    uint32_t c1[WPL][8], c2[WPL][8];
    float nrm = 0.0f;
#pragma unroll
    for (int i = 0; i < WPL; ++i) {
      const int g = lane + 32 * i;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int j = g * 8 + e;
        c1[i][e] = 0;
        c2[i][e] = 0;
        if (g < groups && j < d) {
          const float y = xv[i][e];
          c1[i][e] = quant_code(y, lo, inv, maxc1);
          const float yhat = __fadd_rn(__fmul_rn(step, (float)c1[i][e]), lo);
          const float xh = __fadd_rn(__ldg(mu + j), yhat);
          nrm = __fmaf_rn(xh, xh, nrm);
          if (st.bits2) {
            const float r = __fsub_rn(y, yhat);
            if (st.grid2) {
              // round half to even, clipped to [-2^(B2-1), 2^(B2-1) - 1],
              // kept as the two's complement byte
              const float t = fminf(fmaxf(rintf(__fmul_rn(inv2, r)), -half2), half2 - 1.0f);
              c2[i][e] = (uint32_t)((int)t & 255);
            } else {
              c2[i][e] = quant_code(r, lo2, inv2, (float)st.lev2);
            }
          }
        }
      }
    }
    nrm = warp_sum_bcast(nrm);

    if (out.slots == nullptr) {
      // plain layout: one code per byte
#pragma unroll
      for (int i = 0; i < WPL; ++i) {
        const int g = lane + 32 * i;
        if (g < groups) {
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int j = g * 8 + e;
            if (j < d) {
              out.codes1[v * d + j] = (uint8_t)c1[i][e];
              if (out.codes2) out.codes2[v * d + j] = (uint8_t)c2[i][e];
            }
          }
        }
      }
      if (lane == 0) {
        out.lower[v] = lo;
        out.step[v] = step;
        out.mean_id[v] = (uint8_t)m_star;
      }
    } else {
      const int64_t s = out.slots[v];
      if (s < 0) continue;
      uint32_t* row1 = reinterpret_cast<uint32_t*>(st.codes1 + s * st.stride1);
      const int words1 = st.row1 >> 2;
#pragma unroll
      for (int i = 0; i < WPL; ++i) {
        const int g = lane + 32 * i;
        if (g < groups) {
          if (st.bits1 == 4) {
            uint32_t w = 0;
#pragma unroll
            for (int p = 0; p < 4; ++p) w |= (c1[i][2 * p] << (4 * p)) | (c1[i][2 * p + 1] << (16 + 4 * p));
            row1[g] = w;
          } else {
            row1[2 * g] = c1[i][0] | (c1[i][1] << 8) | (c1[i][2] << 16) | (c1[i][3] << 24);
            row1[2 * g + 1] = c1[i][4] | (c1[i][5] << 8) | (c1[i][6] << 16) | (c1[i][7] << 24);
          }
        }
      }
      const int used1 = st.bits1 == 4 ? groups : 2 * groups;
      for (int w = used1 + lane; w < words1; w += 32) row1[w] = 0u;
      if (st.bits2) {
        uint32_t* row2 = reinterpret_cast<uint32_t*>(st.codes2 + s * st.row2);
#pragma unroll
        for (int i = 0; i < WPL; ++i) {
          const int g = lane + 32 * i;
          if (g < groups) {
            row2[2 * g] = c2[i][0] | (c2[i][1] << 8) | (c2[i][2] << 16) | (c2[i][3] << 24);
            row2[2 * g + 1] = c2[i][4] | (c2[i][5] << 8) | (c2[i][6] << 16) | (c2[i][7] << 24);
          }
        }
        for (int w = 2 * groups + lane; w < (st.row2 >> 2); w += 32) row2[w] = 0u;
      }
      if (lane == 0) {
        st.lower[s] = lo;
        st.step[s] = step;
        st.mean_id[s] = (uint8_t)m_star;
        st.norm2[s] = nrm;
        // the record's trailer: the same constants beside the codes
        *reinterpret_cast<uint4*>(st.codes1 + s * st.stride1 + st.row1) =
            make_uint4(__float_as_uint(lo), __float_as_uint(step), __float_as_uint(nrm), (uint32_t)m_star);
      }
    }
  }
}

// ---- free-slot allocation: the n lowest-numbered free slots ---------------

constexpr int kAllocThreads = 256;
constexpr int kAllocWordsPerThread = 4;
constexpr int kAllocWordsPerBlock = kAllocThreads * kAllocWordsPerThread;

__device__ __forceinline__ uint32_t free_mask(const uint32_t* live, const uint32_t* reserved, int64_t w,
                                              int64_t capacity) {
  const int64_t base = w * 32;
  if (base >= capacity) return 0u;
  uint32_t valid = (capacity - base >= 32) ? 0xffffffffu : ((1u << (capacity - base)) - 1u);
  return ~(live[w] | reserved[w]) & valid;
}

__global__ void __launch_bounds__(kAllocThreads) free_count_kernel(const uint32_t* live, const uint32_t* reserved,
                                                                   int64_t capacity, int64_t nwords,
                                                                   int32_t* block_free) {
  __shared__ int sh[kAllocThreads / 32];
  int cnt = 0;
  const int64_t w0 = (int64_t)blockIdx.x * kAllocWordsPerBlock + threadIdx.x * kAllocWordsPerThread;
#pragma unroll
  for (int i = 0; i < kAllocWordsPerThread; ++i)
    if (w0 + i < nwords) cnt += __popc(free_mask(live, reserved, w0 + i, capacity));
  int total;
  block_exclusive_scan(cnt, sh, total);
  if (threadIdx.x == 0) block_free[blockIdx.x] = total;
}

// One block: exclusive scan of the per-block free counts.  When fewer than n
// slots are free the insert is abandoned as a whole.
__global__ void __launch_bounds__(1024) alloc_scan_kernel(int32_t* block_free, int nblocks, int64_t n,
                                                         int32_t* abort_flag, int32_t* err,
                                                         int64_t* out_ids) {
  __shared__ int sh[32];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nblocks; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int v = i < nblocks ? block_free[i] : 0;
    int total;
    const int ex = block_exclusive_scan(v, sh, total);
    const int64_t c = carry;
    if (i < nblocks) block_free[i] = (int32_t)((c + ex) < (int64_t)INT32_MAX ? (c + ex) : (int64_t)INT32_MAX);
    __syncthreads();
    if (threadIdx.x == 0) carry = c + total;
    __syncthreads();
  }
  const bool full = carry < n;
  if (threadIdx.x == 0) {
    *abort_flag = full ? 1 : 0;
    if (full) set_error(err, LVQ_EFULL);
  }
  if (full)
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) out_ids[i] = -1;
}

__global__ void __launch_bounds__(kAllocThreads) alloc_assign_kernel(const uint32_t* live, const uint32_t* reserved,
                                                                     int64_t capacity,
                                                                     int64_t nwords, const int32_t* block_base,
                                                                     int64_t n, const int32_t* abort_flag,
                                                                     int64_t* out_ids) {
  __shared__ int sh[kAllocThreads / 32];
  if (*abort_flag) return;
  const int64_t base = block_base[blockIdx.x];
  if (base >= n) return;
  const int64_t w0 = (int64_t)blockIdx.x * kAllocWordsPerBlock + threadIdx.x * kAllocWordsPerThread;
  uint32_t masks[kAllocWordsPerThread];
  int cnt = 0;
#pragma unroll
  for (int i = 0; i < kAllocWordsPerThread; ++i) {
    masks[i] = (w0 + i < nwords) ? free_mask(live, reserved, w0 + i, capacity) : 0u;
    cnt += __popc(masks[i]);
  }
  int total;
  int64_t rank = base + block_exclusive_scan(cnt, sh, total);
#pragma unroll
  for (int i = 0; i < kAllocWordsPerThread; ++i) {
    uint32_t m = masks[i];
    while (m && rank < n) {
      const int b = __ffs(m) - 1;
      m &= m - 1;
      out_ids[rank++] = (w0 + i) * 32 + b;
    }
  }
}

// mode 0: make the freshly inserted slots live; mode 1: mark them reserved
// (deferred insert).  Skipped when the allocation was abandoned.
__global__ void publish_kernel(uint32_t* live, uint32_t* reserved, const int64_t* ids, int64_t n,
                               const int32_t* abort_flag, int64_t* n_live, int mode) {
  if (*abort_flag) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = ids[i];
    atomicOr((mode == 0 ? live : reserved) + (s >> 5), 1u << (s & 31));
  }
  if (mode == 0 && blockIdx.x == 0 && threadIdx.x == 0)
    atomicAdd(reinterpret_cast<unsigned long long*>(n_live), (unsigned long long)n);
}

// Publication of deferred inserts: reserved slots become live.  Ids that are
// out of range or not reserved are ignored; the count of newly live slots is
// added to n_live.
__global__ void publish_reserved_kernel(uint32_t* live, uint32_t* reserved, int64_t capacity, const int64_t* ids,
                                        int64_t n, int64_t* n_live) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = ids[i];
    if (s < 0 || s >= capacity) continue;
    const uint32_t bit = 1u << (s & 31);
    const uint32_t old = atomicAnd(reserved + (s >> 5), ~bit);
    if (old & bit) {
      atomicOr(live + (s >> 5), bit);
      atomicAdd(reinterpret_cast<unsigned long long*>(n_live), 1ull);
    }
  }
}

// Deletes clear the live bit; with `hold` (non-null: the reserved bitmap)
// a slot that was live also becomes reserved, so no insert reuses it before
// release_kernel frees it.
__global__ void delete_kernel(uint32_t* live, uint32_t* hold, int64_t capacity, const int64_t* ids, int64_t n,
                              unsigned long long* count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = ids[i];
    if (s < 0 || s >= capacity) continue;
    const uint32_t bit = 1u << (s & 31);
    const uint32_t old = atomicAnd(live + (s >> 5), ~bit);
    if (old & bit) {
      if (hold) atomicOr(hold + (s >> 5), bit);
      atomicAdd(count, 1ull);
    }
  }
}

// Held slots (reserved, not live) among ids become free.
__global__ void release_kernel(const uint32_t* live, uint32_t* reserved, int64_t capacity, const int64_t* ids,
                               int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = ids[i];
    if (s < 0 || s >= capacity) continue;
    const uint32_t bit = 1u << (s & 31);
    if (!(live[s >> 5] & bit)) atomicAnd(reserved + (s >> 5), ~bit);
  }
}

__global__ void delete_finish_kernel(const unsigned long long* count, int64_t* out_n, int64_t* n_live) {
  out_n[0] = (int64_t)count[0];
  n_live[0] -= (int64_t)count[0];
}

__global__ void __launch_bounds__(256) export_kernel(DeviceStore st, const int64_t* ids, int64_t n,
                                                     uint8_t* codes1, uint8_t* codes2, float* lower,
                                                     float* step, uint8_t* mean_id) {
  const int lane = threadIdx.x & 31;
  const int warps = blockDim.x >> 5;
  const int d = st.d;
  for (int64_t v = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5); v < n; v += (int64_t)gridDim.x * warps) {
    const int64_t s = ids[v];
    const bool ok = s >= 0 && s < st.capacity && is_live(st.live, s);
    if (!ok && lane == 0) set_error(st.err, LVQ_ENOTFOUND);
    for (int j = lane; j < d; j += 32) {
      uint32_t c = 0, r = 0;
      if (ok) {
        const uint8_t* row = st.codes1 + s * st.stride1;
        if (st.bits1 == 4) {
          const uint32_t w = reinterpret_cast<const uint32_t*>(row)[j >> 3];
          const int e = j & 7;
          c = (w >> ((e & 1) ? (16 + 4 * (e >> 1)) : (4 * (e >> 1)))) & 0xFu;
        } else {
          c = row[j];
        }
        if (st.bits2) r = st.codes2[s * st.row2 + j];
      }
      codes1[v * d + j] = (uint8_t)c;
      if (codes2 && st.bits2) codes2[v * d + j] = (uint8_t)r;
    }
    if (lane == 0) {
      lower[v] = ok ? st.lower[s] : 0.0f;
      step[v] = ok ? st.step[s] : 0.0f;
      mean_id[v] = ok ? st.mean_id[s] : 0;
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------

cudaError_t launch_encode(const DeviceStore& st, const float* x, int64_t n, const EncodeOut& out,
                          cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int groups = (st.d + 7) / 8;
  const int wpl = (groups + 31) / 32;
  const int threads = 256;
  const int64_t blocks64 = ceil_div(n, threads / 32);
  const int blocks = (int)(blocks64 < 65536 * 8 ? blocks64 : 65536 * 8);
  switch (wpl) {
    case 1: encode_kernel<1><<<blocks, threads, 0, stream>>>(st, x, n, out); break;
    case 2: encode_kernel<2><<<blocks, threads, 0, stream>>>(st, x, n, out); break;
    case 3: encode_kernel<3><<<blocks, threads, 0, stream>>>(st, x, n, out); break;
    case 4: encode_kernel<4><<<blocks, threads, 0, stream>>>(st, x, n, out); break;
    case 5: case 6: case 7: case 8:
      encode_kernel<8><<<blocks, threads, 0, stream>>>(st, x, n, out); break;
    default:
      encode_kernel<16><<<blocks, threads, 0, stream>>>(st, x, n, out); break;
  }
  return cudaGetLastError();
}

// ---- M-LVQ local re-encode ------------------------------------------------------
namespace {

__global__ void __launch_bounds__(256) select_mean_kernel(DeviceStore st, int64_t n_rows, int m, int64_t* list,
                                                          unsigned long long* count) {
  const int lane = threadIdx.x & 31;
  // warp-uniform loop: every lane takes part in each ballot
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n_rows;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = base + lane;
    const bool take = s < n_rows && is_live(st.live, s) && st.mean_id[s] == m;
    const unsigned bal = __ballot_sync(FULL, take);
    if (!bal) continue;
    unsigned long long at = 0;
    if (lane == __ffs(bal) - 1) at = atomicAdd(count, (unsigned long long)__popc(bal));
    at = __shfl_sync(FULL, at, __ffs(bal) - 1);
    if (take) list[at + __popc(bal & ((1u << lane) - 1u))] = s;
  }
}

// The stored record decoded in float32, each operation rounded:
//   y = fl(fl(D c) + l); with a second level y = fl(y + fl(fl(D2 c2) + l2));
//   x = fl(mu + y).  One warp per slot.
__global__ void __launch_bounds__(256) reconstruct_kernel(DeviceStore st, const int64_t* __restrict__ list,
                                                          int64_t n, const float* __restrict__ mu,
                                                          float* __restrict__ x) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= n) return;
  const int64_t s = list[i];
  const float lo = st.lower[s], step = st.step[s];
  const float lo2 = st.grid2 ? 0.0f : __fmul_rn(-step, 0.5f);
  const float step2 = st.grid2 ? __fmul_rn(step, __int_as_float((127 - st.b2) << 23)) : __fdiv_rn(step, (float)st.lev2);
  const uint8_t* r1 = st.codes1 + s * st.stride1;
  const uint8_t* r2 = st.bits2 ? st.codes2 + s * st.row2 : nullptr;
  for (int j = lane; j < st.d; j += 32) {
    uint32_t c;
    if (st.bits1 == 4) {
      // word j/8 holds dim 8w+2p at bits 4p and dim 8w+2p+1 at bits 16+4p
      const uint32_t w = reinterpret_cast<const uint32_t*>(r1)[j >> 3];
      const int e = j & 7;
      c = (w >> ((e & 1) ? 16 + 4 * (e >> 1) : 4 * (e >> 1))) & 0xFu;
    } else {
      c = r1[j];
    }
    float y = __fadd_rn(__fmul_rn(step, (float)c), lo);
    if (r2) {
      const float c2 = st.grid2 ? (float)(int8_t)r2[j] : (float)r2[j];
      y = __fadd_rn(y, __fadd_rn(__fmul_rn(step2, c2), lo2));
    }
    x[i * st.d + j] = __fadd_rn(mu[j], y);
  }
}

}  // namespace

cudaError_t launch_select_mean(const DeviceStore& st, int64_t n_rows, int m, int64_t* list,
                               unsigned long long* count, cudaStream_t stream) {
  if (n_rows <= 0) return cudaSuccess;
  const int64_t b = ceil_div(n_rows, 256);
  select_mean_kernel<<<(unsigned)(b < 4096 ? b : 4096), 256, 0, stream>>>(st, n_rows, m, list, count);
  return cudaGetLastError();
}

cudaError_t launch_reconstruct(const DeviceStore& st, const int64_t* list, int64_t n, const float* mu, float* x,
                               cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  reconstruct_kernel<<<(unsigned)ceil_div(n, 8), 256, 0, stream>>>(st, list, n, mu, x);
  return cudaGetLastError();
}

size_t alloc_scratch_bytes(int64_t capacity) {
  const int64_t nwords = ceil_div(capacity, 32);
  const int64_t nblocks = ceil_div(nwords, kAllocWordsPerBlock);
  return (size_t)round_up(nblocks * 4 + 64, 256);
}

cudaError_t launch_alloc_slots(const DeviceStore& st, int64_t n, int64_t* out_ids, int32_t* scratch,
                               int32_t* abort_flag, cudaStream_t stream) {
  const int64_t nwords = ceil_div(st.capacity, 32);
  const int nblocks = (int)ceil_div(nwords, kAllocWordsPerBlock);
  free_count_kernel<<<nblocks, kAllocThreads, 0, stream>>>(st.live, st.reserved, st.capacity, nwords, scratch);
  alloc_scan_kernel<<<1, 1024, 0, stream>>>(scratch, nblocks, n, abort_flag, st.err, out_ids);
  alloc_assign_kernel<<<nblocks, kAllocThreads, 0, stream>>>(st.live, st.reserved, st.capacity, nwords, scratch, n,
                                                            abort_flag, out_ids);
  return cudaGetLastError();
}

cudaError_t launch_publish(const DeviceStore& st, const int64_t* ids, int64_t n, const int32_t* abort_flag,
                           int64_t* n_live, bool deferred, cudaStream_t stream) {
  const int blocks = (int)(ceil_div(n, 256) < 4096 ? ceil_div(n, 256) : 4096);
  publish_kernel<<<blocks > 0 ? blocks : 1, 256, 0, stream>>>(st.live, st.reserved, ids, n, abort_flag, n_live,
                                                              deferred ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_publish_reserved(const DeviceStore& st, const int64_t* ids, int64_t n, int64_t* n_live,
                                    cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)(ceil_div(n, 256) < 4096 ? ceil_div(n, 256) : 4096);
  publish_reserved_kernel<<<blocks, 256, 0, stream>>>(st.live, st.reserved, st.capacity, ids, n, n_live);
  return cudaGetLastError();
}

cudaError_t launch_delete(const DeviceStore& st, const int64_t* ids, int64_t n, int64_t* out_n,
                          unsigned long long* count, int64_t* n_live, cudaStream_t stream, bool hold) {
  cudaMemsetAsync(count, 0, sizeof(unsigned long long), stream);
  if (n > 0) {
    const int blocks = (int)(ceil_div(n, 256) < 4096 ? ceil_div(n, 256) : 4096);
    delete_kernel<<<blocks, 256, 0, stream>>>(st.live, hold ? st.reserved : nullptr, st.capacity, ids, n, count);
  }
  delete_finish_kernel<<<1, 1, 0, stream>>>(count, out_n, n_live);
  return cudaGetLastError();
}

cudaError_t launch_release(const DeviceStore& st, const int64_t* ids, int64_t n, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)(ceil_div(n, 256) < 4096 ? ceil_div(n, 256) : 4096);
  release_kernel<<<blocks, 256, 0, stream>>>(st.live, st.reserved, st.capacity, ids, n);
  return cudaGetLastError();
}

cudaError_t launch_export(const DeviceStore& st, const int64_t* ids, int64_t n, uint8_t* codes1, uint8_t* codes2,
                          float* lower, float* step, uint8_t* mean_id, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)(ceil_div(n, 8) < 65536 ? ceil_div(n, 8) : 65536);
  export_kernel<<<blocks, 256, 0, stream>>>(st, ids, n, codes1, codes2, lower, step, mean_id);
  return cudaGetLastError();
}

}  // namespace lvq
