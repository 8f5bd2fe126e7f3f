// Float32 LVQ scoring helpers (Sec. 3.2) shared by the CUDA-core kernels.
#pragma once

#include <cuda_fp16.h>

#include "topk.cuh"

namespace lvq {

// Code offset used to centre first-level codes before multiplying them with
// a query: c - 2^(B1-1) lies in [-2^(B1-1), 2^(B1-1) - 1], which halves the
// magnitude of the partial sums.  The offset is folded back into the
// per-vector constant:  <q, l + D c> = (l + off*D) sum(q) + D <q, c - off>.
__host__ __device__ inline float code_offset(int bits1) { return bits1 == 4 ? 8.0f : 128.0f; }

// exact float of (code - off) for the 16-bit integers in the low / high half
__device__ __forceinline__ float lo_centred(uint32_t t, float magic_plus_off) {
  return __uint_as_float(__byte_perm(t, 0x4B000000u, 0x7610)) - magic_plus_off;
}
__device__ __forceinline__ float hi_centred(uint32_t t, float magic_plus_off) {
  return __uint_as_float(__byte_perm(t, 0x4B000000u, 0x7632)) - magic_plus_off;
}
__device__ __forceinline__ float byte_centred(uint32_t w, int i, float magic_plus_off) {
  return __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7440 + i)) - magic_plus_off;
}

// Decode the 8 first-level codes of group g (dims 8g..8g+7) of a stored row
// into floats minus `sub` (sub = 2^23 for the raw code, 2^23 + off centred).
__device__ __forceinline__ void group_codes(const uint8_t* row, int bits1, int g, float sub, float (&c)[8]) {
  if (bits1 == 4) {
    const uint32_t w = __ldg(reinterpret_cast<const uint32_t*>(row) + g);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const uint32_t t = nib_pair(w, p);
      c[2 * p] = lo_centred(t, sub);
      c[2 * p + 1] = hi_centred(t, sub);
    }
  } else {
    const uint2 w = __ldg(reinterpret_cast<const uint2*>(row) + g);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      c[i] = byte_centred(w.x, i, sub);
      c[4 + i] = byte_centred(w.y, i, sub);
    }
  }
}

// The same in two steps: the raw words of group g (one load), then their codes.
__device__ __forceinline__ uint2 group_words(const uint8_t* row, int bits1, int g) {
  if (bits1 == 4) return make_uint2(__ldg(reinterpret_cast<const uint32_t*>(row) + g), 0u);
  return __ldg(reinterpret_cast<const uint2*>(row) + g);
}
__device__ __forceinline__ void words_codes(uint2 w, int bits1, float sub, float (&c)[8]) {
  if (bits1 == 4) {
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const uint32_t t = nib_pair(w.x, p);
      c[2 * p] = lo_centred(t, sub);
      c[2 * p + 1] = hi_centred(t, sub);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      c[i] = byte_centred(w.x, i, sub);
      c[4 + i] = byte_centred(w.y, i, sub);
    }
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// The second level of a slot with step D: its lower bound l2 and step D2,
// and how its code bytes read as numbers.  The text's grid (Sec. 2.2):
// l2 = -D/2, D2 = fl(D / (2^B2 - 1)), unsigned codes.  The App. C listing's
// grid: l2 = 0, D2 = D / 2^B2 (exact), int8 codes, read as excess-128 bytes
// (XOR 0x80) less 128.
struct Resid {
  float lo2, step2;
  uint32_t flip;
  float sub;  // 2^23 (+ 128 for signed codes): byte_centred's magic offset
};
__device__ __forceinline__ Resid resid_of(const DeviceStore& st, float step) {
  Resid r;
  if (st.grid2) {
    r.lo2 = 0.0f;
    r.step2 = __fmul_rn(step, __int_as_float((127 - st.b2) << 23));  // step * 2^-B2
    r.flip = 0x80808080u;
    r.sub = 8388608.0f + 128.0f;
  } else {
    r.lo2 = __fmul_rn(-step, 0.5f);
    r.step2 = __fdiv_rn(step, (float)st.lev2);
    r.flip = 0u;
    r.sub = 8388608.0f;
  }
  return r;
}

// Two-level float32 score of slot s, computed by one warp (result valid in
// every lane).  x2_j = mu_mj + (l + D c_j) + (l2 + D2 c2_j) on the slot's
// residual grid (resid_of); L2: sum (q_j - x2_j)^2, IP: sum q_j x2_j.  q is
// in shared memory.
__device__ __forceinline__ float score2_warp(const DeviceStore& st, int64_t s, const float* qsh) {
  const int lane = threadIdx.x & 31;
  const int d = st.d;
  const int groups = (d + 7) >> 3;
  const float lo = __ldg(st.lower + s), step = __ldg(st.step + s);
  const Resid R = resid_of(st, step);
  const float lo2 = R.lo2, step2 = R.step2;
  const float* mu = st.means + (int64_t)__ldg(st.mean_id + s) * d;
  const uint8_t* row1 = st.codes1 + s * st.stride1;
  const uint8_t* row2 = st.codes2 + s * st.row2;
  float acc = 0.0f;
  for (int g = lane; g < groups; g += 32) {
    float c[8];
    group_codes(row1, st.bits1, g, 8388608.0f, c);
    const uint2 w2 = __ldg(reinterpret_cast<const uint2*>(row2) + g);
    float part = 0.0f;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int j = g * 8 + e;
      if (j < d) {
        const float c2 = byte_centred((e < 4 ? w2.x : w2.y) ^ R.flip, e & 3, R.sub);
        const float x2 = __fadd_rn(__fadd_rn(__fmaf_rn(step, c[e], lo), __fmaf_rn(step2, c2, lo2)), __ldg(mu + j));
        if (st.metric == LVQ_L2) {
          const float df = qsh[j] - x2;
          part = __fmaf_rn(df, df, part);
        } else {
          part = __fmaf_rn(qsh[j], x2, part);
        }
      }
    }
    acc += part;
  }
  return warp_sum(acc);
}

}  // namespace lvq
