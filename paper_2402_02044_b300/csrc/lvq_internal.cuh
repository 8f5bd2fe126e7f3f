// Internal definitions shared by the CUDA sources of the LVQ library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lvq.h"

// ---------------------------------------------------------------------------
// Store layout in HBM (structure of arrays, one entry per slot)
//
//   codes1  [capacity][stride1] one record per slot: row1 bytes of
//                             first-level codes (row1 = ceil(d*B1/8) rounded
//                             up to 16 bytes), then a 16-byte trailer
//                             {l, D, ||x^1||^2 as float32, mean id as u32},
//                             a copy of the per-vector constants below, so
//                             that a gather of one slot reads one record
//                             (stride1 = row1 + 16: 64 B at d = 96 with 4-bit
//                             codes, the paper's padded record size).  4-bit codes: 32-bit word w
//                             holds dims 8w..8w+7 with dim 8w+2p in bits
//                             4p..4p+3 and dim 8w+2p+1 in bits 16+4p..19+4p
//                             (p = 0..3), so (word >> 4p) & 0x000F000F puts
//                             an adjacent pair of dims in the two 16-bit
//                             halves.  8-bit codes: byte j = dim j.  Padding
//                             bytes are zero.
//   codes2  [capacity][row2]  residual codes, byte j = dim j, row2 = d rounded
//                             up to 32 bytes (absent when B2 = 0); unsigned
//                             on the text's grid, two's complement int8 on
//                             the listing's signed grid.
//   lower   [capacity] f32    l(x)
//   step    [capacity] f32    D
//   mean_id [capacity] u8     index of the centring mean
//   norm2   [capacity] f32    ||x^1||^2 of the first-level reconstruction
//                             (used by the tensor-core L2 epilogue)
//   live    [capacity/32] u32 bit s%32 of word s/32: slot s holds a vector
//   reserved[capacity/32] u32 slot s is written by a deferred insert and not
//                             yet published (neither free nor visible)
//   means   [M][d] f32        centring means
// ---------------------------------------------------------------------------

namespace lvq {

constexpr int kMaxD = 4096;
constexpr int kMaxMeans = 256;
constexpr int kMaxK1 = 512;
constexpr int kMaxRerank = 4096;
constexpr int kMaxCand = 65536;

// Device error word values (first error wins)
enum : int32_t { kErrNone = 0 };

struct DeviceStore {
  // bits1 / bits2: the code containers (4- or 8-bit first level, 8-bit
  // residual bytes or 0) that every scan, gather and re-rank unpacks; b1 /
  // b2: the quantisers' bit widths (Sec. 3.3: B1 in 2..8, B2 in 2..8), held
  // in those containers (B1 <= 4 in nibbles, else bytes); lev1 = 2^B1 - 1,
  // lev2 = 2^B2 - 1; grid2: the residual grid (0 the text's Q_{B2,-D/2,D/2},
  // 1 the App. C listing's signed grid, step D/2^B2, codes as int8).
  int d, bits1, bits2, n_means, metric;
  int b1, b2, lev1, lev2, grid2;
  int row1, row2;  // code bytes per slot (first level, residual)
  int stride1;     // bytes per first-level record: row1 + 16-byte trailer
  int64_t capacity;
  uint8_t* codes1;
  uint8_t* codes2;
  float* lower;
  float* step;
  uint8_t* mean_id;
  float* norm2;
  uint32_t* live;
  uint32_t* reserved;
  float* means;
  int32_t* err;  // device error word (lvq_status of the first device error)
};

}  // namespace lvq

struct lvq_store {
  lvq_config cfg;
  int device;
  lvq::DeviceStore ds;
  // A view (lvq_store_view) shares the device arrays, counters and row bound
  // of its base store and owns only its scratch memory, tuning and timing.
  lvq_store* base = nullptr;
  std::atomic<int64_t> rows_bound{0};  // (base only) no live slot at or beyond this index
  lvq_tuning tuning;
  // scratch memory (grown on demand, or pre-sized by lvq_reserve)
  void* ws = nullptr;
  size_t ws_bytes = 0;
  // small device-side counters used by insert / delete
  int64_t* counters = nullptr;
  int sm_count = 0;
  mutable std::mutex mu;      // plan, scratch and tuning of calls
  mutable std::mutex msg_mu;  // last_msg alone: errors are recorded while mu is held
  mutable std::string last_msg;
  // per-kernel timing (lvq_profile_enable)
  struct ProfRec {
    int kind;
    int launches;
    cudaEvent_t a, b;
  };
  bool prof_on = false;
  std::vector<ProfRec> prof;
};

namespace lvq {

__host__ __device__ inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// Raises a kernel's dynamic shared memory limit on the current device, once
// per device: `done` (one per kernel) keeps a bit per device ordinal below
// 64 (the attribute is per device); on higher ordinals it is set every call.
inline cudaError_t max_dyn_smem_once(const void* func, int bytes, std::atomic<uint64_t>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = dev >= 0 && dev < 64 ? (1ull << dev) : 0;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}
__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Ordering of results: an unsigned 64-bit key whose high word is the score
// mapped so that "better" is "smaller" (L2 ascending, IP descending) and
// whose low word is the slot id.  Comparing keys compares (score, id).
__device__ __forceinline__ uint32_t order_bits(float better_small) {
  uint32_t b = __float_as_uint(better_small);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float order_float(uint32_t o) {
  uint32_t b = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
  return __uint_as_float(b);
}
__device__ __forceinline__ uint64_t make_key(float score, uint32_t id, int metric) {
  float s = metric == LVQ_IP ? -score : score;
  return ((uint64_t)order_bits(s) << 32) | id;
}
__device__ __forceinline__ float key_score(uint64_t key, int metric) {
  float s = order_float((uint32_t)(key >> 32));
  return metric == LVQ_IP ? -s : s;
}
constexpr uint64_t kNoKey = ~0ull;

__device__ __forceinline__ void set_error(int32_t* err, int32_t code) { atomicCAS(err, 0, code); }

__device__ __forceinline__ bool is_live(const uint32_t* live, int64_t s) {
  return (__ldg(live + (s >> 5)) >> (s & 31)) & 1u;
}

// 4-bit unpack helpers: (w >> 4p) & 0x000F000F holds dims (2p, 2p+1) of the
// word in the low and high 16-bit halves.
__device__ __forceinline__ uint32_t nib_pair(uint32_t w, int p) { return (w >> (4 * p)) & 0x000F000Fu; }
// exact float of a 16-bit unsigned integer held in the low half
__device__ __forceinline__ float u16_lo_to_f(uint32_t t) {
  return __uint_as_float(__byte_perm(t, 0x4B000000u, 0x7610)) - 8388608.0f;
}
__device__ __forceinline__ float u16_hi_to_f(uint32_t t) {
  return __uint_as_float(__byte_perm(t, 0x4B000000u, 0x7632)) - 8388608.0f;
}
// exact float of byte i (0..3) of w
__device__ __forceinline__ float byte_to_f(uint32_t w, int i) {
  return __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7440 + i)) - 8388608.0f;
}

}  // namespace lvq
