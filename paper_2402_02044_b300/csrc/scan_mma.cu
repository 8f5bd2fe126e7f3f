// First-level scan on the 5th-generation tensor cores (tcgen05), fused with
// top-k1 selection.
//
// <q, x^> = <q, mu_m> + (l + off*D) sum(q) + D * <q, c - off>   (Sec. 3.2)
// The last inner product is a [DB rows x d] . [d x queries] contraction:
// codes minus the offset (-8..7 at 4 bits, -128..127 at 8 bits) are exact in
// float16, the queries are rounded to float16, and the products accumulate in
// float32 in tensor memory (TMEM).  L2 uses ||q||^2 - 2 <q, x^> + ||x^||^2.
//
// One persistent CTA per SM, 10 warps with fixed roles:
//   warp 0      TMA producer: the CTA's query tile (N queries x all dims,
//               float16, 128-byte swizzle, resident while the CTA works on
//               that tile) and 128-row x 64-byte boxes of codes (64-byte
//               swizzle) into a 3-stage ring;
//   warp 1      allocates TMEM and issues tcgen05.mma (M = 128 database
//               rows, N queries, K = 16) with A read from TMEM;
//   warps 2-5   unpack: each thread owns one database row of the tile,
//               turns 4- or 8-bit codes into centred float16 pairs and
//               writes them with tcgen05.st into an A ring in TMEM;
//   warps 6-9   epilogue: tcgen05.ld of the float32 accumulators (double
//               buffered in TMEM), the affine fix-up, and the top-k1
//               threshold filter into per-query candidate buffers.
// Work is the list of (query tile, database tile) units, split evenly
// between the CTAs; a CTA's stretch of one query tile is a "segment" whose
// k1 best keys go to partial[q][segment].
//
// Every wait on an mbarrier is bounded; on expiry the CTA records
// LVQ_ETIMEOUT, stops issuing work, waits (bounded) for its own copies and
// MMAs in flight, frees its TMEM and exits.
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include "kernels.cuh"
#include "score.cuh"
#include "tcgen05.cuh"

namespace lvq {

namespace {

using namespace sm100;

constexpr int kRows = 128;              // database rows per tile (MMA M)
constexpr int kBoxBytes = 64;           // code bytes per row per TMA box
constexpr int kStageBytes = kRows * kBoxBytes;
constexpr int kCodeStages = 3;
constexpr int kWarps = 10;
constexpr int kThreads = kWarps * 32;
constexpr int kTmemCols = 512;
constexpr uint32_t kWaitLimit = 1u << 24;
constexpr int kMinSmem = 120 * 1024;    // keeps one CTA per SM (TMEM is taken whole)
constexpr int kMaxQueryBytes = 196608;

struct MmaArgs {
  DeviceStore st;
  int64_t nq;
  QueryPrep p;
  int k1;
  int64_t n_rows;
  uint64_t* partial;  // [nq][seg_max][k1]
  uint64_t* cand;     // [grid][N][cap]
  int cap;
  int n_kbox;         // code boxes per row
  int qboxes;         // 64-dim float16 query boxes per query row
  int a_stages;       // depth of the A ring in TMEM
  int64_t ntiles;     // database tiles
  int64_t units;      // query tiles x database tiles
  int seg_max;
};

struct Smem {
  // offsets from the 1024-aligned base
  int q, code, bars, misc;
  int total;
};

__host__ __device__ inline Smem smem_layout(int n, int qboxes) {
  Smem s;
  s.q = 0;
  s.code = qboxes * n * 128;
  s.bars = s.code + kCodeStages * kStageBytes;
  s.misc = s.bars + 64 * 8;
  // misc: tmem base (16) + abort (16) + thr[n] u64 + cnt[n] + qsum[n] + qnorm[n] + hist[4][256]
  s.total = s.misc + 32 + n * 8 + n * 4 * 3 + 4 * 256 * 4;
  return s;
}

struct Bars {
  uint64_t *code_full, *code_empty, *a_full, *a_empty, *d_full, *d_empty, *q_full, *q_empty, *mma_done;
};

__device__ __forceinline__ Bars bars_at(uint64_t* b) {
  Bars r;
  r.code_full = b;
  r.code_empty = b + kCodeStages;
  r.a_full = b + 2 * kCodeStages;
  r.a_empty = r.a_full + 8;
  r.d_full = r.a_empty + 8;
  r.d_empty = r.d_full + 2;
  r.q_full = r.d_empty + 2;
  r.q_empty = r.q_full + 1;
  r.mma_done = r.q_empty + 1;
  return r;
}

__device__ __forceinline__ int64_t unit_begin(int64_t units, int c, int grid) { return units * c / grid; }

// first CTA whose stretch of units contains unit u
__device__ __forceinline__ int cta_of_unit(int64_t u, int64_t units, int grid) {
  return (int)(((u + 1) * grid - 1) / units);
}

// centred float16 pairs of one 64-byte box of a row: 4-bit -> 64 pairs, 8-bit -> 32
template <int BITS>
__device__ __forceinline__ void unpack_box(const uint4 (&w)[4], uint32_t (&r)[64]) {
  if (BITS == 4) {
    const __half2 off = __halves2half2(__float2half_rn(1032.0f), __float2half_rn(1032.0f));
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const uint32_t ws[4] = {w[c].x, w[c].y, w[c].z, w[c].w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          const uint32_t h = ((ws[i] >> (4 * p)) & 0x000F000Fu) | 0x64006400u;  // (1024 + c_lo, 1024 + c_hi)
          __half2 v = __hsub2(*reinterpret_cast<const __half2*>(&h), off);
          r[c * 16 + i * 4 + p] = *reinterpret_cast<uint32_t*>(&v);
        }
      }
    }
  } else {
    const __half2 off = __halves2half2(__float2half_rn(1152.0f), __float2half_rn(1152.0f));
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const uint32_t ws[4] = {w[c].x, w[c].y, w[c].z, w[c].w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          const uint32_t h = __byte_perm(ws[i], 0x64646464u, p == 0 ? 0x5140 : 0x5342);  // (1024 + b, 1024 + b')
          __half2 v = __hsub2(*reinterpret_cast<const __half2*>(&h), off);
          r[c * 8 + i * 2 + p] = *reinterpret_cast<uint32_t*>(&v);
        }
      }
    }
  }
}

struct Ctx {
  unsigned char* qs;
  unsigned char* cst;
  Bars B;
  uint32_t tbase;
  volatile int* abort_sh;
  uint64_t* thr;
  int* cnt;
  float* qsum_s;
  float* qnorm_s;
  int* hist;
  volatile int* ep_go;  // [2] epilogue leader's verdicts, read by the 4 epilogue warps after a named barrier
  int64_t u_begin, u_end;
  int cta, grid;
};

// Bounded wait; on expiry record LVQ_ETIMEOUT, tell the other roles, and
// jump to the role's exit (a label `out` in the calling function).
#define LVQ_WAIT(c, bar, par)                            \
  do {                                                   \
    if (!mbar_wait((bar), (par), kWaitLimit)) {          \
      *(c).abort_sh = 1;                                 \
      set_error(a.st.err, LVQ_ETIMEOUT);                 \
      goto out;                                          \
    }                                                    \
  } while (0)

template <int N, int BITS>
__device__ __forceinline__ void producer_role(const CUtensorMap* cmap, const CUtensorMap* qmap, const MmaArgs& a,
                                              const Ctx& c) {
  uint32_t ci = 0, qi = 0;
  int64_t g_cur = -1;
  for (int64_t u = c.u_begin; u < c.u_end && !*c.abort_sh;) {
    const int64_t g = u / a.ntiles, t0 = u % a.ntiles;
    const int64_t t1 = min(a.ntiles, t0 + (c.u_end - u));
    if (g != g_cur) {
      if (qi > 0) LVQ_WAIT(c, c.B.q_empty, (qi - 1) & 1);
      mbar_expect_tx(c.B.q_full, (uint32_t)(a.qboxes * N * 128));
      for (int kb = 0; kb < a.qboxes; ++kb)
        tma_load_2d(c.qs + kb * N * 128, qmap, c.B.q_full, kb * 64, (int)(g * N));
      ++qi;
      g_cur = g;
    }
    for (int64_t t = t0; t < t1; ++t) {
      for (int kb = 0; kb < a.n_kbox; ++kb) {
        const int s = ci % kCodeStages;
        LVQ_WAIT(c, c.B.code_empty + s, ((ci / kCodeStages) & 1) ^ 1);
        mbar_expect_tx(c.B.code_full + s, kStageBytes);
        tma_load_2d(c.cst + s * kStageBytes, cmap, c.B.code_full + s, kb * kBoxBytes, (int)(t * kRows));
        ++ci;
      }
    }
    u += t1 - t0;
  }
out:
  // copies that may still be in flight: the last (up to) 3 code boxes and
  // the last query tile
  for (uint32_t j = 1; j <= (uint32_t)kCodeStages && j <= ci; ++j) {
    const uint32_t k = ci - j;
    mbar_wait(c.B.code_full + k % kCodeStages, (k / kCodeStages) & 1, kWaitLimit);
  }
  if (qi > 0) mbar_wait(c.B.q_full, (qi - 1) & 1, kWaitLimit);
}

template <int N, int BITS>
__device__ __forceinline__ void mma_role(const MmaArgs& a, const Ctx& c) {
  constexpr int kBoxDims = BITS == 4 ? 128 : 64;
  constexpr int kACols = kBoxDims / 2;
  constexpr int kKSteps = kBoxDims / 16;
  constexpr uint32_t kIdesc = idesc_f16_f32(kRows, N);
  const int AS = a.a_stages;
  uint32_t ai = 0, di = 0, qi = 0;
  int64_t g_cur = -1;
  const uint32_t qbase = smem_u32(c.qs);
  for (int64_t u = c.u_begin; u < c.u_end && !*c.abort_sh;) {
    const int64_t g = u / a.ntiles, t0 = u % a.ntiles;
    const int64_t t1 = min(a.ntiles, t0 + (c.u_end - u));
    if (g != g_cur) {
      LVQ_WAIT(c, c.B.q_full, qi & 1);
      ++qi;
      g_cur = g;
      tc_fence_after();
    }
    for (int64_t t = t0; t < t1; ++t) {
      const int db = di & 1;
      LVQ_WAIT(c, c.B.d_empty + db, ((di >> 1) & 1) ^ 1);
      tc_fence_after();
      const uint32_t d_tmem = c.tbase + db * N;
      for (int kb = 0; kb < a.n_kbox; ++kb) {
        const int s = ai % AS;
        LVQ_WAIT(c, c.B.a_full + s, (ai / AS) & 1);
        tc_fence_after();
        const uint32_t a_tmem = c.tbase + 2 * N + s * kACols;
#pragma unroll
        for (int kk = 0; kk < kKSteps; ++kk) {
          const int kg = kb * kBoxDims + kk * 16;  // first dim of this K step
          const uint32_t baddr = qbase + (kg >> 6) * N * 128 + (kg & 63) * 2;
          mma_f16_ts(d_tmem, a_tmem + kk * 8, desc_sw128(baddr), kIdesc, (kb | kk) != 0);
        }
        mma_commit(c.B.a_empty + s);
        ++ai;
      }
      mma_commit(c.B.d_full + db);
      ++di;
    }
    u += t1 - t0;
    mma_commit(c.B.q_empty);
  }
out:
  // all MMAs issued by this thread are complete before TMEM is freed
  mma_commit(c.B.mma_done);
  mbar_wait(c.B.mma_done, 0, kWaitLimit);
}

template <int N, int BITS>
__device__ __forceinline__ void unpack_role(const MmaArgs& a, const Ctx& c, int warp, int lane) {
  constexpr int kBoxDims = BITS == 4 ? 128 : 64;
  constexpr int kACols = kBoxDims / 2;
  const int AS = a.a_stages;
  const int quarter = warp & 3;
  const int row = quarter * 32 + lane;
  const uint32_t lane_base = c.tbase + ((uint32_t)(quarter * 32) << 16);
  uint32_t ci = 0, ai = 0;
  for (int64_t u = c.u_begin; u < c.u_end && !*c.abort_sh;) {
    const int64_t t0 = u % a.ntiles;
    const int64_t t1 = min(a.ntiles, t0 + (c.u_end - u));
    for (int64_t t = t0; t < t1; ++t) {
      for (int kb = 0; kb < a.n_kbox; ++kb) {
        const int s = ci % kCodeStages;
        LVQ_WAIT(c, c.B.code_full + s, (ci / kCodeStages) & 1);
        const uint4* src = reinterpret_cast<const uint4*>(c.cst + s * kStageBytes + row * kBoxBytes);
        uint4 w[4];
        const int sw = (row >> 1) & 3;  // 64-byte swizzle of the TMA box
#pragma unroll
        for (int q = 0; q < 4; ++q) w[q] = src[q ^ sw];
        __syncwarp();
        if (lane == 0) mbar_arrive(c.B.code_empty + s);
        ++ci;
        uint32_t r[64];
        unpack_box<BITS>(w, r);
        const int as = ai % AS;
        LVQ_WAIT(c, c.B.a_empty + as, ((ai / AS) & 1) ^ 1);
        tc_fence_after();
        const uint32_t taddr = lane_base + 2 * N + as * kACols;
        tmem_st_x32<0>(taddr, r);
        if (BITS == 4) tmem_st_x32<32>(taddr + 32, r);
        tmem_st_wait();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(c.B.a_full + as);
        ++ai;
      }
    }
    u += t1 - t0;
  }
out:
  return;
}

template <int N>
__device__ __forceinline__ void load_acc(uint32_t taddr, uint32_t (&v)[N]) {
  if constexpr (N == 16) {
    tmem_ld_x16<0>(taddr, v);
  } else {
    tmem_ld_x32<0>(taddr, v);
    if constexpr (N >= 64) tmem_ld_x32<32>(taddr + 32, v);
    if constexpr (N >= 128) {
      tmem_ld_x32<64>(taddr + 64, v);
      tmem_ld_x32<96>(taddr + 96, v);
    }
  }
}

template <int N, int BITS>
__device__ __forceinline__ void epilogue_role(const MmaArgs& a, const Ctx& c, int warp, int lane) {
  const int quarter = warp & 3;
  const int ew = warp - 6;        // 0..3
  const int et = ew * 32 + lane;  // 0..127
  const int row_in = quarter * 32 + lane;
  const uint32_t lane_base = c.tbase + ((uint32_t)(quarter * 32) << 16);
  const DeviceStore& st = a.st;
  const bool ip = st.metric == LVQ_IP;
  const float off = code_offset(BITS);
  uint64_t* mybuf = a.cand + (int64_t)c.cta * N * a.cap;
  int* myhist = c.hist + ew * 256;
  uint32_t di = 0, pub = 0;
  // The four epilogue warps meet at named barriers, so they must all take the
  // same path: only warp 6 waits on mbarriers and reads the abort flag, and
  // publishes its verdict in shared memory before a barrier.  Verdicts
  // alternate between two slots, so a slot is rewritten only after every
  // warp has passed the barrier that follows its read.
  for (int64_t u = c.u_begin; u < c.u_end;) {
    const int64_t g = u / a.ntiles, t0 = u % a.ntiles;
    const int64_t t1 = min(a.ntiles, t0 + (c.u_end - u));
    const int64_t q0 = g * N;
    if (et < N) {
      const bool real = q0 + et < a.nq;
      c.thr[et] = real ? kNoKey : 0ull;
      c.cnt[et] = 0;
      c.qsum_s[et] = real ? a.p.qsum[q0 + et] : 0.0f;
      c.qnorm_s[et] = real ? a.p.qnorm[q0 + et] : 0.0f;
    }
    if (et == 0) c.ep_go[pub & 1] = !*c.abort_sh;
    named_bar(1, 128);
    if (!c.ep_go[pub++ & 1]) goto out;
    for (int64_t t = t0; t < t1; ++t) {
      const int db = di & 1;
      if (ew == 0) {
        const bool ok = !*c.abort_sh && mbar_wait(c.B.d_full + db, (di >> 1) & 1, kWaitLimit);
        if (!ok && lane == 0) {
          if (!*c.abort_sh) set_error(st.err, LVQ_ETIMEOUT);
          *c.abort_sh = 1;
        }
        __syncwarp();
        if (lane == 0) c.ep_go[pub & 1] = ok;
      }
      named_bar(1, 128);
      if (!c.ep_go[pub++ & 1]) goto out;
      tc_fence_after();
      uint32_t v[N];
      load_acc<N>(lane_base + db * N, v);
      tmem_ld_wait();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(c.B.d_empty + db);
      ++di;
      const int64_t rw = t * kRows + row_in;
      if (rw < a.n_rows && is_live(st.live, rw)) {
        const float lo = __ldg(st.lower + rw), step = __ldg(st.step + rw);
        const int m = __ldg(st.mean_id + rw);
        const float nrm = ip ? 0.0f : __ldg(st.norm2 + rw);
        const float base_ip = __fmaf_rn(off, step, lo);
        const float* cmq = a.p.cm + q0 * st.n_means + m;
#pragma unroll
        for (int n = 0; n < N; ++n) {
          if (q0 + n < a.nq) {
            const float acc = __uint_as_float(v[n]);
            float s = __fmaf_rn(step, acc, __fmaf_rn(base_ip, c.qsum_s[n], __ldg(cmq + n * st.n_means)));
            if (!ip) s = c.qnorm_s[n] + nrm - 2.0f * s;
            const uint64_t key = make_key(s, (uint32_t)rw, st.metric);
            if (key < c.thr[n]) mybuf[n * a.cap + atomicAdd(&c.cnt[n], 1)] = key;
          }
        }
      }
      named_bar(1, 128);
      for (int n = ew; n < N; n += 4) {
        if (c.cnt[n] > a.cap - kRows) {
          uint64_t tk;
          const int kept = warp_select(mybuf + n * a.cap, c.cnt[n], a.k1, myhist, &tk);
          if (lane == 0) {
            c.cnt[n] = kept;
            c.thr[n] = tk;
          }
        }
      }
      named_bar(1, 128);
    }
    {
      // end of this CTA's segment of query tile g: k1 best of each query
      const int seg = c.cta - cta_of_unit(g * a.ntiles, a.units, c.grid);
      if (seg < 0 || seg >= a.seg_max) {
        if (et == 0) set_error(st.err, LVQ_ECUDA);
      } else {
        for (int n = ew; n < N; n += 4) {
          if (q0 + n >= a.nq) continue;
          uint64_t tk;
          const int kept = warp_select(mybuf + n * a.cap, c.cnt[n], a.k1, myhist, &tk);
          uint64_t* dst = a.partial + ((q0 + n) * a.seg_max + seg) * a.k1;
          for (int i = lane; i < a.k1; i += 32) dst[i] = i < kept ? mybuf[n * a.cap + i] : kNoKey;
        }
      }
    }
    named_bar(1, 128);
    u += t1 - t0;
  }
out:
  return;
}

#undef LVQ_WAIT

template <int N, int BITS>
__global__ void __launch_bounds__(kThreads, 1)
    scan_mma_kernel(const __grid_constant__ CUtensorMap cmap, const __grid_constant__ CUtensorMap qmap, MmaArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const Smem L = smem_layout(N, a.qboxes);
  Ctx c;
  c.qs = smem + L.q;
  c.cst = smem + L.code;
  uint64_t* bar_mem = reinterpret_cast<uint64_t*>(smem + L.bars);
  uint32_t* tmem_base_sh = reinterpret_cast<uint32_t*>(smem + L.misc);
  c.abort_sh = reinterpret_cast<volatile int*>(smem + L.misc + 16);
  c.thr = reinterpret_cast<uint64_t*>(smem + L.misc + 32);
  c.cnt = reinterpret_cast<int*>(c.thr + N);
  c.qsum_s = reinterpret_cast<float*>(c.cnt + N);
  c.qnorm_s = c.qsum_s + N;
  c.hist = reinterpret_cast<int*>(c.qnorm_s + N);
  c.ep_go = reinterpret_cast<volatile int*>(smem + L.misc + 20);  // two ints
  c.B = bars_at(bar_mem);
  c.grid = gridDim.x;
  c.cta = blockIdx.x;
  c.u_begin = unit_begin(a.units, c.cta, c.grid);
  c.u_end = unit_begin(a.units, c.cta + 1, c.grid);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kCodeStages; ++i) {
      mbar_init(c.B.code_full + i, 1);
      mbar_init(c.B.code_empty + i, 4);
    }
    for (int i = 0; i < a.a_stages; ++i) {
      mbar_init(c.B.a_full + i, 4);
      mbar_init(c.B.a_empty + i, 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(c.B.d_full + i, 1);
      mbar_init(c.B.d_empty + i, 4);
    }
    mbar_init(c.B.q_full, 1);
    mbar_init(c.B.q_empty, 1);
    mbar_init(c.B.mma_done, 1);
    *c.abort_sh = 0;
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(tmem_base_sh, kTmemCols);
  if (warp == 0 && lane == 0) {
    prefetch_tmap(&cmap);
    prefetch_tmap(&qmap);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  c.tbase = *tmem_base_sh;

  if (warp == 0) {
    if (lane == 0) producer_role<N, BITS>(&cmap, &qmap, a, c);
  } else if (warp == 1) {
    if (lane == 0) mma_role<N, BITS>(a, c);
  } else if (warp < 6) {
    unpack_role<N, BITS>(a, c, warp, lane);
  } else {
    epilogue_role<N, BITS>(a, c, warp, lane);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(c.tbase, kTmemCols);
}

// ---- host side -------------------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

int max_n_tile(const DeviceStore& st) {
  const int qboxes = (int)ceil_div(st.row1, kBoxBytes) * (st.bits1 == 4 ? 2 : 1);
  int n = 128;
  while (n > 16 && qboxes * n * 128 > kMaxQueryBytes) n >>= 1;
  return qboxes * n * 128 <= kMaxQueryBytes ? n : 0;
}

template <int N, int BITS>
cudaError_t launch_nb(const CUtensorMap& cm, const CUtensorMap& qm, const MmaArgs& a, int grid, size_t smem,
                      cudaStream_t stream) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(scan_mma_kernel<N, BITS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         232448);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  scan_mma_kernel<N, BITS><<<grid, kThreads, smem, stream>>>(cm, qm, a);
  return cudaGetLastError();
}

}  // namespace

bool mma_supported(const DeviceStore& st) {
  return (st.bits1 == 4 || st.bits1 == 8) && max_n_tile(st) > 0 && encode_fn() != nullptr;
}

int mma_tile_limit(const DeviceStore& st) { return max_n_tile(st); }

size_t mma_scan_cand_bytes(int grid, int n_tile, int k1) {
  return (size_t)grid * n_tile * pow2_at_least(k1 + kRows) * 8;
}

int mma_seg_max(int grid, int64_t groups) { return (int)ceil_div(grid, groups) + 1; }

cudaError_t launch_scan_mma(const DeviceStore& st, int64_t nq, const QueryPrep& p, int n_tile, const ScanPlan& plan,
                            cudaStream_t stream) {
  if (nq <= 0) return cudaSuccess;
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  const int qboxes = p.kq / 64;
  MmaArgs a;
  a.st = st;
  a.nq = nq;
  a.p = p;
  a.k1 = plan.k1;
  a.n_rows = plan.n_rows;
  a.partial = plan.partial;
  a.cand = plan.cand;
  a.cap = pow2_at_least(plan.k1 + kRows);
  a.n_kbox = (int)ceil_div(st.row1, kBoxBytes);
  a.qboxes = qboxes;
  const int acols = st.bits1 == 4 ? 64 : 32;
  a.a_stages = (kTmemCols - 2 * n_tile) / acols;
  if (a.a_stages > 8) a.a_stages = 8;
  a.ntiles = ceil_div(plan.n_rows > 0 ? plan.n_rows : 1, kRows);
  const int64_t groups = p.nq_pad / n_tile;
  a.units = groups * a.ntiles;
  const int grid = plan.grid;
  a.seg_max = plan.splits;

  CUtensorMap cm, qm;
  {
    cuuint64_t dims[2] = {(cuuint64_t)st.row1, (cuuint64_t)st.capacity};
    cuuint64_t strides[1] = {(cuuint64_t)st.row1};
    cuuint32_t box[2] = {(cuuint32_t)kBoxBytes, (cuuint32_t)kRows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(&cm, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, st.codes1, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  {
    cuuint64_t dims[2] = {(cuuint64_t)p.kq, (cuuint64_t)p.nq_pad};
    cuuint64_t strides[1] = {(cuuint64_t)p.kq * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)n_tile};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(&qm, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, p.q16, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaMemsetAsync(plan.partial, 0xFF, (size_t)nq * a.seg_max * plan.k1 * 8, stream);
  if (e != cudaSuccess) return e;
  const Smem L = smem_layout(n_tile, qboxes);
  size_t smem = (size_t)L.total + 1024;
  if (smem < (size_t)kMinSmem) smem = kMinSmem;
  if (smem > 232448) return cudaErrorInvalidConfiguration;
  const bool b4 = st.bits1 == 4;
  switch (n_tile) {
    case 16: return b4 ? launch_nb<16, 4>(cm, qm, a, grid, smem, stream) : launch_nb<16, 8>(cm, qm, a, grid, smem, stream);
    case 32: return b4 ? launch_nb<32, 4>(cm, qm, a, grid, smem, stream) : launch_nb<32, 8>(cm, qm, a, grid, smem, stream);
    case 64: return b4 ? launch_nb<64, 4>(cm, qm, a, grid, smem, stream) : launch_nb<64, 8>(cm, qm, a, grid, smem, stream);
    case 128: return b4 ? launch_nb<128, 4>(cm, qm, a, grid, smem, stream) : launch_nb<128, 8>(cm, qm, a, grid, smem, stream);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lvq
