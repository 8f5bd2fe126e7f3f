// First-level scan on the 5th-generation tensor cores (tcgen05), fused with
// top-k1 selection.
//
// <q, x^> = <q, mu_m> + l sum(q) + D <q, c>   (Sec. 3.2)
// The last inner product is a [DB rows x d] . [d x queries] contraction run
// on the tensor cores with float32 accumulation in tensor memory (TMEM).  A
// code reaches them as the float16 1024 + c (4-bit codes in the upper nibble
// of a byte as 1024 + 16c, with the matching query dims pre-scaled by 1/16):
// OR-ing the code into the mantissa of 1024 is one LOP3 per pair of codes.
// The queries are rounded to float16; the offset is removed afterwards,
// <q16, c> = acc - 1024 sum(q16).  L2 uses ||q||^2 - 2 <q, x^> + ||x^||^2.
//
// One persistent CTA per SM, 18 or 19 warps with fixed roles:
//   warp 0      TMA producer: the CTA's query tile (N queries x all dims,
//               float16, 128-byte swizzle, resident while the CTA works on
//               that tile) and 128-row x 64-byte boxes of codes (64-byte
//               swizzle) into a ring of 3 to 16 stages;
//   warp 1      allocates TMEM and issues tcgen05.mma (M = 128 database
//               rows, N queries, K = 16) with A read from TMEM;
//               both run as whole warps: every lane waits on the
//               mbarriers, one elected lane issues;
//   warps 2-9   unpack, two per TMEM lane quarter taking alternate code
//               boxes (one box's tcgen05.st completes while the other's
//               codes are read and converted): each thread owns one
//               database row of the tile, turns 4- or 8-bit codes into
//               float16 pairs and writes them with tcgen05.st into an A
//               ring in TMEM;
//   warps 10-17 epilogue (two per TMEM lane quarter, each taking half of the
//               query columns): tcgen05.ld of the float32 accumulators
//               (double buffered in TMEM) 8 to 32 columns at a time, a cheap
//               per-query filter, then the exact key and the top-k1
//               threshold test for the few rows that pass it;
//   warp 18     (query tiles of up to 64) bound: lowers each query's
//               shared bound (below).
// Work is a list of jobs (a query tile x a database segment), dealt evenly
// between the CTAs; a CTA's stretch of one query tile is a "segment" whose
// k1 best keys go to partial[q][segment].
//
// The filter's bound for a query is the lowest of (a) its own buffer's
// k1-th key, (b) the shared per-query bound, which every CTA lowers to its
// buffer's k1-th key when it cuts the buffer, and (c) a union bound: every
// exact key also lowers, in global memory, the lowest key of its (segment,
// id mod J) row set, J = ceil(k1 / segments); the bound warp takes the k1-th
// lowest of a query's segments x J such keys, all of distinct rows, so at
// least k1 rows lie at or below it.  Unlike (a) and (b), which stand for one
// CTA's share of the rows, (c) stands for all rows scanned so far.
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
constexpr int kMaxCodeStages = 16;
// the bound warp runs with query tiles of up to 64 (measured on B300: it
// makes 16- and 64-query scans 1.2x and 1.6x faster, while a full 128-query
// tile is held up by a 19th warp even when it idles, and its own bound
// rarely beats the segments' by then)
template <int N>
constexpr int warps_of() {
  return N <= 64 ? 19 : 18;
}
constexpr int kUnpackWarps = 8;         // warps 2-9
constexpr int kEpiWarp0 = 2 + kUnpackWarps;  // first of the 8 epilogue warps
constexpr int kBoundWarp = kEpiWarp0 + 8;       // the bound warp
constexpr int kEpiThreads = 256;

constexpr int kTmemCols = 512;
constexpr uint32_t kWaitLimit = 1u << 24;
constexpr int kMinSmem = 120 * 1024;    // keeps one CTA per SM (TMEM is taken whole)
constexpr int kHistInts = 64;           // 6-bit-digit radix histogram of one warp
// epilogue warps that cut candidate buffers: all eight with query tiles of up
// to 64 (whose CTAs start with loose bounds and cut often), four with 128
// (whose shared memory has no room for more histograms)
__host__ __device__ constexpr int compact_warps(int n) { return n <= 64 ? 8 : 4; }
constexpr int kMetaAhead = 4;           // tiles between the L2 prefetch of row constants and their use

struct MmaArgs {
  DeviceStore st;
  int cm_table;       // <q, mu_m> of the query tile in shared memory: 0 no, 1 float16, 2 float32
  int64_t nq;
  QueryPrep p;
  int k1;
  int64_t n_rows;
  uint64_t* partial;  // [nq][segs][k1]: keys of each (query, database segment)
  int* counts;        // [nq][segs] keys written per list
  uint64_t* gthr;     // [nq] lowest k1-th key any job has found (bounds the global k1-th)
  uint64_t* cand;     // [grid][N][cap]
  int cap;
  int n_kbox;         // code boxes per row
  int qboxes;         // 64-dim float16 query boxes per query row
  int a_stages;       // depth of the A ring in TMEM
  int code_stages;    // depth of the code-box ring in shared memory
  int64_t ntiles;     // database tiles
  int64_t groups;     // query tiles
  int segs;           // database segments (equal ranges of tiles)
  int64_t jobs;       // groups x segs; job j = (query tile j % groups, segment j / groups)
  uint32_t wait_limit;  // polls of a pipeline wait before the CTA gives up (drains use kWaitLimit)
  uint64_t* seg_best;   // [nq][segs][best_j]: lowest key of the rows of a segment with id = i mod best_j
  int best_j;           // 0: no such keys kept
};

struct Smem {
  // offsets from the 1024-aligned base
  int q, code, bars, misc, cm;
  int total;
};

// The small per-CTA state comes first, at offsets that depend on n only,
// so that the epilogue reaches it from the base with constant offsets
// (fewer registers held across its loop); the query tile (1024-byte
// aligned for its swizzle) and the code stages follow.
//   misc: tmem base, abort, verdicts (32 B) + thr[n] u64 + fq[n] float4 +
//         qnorm[n] + cmabs[n] + hist[compact_warps(n)][kHistInts]; then the mbarriers
//         (64 x 8 B) and <q, mu_m> of the tile (cm_bytes, when held)
__host__ __device__ inline Smem smem_layout(int n, int qboxes, int stages, int cm_bytes) {
  Smem s;
  s.misc = 0;
  s.bars = 32 + n * 8 + n * 16 + n * 4 * 2 + compact_warps(n) * kHistInts * 4;
  s.cm = s.bars + 64 * 8;
  s.q = (s.cm + cm_bytes + 1023) / 1024 * 1024;
  s.code = s.q + qboxes * n * 128;
  s.total = s.code + stages * kStageBytes;
  return s;
}

struct Bars {
  uint64_t *code_full, *code_empty, *a_full, *a_empty, *d_full, *d_empty, *q_full, *q_empty, *mma_done;
};

__device__ __forceinline__ Bars bars_at(uint64_t* b) {
  Bars r;
  r.code_full = b;
  r.code_empty = b + kMaxCodeStages;
  r.a_full = b + 2 * kMaxCodeStages;
  r.a_empty = r.a_full + 8;
  r.d_full = r.a_empty + 8;
  r.d_empty = r.d_full + 2;
  r.q_full = r.d_empty + 2;
  r.q_empty = r.q_full + 1;
  r.mma_done = r.q_empty + 1;
  return r;
}

// A position in a ring of n stages: the stage and the parity of its phase,
// advanced without divisions.
struct RingPos {
  int stage = 0;
  uint32_t phase = 0;
  __device__ __forceinline__ void advance(int by, int n) {
    stage += by;
    while (stage >= n) {
      stage -= n;
      phase ^= 1u;
    }
  }
};

// Jobs are dealt round-robin: CTA c takes jobs c, c + grid, ...  At any time
// the CTAs then work on one or two neighbouring database segments for many
// query tiles, so a code tile read from HBM is reused from L2.
struct Job {
  int64_t g, t0, t1;  // query tile, database tiles [t0, t1)
  int s;              // segment
};
__device__ __forceinline__ Job job_of(const MmaArgs& a, int64_t j) {
  Job r;
  r.g = j % a.groups;
  r.s = (int)(j / a.groups);
  r.t0 = a.ntiles * r.s / a.segs;
  r.t1 = a.ntiles * (r.s + 1) / a.segs;
  return r;
}

// float16 pairs of half of a 64-byte box of a row (32 bytes, chunks 2h and
// 2h+1): 4-bit -> 32 pairs (64 dims), 8-bit -> 16 pairs (32 dims, in r[0..15]).
// 4-bit word (dims 8g..8g+7): the pair (2p, 2p+1) sits in bits 4p and 16+4p;
// pairs 0 and 2 become (1024 + c, 1024 + c'), pairs 1 and 3 (1024 + 16c, ...).
template <int BITS>
__device__ __forceinline__ void unpack_half(const uint4 (&w)[4], int h, uint32_t (&r)[32]) {
#pragma unroll
  for (int cc = 0; cc < 2; ++cc) {
    const uint4 q = w[2 * h + cc];
    const uint32_t ws[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (BITS == 4) {
        const uint32_t hi = ws[i] >> 8;
        r[cc * 16 + i * 4 + 0] = (ws[i] & 0x000F000Fu) | 0x64006400u;
        r[cc * 16 + i * 4 + 1] = (ws[i] & 0x00F000F0u) | 0x64006400u;
        r[cc * 16 + i * 4 + 2] = (hi & 0x000F000Fu) | 0x64006400u;
        r[cc * 16 + i * 4 + 3] = (hi & 0x00F000F0u) | 0x64006400u;
      } else {
        r[cc * 8 + i * 2 + 0] = __byte_perm(ws[i], 0x64646464u, 0x5140);  // (1024 + b0, 1024 + b1)
        r[cc * 8 + i * 2 + 1] = __byte_perm(ws[i], 0x64646464u, 0x5342);  // (1024 + b2, 1024 + b3)
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
  uint64_t* thr;    // [N] exact key threshold (insert when key < thr)
  float4* fq;       // [N] {sum(q), 1024 sum(q16), bound, count}: a row may enter only if its
                    //     filter value plus <q, mu_m> exceeds bound; count = keys buffered
  float* qnorm_s;
  float* cmabs_s;   // [N] max_m |<q, mu_m>|
  int* hist;        // [compact_warps(N)][kHistInts] radix histograms of the compacting warps
  __half* cm16;     // [N][M] <q, mu_m> in float16, or null
  float* cm32;      // [N][M] <q, mu_m> in float32, or null
  volatile int* ep_go;  // [2] epilogue leader's verdicts, read by the 4 epilogue warps after a named barrier
  volatile int* bw_job;  // the epilogue's current job for the bound warp (-1 none yet, -2 finished)
  int cta, grid;
};

// Bounded wait by a whole warp, whose lanes share the verdict; on expiry
// record LVQ_ETIMEOUT, tell the other roles, and jump to the role's exit (a
// label `out` in the calling function, which has `lane` and `a` in scope).
#define LVQ_WAIT_WARP(c, bar, par)                                     \
  do {                                                                 \
    if (!__all_sync(kFull, mbar_wait((bar), (par), a.wait_limit))) {   \
      if (lane == 0) {                                                 \
        *(c).abort_sh = 1;                                             \
        set_error(a.st.err, LVQ_ETIMEOUT);                             \
      }                                                                \
      goto out;                                                        \
    }                                                                  \
  } while (0)

// Run by the whole warp 0, like the MMA role: every lane waits, one elected
// lane issues the copies.
template <int N, int BITS>
__device__ __forceinline__ void producer_role(const CUtensorMap* cmap, const CUtensorMap* qmap, const MmaArgs& a,
                                              const Ctx& c, int lane) {
  uint32_t ci = 0, qi = 0;
  RingPos cp;  // code ring position of box ci
  int64_t g_cur = -1;
  for (int64_t j = c.cta; j < a.jobs && !__any_sync(kFull, *c.abort_sh); j += c.grid) {
    const Job jb = job_of(a, j);
    const int64_t g = jb.g, t0 = jb.t0, t1 = jb.t1;
    if (g != g_cur) {
      if (qi > 0) LVQ_WAIT_WARP(c, c.B.q_empty, (qi - 1) & 1);
      if (elect_one()) {
        mbar_expect_tx(c.B.q_full, (uint32_t)(a.qboxes * N * 128));
        for (int kb = 0; kb < a.qboxes; ++kb)
          tma_load_2d(c.qs + kb * N * 128, qmap, c.B.q_full, kb * 64, (int)(g * N));
      }
      __syncwarp();
      ++qi;
      g_cur = g;
    }
    for (int64_t t = t0; t < t1; ++t) {
      for (int kb = 0; kb < a.n_kbox; ++kb) {
        const int s = cp.stage;
        LVQ_WAIT_WARP(c, c.B.code_empty + s, cp.phase ^ 1);
        if (elect_one()) {
          mbar_expect_tx(c.B.code_full + s, kStageBytes);
          tma_load_2d(c.cst + s * kStageBytes, cmap, c.B.code_full + s, kb * kBoxBytes, (int)(t * kRows));
        }
        __syncwarp();
        ++ci;
        cp.advance(1, a.code_stages);
      }
    }
  }
out:
  // copies that may still be in flight: the last (up to) code_stages code
  // boxes and the last query tile
  for (uint32_t j = 1; j <= (uint32_t)a.code_stages && j <= ci; ++j) {
    const uint32_t k = ci - j;
    (void)__all_sync(kFull, mbar_wait(c.B.code_full + k % a.code_stages, (k / a.code_stages) & 1, kWaitLimit));
  }
  if (qi > 0) (void)__all_sync(kFull, mbar_wait(c.B.q_full, (qi - 1) & 1, kWaitLimit));
}

// Run by the whole warp 1: every lane waits on the mbarriers and one elected
// lane (elect.sync) issues the MMAs and commits.  Measured on B300, a
// converged warp issues back-to-back M = 128, K = 16 MMAs at the full rate
// (64 cycles each at N = 128) with a wait and a commit every 8 of them,
// where a lone thread in a divergent branch took 90 cycles per MMA (and 59
// at N <= 64 even without waits, against 19 from a converged warp).
template <int N, int BITS>
__device__ __forceinline__ void mma_role(const MmaArgs& a, const Ctx& c, int lane) {
  constexpr int kBoxDims = BITS == 4 ? 128 : 64;
  constexpr int kACols = kBoxDims / 2;
  constexpr int kKSteps = kBoxDims / 16;
  constexpr uint32_t kIdesc = idesc_f16_f32(kRows, N);
  const int AS = a.a_stages;
  uint32_t di = 0, qi = 0;
  RingPos ap;  // A ring position
  int64_t g_cur = -1;
  const uint32_t qbase = smem_u32(c.qs);
  // a bounded wait whose verdict the whole warp shares
  for (int64_t j = c.cta; j < a.jobs && !__any_sync(kFull, *c.abort_sh); j += c.grid) {
    const Job jb = job_of(a, j);
    const int64_t g = jb.g, t0 = jb.t0, t1 = jb.t1;
    if (g != g_cur) {
      LVQ_WAIT_WARP(c, c.B.q_full, qi & 1);
      ++qi;
      g_cur = g;
      tc_fence_after();
    }
    for (int64_t t = t0; t < t1; ++t) {
      const int db = di & 1;
      LVQ_WAIT_WARP(c, c.B.d_empty + db, ((di >> 1) & 1) ^ 1);
      tc_fence_after();
      const uint32_t d_tmem = c.tbase + db * N;
      for (int kb = 0; kb < a.n_kbox; ++kb) {
        const int s = ap.stage;
        LVQ_WAIT_WARP(c, c.B.a_full + s, ap.phase);
        tc_fence_after();
        const uint32_t a_tmem = c.tbase + 2 * N + s * kACols;
        // K step kk of this box reads query dims kg .. kg+15, kg = kb*box + 16kk:
        // 64-dim query box kg/64 (N x 128 bytes each), byte offset 2*(kg%64)
        const uint64_t d0 = desc_sw128(qbase + (uint32_t)(kb * kBoxDims / 64) * N * 128);
        if (elect_one()) {
#pragma unroll
          for (int kk = 0; kk < kKSteps; ++kk) {
            const uint32_t off16 = (uint32_t)((kk * 16 / 64) * N * 128 + ((kk * 16) % 64) * 2) >> 4;
            mma_f16_ts(d_tmem, a_tmem + kk * 8, d0 + off16, kIdesc, (kb | kk) != 0);
          }
          mma_commit(c.B.a_empty + s);
        }
        __syncwarp();
        ap.advance(1, AS);
      }
      if (elect_one()) mma_commit(c.B.d_full + db);
      __syncwarp();
      ++di;
    }
    if (elect_one()) mma_commit(c.B.q_empty);
    __syncwarp();
  }
out:
  // all MMAs issued by this warp are complete before TMEM is freed
  if (elect_one()) mma_commit(c.B.mma_done);
  __syncwarp();
  (void)__all_sync(kFull, mbar_wait(c.B.mma_done, 0, kWaitLimit));
}

template <int N, int BITS>
__device__ __forceinline__ void unpack_role(const MmaArgs& a, const Ctx& c, int warp, int lane) {
  constexpr int kBoxDims = BITS == 4 ? 128 : 64;
  constexpr int kACols = kBoxDims / 2;
  const int AS = a.a_stages;
  const int quarter = warp & 3;
  const int row = quarter * 32 + lane;
  const uint32_t lane_base = c.tbase + ((uint32_t)(quarter * 32) << 16);
  // the two warps of a lane quarter take alternate boxes: this warp's boxes
  // are the CTA's boxes number `parity`, parity + 2, ...
  const int parity = (warp - 2) >> 2;
  RingPos cp, ap;  // ring positions of this warp's next box
  cp.advance(parity, a.code_stages);
  ap.advance(parity, AS);
  int skip = parity;  // boxes to pass before this warp's next one
  for (int64_t j = c.cta; j < a.jobs && !__any_sync(kFull, *c.abort_sh); j += c.grid) {
    const Job jb = job_of(a, j);
    const int64_t t0 = jb.t0, t1 = jb.t1;
    for (int64_t t = t0; t < t1; ++t) {
      for (int kb = 0; kb < a.n_kbox; ++kb) {
        if (skip) {
          --skip;
          continue;
        }
        skip = 1;
        const int s = cp.stage;
        LVQ_WAIT_WARP(c, c.B.code_full + s, cp.phase);
        const uint4* src = reinterpret_cast<const uint4*>(c.cst + s * kStageBytes + row * kBoxBytes);
        uint4 w[4];
        const int sw = (row >> 1) & 3;  // 64-byte swizzle of the TMA box
#pragma unroll
        for (int q = 0; q < 4; ++q) w[q] = src[q ^ sw];
        __syncwarp();
        if (lane == 0) mbar_arrive(c.B.code_empty + s);
        const int as = ap.stage;
        LVQ_WAIT_WARP(c, c.B.a_empty + as, ap.phase ^ 1);
        tc_fence_after();
        const uint32_t taddr = lane_base + 2 * N + as * kACols;
        // tcgen05.st reads its source registers after issue: a register set
        // is rewritten only after tcgen05.wait::st (one set of 32 live at a
        // time; the other warp of the quarter covers the store latency)
        uint32_t r[32];
        if (BITS == 4) {
          unpack_half<BITS>(w, 0, r);
          tmem_st_x32<0>(taddr, r);
          tmem_st_wait();
          unpack_half<BITS>(w, 1, r);
          tmem_st_x32<0>(taddr + 32, r);
        } else {
          uint32_t r2[32];
          unpack_half<BITS>(w, 0, r);
          unpack_half<BITS>(w, 1, r2);
#pragma unroll
          for (int i = 0; i < 16; ++i) r[16 + i] = r2[i];
          tmem_st_x32<0>(taddr, r);
        }
        tmem_st_wait();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(c.B.a_full + as);
        cp.advance(2, a.code_stages);
        ap.advance(2, AS);
      }
    }
  }
out:
  return;
}

// Per-row constants of a database tile, loaded one tile ahead.
struct RowMeta {
  float lo, step, neg_h, nrm;
  int m;
  bool valid;
};

__device__ __forceinline__ RowMeta load_meta(const MmaArgs& a, int64_t rw, bool ip) {
  RowMeta r;
  r.valid = rw < a.n_rows && is_live(a.st.live, rw);
  const int64_t s = r.valid ? rw : 0;
  r.lo = __ldg(a.st.lower + s);
  r.step = __ldg(a.st.step + s);
  r.m = __ldg(a.st.mean_id + s);
  r.nrm = ip ? 0.0f : __ldg(a.st.norm2 + s);
  r.neg_h = -0.5f * r.nrm;
  return r;
}

// Fetch the line holding p into L2 (a hint: no data returns).
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// CM: how <q, mu_m> of the query tile is held in shared memory: 0 not at
// all, 1 float16, 2 float32.
// A threshold key's score as a bound on the filter value (plus <q, mu_m>
// when the table is held; less max |<q, mu_m>| when not), less a margin for
// rounding.
__device__ __forceinline__ float bound_of(uint64_t tk, float qn, float cmabs, bool ip, int cm_table) {
  const float ts = key_score(tk, ip ? LVQ_IP : LVQ_L2);
  float b = ip ? ts : 0.5f * (qn - ts);
  b -= 1e-5f * (fabsf(ts) + qn + cmabs) + 1e-30f;
  if (cm_table == 0) b -= cmabs;
  return b;
}

// A bound on the k-th lowest key of a query from the lowest keys of P <= 256
// disjoint row sets (kNoKey where a set has none): the smallest score word
// T such that at least k of the P keys have a score word <= T, as the key
// (T, any id).  At least k distinct rows then have keys at or below it, so
// the query's k-th lowest key over all rows is too.  kNoKey when fewer than
// k keys exist.  Called by a whole warp.
__device__ __noinline__ uint64_t union_bound(const uint64_t* keys, int P, int k, int lane) {
  uint32_t v[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int at = lane + 32 * i;
    v[i] = at < P ? (uint32_t)(__ldcg(keys + at) >> 32) : 0xFFFFFFFFu;
  }
  uint32_t lo = 0, hi = 0xFFFFFFFFu;
  while (lo < hi) {
    const uint32_t mid = lo + (hi - lo) / 2;
    int c = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) c += v[i] <= mid ? 1 : 0;
    if ((int)__reduce_add_sync(kFull, (unsigned)c) >= k)
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo == 0xFFFFFFFFu ? kNoKey : (((uint64_t)lo << 32) | 0xFFFFFFFFull);
}

// Candidate-buffer selections, kept out of line: they run rarely and their
// register arrays would otherwise share the epilogue's register budget.
__device__ __noinline__ int prune_keys(uint64_t* buf, int n, int k, int keep_max, int* hist, uint64_t* thr) {
  return warp_prune(buf, n, k, keep_max, hist, thr);
}
__device__ __noinline__ int select_keys(uint64_t* buf, int n, int k, int* hist, uint64_t* thr) {
  return warp_select6(buf, n, k, hist, thr);
}

template <int N, int BITS, int CM>
__device__ __forceinline__ void epilogue_role(const MmaArgs& a, const Ctx& c, int warp, int lane) {
  const int quarter = warp & 3;
  const int ew = warp - kEpiWarp0;  // 0..7
  const int et = ew * 32 + lane;    // 0..255
  const int row_in = quarter * 32 + lane;
  // columns of this warp: warps 0-3 the first half, 4-7 the second
  constexpr int kHalf = N / 2;
  const int col0 = (ew >> 2) * kHalf;
  const int col1 = col0 + kHalf <= N ? col0 + kHalf : N;
  const uint32_t lane_base = c.tbase + ((uint32_t)(quarter * 32) << 16);
  const DeviceStore& st = a.st;
  const bool ip = st.metric == LVQ_IP;
  uint64_t* mybuf = a.cand + (int64_t)c.cta * N * a.cap;
  constexpr int kCW = compact_warps(N);
  int* myhist = c.hist + (ew & (kCW - 1)) * kHistInts;  // used by warps 0 .. kCW-1
  uint32_t di = 0, pub = 0;
  // The eight epilogue warps meet at named barriers, so they must all take
  // the same path: only the first waits on mbarriers and reads the abort
  // flag, and publishes its verdict in shared memory before a barrier.
  // Verdicts alternate between two slots, so a slot is rewritten only after
  // every warp has passed the barrier that follows its read.
  for (int64_t j = c.cta; j < a.jobs; j += c.grid) {
    const Job jb = job_of(a, j);
    const int64_t g = jb.g, t0 = jb.t0, t1 = jb.t1;
    const int64_t q0 = g * N;
    if (N <= 64 && et == 0) *c.bw_job = (int)j;
    if (et < N) {
      const bool real = q0 + et < a.nq;
      float cmabs = 0.0f;
      if (real)
        for (int m = 0; m < st.n_means; ++m) cmabs = fmaxf(cmabs, fabsf(a.p.cm[(q0 + et) * st.n_means + m]));
      c.cmabs_s[et] = cmabs;
      const float qn = real ? a.p.qnorm[q0 + et] : 0.0f;
      c.qnorm_s[et] = qn;
      // absent queries take nothing (bound +inf); real ones start from the
      // global bound of earlier jobs (everything, -inf, while there is none)
      const uint64_t gt = real ? *reinterpret_cast<volatile uint64_t*>(a.gthr + q0 + et) : 0ull;
      c.thr[et] = gt;
      float b = real ? __int_as_float(0xff800000) : __int_as_float(0x7f800000);
      if (real && gt != kNoKey) b = bound_of(gt, qn, cmabs, ip, CM);
      c.fq[et] = make_float4(real ? a.p.qsum[q0 + et] : 0.0f, real ? 1024.0f * a.p.q16sum[q0 + et] : 0.0f, b, 0.0f);
    }
    if (CM) {
      for (int i = et; i < N * st.n_means; i += kEpiThreads) {
        const int n = i / st.n_means;
        const float v = q0 + n < a.nq ? a.p.cm[q0 * st.n_means + i] : 0.0f;
        if (CM == 2) c.cm32[i] = v;
        else c.cm16[i] = __float2half_rn(v);
      }
    }
    if (et == 0) c.ep_go[pub & 1] = !*c.abort_sh;
    named_bar(1, kEpiThreads);
    if (!c.ep_go[pub++ & 1]) goto out;
    RowMeta nxt = load_meta(a, t0 * kRows + row_in, ip);
    // The shared bound is read again every tile (the value read one tile ago
    // is applied, so the load's latency hides behind a tile): once any CTA
    // has cut a query's buffer, every other CTA filters with the k1-th best
    // of all rows scanned so far instead of its own.
    uint64_t pend = kNoKey;
    for (int64_t t = t0; t < t1; ++t) {
      const int db = di & 1;
      if (et < N && q0 + et < a.nq) {
        if (pend < c.thr[et]) {
          c.thr[et] = pend;
          c.fq[et].z = bound_of(pend, c.qnorm_s[et], c.cmabs_s[et], ip, CM);
        }
        pend = *reinterpret_cast<volatile uint64_t*>(a.gthr + q0 + et);
      }
      if (ew == 0) {
        const bool ok = !*c.abort_sh && mbar_wait(c.B.d_full + db, (di >> 1) & 1, a.wait_limit);
        if (!ok && lane == 0) {
          if (!*c.abort_sh) set_error(st.err, LVQ_ETIMEOUT);
          *c.abort_sh = 1;
        }
        __syncwarp();
        if (lane == 0) c.ep_go[pub & 1] = ok;
      }
      named_bar(1, kEpiThreads);
      if (!c.ep_go[pub++ & 1]) goto out;
      tc_fence_after();
      const RowMeta cur = nxt;
      if (t + 1 < t1) nxt = load_meta(a, (t + 1) * kRows + row_in, ip);
      // With up to 64 queries a tile takes only a few microseconds, and the
      // codes stream from HBM: the per-row constants of the tile kMetaAhead
      // tiles on are fetched into L2 now, so that the loads one tile ahead
      // wait on L2 rather than HBM (one line per lane: 4 lines of each float
      // array, the mean ids, the live words).
      if (N <= 64 && et < 14 && t + kMetaAhead < t1) {
        const int64_t r0 = (t + kMetaAhead) * kRows + (et & 3) * 32;
        const int64_t r = r0 < a.n_rows ? r0 : a.n_rows - 1;
        if (et < 4) prefetch_l2(st.lower + r);
        else if (et < 8) prefetch_l2(st.step + r);
        else if (et < 12) { if (!ip) prefetch_l2(st.norm2 + r); }
        else if (et == 12) prefetch_l2(st.mean_id + r);
        else prefetch_l2(st.live + (r >> 5));
      }
      const int64_t rw = t * kRows + row_in;
      const float* cm_row = a.p.cm + q0 * st.n_means + cur.m;
      const __half* cm16_row = c.cm16 + cur.m;
      const float* cm32_row = c.cm32 + cur.m;
      // This warp's columns, 32 at a time from TMEM.  The filter value
      // D <q16, c> + l sum(q) - ||x^||^2 / 2 (IP: no norm term), plus
      // <q, mu_m> (the shared-memory copy; 0 when not held), is compared with
      // fq[n].z, the query's threshold minus a rounding margin (minus
      // max_m |<q, mu_m>| without the copy): rows below it cannot beat the
      // threshold.  The rows that pass get their exact key (with the same
      // <q, mu_m>) and the exact test.
      constexpr int kPart = kHalf < 32 ? kHalf : 32;  // columns per TMEM read
      uint64_t pass = 0;
#pragma unroll
      for (int part = 0; part < kHalf / kPart; ++part) {
        uint32_t v[kPart];
        if constexpr (kPart == 8) {
          tmem_ld_x8<0>(lane_base + db * N + col0, v);
        } else if constexpr (kPart == 16) {
          tmem_ld_x16<0>(lane_base + db * N + col0, v);
        } else {
          tmem_ld_x32<0>(lane_base + db * N + col0 + part * 32, v);
        }
        tmem_ld_wait();
        if (col0 < col1) {
#pragma unroll
          for (int j = 0; j < kPart; ++j) {
            const int n = col0 + part * kPart + j;
            const float4 f = c.fq[n];
            const float acc = __uint_as_float(v[j]) - f.y;
            float fv = __fmaf_rn(cur.lo, f.x, __fmaf_rn(cur.step, acc, cur.neg_h));
            if (CM == 2) fv += cm32_row[n * st.n_means];
            if (CM == 1) fv += __half2float(cm16_row[n * st.n_means]);
            pass |= (uint64_t)(fv > f.z ? 1u : 0u) << (part * kPart + j);
          }
        }
      }
      if (!cur.valid) pass = 0;
      // Columns where some row of the warp passed, one at a time
      // (warp-uniform), re-read from TMEM: the exact key and the exact test.
      uint64_t any = pass;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) any |= __shfl_xor_sync(kFull, any, o);
      while (any) {
        const int j = __ffsll((long long)any) - 1;
        any &= any - 1;
        const int n = col0 + j;
        const uint32_t raw = tmem_ld_x1(lane_base + db * N + n);
        tmem_ld_wait();
        if ((pass >> j) & 1ull) {
          const float4 f = c.fq[n];
          const float acc = __uint_as_float(raw) - f.y;
          const float cmv = CM == 2 ? cm32_row[n * st.n_means]
                            : CM == 1 ? __half2float(cm16_row[n * st.n_means]) : __ldg(cm_row + n * st.n_means);
          float sc = __fmaf_rn(cur.step, acc, __fmaf_rn(cur.lo, f.x, cmv));
          if (!ip) sc = c.qnorm_s[n] + cur.nrm - 2.0f * sc;
          const uint64_t key = make_key(sc, (uint32_t)rw, st.metric);
          if (key < c.thr[n]) mybuf[n * a.cap + atomicAdd(reinterpret_cast<int*>(&c.fq[n].w), 1)] = key;
          if (N <= 64 && a.best_j && q0 + n < a.nq)
            atomicMin(reinterpret_cast<unsigned long long*>(a.seg_best) +
                          ((q0 + n) * a.segs + jb.s) * a.best_j + (int)(rw % a.best_j),
                      (unsigned long long)key);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(c.B.d_empty + db);
      ++di;
      named_bar(1, kEpiThreads);
      if (ew < kCW) {
        // warps 0 .. kCW-1 compact the buffers that may not take another
        // tile: warp ew owns queries ew, ew + kCW, ... (one per lane), and only
        // those whose buffer is full are visited
        const int nl = ew + kCW * lane;
        uint32_t full = __ballot_sync(kFull, nl < N && __float_as_int(c.fq[nl < N ? nl : 0].w) > a.cap - kRows);
        while (full) {
          const int n = ew + kCW * (__ffs((int)full) - 1);
          full &= full - 1;
          const int cnt = __float_as_int(c.fq[n].w);
          {
            uint64_t tk;
            const int kept = prune_keys(mybuf + n * a.cap, cnt, a.k1, a.k1 + (a.cap - kRows - a.k1) / 2, myhist, &tk);
            if (lane == 0) {
              c.fq[n].w = __int_as_float(kept);
              // the bound only tightens (it may already be the shared one)
              if (tk < c.thr[n]) {
                c.thr[n] = tk;
                atomicMin(reinterpret_cast<unsigned long long*>(a.gthr + q0 + n), tk);
                c.fq[n].z = bound_of(tk, c.qnorm_s[n], c.cmabs_s[n], ip, CM);
              }
            }
            __syncwarp();
          }
        }
      }
      named_bar(1, kEpiThreads);
    }
    if (ew < kCW) {
      // end of job: the k1 best of each query in segment jb.s; its k1-th key
      // bounds every job, and only keys at or below the bound are kept
      for (int n = ew; n < N; n += kCW) {
        if (q0 + n >= a.nq) continue;
        uint64_t tk;
        uint64_t* b0 = mybuf + n * a.cap;
        const int kept = select_keys(b0, __float_as_int(c.fq[n].w), a.k1, myhist, &tk);
        if (lane == 0 && kept == a.k1) atomicMin(reinterpret_cast<unsigned long long*>(a.gthr + q0 + n), tk);
        __syncwarp();
        const uint64_t gt = *reinterpret_cast<volatile uint64_t*>(a.gthr + q0 + n);
        uint64_t* dst = a.partial + ((q0 + n) * a.segs + jb.s) * a.k1;
        int pos = 0;
        for (int base = 0; base < kept; base += 32) {
          const uint64_t v = base + lane < kept ? b0[base + lane] : kNoKey;
          const bool keep = base + lane < kept && v <= gt;
          const unsigned m = __ballot_sync(kFull, keep);
          if (keep) dst[pos + __popc(m & ((1u << lane) - 1u))] = v;
          pos += __popc(m);
        }
        if (lane == 0) a.counts[(q0 + n) * a.segs + jb.s] = pos;
      }
    }
    named_bar(1, kEpiThreads);
  }
out:
  if (N <= 64 && et == 0) *c.bw_job = -2;
  return;
}

// The bound warp: while the epilogue works on a job, it takes the job's
// queries in turn and lowers each one's shared bound to the union bound of
// the lowest keys every segment has found so far (union_bound).  It waits on
// nothing: it reads the epilogue's job index, and stops when the epilogue
// marks its exit (or after a pass limit).
template <int N>
__device__ __forceinline__ void bound_role(const MmaArgs& a, const Ctx& c, int lane) {
  if (!a.best_j) return;
  const int P = a.segs * a.best_j;
  for (uint32_t pass = 0; pass < (1u << 24); ++pass) {
    const int jv = __shfl_sync(kFull, *c.bw_job, 0);
    if (jv == -2) return;
    if (jv < 0) {
      __nanosleep(256);
      continue;
    }
    const int64_t q0 = job_of(a, jv).g * N;
    for (int n = 0; n < N && q0 + n < a.nq; ++n) {
      const uint64_t b = union_bound(a.seg_best + (q0 + n) * P, P, a.k1, lane);
      if (lane == 0 && b != kNoKey) atomicMin(reinterpret_cast<unsigned long long*>(a.gthr + q0 + n), b);
    }
  }
}

#undef LVQ_WAIT_WARP

template <int N, int BITS, int CM>
__global__ void __launch_bounds__(warps_of<N>() * 32, 1)
    scan_mma_kernel(const __grid_constant__ CUtensorMap cmap, const __grid_constant__ CUtensorMap qmap, MmaArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const Smem L = smem_layout(N, a.qboxes, a.code_stages, a.cm_table * N * a.st.n_means * 2);
  Ctx c;
  c.qs = smem + L.q;
  c.cst = smem + L.code;
  uint64_t* bar_mem = reinterpret_cast<uint64_t*>(smem + L.bars);
  uint32_t* tmem_base_sh = reinterpret_cast<uint32_t*>(smem + L.misc);
  c.abort_sh = reinterpret_cast<volatile int*>(smem + L.misc + 16);
  c.thr = reinterpret_cast<uint64_t*>(smem + L.misc + 32);
  c.fq = reinterpret_cast<float4*>(c.thr + N);
  c.qnorm_s = reinterpret_cast<float*>(c.fq + N);
  c.cmabs_s = c.qnorm_s + N;
  c.hist = reinterpret_cast<int*>(c.cmabs_s + N);
  c.cm16 = reinterpret_cast<__half*>(smem + L.cm);  // used when CM == 1
  c.cm32 = reinterpret_cast<float*>(smem + L.cm);   // used when CM == 2
  c.ep_go = reinterpret_cast<volatile int*>(smem + L.misc + 20);  // two ints
  c.bw_job = reinterpret_cast<volatile int*>(smem + L.misc + 28);
  c.B = bars_at(bar_mem);
  c.grid = gridDim.x;
  c.cta = blockIdx.x;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < a.code_stages; ++i) {
      mbar_init(c.B.code_full + i, 1);
      mbar_init(c.B.code_empty + i, 4);
    }
    for (int i = 0; i < a.a_stages; ++i) {
      mbar_init(c.B.a_full + i, 4);
      mbar_init(c.B.a_empty + i, 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(c.B.d_full + i, 1);
      mbar_init(c.B.d_empty + i, 8);
    }
    mbar_init(c.B.q_full, 1);
    mbar_init(c.B.q_empty, 1);
    mbar_init(c.B.mma_done, 1);
    *c.abort_sh = 0;
    *c.bw_job = -1;
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
    producer_role<N, BITS>(&cmap, &qmap, a, c, lane);
  } else if (warp == 1) {
    mma_role<N, BITS>(a, c, lane);
  } else if (warp < kEpiWarp0) {
    unpack_role<N, BITS>(a, c, warp, lane);
  } else if (warp < kBoundWarp) {
    epilogue_role<N, BITS, CM>(a, c, warp, lane);
  } else if (N <= 64) {
    bound_role<N>(a, c, lane);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(c.tbase, kTmemCols);
}

// ---- host side -------------------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  // looked up once per process (thread-safe initialisation of a local static)
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    return nullptr;
  }();
  return fn;
}

// candidate buffer per (CTA, query): room for k1 kept keys, a tile of new
// ones, and slack so that compactions are rare; at most 1024 keys (the
// radix select holds them in registers)
int mma_cap(int k1) {
  const int c = 2 * pow2_at_least(k1 + kRows);
  return c <= 1024 ? c : 1024;
}

int max_n_tile(const DeviceStore& st) {
  // the largest query tile whose queries fit in shared memory beside three
  // code stages (and, below 128 queries, a float32 table of <q, mu_m>)
  const int qboxes = (int)ceil_div(st.row1, kBoxBytes) * (st.bits1 == 4 ? 2 : 1);
  for (int n = 128; n >= 16; n >>= 1) {
    const int cm = n < 128 ? n * st.n_means * 4 : 0;
    if ((size_t)smem_layout(n, qboxes, 3, cm).total + 1024 <= 232448) return n;
  }
  return 0;
}

template <int N, int BITS, int CM>
cudaError_t launch_nbc(const CUtensorMap& cm, const CUtensorMap& qm, const MmaArgs& a, int grid, size_t smem,
                       cudaStream_t stream) {
  static std::atomic<uint64_t> attr{0};
  const cudaError_t e = max_dyn_smem_once((const void*)scan_mma_kernel<N, BITS, CM>, 232448, attr);
  if (e != cudaSuccess) return e;
  scan_mma_kernel<N, BITS, CM><<<grid, warps_of<N>() * 32, smem, stream>>>(cm, qm, a);
  return cudaGetLastError();
}

// Query tiles of up to 64 queries always hold <q, mu_m> in float32 (it fits
// for M <= 256); 128-query tiles hold it as space allows.
template <int N, int BITS>
cudaError_t launch_nb(const CUtensorMap& cm, const CUtensorMap& qm, const MmaArgs& a, int grid, size_t smem,
                      cudaStream_t stream) {
  if constexpr (N < 128) {
    return launch_nbc<N, BITS, 2>(cm, qm, a, grid, smem, stream);
  } else {
    switch (a.cm_table) {
      case 2: return launch_nbc<N, BITS, 2>(cm, qm, a, grid, smem, stream);
      case 1: return launch_nbc<N, BITS, 1>(cm, qm, a, grid, smem, stream);
      default: return launch_nbc<N, BITS, 0>(cm, qm, a, grid, smem, stream);
    }
  }
}

}  // namespace

// Tensor map of the first-level codes: 128-row x 64-byte boxes, 64-byte
// swizzle (shared by the tensor-core and the small-batch scans).
cudaError_t encode_code_map(const DeviceStore& st, CUtensorMap* cm, int box_bytes) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  if (box_bytes != 64 && box_bytes != 128) return cudaErrorInvalidValue;
  cuuint64_t dims[2] = {(cuuint64_t)st.row1, (cuuint64_t)st.capacity};
  cuuint64_t strides[1] = {(cuuint64_t)st.stride1};  // records: codes, then a 16-byte trailer
  cuuint32_t box[2] = {(cuuint32_t)box_bytes, (cuuint32_t)kRows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(cm, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, st.codes1, dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, box_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

bool mma_supported(const DeviceStore& st) {
  return (st.bits1 == 4 || st.bits1 == 8) && max_n_tile(st) > 0 && encode_fn() != nullptr;
}

int mma_tile_limit(const DeviceStore& st) { return max_n_tile(st); }

size_t mma_scan_cand_bytes(int grid, int n_tile, int k1) { return (size_t)grid * n_tile * mma_cap(k1) * 8; }

int mma_segments(int grid, int64_t groups, int64_t ntiles) {
  // groups x segments a multiple of grid: every CTA gets as many jobs
  int64_t x = groups, y = grid;
  while (y) {
    const int64_t t = x % y;
    x = y;
    y = t;
  }
  int64_t segs = grid / x;
  if (segs > ntiles) segs = ntiles;
  return (int)(segs < 1 ? 1 : segs);
}

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
  a.cap = mma_cap(plan.k1);
  a.n_kbox = (int)ceil_div(st.row1, kBoxBytes);
  a.qboxes = qboxes;
  const int acols = st.bits1 == 4 ? 64 : 32;
  a.a_stages = (kTmemCols - 2 * n_tile) / acols;
  if (a.a_stages > 8) a.a_stages = 8;
  a.ntiles = ceil_div(plan.n_rows > 0 ? plan.n_rows : 1, kRows);
  a.groups = p.nq_pad / n_tile;
  a.segs = plan.splits;
  a.jobs = a.groups * a.segs;
  a.counts = plan.counts;
  a.gthr = plan.gthr;
  a.wait_limit = plan.wait_polls > 0 ? plan.wait_polls : kWaitLimit;
  a.seg_best = plan.seg_best;
  a.best_j = plan.seg_best ? plan.best_j : 0;
  if (!a.counts || !a.gthr || a.segs < 1 || a.segs > a.ntiles) return cudaErrorInvalidValue;
  const int grid = plan.grid;

  CUtensorMap cm, qm;
  {
    const cudaError_t e = encode_code_map(st, &cm, kBoxBytes);
    if (e != cudaSuccess) return e;
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
  cudaError_t e = cudaMemsetAsync(plan.gthr, 0xFF, (size_t)nq * 8, stream);
  if (e != cudaSuccess) return e;
  if (a.best_j) {
    e = cudaMemsetAsync(a.seg_best, 0xFF, (size_t)nq * a.segs * a.best_j * 8, stream);
    if (e != cudaSuccess) return e;
  }
  // as many code stages as shared memory allows (more bytes in flight for
  // narrow query tiles)
  // The table of <q, mu_m> is held in float32 when it fits beside three
  // code stages, else in float16 (scores then carry its rounding, at most
  // 2^-11 |<q, mu_m>|), else not at all.
  a.cm_table = 0;
  for (int w = 2; w >= 1 && !a.cm_table; --w)
    if ((size_t)smem_layout(n_tile, qboxes, 3, n_tile * st.n_means * 2 * w).total + 1024 <= 232448) a.cm_table = w;
  if (n_tile < 128 && a.cm_table != 2) return cudaErrorInvalidConfiguration;  // narrow tiles always hold float32
  const int cmb = n_tile * st.n_means * 2 * a.cm_table;
  a.code_stages = kMaxCodeStages;
  while (a.code_stages > 2 && (size_t)smem_layout(n_tile, qboxes, a.code_stages, cmb).total + 1024 > 232448)
    --a.code_stages;
  const Smem L = smem_layout(n_tile, qboxes, a.code_stages, cmb);
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
