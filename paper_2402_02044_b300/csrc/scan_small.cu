// First-level scan of small query batches (1 to 4 queries) on CUDA cores.
//
// A small batch reads every code byte once for a few dot products, so the
// scan is bound by HBM, not by arithmetic, and is not reshaped into a
// matrix product.  Each query is rounded to 16-bit integers,
//   q ~ s * (256 hi + lo),  s = max|q| / 32767,  hi a signed, lo an unsigned byte,
// and <q, c> ~ s * (256 sum hi_j c_j + sum lo_j c_j) is accumulated exactly
// in 32-bit integers with dp4a (four byte products per instruction).  4-bit
// codes become bytes with one mask each: (w & 0x0F0F0F0F) holds dims
// (0, 4, 1, 5) of an 8-dim code word and ((w >> 4) & 0x0F0F0F0F) dims
// (2, 6, 3, 7); the query bytes are stored in the same order.  Then
//   IP: s = <q, mu_m> + l sum(q) + D <q, c>;   L2: ||q||^2 + ||x^||^2 - 2 s.
//
// One persistent CTA per SM scans a contiguous range of database tiles.
// One thread of warp 0 streams each tile's 128-byte code boxes with TMA into
// one ring per consumer group; each group (four warps, 128 threads) takes
// every G-th tile and runs without waiting for the others.  A thread scores
// one row of a 128-row tile, or, when the batch has two or more queries, two
// rows of a 256-row tile: the query bytes come from shared memory (a 128-bit
// broadcast read costs four shared-memory wavefronts, which bound the scan
// once there are several queries), and each read then serves two rows.  Per
// query and group, scores below a running threshold (the lowest of the
// groups') go to a candidate buffer in shared memory, which a warp cuts back
// to the k1 best when it fills; at the end each CTA's k1 best of the union go
// to partial[q][cta][.].
#include <cudaTypedefs.h>

#include "kernels.cuh"
#include "score.cuh"
#include "tcgen05.cuh"

namespace lvq {

namespace {

using namespace sm100;

constexpr int kRows = 128;
constexpr int kBoxBytes = 128;  // 128-byte swizzle: chunk c of row r sits at c ^ (r & 7)
constexpr int kChunks = kBoxBytes / 16;
constexpr int kStageBytes = kRows * kBoxBytes;
constexpr int kMaxRingStages = 8;  // per ring; two rings
// groups of 4 consumer warps (one 128-row tile each at a time) + 1 producer warp
__host__ __device__ constexpr int small_threads(int groups) { return 32 * (1 + 4 * groups); }
constexpr uint32_t kWaitLimit = 1u << 24;
constexpr int kSmemLimit = 232448;

struct SmallArgs {
  DeviceStore st;
  int64_t nq;
  const uint32_t* qw;   // [nq][4][Wp]: A-hi, B-hi, A-lo, B-lo bytes per code word
  const float* qscale;  // [nq]
  QueryPrep p;
  int Wp;               // code words per row, padded to whole boxes
  int n_kbox;
  int stages;           // ring stages per ring
  int k1, cap;
  int64_t n_rows, ntiles;
  uint64_t* partial;    // [nq][gridDim.x][k1]
  int* counts;          // [nq][gridDim.x] keys written per list
  uint64_t* gthr;       // [nq] lowest k1-th key any CTA has found (bounds the global k1-th)
};

__device__ __forceinline__ int dp4a_us(uint32_t a, uint32_t b, int c) {
  int d;
  asm("dp4a.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ uint32_t dp4a_uu(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("dp4a.u32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

// Cuts a candidate buffer to its k best (kept out of line: the scan loop
// and the select do not share registers).
__device__ __noinline__ int select_k(uint64_t* buf, int n, int k, int* hist, uint64_t* thr) {
  return warp_select6(buf, n, k, hist, thr);
}

struct SmallSmem {
  int ring, qw, fq, thr, cnt, cm, cand, hist, bars, total;
};

__host__ __device__ inline int align_up(int x, int a) { return (x + a - 1) / a * a; }

// cand: [QB][G groups][cap] keys; thr, cnt: [G][QB]; hist: 64 ints per consumer warp
__host__ __device__ inline SmallSmem small_layout(int qb, int G, int Wp, int M, int cap, int stages, int rpt) {
  SmallSmem s;
  s.ring = 0;
  s.qw = s.ring + G * stages * kStageBytes * rpt;
  s.fq = s.qw + qb * 4 * Wp * 4;
  s.thr = s.fq + qb * 16;
  s.cnt = s.thr + G * qb * 8;
  s.cm = align_up(s.cnt + G * qb * 4 + 16, 16);
  s.cand = align_up(s.cm + qb * M * 4, 16);
  s.hist = s.cand + qb * G * cap * 8;
  s.bars = align_up(s.hist + 4 * G * 64 * 4, 16);
  s.total = s.bars + 2 * G * stages * 8;
  return s;
}

// QB: query slots (nq <= QB); BITS: first-level code width; G: consumer
// groups; RPT: rows per consumer thread (a tile is RPT x 128 rows, thread i
// of a group scores rows i, i + 128, .. of it).
template <int QB, int BITS, int G, int RPT>
__global__ void __launch_bounds__(small_threads(G), 1)
    scan_small_kernel(const __grid_constant__ CUtensorMap cmap, SmallArgs a) {
  constexpr int kThreads = small_threads(G);
  constexpr int kTR = kRows * RPT;              // rows per tile
  constexpr int kStageB = kStageBytes * RPT;    // bytes per ring stage (RPT boxes)
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const DeviceStore& st = a.st;
  const int RS = a.stages;
  const SmallSmem L = small_layout(QB, G, a.Wp, st.n_means, a.cap, RS, RPT);
  unsigned char* ring = smem + L.ring;
  uint32_t* qw = reinterpret_cast<uint32_t*>(smem + L.qw);
  float4* fq = reinterpret_cast<float4*>(smem + L.fq);  // {sum q, s, 0, ||q||^2}
  uint64_t* thr = reinterpret_cast<uint64_t*>(smem + L.thr);
  int* cnt = reinterpret_cast<int*>(smem + L.cnt);
  volatile int* abort_sh = cnt + G * QB;
  float* cmt = reinterpret_cast<float*>(smem + L.cm);
  uint64_t* cand = reinterpret_cast<uint64_t*>(smem + L.cand);
  int* hist = reinterpret_cast<int*>(smem + L.hist);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.bars);  // [G][RS]
  uint64_t* empty = full + G * RS;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t t_begin = a.ntiles * blockIdx.x / gridDim.x;
  const int64_t t_end = a.ntiles * (blockIdx.x + 1) / gridDim.x;
  const bool ip = st.metric == LVQ_IP;
  const int M = st.n_means;
  const int cap = a.cap;

  if (threadIdx.x == 0) {
    for (int i = 0; i < G * RS; ++i) {
      mbar_init(full + i, 1);
      mbar_init(empty + i, 4);
    }
    *abort_sh = 0;
    fence_mbar_init();
  }
  for (int i = threadIdx.x; i < QB * 4 * a.Wp; i += kThreads) {
    const int q = i / (4 * a.Wp);
    qw[i] = q < a.nq ? a.qw[i] : 0u;
  }
  for (int i = threadIdx.x; i < QB * M; i += kThreads) {
    const int q = i / M;
    cmt[i] = q < a.nq ? a.p.cm[i] : 0.0f;
  }
  if (threadIdx.x < G * QB) {
    const int q = threadIdx.x % QB;
    thr[threadIdx.x] = kNoKey;
    cnt[threadIdx.x] = 0;
    if (threadIdx.x < QB) {
      const bool real = q < a.nq;
      fq[q] = make_float4(real ? a.p.qsum[q] : 0.0f, real ? a.qscale[q] : 0.0f, 0.0f, real ? a.p.qnorm[q] : 0.0f);
    }
  }
  __syncthreads();

  if (warp == 0) {
    // ------------------------------------------------------------- producer
    // Ring g carries the boxes of local tiles g, g + 2, ...; one thread keeps
    // both rings full, refilling whichever has a free stage.
    if (lane == 0) {
      prefetch_tmap(&cmap);
      int64_t next_t[G];
      int next_kb[G];
      uint32_t fills[G];
#pragma unroll
      for (int g = 0; g < G; ++g) {
        next_t[g] = t_begin + g;
        next_kb[g] = 0;
        fills[g] = 0u;
      }
      uint32_t idle = 0;
      while (!*abort_sh) {
        bool left = false, moved = false;
#pragma unroll
        for (int g = 0; g < G; ++g) {
          if (next_t[g] >= t_end) continue;
          left = true;
          const uint32_t ci = fills[g];
          const int s = g * RS + (int)(ci % RS);
          if (!mbar_test_wait(empty + s, ((ci / RS) & 1) ^ 1)) continue;
          mbar_expect_tx(full + s, kStageB);
#pragma unroll
          for (int pr = 0; pr < RPT; ++pr)
            tma_load_2d(ring + s * kStageB + pr * kStageBytes, &cmap, full + s, next_kb[g] * kBoxBytes,
                        (int)(next_t[g] * kTR + pr * kRows));
          fills[g] = ci + 1;
          if (++next_kb[g] == a.n_kbox) {
            next_kb[g] = 0;
            next_t[g] += G;
          }
          moved = true;
        }
        if (!left) break;
        if (moved) {
          idle = 0;
        } else if (++idle > kWaitLimit) {
          *abort_sh = 1;
          set_error(st.err, LVQ_ETIMEOUT);
          break;
        } else {
          __nanosleep(32);
        }
      }
      // let the copies still in flight land before the CTA can exit
      for (int g = 0; g < G; ++g)
        for (uint32_t j = 1; j <= (uint32_t)RS && j <= fills[g]; ++j) {
          const uint32_t k = fills[g] - j;
          mbar_wait(full + g * RS + k % RS, (k / RS) & 1, kWaitLimit);
        }
    }
  } else {
    // ------------------------------------------------------------ consumers
    const int cw = warp - 1;        // 0..7
    const int g = cw >> 2;          // group: local tiles g, g + G, ...
    const int wq = cw & 3;          // warp within the group
    const int row = wq * 32 + lane;
    const int sw = row & 7;  // 128-byte swizzle of the box: chunk c sits at c ^ sw
    uint64_t* my_thr = thr + g * QB;
    int* my_cnt = cnt + g * QB;
    uint32_t used = 0;              // boxes taken from this group's ring
    bool go = true;
    for (int64_t t = t_begin + g; t < t_end; t += G) {
      // the global bound as of this tile's start, read now and used after it
      uint64_t gt_tile = kNoKey;
      if (wq < QB && wq < a.nq && lane == 0) gt_tile = *reinterpret_cast<volatile uint64_t*>(a.gthr + wq);
      if (go) {
        // four independent accumulator chains per query: A/B halves (4-bit)
        // or even/odd words (8-bit), high and low query bytes
        int hi[RPT][QB][2];
        uint32_t lo[RPT][QB][2];
#pragma unroll
        for (int pr = 0; pr < RPT; ++pr)
#pragma unroll
          for (int q = 0; q < QB; ++q) {
            hi[pr][q][0] = hi[pr][q][1] = 0;
            lo[pr][q][0] = lo[pr][q][1] = 0u;
          }
        // per-row constants and the live bits, all loaded now and first used
        // after the boxes (no load waits on another)
        int64_t rw[RPT];
        bool in_range[RPT];
        uint32_t live_w[RPT];
        float lo_r[RPT], step_r[RPT], nrm[RPT];
        int m_r[RPT];
#pragma unroll
        for (int pr = 0; pr < RPT; ++pr) {
          rw[pr] = t * kTR + pr * kRows + row;
          in_range[pr] = rw[pr] < a.n_rows;
          const int64_t ms = in_range[pr] ? rw[pr] : 0;
          live_w[pr] = __ldg(st.live + (ms >> 5));
          lo_r[pr] = __ldg(st.lower + ms);
          step_r[pr] = __ldg(st.step + ms);
          m_r[pr] = __ldg(st.mean_id + ms);
          nrm[pr] = ip ? 0.0f : __ldg(st.norm2 + ms);
        }
        for (int kb = 0; kb < a.n_kbox; ++kb, ++used) {
          const int s = g * RS + (int)(used % RS);
          if (!mbar_wait(full + s, (used / RS) & 1, kWaitLimit)) {
            if (lane == 0) {
              *abort_sh = 1;
              set_error(st.err, LVQ_ETIMEOUT);
            }
            go = false;
            break;
          }
          uint4 w[RPT][kChunks];
#pragma unroll
          for (int pr = 0; pr < RPT; ++pr) {
            const uint4* src =
                reinterpret_cast<const uint4*>(ring + s * kStageB + pr * kStageBytes + row * kBoxBytes);
#pragma unroll
            for (int c = 0; c < kChunks; ++c) w[pr][c] = src[c ^ sw];
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(empty + s);
#pragma unroll
          for (int c = 0; c < kChunks; ++c) {
            const int word0 = kb * (kBoxBytes / 4) + c * 4;
#pragma unroll
            for (int q = 0; q < QB; ++q) {
              const uint32_t* qq = qw + q * 4 * a.Wp + word0;
              const uint4 ah = *reinterpret_cast<const uint4*>(qq);
              const uint4 al = *reinterpret_cast<const uint4*>(qq + 2 * a.Wp);
              const uint32_t ahs[4] = {ah.x, ah.y, ah.z, ah.w};
              const uint32_t als[4] = {al.x, al.y, al.z, al.w};
              if (BITS == 4) {
                const uint4 bh = *reinterpret_cast<const uint4*>(qq + a.Wp);
                const uint4 bl = *reinterpret_cast<const uint4*>(qq + 3 * a.Wp);
                const uint32_t bhs[4] = {bh.x, bh.y, bh.z, bh.w};
                const uint32_t bls[4] = {bl.x, bl.y, bl.z, bl.w};
#pragma unroll
                for (int pr = 0; pr < RPT; ++pr) {
                  const uint32_t ws[4] = {w[pr][c].x, w[pr][c].y, w[pr][c].z, w[pr][c].w};
#pragma unroll
                  for (int i = 0; i < 4; ++i) {
                    const uint32_t A = ws[i] & 0x0F0F0F0Fu;
                    const uint32_t B = (ws[i] >> 4) & 0x0F0F0F0Fu;
                    hi[pr][q][0] = dp4a_us(A, ahs[i], hi[pr][q][0]);
                    hi[pr][q][1] = dp4a_us(B, bhs[i], hi[pr][q][1]);
                    lo[pr][q][0] = dp4a_uu(A, als[i], lo[pr][q][0]);
                    lo[pr][q][1] = dp4a_uu(B, bls[i], lo[pr][q][1]);
                  }
                }
              } else {
#pragma unroll
                for (int pr = 0; pr < RPT; ++pr) {
                  const uint32_t ws[4] = {w[pr][c].x, w[pr][c].y, w[pr][c].z, w[pr][c].w};
#pragma unroll
                  for (int i = 0; i < 4; ++i) {
                    hi[pr][q][i & 1] = dp4a_us(ws[i], ahs[i], hi[pr][q][i & 1]);
                    lo[pr][q][i & 1] = dp4a_uu(ws[i], als[i], lo[pr][q][i & 1]);
                  }
                }
              }
            }
          }
        }
#pragma unroll
        for (int pr = 0; pr < RPT; ++pr) {
          const bool valid = in_range[pr] && ((live_w[pr] >> (rw[pr] & 31)) & 1u);
          if (go && valid) {
#pragma unroll
            for (int q = 0; q < QB; ++q) {
              if (q < a.nq) {
                const float4 f = fq[q];
                const float h = (float)(hi[pr][q][0] + hi[pr][q][1]);
                const float l = (float)lo[pr][q][0] + (float)lo[pr][q][1];
                const float dot = f.y * __fmaf_rn(256.0f, h, l);
                float sc = __fmaf_rn(step_r[pr], dot, __fmaf_rn(lo_r[pr], f.x, cmt[q * M + m_r[pr]]));
                if (!ip) sc = f.w + nrm[pr] - 2.0f * sc;
                const uint64_t key = make_key(sc, (uint32_t)rw[pr], st.metric);
                // every group's threshold bounds the CTA's k1-th best
                uint64_t tq = thr[q];
#pragma unroll
                for (int h = 1; h < G; ++h) tq = thr[h * QB + q] < tq ? thr[h * QB + q] : tq;
                if (key < tq) cand[(q * G + g) * cap + atomicAdd(&my_cnt[q], 1)] = key;
              }
            }
          }
        }
      }
      named_bar(1 + g, 128);
      go = go && !*abort_sh;
      if (wq < QB && wq < a.nq) {
        // a buffer without room for another tile is cut to the k1 best, whose
        // k1-th key bounds every CTA's search
        if (my_cnt[wq] > cap - kTR) {
          uint64_t tk;
          const int kept = select_k(cand + (wq * G + g) * cap, my_cnt[wq], a.k1, hist + cw * 64, &tk);
          if (lane == 0) {
            my_cnt[wq] = kept;
            if (tk < my_thr[wq]) my_thr[wq] = tk;
            if (tk != kNoKey) atomicMin(reinterpret_cast<unsigned long long*>(a.gthr + wq), tk);
          }
          __syncwarp();
        }
        if (lane == 0 && gt_tile < my_thr[wq]) my_thr[wq] = gt_tile;
        __syncwarp();
      }
      named_bar(1 + g, 128);
    }
    named_bar(1 + G, 4 * G * 32);
    // the CTA's k1 best of each query: the other groups' keys moved behind
    // group 0's (each move only writes below the next buffer's start)
    if (cw < QB && cw < a.nq) {
      const int q = cw;
      uint64_t* b0 = cand + (q * G) * cap;
      int n = cnt[q];
      for (int h = 1; h < G; ++h) {
        const int nh = cnt[h * QB + q];
        for (int base = 0; base < nh; base += 32) {
          const uint64_t v = base + lane < nh ? b0[h * cap + base + lane] : 0ull;
          __syncwarp();
          if (base + lane < nh) b0[n + base + lane] = v;
          __syncwarp();
        }
        n += nh;
      }
      uint64_t tk;
      const int kept = select_k(b0, n, a.k1, hist + cw * 64, &tk);
      if (lane == 0 && kept == a.k1) atomicMin(reinterpret_cast<unsigned long long*>(a.gthr + q), tk);
      __syncwarp();
      // only keys at or below the global bound can be among the k1 best
      const uint64_t gt = *reinterpret_cast<volatile uint64_t*>(a.gthr + q);
      uint64_t* dst = a.partial + ((int64_t)q * gridDim.x + blockIdx.x) * a.k1;
      int pos = 0;
      for (int base = 0; base < kept; base += 32) {
        const uint64_t v = base + lane < kept ? b0[base + lane] : kNoKey;
        const bool keep = base + lane < kept && v <= gt;
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (keep) dst[pos + __popc(m & ((1u << lane) - 1u))] = v;
        pos += __popc(m);
      }
      if (lane == 0) a.counts[(int64_t)q * gridDim.x + blockIdx.x] = pos;
    }
  }
}

// Rounds each query to 16-bit integers and lays its bytes out in code-word
// order (one warp per query).
__global__ void __launch_bounds__(256) small_prep_kernel(DeviceStore st, const float* __restrict__ q, int64_t nq,
                                                         int Wp, uint32_t* __restrict__ qw,
                                                         float* __restrict__ qscale, uint64_t* __restrict__ gthr) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= nq) return;
  const int d = st.d;
  const float* qi = q + i * d;
  float mx = 0.0f;
  for (int j = lane; j < d; j += 32) mx = fmaxf(mx, fabsf(qi[j]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const float s = mx > 0.0f ? mx / 32767.0f : 1.0f;
  const float inv = mx > 0.0f ? 32767.0f / mx : 0.0f;
  if (lane == 0) {
    qscale[i] = s;
    gthr[i] = kNoKey;
  }
  uint32_t* out = qw + i * 4 * Wp;
  auto qint = [&](int j) -> int {
    return j < d ? max(-32767, min(32767, __float2int_rn(qi[j] * inv))) : 0;
  };
  for (int w = lane; w < Wp; w += 32) {
    uint32_t ah = 0, bh = 0, al = 0, bl = 0;
    if (st.bits1 == 4) {
      const int oa[4] = {0, 4, 1, 5}, ob[4] = {2, 6, 3, 7};
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int va = qint(8 * w + oa[b]), vb = qint(8 * w + ob[b]);
        ah |= (uint32_t)((va >> 8) & 255) << (8 * b);
        al |= (uint32_t)(va & 255) << (8 * b);
        bh |= (uint32_t)((vb >> 8) & 255) << (8 * b);
        bl |= (uint32_t)(vb & 255) << (8 * b);
      }
    } else {
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int va = qint(4 * w + b);
        ah |= (uint32_t)((va >> 8) & 255) << (8 * b);
        al |= (uint32_t)(va & 255) << (8 * b);
      }
    }
    out[w] = ah;
    out[Wp + w] = bh;
    out[2 * Wp + w] = al;
    out[3 * Wp + w] = bl;
  }
}

template <int QB, int BITS, int G, int RPT>
cudaError_t launch_qb(const CUtensorMap& cm, const SmallArgs& a, int grid, size_t smem, cudaStream_t stream) {
  static std::atomic<uint64_t> attr{0};
  const cudaError_t e = max_dyn_smem_once((const void*)scan_small_kernel<QB, BITS, G, RPT>, kSmemLimit, attr);
  if (e != cudaSuccess) return e;
  scan_small_kernel<QB, BITS, G, RPT><<<grid, small_threads(G), smem, stream>>>(cm, a);
  return cudaGetLastError();
}

// a buffer is cut when it may not take another tile (more than cap - tile
// rows keys), so k1 kept keys and one tile of new ones always fit
int small_cap(int k1, int rpt) { return pow2_at_least(k1 + kRows * rpt); }
int small_wp(const DeviceStore& st) { return (int)ceil_div(st.row1, kBoxBytes) * (kBoxBytes / 4); }
int small_qb(int64_t nq) { return nq <= 1 ? 1 : nq <= 2 ? 2 : nq <= 3 ? 3 : 4; }
// consumer groups: more warps hide more load latency, while the registers of
// more queries allow fewer of them (4, 3 and 2 groups for 1, 2 and 3-4 slots)
int small_groups(int qb, int rpt) { return qb <= 1 ? 4 : qb <= 2 ? 3 : 2; }

// ring stages per ring: as many as shared memory holds, up to kMaxRingStages;
// 0 when not even two fit
int small_stages(const DeviceStore& st, int qb, int k1, int rpt) {
  const int G = small_groups(qb, rpt);
  for (int rs = kMaxRingStages; rs >= 2; --rs)
    if (small_layout(qb, G, small_wp(st), st.n_means, small_cap(k1, rpt), rs, rpt).total + 1024 <= kSmemLimit)
      return rs;
  return 0;
}

// rows per consumer thread: with one query each code word meets one query
// word either way; with more, two rows per thread halve the query words read
// from shared memory per row (when the larger buffers and stages fit)
int small_rpt(const DeviceStore& st, int64_t nq, int k1) {
  const int qb = small_qb(nq);
  return qb >= 2 && small_stages(st, qb, k1, 2) > 0 ? 2 : 1;
}

}  // namespace

bool small_supported(const DeviceStore& st, int64_t nq, int k1) {
  if (nq < 1 || nq > kSmallMaxQ || k1 < 1 || k1 > 1024) return false;
  if (st.bits1 != 4 && st.bits1 != 8) return false;
  if (!mma_supported(st)) return false;  // needs the CUDA driver's tensor-map encoder too
  return small_stages(st, small_qb(nq), k1, small_rpt(st, nq, k1)) > 0;
}

// scratch: rounded queries [nq][4][Wp] u32 | scales [nq] f32 | global bounds [nq] u64 (8-byte aligned)
size_t small_scratch_bytes(const DeviceStore& st, int64_t nq) {
  return (size_t)nq * 4 * small_wp(st) * 4 + (size_t)nq * 8 + (size_t)nq * 8 + 256;
}
static uint64_t* small_gthr(void* scratch, const DeviceStore& st, int64_t nq) {
  const size_t off = (size_t)nq * 4 * small_wp(st) * 4 + (size_t)nq * 8;
  return reinterpret_cast<uint64_t*>(static_cast<char*>(scratch) + off);
}

int small_grid(const DeviceStore& st, int64_t n_rows, int64_t nq, int k1, int sm_count) {
  const int64_t ntiles = ceil_div(n_rows > 0 ? n_rows : 1, (int64_t)kRows * small_rpt(st, nq, k1));
  return (int)(ntiles < sm_count ? ntiles : sm_count);
}

cudaError_t launch_small_prep(const DeviceStore& st, const float* q, int64_t nq, void* scratch, cudaStream_t stream) {
  if (nq <= 0) return cudaSuccess;
  const int Wp = small_wp(st);
  uint32_t* qw = reinterpret_cast<uint32_t*>(scratch);
  float* qscale = reinterpret_cast<float*>(qw + nq * 4 * Wp);
  small_prep_kernel<<<(unsigned)ceil_div(nq, 8), 256, 0, stream>>>(st, q, nq, Wp, qw, qscale,
                                                                     small_gthr(scratch, st, nq));
  return cudaGetLastError();
}

cudaError_t launch_scan_small(const DeviceStore& st, int64_t nq, const QueryPrep& p, const void* scratch,
                              const ScanPlan& plan, cudaStream_t stream) {
  if (nq <= 0) return cudaSuccess;
  if (nq > kSmallMaxQ || plan.splits != plan.grid) return cudaErrorInvalidValue;
  SmallArgs a;
  a.st = st;
  a.nq = nq;
  a.p = p;
  a.Wp = small_wp(st);
  const uint32_t* qw = reinterpret_cast<const uint32_t*>(scratch);
  a.qw = qw;
  a.qscale = reinterpret_cast<const float*>(qw + nq * 4 * a.Wp);
  a.n_kbox = (int)ceil_div(st.row1, kBoxBytes);
  a.k1 = plan.k1;
  const int qb = small_qb(nq), rpt = small_rpt(st, nq, plan.k1);
  a.cap = small_cap(plan.k1, rpt);
  a.n_rows = plan.n_rows;
  a.ntiles = ceil_div(plan.n_rows > 0 ? plan.n_rows : 1, (int64_t)kRows * rpt);
  a.partial = plan.partial;
  a.counts = plan.counts;
  a.gthr = small_gthr(const_cast<void*>(scratch), st, nq);
  if (!a.counts) return cudaErrorInvalidValue;
  a.stages = small_stages(st, qb, plan.k1, rpt);
  if (a.stages == 0) return cudaErrorInvalidValue;
  CUtensorMap cm;
  cudaError_t e = encode_code_map(st, &cm, kBoxBytes);
  if (e != cudaSuccess) return e;
  const size_t smem =
      (size_t)small_layout(qb, small_groups(qb, rpt), a.Wp, st.n_means, a.cap, a.stages, rpt).total + 1024;
  const int grid = plan.grid;
  const bool b4 = st.bits1 == 4;
  switch (qb) {
    case 1:
      return b4 ? launch_qb<1, 4, 4, 1>(cm, a, grid, smem, stream) : launch_qb<1, 8, 4, 1>(cm, a, grid, smem, stream);
    case 2:
      if (rpt == 2)
        return b4 ? launch_qb<2, 4, 3, 2>(cm, a, grid, smem, stream) : launch_qb<2, 8, 3, 2>(cm, a, grid, smem, stream);
      return b4 ? launch_qb<2, 4, 3, 1>(cm, a, grid, smem, stream) : launch_qb<2, 8, 3, 1>(cm, a, grid, smem, stream);
    case 3:
      if (rpt == 2)
        return b4 ? launch_qb<3, 4, 2, 2>(cm, a, grid, smem, stream) : launch_qb<3, 8, 2, 2>(cm, a, grid, smem, stream);
      return b4 ? launch_qb<3, 4, 2, 1>(cm, a, grid, smem, stream) : launch_qb<3, 8, 2, 1>(cm, a, grid, smem, stream);
    default:
      if (rpt == 2)
        return b4 ? launch_qb<4, 4, 2, 2>(cm, a, grid, smem, stream) : launch_qb<4, 8, 2, 2>(cm, a, grid, smem, stream);
      return b4 ? launch_qb<4, 4, 2, 1>(cm, a, grid, smem, stream) : launch_qb<4, 8, 2, 1>(cm, a, grid, smem, stream);
  }
}

}  // namespace lvq
