// Top-k selection on 64-bit (score, id) keys.
//
// The scans and merges keep, per query, a "candidate buffer": keys better
// than a running threshold are appended; when the buffer may overflow, one
// warp finds the k-th smallest key by a most-significant-digit radix select
// (8-bit digits, a 256-bin histogram in shared memory), keeps the keys not
// above it and makes it the new threshold.  Final lists are sorted by a
// bitonic sort in shared memory.
#pragma once

#include "lvq_internal.cuh"

namespace lvq {

constexpr unsigned kFull = 0xffffffffu;

__host__ __device__ inline int pow2_at_least(int v) {
  int p = 32;
  while (p < v) p <<= 1;
  return p;
}

// Radix select on keys held in registers: key i of the warp's n keys is
// v[i / 32] of lane i % 32 (E registers per lane, n <= 32 * E; entries at
// or beyond n hold kNoKey and are never counted).  Returns the k-th smallest
// (1-based, 1 <= k <= n) of the n distinct keys, using 8-bit digits from the
// most significant one and a 256-bin histogram in shared memory.  hist: 288
// ints owned by the warp; bin b lives at b + b/8 so that lane l reading its
// bins 8l..8l+7 touches banks 9l..9l+7 (mod 32): no bank conflicts.
template <int E>
__device__ __forceinline__ uint64_t warp_kth_regs(const uint64_t (&v)[E], int n, int k, int* hist) {
  const int lane = threadIdx.x & 31;
  uint64_t prefix = 0, mask = 0;
  for (int shift = 56; shift >= 0; shift -= 8) {
    for (int i = lane; i < 288; i += 32) hist[i] = 0;
    __syncwarp();
#pragma unroll
    for (int e = 0; e < E; ++e) {
      if (e * 32 + lane < n && (v[e] & mask) == prefix) {
        const int b = (int)((v[e] >> shift) & 255u);
        atomicAdd(&hist[b + (b >> 3)], 1);
      }
    }
    __syncwarp();
    int c[8], s = 0;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      c[e] = hist[lane * 9 + e];
      s += c[e];
    }
    int incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    const int excl = incl - s;
    const bool mine = excl < k && k <= incl;
    const int src = __ffs(__ballot_sync(kFull, mine)) - 1;
    int bin = 0, before = 0, inbin = 0;
    if (mine) {
      int run = excl;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        if (run < k && k <= run + c[e] && inbin == 0) {
          bin = lane * 8 + e;
          before = run;
          inbin = c[e];
        }
        run += c[e];
      }
    }
    bin = __shfl_sync(kFull, bin, src);
    before = __shfl_sync(kFull, before, src);
    inbin = __shfl_sync(kFull, inbin, src);
    k -= before;
    prefix |= (uint64_t)bin << shift;
    mask |= 255ull << shift;
    __syncwarp();
    if (inbin == 1) {
      // a single key carries this prefix: it is the answer
      uint64_t r = 0;
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (e * 32 + lane < n && (v[e] & mask) == prefix) r = v[e];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const uint64_t y = __shfl_xor_sync(kFull, r, o);
        r = r > y ? r : y;
      }
      return (r & mask) == prefix ? r : prefix;
    }
  }
  return prefix;
}

__device__ __forceinline__ uint64_t warp_min64(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t y = __shfl_xor_sync(kFull, v, o);
    v = v < y ? v : y;
  }
  return v;
}
__device__ __forceinline__ uint64_t warp_max64(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t y = __shfl_xor_sync(kFull, v, o);
    v = v > y ? v : y;
  }
  return v;
}

// The same select with 6-bit digits (64 bins: hist of 64 ints, lane l owning
// bins 2l and 2l+1), for kernels short of shared memory.  The bits that all
// keys share (the common prefix of the smallest and the largest) are skipped,
// and lanes that fall in the same bin add to it once (warp-aggregated), so
// keys with close scores do not serialise on one shared-memory counter.
template <int E>
__device__ __forceinline__ uint64_t warp_kth_regs6(const uint64_t (&v)[E], int n, int k, int* hist) {
  const int lane = threadIdx.x & 31;
  uint64_t lo = kNoKey, hi = 0;
#pragma unroll
  for (int e = 0; e < E; ++e)
    if (e * 32 + lane < n) {
      lo = v[e] < lo ? v[e] : lo;
      hi = v[e] > hi ? v[e] : hi;
    }
  lo = warp_min64(lo);
  hi = warp_max64(hi);
  if (lo == hi) return lo;
  const int top = 63 - __clzll((long long)(lo ^ hi));  // highest bit where keys differ
  uint64_t mask = top == 63 ? 0ull : ~((2ull << top) - 1ull);
  uint64_t prefix = lo & mask;
  for (int low = top - 5; low > -6; low -= 6) {
    const int sh = low > 0 ? low : 0;
    const int width = low >= 0 ? 6 : 6 + low;
    const uint64_t dmask = (1ull << width) - 1ull;
    hist[lane] = 0;
    hist[lane + 32] = 0;
    __syncwarp();
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const bool in = e * 32 + lane < n && (v[e] & mask) == prefix;
      const int b = in ? (int)((v[e] >> sh) & dmask) : 64 + lane;  // lanes out get distinct dummies
      const unsigned same = __match_any_sync(kFull, b);
      if (in && (__ffs(same) - 1) == lane) atomicAdd(&hist[b], __popc(same));
    }
    __syncwarp();
    const int c0 = hist[2 * lane], c1 = hist[2 * lane + 1];
    const int s = c0 + c1;
    int incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    const int excl = incl - s;
    const bool mine = excl < k && k <= incl;
    const int src = __ffs(__ballot_sync(kFull, mine)) - 1;
    int bin = 0, before = 0, inbin = 0;
    if (mine) {
      if (k <= excl + c0) {
        bin = 2 * lane;
        before = excl;
        inbin = c0;
      } else {
        bin = 2 * lane + 1;
        before = excl + c0;
        inbin = c1;
      }
    }
    bin = __shfl_sync(kFull, bin, src);
    before = __shfl_sync(kFull, before, src);
    inbin = __shfl_sync(kFull, inbin, src);
    k -= before;
    prefix |= (uint64_t)bin << sh;
    mask |= dmask << sh;
    __syncwarp();
    if (inbin == 1) {
      uint64_t r = 0;
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (e * 32 + lane < n && (v[e] & mask) == prefix) r = v[e];
      return warp_max64(r) | prefix;
    }
  }
  return prefix;
}

// Keep the k smallest of the n distinct keys buf[0..n) at buf[0..kept),
// unsorted; returns kept = min(n, k) and sets *thr to the k-th smallest key
// when n >= k (else kNoKey).  One whole warp; n <= 32 * E.
template <int E>
__device__ __forceinline__ int warp_select_e(uint64_t* buf, int n, int k, int* hist, uint64_t* thr) {
  const int lane = threadIdx.x & 31;
  uint64_t v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) v[e] = e * 32 + lane < n ? buf[e * 32 + lane] : kNoKey;
  if (n <= k) {
    *thr = (n == k && k > 0) ? warp_kth_regs<E>(v, n, k, hist) : kNoKey;
    __syncwarp();
    return n;
  }
  const uint64_t t = warp_kth_regs<E>(v, n, k, hist);
  int pos = 0;
  __syncwarp();
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const bool keep = e * 32 + lane < n && v[e] <= t;
    const unsigned bal = __ballot_sync(kFull, keep);
    if (keep) buf[pos + __popc(bal & ((1u << lane) - 1u))] = v[e];
    pos += __popc(bal);
  }
  __syncwarp();
  *thr = t;
  return pos;
}

// k-th smallest of the n distinct keys buf[0..n) by the same radix select,
// reading the keys from memory on every pass (no registers held; for large
// buffers in register-bound kernels).
__device__ __forceinline__ uint64_t warp_kth_mem(const uint64_t* buf, int n, int k, int* hist) {
  const int lane = threadIdx.x & 31;
  uint64_t prefix = 0, mask = 0;
  for (int shift = 56; shift >= 0; shift -= 8) {
    for (int i = lane; i < 288; i += 32) hist[i] = 0;
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
      const uint64_t key = buf[i];
      if ((key & mask) == prefix) {
        const int b = (int)((key >> shift) & 255u);
        atomicAdd(&hist[b + (b >> 3)], 1);
      }
    }
    __syncwarp();
    int c[8], s = 0;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      c[e] = hist[lane * 9 + e];
      s += c[e];
    }
    int incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    const int excl = incl - s;
    const bool mine = excl < k && k <= incl;
    const int src = __ffs(__ballot_sync(kFull, mine)) - 1;
    int bin = 0, before = 0;
    if (mine) {
      int run = excl;
      bool found = false;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        if (!found && run < k && k <= run + c[e]) {
          bin = lane * 8 + e;
          before = run;
          found = true;
        }
        run += c[e];
      }
    }
    bin = __shfl_sync(kFull, bin, src);
    before = __shfl_sync(kFull, before, src);
    k -= before;
    prefix |= (uint64_t)bin << shift;
    mask |= 255ull << shift;
    __syncwarp();
  }
  return prefix;
}

__device__ __forceinline__ int warp_select_mem(uint64_t* buf, int n, int k, int* hist, uint64_t* thr) {
  const int lane = threadIdx.x & 31;
  if (n <= k) {
    *thr = (n == k && k > 0) ? warp_kth_mem(buf, n, k, hist) : kNoKey;
    __syncwarp();
    return n;
  }
  const uint64_t t = warp_kth_mem(buf, n, k, hist);
  int pos = 0;
  for (int base = 0; base < n; base += 32) {
    const int i = base + lane;
    const uint64_t key = i < n ? buf[i] : kNoKey;
    const bool keep = i < n && key <= t;
    const unsigned bal = __ballot_sync(kFull, keep);
    __syncwarp();
    if (keep) buf[pos + __popc(bal & ((1u << lane) - 1u))] = key;
    pos += __popc(bal);
    __syncwarp();
  }
  *thr = t;
  return pos;
}

// Up to 512 keys in registers, more from memory (for register-bound kernels).
__device__ __forceinline__ int warp_select_small(uint64_t* buf, int n, int k, int* hist, uint64_t* thr) {
  if (n <= 256) return warp_select_e<8>(buf, n, k, hist, thr);
  if (n <= 512) return warp_select_e<16>(buf, n, k, hist, thr);
  return warp_select_mem(buf, n, k, hist, thr);
}

// As warp_select_e with 6-bit digits (hist: 64 ints).
template <int E>
__device__ __forceinline__ int warp_select_e6(uint64_t* buf, int n, int k, int* hist, uint64_t* thr) {
  const int lane = threadIdx.x & 31;
  uint64_t v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) v[e] = e * 32 + lane < n ? buf[e * 32 + lane] : kNoKey;
  if (n <= k) {
    *thr = (n == k && k > 0) ? warp_kth_regs6<E>(v, n, k, hist) : kNoKey;
    __syncwarp();
    return n;
  }
  const uint64_t t = warp_kth_regs6<E>(v, n, k, hist);
  int pos = 0;
  __syncwarp();
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const bool keep = e * 32 + lane < n && v[e] <= t;
    const unsigned bal = __ballot_sync(kFull, keep);
    if (keep) buf[pos + __popc(bal & ((1u << lane) - 1u))] = v[e];
    pos += __popc(bal);
  }
  __syncwarp();
  *thr = t;
  return pos;
}

// Ascending bitonic sort of one key per lane across the warp.
__device__ __forceinline__ uint64_t warp_sort32(uint64_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const uint64_t o = __shfl_xor_sync(kFull, v, j);
      const bool up = (lane & k) == 0;
      const bool lower = (lane & j) == 0;
      v = (up == lower) ? (v < o ? v : o) : (v < o ? o : v);
    }
  }
  return v;
}

// Forward declaration (defined below): exact select of keys in memory.
__device__ __forceinline__ int warp_select_mem6(uint64_t* buf, int n, int k, int* hist, uint64_t* thr);

// Approximate pruning of a candidate buffer of n distinct keys: find a
// threshold T among 32 sampled keys such that between k and keep_max keys
// are below T, keep those (unsorted) and return their number; *thr = T, a
// valid insertion threshold (at least k kept keys beat it).  Falls back to
// the exact select when no sampled key qualifies.  Up to 512 keys are held
// in registers; a larger buffer (k1 above 128 gives buffers of 1024) is cut
// exactly to its k best from memory.  hist: 64 ints.
__device__ __forceinline__ int warp_prune(uint64_t* buf, int n, int k, int keep_max, int* hist, uint64_t* thr) {
  const int lane = threadIdx.x & 31;
  if (n <= keep_max) {
    *thr = kNoKey;
    return -1;  // nothing to do
  }
  if (n > 512) return warp_select_mem6(buf, n, k, hist, thr);
  uint64_t v[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) v[e] = e * 32 + lane < n ? buf[e * 32 + lane] : kNoKey;
  // sample: lane l takes key l * n / 32 (spread over the buffer)
  const int si = (lane * n) >> 5;
  uint64_t smp = kNoKey;
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    const uint64_t x = __shfl_sync(kFull, v[e], si & 31);
    if (e == (si >> 5)) smp = x;
  }
  smp = warp_sort32(smp);
  // count of keys below sample j, by binary search on j
  auto count_below = [&](uint64_t t) {
    int c = 0;
#pragma unroll
    for (int e = 0; e < 16; ++e) c += __popc(__ballot_sync(kFull, e * 32 + lane < n && v[e] < t));
    return c;
  };
  int lo_j = 0, hi_j = 31;
  uint64_t t = kNoKey;
  bool found = false;
  for (int it = 0; it < 6 && lo_j <= hi_j; ++it) {
    const int mid = (lo_j + hi_j) >> 1;
    const uint64_t tm = __shfl_sync(kFull, smp, mid);
    const int c = count_below(tm);
    if (c < k) lo_j = mid + 1;
    else if (c > keep_max) hi_j = mid - 1;
    else {
      t = tm;
      found = true;
      break;
    }
  }
  if (!found) {
    // exact k-th smallest; keep the k best
    t = warp_kth_regs6<16>(v, n, k, hist);
    int pos = 0;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const bool keep = e * 32 + lane < n && v[e] <= t;
      const unsigned bal = __ballot_sync(kFull, keep);
      if (keep) buf[pos + __popc(bal & ((1u << lane) - 1u))] = v[e];
      pos += __popc(bal);
    }
    __syncwarp();
    *thr = t;
    return pos;
  }
  int pos = 0;
  __syncwarp();
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    const bool keep = e * 32 + lane < n && v[e] < t;
    const unsigned bal = __ballot_sync(kFull, keep);
    if (keep) buf[pos + __popc(bal & ((1u << lane) - 1u))] = v[e];
    pos += __popc(bal);
  }
  __syncwarp();
  *thr = t;
  return pos;
}

// warp_select6 for keys in shared memory (any n): 6-bit digits from the
// highest bit where the keys differ, histogram increments aggregated over
// lanes holding the same digit, stop once the k-th key's bin holds one key.
__device__ __forceinline__ int warp_select_mem6(uint64_t* buf, int n, int k, int* hist, uint64_t* thr) {
  const int lane = threadIdx.x & 31;
  if (n <= k) {
    uint64_t t = kNoKey;
    if (n == k && k > 0) {
      uint64_t m = 0;
      for (int i = lane; i < n; i += 32) m = buf[i] > m ? buf[i] : m;
      t = warp_max64(m);
    }
    *thr = t;
    __syncwarp();
    return n;
  }
  uint64_t lo = kNoKey, hi = 0;
  for (int i = lane; i < n; i += 32) {
    const uint64_t key = buf[i];
    lo = key < lo ? key : lo;
    hi = key > hi ? key : hi;
  }
  lo = warp_min64(lo);
  hi = warp_max64(hi);
  uint64_t t = lo;
  if (lo != hi) {
    const int top = 63 - __clzll((long long)(lo ^ hi));
    uint64_t mask = top == 63 ? 0ull : ~((2ull << top) - 1ull);
    uint64_t prefix = lo & mask;
    int kk = k;
    bool done = false;
    for (int low = top - 5; low > -6 && !done; low -= 6) {
      const int sh = low > 0 ? low : 0;
      const int width = low >= 0 ? 6 : 6 + low;
      const uint64_t dmask = (1ull << width) - 1ull;
      hist[lane] = 0;
      hist[lane + 32] = 0;
      __syncwarp();
      const int rounds = (n + 31) >> 5;
      for (int r = 0; r < rounds; ++r) {
        const int i = r * 32 + lane;
        const uint64_t key = i < n ? buf[i] : 0ull;
        const bool in = i < n && (key & mask) == prefix;
        const int b = in ? (int)((key >> sh) & dmask) : 64 + lane;
        const unsigned same = __match_any_sync(kFull, b);
        if (in && (__ffs(same) - 1) == lane) atomicAdd(&hist[b], __popc(same));
      }
      __syncwarp();
      const int c0 = hist[2 * lane], c1 = hist[2 * lane + 1];
      const int sum = c0 + c1;
      int incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      const int excl = incl - sum;
      const bool mine = excl < kk && kk <= incl;
      const int src = __ffs(__ballot_sync(kFull, mine)) - 1;
      int bin = 0, before = 0, inbin = 0;
      if (mine) {
        if (kk <= excl + c0) {
          bin = 2 * lane;
          before = excl;
          inbin = c0;
        } else {
          bin = 2 * lane + 1;
          before = excl + c0;
          inbin = c1;
        }
      }
      bin = __shfl_sync(kFull, bin, src);
      before = __shfl_sync(kFull, before, src);
      inbin = __shfl_sync(kFull, inbin, src);
      kk -= before;
      prefix |= (uint64_t)bin << sh;
      mask |= dmask << sh;
      __syncwarp();
      if (inbin == 1) {
        // the k-th key is the only one left under the prefix
        uint64_t m = 0;
        for (int i = lane; i < n; i += 32) {
          const uint64_t key = buf[i];
          if ((key & mask) == prefix) m = key;
        }
        prefix = warp_max64(m) | prefix;
        done = true;
      }
    }
    t = prefix;
  }
  int pos = 0;
  for (int base = 0; base < n; base += 32) {
    const int i = base + lane;
    const uint64_t key = i < n ? buf[i] : kNoKey;
    const bool keep = i < n && key <= t;
    const unsigned bal = __ballot_sync(kFull, keep);
    __syncwarp();
    if (keep) buf[pos + __popc(bal & ((1u << lane) - 1u))] = key;
    pos += __popc(bal);
    __syncwarp();
  }
  *thr = t;
  return pos;
}

// 6-bit-digit select (hist: 64 ints): up to 512 keys in registers, more
// from memory.
__device__ __forceinline__ int warp_select6(uint64_t* buf, int n, int k, int* hist, uint64_t* thr) {
  if (n <= 256) return warp_select_e6<8>(buf, n, k, hist, thr);
  if (n <= 512) return warp_select_e6<16>(buf, n, k, hist, thr);
  return warp_select_mem6(buf, n, k, hist, thr);
}

// Runtime dispatch on the number of keys (held in registers); n <= 1024.
__device__ __forceinline__ int warp_select(uint64_t* buf, int n, int k, int* hist, uint64_t* thr) {
  if (n <= 256) return warp_select_e<8>(buf, n, k, hist, thr);
  if (n <= 512) return warp_select_e<16>(buf, n, k, hist, thr);
  return warp_select_e<32>(buf, n, k, hist, thr);
}

// Ascending bitonic sort of keys[0..n) in shared memory, n a power of two;
// called by all threads of the block.
__device__ __forceinline__ void block_sort(uint64_t* keys, int n) {
  for (int k = 2; k <= n; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      __syncthreads();
      for (int t = threadIdx.x; t < (n >> 1); t += blockDim.x) {
        const int i = 2 * t - (t & (j - 1));  // lower index of the pair
        const int p = i + j;
        const bool up = (i & k) == 0;
        const uint64_t a = keys[i], b = keys[p];
        if ((a > b) == up) {
          keys[i] = b;
          keys[p] = a;
        }
      }
    }
  }
  __syncthreads();
}

__device__ __forceinline__ int block_exclusive_scan(int v, int* sh, int& total) {
  // sh: blockDim/32 ints of shared memory
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int s = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, s, o);
      if (lane >= o) s += y;
    }
    if (lane < (int)(blockDim.x >> 5)) sh[lane] = s;
  }
  __syncthreads();
  const int before = (wid ? sh[wid - 1] : 0) + x - v;
  total = sh[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before;
}

// Cut buf[0..n) (n <= cap, cap a power of two) to its k best distinct keys,
// sorted, in place; returns how many were kept and sets *thr to the k-th key
// (kNoKey if fewer than k).  Called by all threads; sh: blockDim/32 + 1 ints.
// Each chunk of the sorted keys is read before any survivor of it is written
// (survivors only move down), so the compaction needs no second buffer.
__device__ __forceinline__ int block_select_dedupe(uint64_t* buf, int cap, int n, int k, int* sh, uint64_t* thr) {
  for (int i = n + threadIdx.x; i < cap; i += blockDim.x) buf[i] = kNoKey;
  block_sort(buf, cap);
  int written = 0;
  uint64_t prev_last = kNoKey;  // the previous chunk's last key, read before it was overwritten
  for (int base = 0; base < cap && written < k; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const uint64_t key = i < cap ? buf[i] : kNoKey;
    const uint64_t prev = threadIdx.x == 0 ? prev_last : (i < cap ? buf[i - 1] : kNoKey);
    const uint64_t last = buf[(base + (int)blockDim.x < cap ? base + (int)blockDim.x : cap) - 1];
    const bool keep = i < cap && key != kNoKey && key != prev;
    prev_last = last;
    int total;
    const int pos = written + block_exclusive_scan(keep ? 1 : 0, sh, total);  // ends with a barrier
    if (keep && pos < k) buf[pos] = key;
    written += total;
    __syncthreads();
  }
  const int kept = written < k ? written : k;
  *thr = (kept == k && k > 0) ? buf[k - 1] : kNoKey;
  __syncthreads();
  return kept;
}

// Write the k best of the sorted keys[0..n) (repeats skipped) as (id, score),
// padding with (-1, +/-inf).  Called by all threads of the block; sh_pos:
// k + 1 ints of shared memory.
__device__ __forceinline__ void write_results(const uint64_t* keys, int n, int k, int metric, int64_t* out_ids,
                                              float* out_scores, int* sh_pos) {
  // one warp finds the positions of the first k distinct keys (repeats are
  // adjacent in sorted order), 32 keys per step
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    int w = 0;
    bool done = false;
    for (int base = 0; base < n && !done && w < k; base += 32) {
      const int i = base + lane;
      const uint64_t key = i < n ? keys[i] : kNoKey;
      const bool keep = i < n && key != kNoKey && (i == 0 || key != keys[i - 1]);
      const unsigned bal = __ballot_sync(kFull, keep);
      const int pos = w + __popc(bal & ((1u << lane) - 1u));
      if (keep && pos < k) sh_pos[pos] = i;
      w += __popc(bal);
      done = __any_sync(kFull, i < n && key == kNoKey);
    }
    if (lane == 0) sh_pos[k] = w < k ? w : k;
  }
  __syncthreads();
  const int w = sh_pos[k];
  const float pad = metric == LVQ_IP ? __int_as_float(0xff800000) : __int_as_float(0x7f800000);
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    if (i < w) {
      const uint64_t key = keys[sh_pos[i]];
      out_ids[i] = (int64_t)(uint32_t)key;
      out_scores[i] = key_score(key, metric);
    } else {
      out_ids[i] = -1;
      out_scores[i] = pad;
    }
  }
  __syncthreads();
}

}  // namespace lvq
