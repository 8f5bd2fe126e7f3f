// The C ABI declared in include/lvq.h: argument checks, store memory, scratch
// sizing and the order of kernel launches of each call.
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "kernels.cuh"
#include "topk.cuh"

using namespace lvq;

namespace {

constexpr size_t kAlign = 256;

// An NVTX range around the host side of one C-ABI call (the launches it
// enqueues), named after the entry point, for timelines in profilers.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};
#define LVQ_RANGE() NvtxRange nvtx_range_(__func__)
constexpr int64_t kReencodeChunk = 65536;  // rows reconstructed and re-encoded per pass

// counters block layout (device, int64 words)
enum { kCtrLive = 0, kCtrAbort = 1, kCtrDelCount = 2, kCtrWords = 4 };

lvq_status fail(const lvq_store* s, lvq_status code, const char* msg) {
  if (s) {
    std::lock_guard<std::mutex> g(s->msg_mu);
    s->last_msg = msg;
  }
  return code;
}

lvq_status cuda_fail(const lvq_store* s, cudaError_t e, const char* where) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
  return fail(s, e == cudaErrorMemoryAllocation ? LVQ_ENOMEM : LVQ_ECUDA, buf);
}

#define LVQ_CUDA(s, call, where)                      \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(s, e_, where); \
  } while (0)

// Scratch memory of one call, carved from the store's workspace.
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  template <class T>
  T* take(size_t count) {
    T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
    off += (count * sizeof(T) + kAlign - 1) / kAlign * kAlign;
    return p;
  }
};

lvq_status ensure_ws(lvq_store* s, size_t bytes) {
  if (bytes <= s->ws_bytes) return LVQ_OK;
  if (s->ws) {
    cudaError_t e = cudaFree(s->ws);
    s->ws = nullptr;
    s->ws_bytes = 0;
    if (e != cudaSuccess) return cuda_fail(s, e, "cudaFree(workspace)");
  }
  const size_t want = bytes + bytes / 4 + (1 << 20);
  cudaError_t e = cudaMalloc(&s->ws, want);
  if (e != cudaSuccess) {
    s->ws = nullptr;
    return cuda_fail(s, e, "cudaMalloc(workspace)");
  }
  s->ws_bytes = want;
  return LVQ_OK;
}

lvq_store* root_of(const lvq_store* s) { return const_cast<lvq_store*>(s->base ? s->base : s); }

bool valid_stream_device(const lvq_store* s) {
  int dev = -1;
  return cudaGetDevice(&dev) == cudaSuccess && dev == s->device;
}

int pick_qb(const lvq_store* s, int64_t nq) {
  if (s->tuning.fp32_q > 0) return s->tuning.fp32_q;
  if (nq >= 16) return 16;
  int qb = 1;
  while (qb < nq) qb <<= 1;
  return qb;
}

int pick_mma_n(const lvq_store* s, int64_t nq) {
  int n;
  if (s->tuning.mma_n > 0) n = s->tuning.mma_n;
  else if (nq <= 16) n = 16;
  else if (nq <= 32) n = 32;
  else if (nq <= 64) n = 64;
  else n = 128;
  const int lim = mma_tile_limit(s->ds);
  return n > lim ? lim : n;
}

// First-level scan kernels.
enum ScanPath { kPathFp32 = 0, kPathMma = 1, kPathSmall = 2 };

// Layout of the scratch memory of a first-level scan.
struct ScanScratch {
  QueryPrep prep;
  ScanPlan plan;
  int qb = 0, n_tile = 0;
  int path = kPathFp32;
  void* small = nullptr;  // rounded queries of the small-batch scan
};

// n_rows: the rows to scan (a snapshot of the store's row bound, taken once
// per call so that the sizing and the layout of a plan always agree).
size_t plan_scan(const lvq_store* s, int64_t nq, int k1, int path, int64_t n_rows, void* base, ScanScratch* out) {
  const DeviceStore& st = s->ds;
  const bool mma = path == kPathMma;
  Carver c(base);
  ScanScratch sc;
  sc.path = path;
  sc.prep.qsum = c.take<float>(nq);
  sc.prep.qnorm = c.take<float>(nq);
  sc.prep.cm = c.take<float>((size_t)nq * st.n_means);
  sc.prep.q16 = nullptr;
  sc.prep.q16sum = nullptr;
  sc.prep.nq_pad = nq;
  sc.prep.kq = 0;
  int grid, tiles_rows;
  int64_t groups;
  if (mma) {
    sc.n_tile = pick_mma_n(s, nq);
    sc.prep.nq_pad = round_up(nq, sc.n_tile);
    // K is padded to whole 64-byte code boxes (128 dims at 4 bits, 64 at 8)
    const int box_dims = st.bits1 == 4 ? 128 : 64;
    sc.prep.kq = (int)ceil_div(st.row1, 64) * box_dims;
    sc.prep.q16 = c.take<uint16_t>((size_t)sc.prep.nq_pad * sc.prep.kq);
    sc.prep.q16sum = c.take<float>(nq);
    grid = s->sm_count;
    tiles_rows = 128;
    groups = sc.prep.nq_pad / sc.n_tile;
  } else if (path == kPathSmall) {
    sc.small = c.take<unsigned char>(small_scratch_bytes(st, nq));
    grid = small_grid(st, n_rows, nq, k1, s->sm_count);
    tiles_rows = 128;
    groups = 1;
  } else {
    sc.qb = pick_qb(s, nq);
    grid = fp32_scan_grid(st, sc.qb, s->sm_count);
    tiles_rows = 256;
    groups = ceil_div(nq, sc.qb);
  }
  const int64_t ntiles = ceil_div(n_rows > 0 ? n_rows : 1, tiles_rows);
  int splits;
  if (mma) {
    // jobs (query tile x database segment) dealt round-robin to the CTAs
    int g = s->tuning.mma_ctas > 0 ? s->tuning.mma_ctas : grid;
    if (g < 1) g = 1;
    splits = mma_segments(g, groups, ntiles);
    const int64_t jobs = groups * splits;
    sc.plan.grid = (int)(jobs < g ? jobs : g);
  } else if (path == kPathSmall) {
    // one contiguous range of tiles per CTA; each CTA writes its own list
    sc.plan.grid = grid;
    splits = grid;
  } else {
    splits = s->tuning.fp32_splits;
    if (splits <= 0) splits = (int)ceil_div((int64_t)grid * 2, groups);
    if (splits > ntiles) splits = (int)ntiles;
    if (splits < 1) splits = 1;
    sc.plan.grid = (int)(groups * splits < grid ? groups * splits : grid);
  }
  sc.plan.splits = splits;
  sc.plan.wait_polls = (uint32_t)s->tuning.wait_polls;
  sc.plan.n_rows = n_rows;
  sc.plan.k1 = k1;
  sc.plan.partial = c.take<uint64_t>((size_t)nq * splits * k1);
  sc.plan.counts = path != kPathFp32 ? c.take<int>((size_t)nq * splits) : nullptr;
  sc.plan.gthr = mma ? c.take<uint64_t>((size_t)nq) : nullptr;
  if (mma) {
    // enough keys of distinct rows per query that their k1-th lowest can bound
    // the search: ceil(k1 / segments) per segment, at most 256 per query (the
    // bound warp runs with query tiles of up to 64)
    const int j = (int)ceil_div(k1, splits);
    sc.plan.best_j = (int64_t)splits * j <= 256 && sc.n_tile <= 64 ? j : 0;
    sc.plan.seg_best = sc.plan.best_j ? c.take<uint64_t>((size_t)nq * splits * sc.plan.best_j) : nullptr;
  }
  const size_t cand = mma                  ? mma_scan_cand_bytes(sc.plan.grid, sc.n_tile, k1)
                     : path == kPathSmall ? 0
                                          : fp32_scan_cand_bytes(sc.plan.grid, sc.qb, k1);
  sc.plan.cand = c.take<uint64_t>(cand / 8);
  if (out) *out = sc;
  return c.off;
}

// Brackets the launches of one kernel kind with events when profiling is on.
struct Prof {
  lvq_store* s;
  cudaStream_t st;
  int kind, launches;
  cudaEvent_t a = nullptr, b = nullptr;
  Prof(const lvq_store* s_, cudaStream_t st_, int kind_, int launches_ = 1)
      : s(const_cast<lvq_store*>(s_)), st(st_), kind(kind_), launches(launches_) {
    if (s->prof_on && cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess)
      cudaEventRecord(a, st);
  }
  ~Prof() {
    if (a && b) {
      cudaEventRecord(b, st);
      s->prof.push_back({kind, launches, a, b});
    }
  }
};

lvq_status check_q(const lvq_store* s, const void* q, int64_t nq) {
  if (!s) return LVQ_EINVAL;
  if (nq < 0) return fail(s, LVQ_EINVAL, "nq < 0");
  if (nq > 0 && !q) return fail(s, LVQ_EINVAL, "null query pointer");
  if (nq > (int64_t)INT32_MAX) return fail(s, LVQ_EINVAL, "nq too large");
  if (!valid_stream_device(s)) return fail(s, LVQ_EINVAL, "current device differs from the store's device");
  return LVQ_OK;
}

lvq_status first_level(lvq_store* s, const float* q, int64_t nq, int k1, int k, bool rerank, int precision,
                       int64_t* out_ids, float* out_scores, cudaStream_t stream) {
  const DeviceStore& st = s->ds;
  int path;
  if (precision == LVQ_FP32) {
    path = kPathFp32;
  } else if (precision == LVQ_FP16_MMA) {
    if (!mma_supported(st)) return fail(s, LVQ_EINVAL, "tensor-core scan unavailable for this store");
    path = kPathMma;
  } else if (precision == LVQ_INT16) {
    if (!small_supported(st, nq, k1) && nq > 0)
      return fail(s, LVQ_EINVAL, "integer scan takes 1 to 4 queries of a 4- or 8-bit store");
    path = kPathSmall;
  } else if (precision == LVQ_AUTO) {
    path = small_supported(st, nq, k1) ? kPathSmall : mma_supported(st) ? kPathMma : kPathFp32;
  } else {
    return fail(s, LVQ_EINVAL, "unknown precision");
  }
  std::lock_guard<std::mutex> g(s->mu);
  const int64_t n_rows = root_of(s)->rows_bound.load();
  const size_t need = plan_scan(s, nq, k1, path, n_rows, nullptr, nullptr);
  lvq_status rc = ensure_ws(s, need);
  if (rc != LVQ_OK) return rc;
  ScanScratch sc;
  plan_scan(s, nq, k1, path, n_rows, s->ws, &sc);
  cudaError_t e;
  {
    Prof p(s, stream, LVQ_K_PREP, path == kPathSmall ? 2 : 1);
    e = launch_prep_queries(st, q, nq, sc.prep, stream);
    if (e == cudaSuccess && path == kPathSmall) e = launch_small_prep(st, q, nq, sc.small, stream);
  }
  if (e != cudaSuccess) return cuda_fail(s, e, "prep_queries");
  static const int kind[3] = {LVQ_K_SCAN_FP32, LVQ_K_SCAN_MMA, LVQ_K_SCAN_SMALL};
  static const char* name[3] = {"scan_fp32", "scan_mma", "scan_small"};
  {
    Prof p(s, stream, kind[path]);
    if (path == kPathMma) e = launch_scan_mma(st, nq, sc.prep, sc.n_tile, sc.plan, stream);
    else if (path == kPathSmall) e = launch_scan_small(st, nq, sc.prep, sc.small, sc.plan, stream);
    else e = launch_scan_fp32(st, q, nq, sc.prep, sc.qb, sc.plan, stream);
  }
  if (e != cudaSuccess) return cuda_fail(s, e, name[path]);
  {
    Prof p(s, stream, LVQ_K_MERGE);
    e = launch_merge_rerank(st, q, nq, sc.prep, sc.plan.partial, sc.plan.splits, k1, k, rerank, out_ids,
                            out_scores, stream, sc.plan.counts, s->sm_count);
  }
  if (e != cudaSuccess) return cuda_fail(s, e, "merge_rerank");
  return LVQ_OK;
}

// ---- scratch of lvq_search_exhaustive_static -----------------------------------
// A file-scope device array, one per device (module global), so the call
// allocates nothing: 4 MiB holds the largest small-batch plan (4 queries,
// k1 = 512, one 512-key list per CTA on up to ~240 SMs, <q, mu_m> for 256
// means, rounded queries of d = 4096).  No byte of it needs to start at
// zero: every byte a call reads was written earlier in the same call.
constexpr size_t kStaticScratchBytes = size_t(4) << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_addr[kMaxDevices] = {};

}  // namespace

extern "C" {

const char* lvq_status_string(lvq_status st) {
  switch (st) {
    case LVQ_OK: return "ok";
    case LVQ_EINVAL: return "invalid argument";
    case LVQ_ENOMEM: return "out of device memory";
    case LVQ_EFULL: return "store full";
    case LVQ_ENOTFOUND: return "id not live";
    case LVQ_ECUDA: return "CUDA error";
    case LVQ_ETIMEOUT: return "device wait timed out";
    case LVQ_EBUSY: return "busy";
  }
  return "unknown status";
}

lvq_status lvq_create(const lvq_config* cfg, const float* means_host, lvq_store** out) {
  if (!cfg || !means_host || !out) return LVQ_EINVAL;
  *out = nullptr;
  if (cfg->d < 1 || cfg->d > kMaxD) return LVQ_EINVAL;
  if (cfg->bits1 < 2 || cfg->bits1 > 8) return LVQ_EINVAL;
  if (cfg->bits2 != 0 && (cfg->bits2 < 2 || cfg->bits2 > 8)) return LVQ_EINVAL;
  if (cfg->n_means < 1 || cfg->n_means > kMaxMeans) return LVQ_EINVAL;
  if (cfg->metric != LVQ_L2 && cfg->metric != LVQ_IP) return LVQ_EINVAL;
  if ((cfg->flags & ~LVQ_FLAG_LISTING_RESIDUAL) != 0) return LVQ_EINVAL;
  if (cfg->capacity < 1 || cfg->capacity > (int64_t)INT32_MAX) return LVQ_EINVAL;
  lvq_store* s = new (std::nothrow) lvq_store();
  if (!s) return LVQ_ENOMEM;
  s->cfg = *cfg;
  memset(&s->tuning, 0, sizeof(s->tuning));
  DeviceStore& st = s->ds;
  memset(&st, 0, sizeof(st));
  st.d = cfg->d;
  // codes live in 4-bit (B1 <= 4) or 8-bit containers; residuals in bytes
  st.bits1 = cfg->bits1 <= 4 ? 4 : 8;
  st.bits2 = cfg->bits2 ? 8 : 0;
  st.b1 = cfg->bits1;
  st.b2 = cfg->bits2;
  st.lev1 = (1 << cfg->bits1) - 1;
  st.lev2 = cfg->bits2 ? (1 << cfg->bits2) - 1 : 0;
  st.grid2 = (cfg->flags & LVQ_FLAG_LISTING_RESIDUAL) && cfg->bits2 ? 1 : 0;
  st.n_means = cfg->n_means;
  st.metric = cfg->metric;
  st.capacity = cfg->capacity;
  st.row1 = (int)round_up(ceil_div((int64_t)cfg->d * st.bits1, 8), 16);
  st.stride1 = st.row1 + 16;
  st.row2 = cfg->bits2 ? (int)round_up(cfg->d, 32) : 0;
  const int64_t cap = cfg->capacity;
  cudaError_t e = cudaGetDevice(&s->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device);
  auto A = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes > 0 ? bytes : 16);
  };
  A((void**)&st.codes1, (size_t)cap * st.stride1);
  if (st.bits2) A((void**)&st.codes2, (size_t)cap * st.row2);
  A((void**)&st.lower, (size_t)cap * 4);
  A((void**)&st.step, (size_t)cap * 4);
  A((void**)&st.norm2, (size_t)cap * 4);
  A((void**)&st.mean_id, (size_t)round_up(cap, 16));
  A((void**)&st.live, (size_t)round_up(ceil_div(cap, 32) * 4, 16));
  A((void**)&st.reserved, (size_t)round_up(ceil_div(cap, 32) * 4, 16));
  A((void**)&st.means, (size_t)cfg->n_means * cfg->d * 4);
  A((void**)&st.err, 16);
  A((void**)&s->counters, kCtrWords * 8 + alloc_scratch_bytes(cap));
  if (e == cudaSuccess) e = cudaMemset(st.live, 0, (size_t)round_up(ceil_div(cap, 32) * 4, 16));
  if (e == cudaSuccess) e = cudaMemset(st.reserved, 0, (size_t)round_up(ceil_div(cap, 32) * 4, 16));
  if (e == cudaSuccess) e = cudaMemset(st.err, 0, 16);
  if (e == cudaSuccess) e = cudaMemset(s->counters, 0, kCtrWords * 8);
  if (e == cudaSuccess) e = cudaMemset(st.codes1, 0, (size_t)cap * st.stride1);
  if (e == cudaSuccess) e = cudaMemcpy(st.means, means_host, (size_t)cfg->n_means * cfg->d * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    lvq_status rc = e == cudaErrorMemoryAllocation ? LVQ_ENOMEM : LVQ_ECUDA;
    lvq_destroy(s);
    return rc;
  }
  *out = s;
  return LVQ_OK;
}

lvq_status lvq_destroy(lvq_store* s) {
  if (!s) return LVQ_EINVAL;
  cudaDeviceSynchronize();
  for (auto& r : s->prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  if (s->base) {  // a view owns only its scratch memory
    if (s->ws) cudaFree(s->ws);
    delete s;
    return LVQ_OK;
  }
  DeviceStore& st = s->ds;
  void* ptrs[] = {st.codes1, st.codes2,  st.lower, st.step,     st.norm2, st.mean_id,
                  st.live,   st.reserved, st.means, st.err,     s->counters, s->ws};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete s;
  return LVQ_OK;
}

lvq_status lvq_store_view(const lvq_store* base, lvq_store** out) {
  if (!base || !out) return LVQ_EINVAL;
  *out = nullptr;
  lvq_store* b = root_of(base);
  lvq_store* v = new (std::nothrow) lvq_store();
  if (!v) return LVQ_ENOMEM;
  v->cfg = b->cfg;
  v->device = b->device;
  v->ds = b->ds;
  v->base = b;
  v->counters = b->counters;
  v->sm_count = b->sm_count;
  memset(&v->tuning, 0, sizeof(v->tuning));
  *out = v;
  return LVQ_OK;
}

lvq_status lvq_encode(const lvq_store* s, const float* x, int64_t n, uint8_t* codes1, uint8_t* codes2,
                      float* lower, float* step, uint8_t* mean_id, lvq_stream_t stream) {
  LVQ_RANGE();
  if (!s) return LVQ_EINVAL;
  if (n < 0) return fail(s, LVQ_EINVAL, "n < 0");
  if (n == 0) return LVQ_OK;
  if (!x || !codes1 || !lower || !step || !mean_id) return fail(s, LVQ_EINVAL, "null pointer");
  if (s->ds.bits2 && !codes2) return fail(s, LVQ_EINVAL, "codes2 required when bits2 > 0");
  if (!valid_stream_device(s)) return fail(s, LVQ_EINVAL, "current device differs from the store's device");
  EncodeOut o;
  o.codes1 = codes1;
  o.codes2 = s->ds.bits2 ? codes2 : nullptr;
  o.lower = lower;
  o.step = step;
  o.mean_id = mean_id;
  LVQ_CUDA(s, launch_encode(s->ds, x, n, o, (cudaStream_t)stream), "encode");
  return LVQ_OK;
}

static lvq_status insert_impl(lvq_store* s, const float* x, int64_t n, int64_t* out_ids, lvq_stream_t stream,
                              bool deferred) {
  NvtxRange nvtx_range_(deferred ? "lvq_insert_deferred" : "lvq_insert");
  if (!s) return LVQ_EINVAL;
  if (n < 0 || n > s->ds.capacity) return fail(s, LVQ_EINVAL, "n out of range");
  if (n == 0) return LVQ_OK;
  if (!x || !out_ids) return fail(s, LVQ_EINVAL, "null pointer");
  if (!valid_stream_device(s)) return fail(s, LVQ_EINVAL, "current device differs from the store's device");
  lvq_store* r = root_of(s);
  cudaStream_t st = (cudaStream_t)stream;
  int64_t* ctr = r->counters;
  int32_t* abort_flag = reinterpret_cast<int32_t*>(ctr + kCtrAbort);
  int32_t* scratch = reinterpret_cast<int32_t*>(ctr + kCtrWords);
  {
    Prof p(s, st, LVQ_K_INSERT, 5);
    LVQ_CUDA(s, launch_alloc_slots(r->ds, n, out_ids, scratch, abort_flag, st), "alloc_slots");
    EncodeOut o;
    o.slots = out_ids;
    o.abort_flag = abort_flag;
    LVQ_CUDA(s, launch_encode(r->ds, x, n, o, st), "encode(insert)");
    LVQ_CUDA(s, launch_publish(r->ds, out_ids, n, abort_flag, ctr + kCtrLive, deferred, st), "publish");
  }
  // the n lowest free slots lie below (live + reserved + n) <= bound + n
  int64_t cur = r->rows_bound.load();
  int64_t nxt;
  do {
    nxt = cur + n < s->ds.capacity ? cur + n : s->ds.capacity;
  } while (!r->rows_bound.compare_exchange_weak(cur, nxt));
  return LVQ_OK;
}

lvq_status lvq_insert(lvq_store* s, const float* x, int64_t n, int64_t* out_ids, lvq_stream_t stream) {
  return insert_impl(s, x, n, out_ids, stream, false);
}

lvq_status lvq_insert_deferred(lvq_store* s, const float* x, int64_t n, int64_t* out_ids, lvq_stream_t stream) {
  return insert_impl(s, x, n, out_ids, stream, true);
}

lvq_status lvq_publish(lvq_store* s, const int64_t* ids, int64_t n, lvq_stream_t stream) {
  LVQ_RANGE();
  if (!s) return LVQ_EINVAL;
  if (n < 0) return fail(s, LVQ_EINVAL, "n < 0");
  if (n == 0) return LVQ_OK;
  if (!ids) return fail(s, LVQ_EINVAL, "null pointer");
  if (!valid_stream_device(s)) return fail(s, LVQ_EINVAL, "current device differs from the store's device");
  Prof p(s, (cudaStream_t)stream, LVQ_K_INSERT);
  LVQ_CUDA(s, launch_publish_reserved(root_of(s)->ds, ids, n, root_of(s)->counters + kCtrLive, (cudaStream_t)stream),
           "publish_reserved");
  return LVQ_OK;
}

lvq_status lvq_delete(lvq_store* s, const int64_t* ids, int64_t n, int64_t* out_n_deleted, lvq_stream_t stream) {
  LVQ_RANGE();
  if (!s) return LVQ_EINVAL;
  if (n < 0) return fail(s, LVQ_EINVAL, "n < 0");
  if (!out_n_deleted || (n > 0 && !ids)) return fail(s, LVQ_EINVAL, "null pointer");
  if (!valid_stream_device(s)) return fail(s, LVQ_EINVAL, "current device differs from the store's device");
  int64_t* ctr = root_of(s)->counters;
  Prof p(s, (cudaStream_t)stream, LVQ_K_DELETE, n > 0 ? 2 : 1);
  LVQ_CUDA(s,
           launch_delete(root_of(s)->ds, ids, n, out_n_deleted,
                         reinterpret_cast<unsigned long long*>(ctr + kCtrDelCount), ctr + kCtrLive,
                         (cudaStream_t)stream, false),
           "delete");
  return LVQ_OK;
}

lvq_status lvq_delete_hold(lvq_store* s, const int64_t* ids, int64_t n, int64_t* out_n_deleted,
                           lvq_stream_t stream) {
  LVQ_RANGE();
  if (!s) return LVQ_EINVAL;
  if (n < 0) return fail(s, LVQ_EINVAL, "n < 0");
  if (!out_n_deleted || (n > 0 && !ids)) return fail(s, LVQ_EINVAL, "null pointer");
  if (!valid_stream_device(s)) return fail(s, LVQ_EINVAL, "current device differs from the store's device");
  int64_t* ctr = root_of(s)->counters;
  Prof p(s, (cudaStream_t)stream, LVQ_K_DELETE, n > 0 ? 2 : 1);
  LVQ_CUDA(s,
           launch_delete(root_of(s)->ds, ids, n, out_n_deleted,
                         reinterpret_cast<unsigned long long*>(ctr + kCtrDelCount), ctr + kCtrLive,
                         (cudaStream_t)stream, true),
           "delete_hold");
  return LVQ_OK;
}

lvq_status lvq_release(lvq_store* s, const int64_t* ids, int64_t n, lvq_stream_t stream) {
  LVQ_RANGE();
  if (!s) return LVQ_EINVAL;
  if (n < 0) return fail(s, LVQ_EINVAL, "n < 0");
  if (n > 0 && !ids) return fail(s, LVQ_EINVAL, "null pointer");
  if (!valid_stream_device(s)) return fail(s, LVQ_EINVAL, "current device differs from the store's device");
  LVQ_CUDA(s, launch_release(root_of(s)->ds, ids, n, (cudaStream_t)stream), "release");
  return LVQ_OK;
}

lvq_status lvq_live_words(const lvq_store* s, int64_t* out_words) {
  if (!s || !out_words) return LVQ_EINVAL;
  *out_words = (s->ds.capacity + 31) / 32;
  return LVQ_OK;
}

lvq_status lvq_snapshot_live(const lvq_store* s, uint32_t* dst, lvq_stream_t stream) {
  LVQ_RANGE();
  if (!s) return LVQ_EINVAL;
  lvq_store* m = const_cast<lvq_store*>(s);
  if (!dst) return fail(m, LVQ_EINVAL, "null pointer");
  if (!valid_stream_device(s)) return fail(m, LVQ_EINVAL, "current device differs from the store's device");
  const lvq_store* r = root_of(s);
  LVQ_CUDA(m,
           cudaMemcpyAsync(dst, r->ds.live, (size_t)((r->ds.capacity + 31) / 32) * 4, cudaMemcpyDeviceToDevice,
                           (cudaStream_t)stream),
           "snapshot_live");
  return LVQ_OK;
}

lvq_status lvq_view_set_live(lvq_store* view, const uint32_t* live) {
  if (!view) return LVQ_EINVAL;
  if (!view->base) return fail(view, LVQ_EINVAL, "not a view");
  std::lock_guard<std::mutex> g(view->mu);
  view->ds.live = live ? const_cast<uint32_t*>(live) : root_of(view)->ds.live;
  return LVQ_OK;
}

lvq_status lvq_update_mean(lvq_store* s, int32_t m, const float* new_mean, int64_t* out_count, lvq_stream_t stream) {
  LVQ_RANGE();
  if (!s) return LVQ_EINVAL;
  if (!new_mean || !out_count) return fail(s, LVQ_EINVAL, "null pointer");
  if (m < 0 || m >= s->ds.n_means) return fail(s, LVQ_EINVAL, "mean index out of range");
  if (!valid_stream_device(s)) return fail(s, LVQ_EINVAL, "current device differs from the store's device");
  const DeviceStore& st = root_of(s)->ds;
  const cudaStream_t str = (cudaStream_t)stream;
  std::lock_guard<std::mutex> g(s->mu);
  const int64_t n_rows = root_of(s)->rows_bound.load();
  const int64_t chunk = n_rows < kReencodeChunk ? (n_rows > 0 ? n_rows : 1) : kReencodeChunk;
  Carver sizer(nullptr);
  sizer.take<int64_t>((size_t)(n_rows > 0 ? n_rows : 1));
  sizer.take<unsigned long long>(1);
  sizer.take<float>((size_t)st.d);
  sizer.take<float>((size_t)chunk * st.d);
  lvq_status rc = ensure_ws(s, sizer.off);
  if (rc != LVQ_OK) return rc;
  Carver c(s->ws);
  int64_t* list = c.take<int64_t>((size_t)(n_rows > 0 ? n_rows : 1));
  unsigned long long* cnt = c.take<unsigned long long>(1);
  float* old_mu = c.take<float>((size_t)st.d);
  float* xbuf = c.take<float>((size_t)chunk * st.d);
  float* mu_m = st.means + (int64_t)m * st.d;
  // the old centre is kept for the reconstructions, then replaced
  LVQ_CUDA(s, cudaMemsetAsync(cnt, 0, sizeof(*cnt), str), "memset");
  LVQ_CUDA(s, cudaMemcpyAsync(old_mu, mu_m, (size_t)st.d * 4, cudaMemcpyDeviceToDevice, str), "copy centre");
  LVQ_CUDA(s, launch_select_mean(st, n_rows, m, list, cnt, str), "select_mean");
  LVQ_CUDA(s, cudaMemcpyAsync(mu_m, new_mean, (size_t)st.d * 4, cudaMemcpyDeviceToDevice, str), "copy centre");
  unsigned long long count = 0;
  LVQ_CUDA(s, cudaMemcpyAsync(&count, cnt, sizeof(count), cudaMemcpyDeviceToHost, str), "copy count");
  LVQ_CUDA(s, cudaStreamSynchronize(str), "synchronize");
  for (int64_t off = 0; off < (int64_t)count; off += chunk) {
    const int64_t nb = (int64_t)count - off < chunk ? (int64_t)count - off : chunk;
    LVQ_CUDA(s, launch_reconstruct(st, list + off, nb, old_mu, xbuf, str), "reconstruct");
    EncodeOut out;
    out.slots = list + off;
    out.force_mean = m;
    LVQ_CUDA(s, launch_encode(st, xbuf, nb, out, str), "encode");
  }
  *out_count = (int64_t)count;
  return LVQ_OK;
}

lvq_status lvq_search_graph(const lvq_store* cs, const float* q, int64_t nq, const int32_t* graph, int64_t n_graph,
                            int32_t R, const int64_t* starts, int32_t n_starts, int32_t L, int32_t max_expand,
                            int32_t k1, int32_t k, int64_t* out_ids, float* out_scores, lvq_stream_t stream) {
  LVQ_RANGE();
  lvq_status rc = check_q(cs, q, nq);
  if (rc != LVQ_OK) return rc;
  lvq_store* s = const_cast<lvq_store*>(cs);
  const DeviceStore& st = s->ds;
  if (k < 1 || k > kMaxK1) return fail(s, LVQ_EINVAL, "k out of range");
  if (k1 < 0 || k1 > kMaxK1 || (k1 > 0 && k1 < k)) return fail(s, LVQ_EINVAL, "k1 out of range");
  if (R < 1 || R > 256 || n_graph < 1 || n_graph > st.capacity) return fail(s, LVQ_EINVAL, "graph shape out of range");
  if (L < 1 || L > 1024 || L < k || L < k1) return fail(s, LVQ_EINVAL, "L must be at least k and k1 (and at most 1024)");
  if (n_starts < 1 || n_starts > L) return fail(s, LVQ_EINVAL, "n_starts out of range (1 .. L)");
  if (max_expand < 0) return fail(s, LVQ_EINVAL, "max_expand < 0");
  if (nq > 0 && (!graph || !starts || !out_ids || !out_scores)) return fail(s, LVQ_EINVAL, "null pointer");
  if (nq == 0) return LVQ_OK;
  const int expand = max_expand > 0 ? max_expand : 4 * L;
  if (beam_smem(st, L, R, beam_set_slots(n_starts, R, expand)) > 220 * 1024)
    return fail(s, LVQ_EINVAL, "the seen-set of L, R and max_expand does not fit in shared memory");
  const bool two = st.bits2 && k1 > 0;
  const int kk1 = two ? k1 : k;
  std::lock_guard<std::mutex> g(s->mu);
  Carver sizer(nullptr);
  sizer.take<uint64_t>((size_t)nq * kk1);
  sizer.take<int64_t>((size_t)nq * kk1);
  rc = ensure_ws(s, sizer.off);
  if (rc != LVQ_OK) return rc;
  Carver c(s->ws);
  uint64_t* keys = c.take<uint64_t>((size_t)nq * kk1);
  int64_t* ids = c.take<int64_t>((size_t)nq * kk1);
  const cudaStream_t str = (cudaStream_t)stream;
  {
    Prof p(s, str, LVQ_K_GATHER, 2);
    LVQ_CUDA(s, launch_beam(st, q, nq, graph, n_graph, R, starts, n_starts, L, expand, kk1, keys, ids, str), "beam");
  }
  if (two) {
    QueryPrep none{};
    Prof p(s, str, LVQ_K_RERANK);
    LVQ_CUDA(s, launch_rerank(st, q, nq, none, ids, kk1, k, out_ids, out_scores, str), "rerank");
  } else {
    LVQ_CUDA(s, launch_keys_to_results(keys, nq, kk1, k, st.metric, out_ids, out_scores, str), "results");
  }
  return LVQ_OK;
}

lvq_status lvq_search_exhaustive(const lvq_store* cs, const float* q, int64_t nq, int32_t k1, int32_t k,
                                 int32_t precision, int64_t* out_ids, float* out_scores, lvq_stream_t stream) {
  LVQ_RANGE();
  lvq_status rc = check_q(cs, q, nq);
  if (rc != LVQ_OK) return rc;
  lvq_store* s = const_cast<lvq_store*>(cs);
  if (k < 1 || k > kMaxK1) return fail(s, LVQ_EINVAL, "k out of range");
  if (k1 < 0 || k1 > kMaxK1 || (k1 > 0 && k1 < k)) return fail(s, LVQ_EINVAL, "k1 out of range");
  if (nq > 0 && (!out_ids || !out_scores)) return fail(s, LVQ_EINVAL, "null output pointer");
  if (nq == 0) return LVQ_OK;
  const bool two = s->ds.bits2 && k1 > 0;
  return first_level(s, q, nq, two ? k1 : k, k, two, precision, out_ids, out_scores, (cudaStream_t)stream);
}

lvq_status lvq_search_exhaustive_static(const lvq_store* cs, const float* q, int64_t nq, int32_t k1, int32_t k,
                                        int64_t* out_ids, float* out_scores, lvq_stream_t stream) {
  LVQ_RANGE();
  lvq_status rc = check_q(cs, q, nq);
  if (rc != LVQ_OK) return rc;
  lvq_store* s = const_cast<lvq_store*>(cs);
  if (k < 1 || k > kMaxK1) return fail(s, LVQ_EINVAL, "k out of range");
  if (k1 < 0 || k1 > kMaxK1 || (k1 > 0 && k1 < k)) return fail(s, LVQ_EINVAL, "k1 out of range");
  if (nq < 1 || nq > kSmallMaxQ)
    return fail(s, LVQ_EINVAL, "lvq_search_exhaustive_static takes 1 to 4 queries per call");
  if (!out_ids || !out_scores) return fail(s, LVQ_EINVAL, "null output pointer");
  const DeviceStore& st = s->ds;
  const bool two = st.bits2 && k1 > 0;
  const int kk1 = two ? k1 : k;
  if (!small_supported(st, nq, kk1))
    return fail(s, LVQ_EINVAL, "lvq_search_exhaustive_static: the integer scan does not take this store or k1");
  // the scratch address on this device; the first call on a device looks it up
  if (s->device < 0 || s->device >= kMaxDevices) return fail(s, LVQ_EINVAL, "device ordinal out of range");
  void* base;
  {
    std::lock_guard<std::mutex> g(g_static_mu);
    if (!g_static_addr[s->device]) {
      void* a = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&a, g_static_scratch);
      if (e != cudaSuccess || !a) return cuda_fail(s, e != cudaSuccess ? e : cudaErrorInvalidSymbol, "cudaGetSymbolAddress");
      g_static_addr[s->device] = a;
    }
    base = g_static_addr[s->device];
  }
  std::lock_guard<std::mutex> g(s->mu);
  // one snapshot of the row bound sizes and lays out the plan: an insert on
  // another thread cannot enlarge it between the check and the launch
  const int64_t n_rows = root_of(s)->rows_bound.load();
  const size_t need = plan_scan(s, nq, kk1, kPathSmall, n_rows, nullptr, nullptr);
  if (need > kStaticScratchBytes) {
    char msg[160];
    snprintf(msg, sizeof msg, "lvq_search_exhaustive_static: plan needs %zu bytes of scratch, the static array holds %zu",
             need, kStaticScratchBytes);
    return fail(s, LVQ_EINVAL, msg);
  }
  ScanScratch sc;
  plan_scan(s, nq, kk1, kPathSmall, n_rows, base, &sc);
  const cudaStream_t str = (cudaStream_t)stream;
  cudaError_t e = launch_prep_queries(st, q, nq, sc.prep, str);
  if (e == cudaSuccess) e = launch_small_prep(st, q, nq, sc.small, str);
  if (e != cudaSuccess) return cuda_fail(s, e, "prep_queries");
  e = launch_scan_small(st, nq, sc.prep, sc.small, sc.plan, str);
  if (e != cudaSuccess) return cuda_fail(s, e, "scan_small");
  e = launch_merge_rerank(st, q, nq, sc.prep, sc.plan.partial, sc.plan.splits, kk1, k, two, out_ids, out_scores, str,
                          sc.plan.counts, s->sm_count);
  if (e != cudaSuccess) return cuda_fail(s, e, "merge_rerank");
  return LVQ_OK;
}

lvq_status lvq_search_first_level(const lvq_store* cs, const float* q, int64_t nq, int32_t k1, int32_t precision,
                                  int64_t* out_ids, float* out_scores, lvq_stream_t stream) {
  LVQ_RANGE();
  lvq_status rc = check_q(cs, q, nq);
  if (rc != LVQ_OK) return rc;
  lvq_store* s = const_cast<lvq_store*>(cs);
  if (k1 < 1 || k1 > kMaxK1) return fail(s, LVQ_EINVAL, "k1 out of range");
  if (nq > 0 && (!out_ids || !out_scores)) return fail(s, LVQ_EINVAL, "null output pointer");
  if (nq == 0) return LVQ_OK;
  return first_level(s, q, nq, k1, k1, false, precision, out_ids, out_scores, (cudaStream_t)stream);
}

lvq_status lvq_search_candidates(const lvq_store* cs, const float* q, int64_t nq, const int64_t* cand,
                                 int32_t n_cand, int32_t k1, int32_t k, int64_t* out_ids, float* out_scores,
                                 lvq_stream_t stream) {
  LVQ_RANGE();
  lvq_status rc = check_q(cs, q, nq);
  if (rc != LVQ_OK) return rc;
  lvq_store* s = const_cast<lvq_store*>(cs);
  if (n_cand < 1 || n_cand > kMaxCand) return fail(s, LVQ_EINVAL, "n_cand out of range");
  if (k < 1 || k > kMaxK1) return fail(s, LVQ_EINVAL, "k out of range");
  if (k1 < 0 || k1 > kMaxK1 || (k1 > 0 && k1 < k)) return fail(s, LVQ_EINVAL, "k1 out of range");
  if (nq > 0 && (!cand || !out_ids || !out_scores)) return fail(s, LVQ_EINVAL, "null pointer");
  if (nq == 0) return LVQ_OK;
  const DeviceStore& st = s->ds;
  const bool two = st.bits2 && k1 > 0;
  std::lock_guard<std::mutex> g(s->mu);
  Carver c0(nullptr);
  c0.take<float>(nq);
  c0.take<float>(nq);
  c0.take<float>((size_t)nq * st.n_means);
  if (two) {
    c0.take<int64_t>((size_t)nq * k1);
    c0.take<float>((size_t)nq * k1);
  }
  rc = ensure_ws(s, c0.off);
  if (rc != LVQ_OK) return rc;
  Carver c(s->ws);
  QueryPrep p;
  p.qsum = c.take<float>(nq);
  p.qnorm = c.take<float>(nq);
  p.cm = c.take<float>((size_t)nq * st.n_means);
  p.q16 = nullptr;
  p.q16sum = nullptr;
  p.nq_pad = nq;
  p.kq = 0;
  cudaStream_t str = (cudaStream_t)stream;
  {
    Prof pr(s, str, LVQ_K_PREP);
    LVQ_CUDA(s, launch_prep_queries(st, q, nq, p, str), "prep_queries");
  }
  if (!two) {
    Prof pg(s, str, LVQ_K_GATHER);
    LVQ_CUDA(s, launch_gather(st, q, nq, p, cand, n_cand, k, out_ids, out_scores, str), "gather");
    return LVQ_OK;
  }
  // first level: the k1 best distinct candidates per query; then both levels
  // re-rank them, every query's candidates in flight at once
  int64_t* ids1 = c.take<int64_t>((size_t)nq * k1);
  float* sc1 = c.take<float>((size_t)nq * k1);
  {
    Prof pg(s, str, LVQ_K_GATHER);
    LVQ_CUDA(s, launch_gather(st, q, nq, p, cand, n_cand, k1, ids1, sc1, str), "gather");
  }
  Prof pr(s, str, LVQ_K_RERANK);
  LVQ_CUDA(s, launch_rerank(st, q, nq, p, ids1, k1, k, out_ids, out_scores, str), "rerank");
  return LVQ_OK;
}

lvq_status lvq_rerank(const lvq_store* cs, const float* q, int64_t nq, const int64_t* ids, int32_t k1, int32_t k,
                      int64_t* out_ids, float* out_scores, lvq_stream_t stream) {
  LVQ_RANGE();
  lvq_status rc = check_q(cs, q, nq);
  if (rc != LVQ_OK) return rc;
  lvq_store* s = const_cast<lvq_store*>(cs);
  if (!s->ds.bits2) return fail(s, LVQ_EINVAL, "store has no residual level");
  if (k1 < 1 || k1 > kMaxRerank || k < 1 || k > k1 || k > kMaxK1) return fail(s, LVQ_EINVAL, "k1/k out of range");
  if (nq > 0 && (!ids || !out_ids || !out_scores)) return fail(s, LVQ_EINVAL, "null pointer");
  if (nq == 0) return LVQ_OK;
  QueryPrep p{};
  Prof pr(s, (cudaStream_t)stream, LVQ_K_RERANK);
  LVQ_CUDA(s, launch_rerank(s->ds, q, nq, p, ids, k1, k, out_ids, out_scores, (cudaStream_t)stream), "rerank");
  return LVQ_OK;
}

lvq_status lvq_export(const lvq_store* s, const int64_t* ids, int64_t n, uint8_t* codes1, uint8_t* codes2,
                      float* lower, float* step, uint8_t* mean_id, lvq_stream_t stream) {
  LVQ_RANGE();
  if (!s) return LVQ_EINVAL;
  if (n < 0) return fail(s, LVQ_EINVAL, "n < 0");
  if (n == 0) return LVQ_OK;
  if (!ids || !codes1 || !lower || !step || !mean_id) return fail(s, LVQ_EINVAL, "null pointer");
  if (!valid_stream_device(s)) return fail(s, LVQ_EINVAL, "current device differs from the store's device");
  LVQ_CUDA(s, launch_export(s->ds, ids, n, codes1, codes2, lower, step, mean_id, (cudaStream_t)stream), "export");
  return LVQ_OK;
}

lvq_status lvq_stats(const lvq_store* s, int64_t* n_live_host, lvq_stream_t stream) {
  if (!s || !n_live_host) return LVQ_EINVAL;
  LVQ_CUDA(s, cudaStreamSynchronize((cudaStream_t)stream), "cudaStreamSynchronize");
  int64_t live = 0;
  int32_t err = 0;
  LVQ_CUDA(s, cudaMemcpy(&live, root_of(s)->counters + kCtrLive, 8, cudaMemcpyDeviceToHost), "read counters");
  LVQ_CUDA(s, cudaMemcpy(&err, s->ds.err, 4, cudaMemcpyDeviceToHost), "read error word");
  *n_live_host = live;
  if (err) {
    LVQ_CUDA(s, cudaMemset(s->ds.err, 0, 4), "clear error word");
    return fail(s, (lvq_status)err, lvq_status_string((lvq_status)err));
  }
  return LVQ_OK;
}

lvq_status lvq_reserve(lvq_store* s, int64_t max_nq, int32_t max_k1, int32_t max_cand) {
  if (!s || max_nq < 0 || max_k1 < 1 || max_k1 > kMaxK1 || max_cand < 0) return LVQ_EINVAL;
  (void)max_cand;
  std::lock_guard<std::mutex> g(s->mu);
  // sized for a full store: later inserts cannot outgrow the reservation
  const int64_t n_rows = s->ds.capacity;
  size_t need = plan_scan(s, max_nq, max_k1, kPathFp32, n_rows, nullptr, nullptr);
  if (mma_supported(s->ds)) {
    const size_t m = plan_scan(s, max_nq, max_k1, kPathMma, n_rows, nullptr, nullptr);
    if (m > need) need = m;
  }
  const int64_t small_nq = max_nq < kSmallMaxQ ? max_nq : kSmallMaxQ;
  if (small_supported(s->ds, small_nq, max_k1)) {
    const size_t m = plan_scan(s, small_nq, max_k1, kPathSmall, n_rows, nullptr, nullptr);
    if (m > need) need = m;
  }
  return ensure_ws(s, need);
}

lvq_status lvq_set_tuning(lvq_store* s, const lvq_tuning* t) {
  if (!s || !t) return LVQ_EINVAL;
  if (t->mma_n != 0 && t->mma_n != 16 && t->mma_n != 32 && t->mma_n != 64 && t->mma_n != 128) return LVQ_EINVAL;
  if (t->fp32_q != 0 && t->fp32_q != 1 && t->fp32_q != 2 && t->fp32_q != 4 && t->fp32_q != 8 && t->fp32_q != 16)
    return LVQ_EINVAL;
  if (t->mma_ctas < 0 || t->fp32_splits < 0 || t->wait_polls < 0) return LVQ_EINVAL;
  std::lock_guard<std::mutex> g(s->mu);
  s->tuning = *t;
  return LVQ_OK;
}

lvq_status lvq_get_tuning(const lvq_store* s, lvq_tuning* t) {
  if (!s || !t) return LVQ_EINVAL;
  std::lock_guard<std::mutex> g(s->mu);
  *t = s->tuning;
  return LVQ_OK;
}

lvq_status lvq_profile_enable(lvq_store* s, int32_t on) {
  if (!s) return LVQ_EINVAL;
  std::lock_guard<std::mutex> g(s->mu);
  s->prof_on = on != 0;
  return LVQ_OK;
}

lvq_status lvq_profile_read(lvq_store* s, double* ms, int64_t* launches, int32_t n_kinds) {
  if (!s || !ms || !launches || n_kinds < 1 || n_kinds > LVQ_KERNEL_KINDS) return LVQ_EINVAL;
  std::lock_guard<std::mutex> g(s->mu);
  LVQ_CUDA(s, cudaDeviceSynchronize(), "cudaDeviceSynchronize");
  for (int i = 0; i < n_kinds; ++i) {
    ms[i] = 0.0;
    launches[i] = 0;
  }
  for (auto& r : s->prof) {
    float t = 0.0f;
    if (r.kind < n_kinds && cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
      ms[r.kind] += t;
      launches[r.kind] += r.launches;
    }
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  s->prof.clear();
  return LVQ_OK;
}

lvq_status lvq_last_error(const lvq_store* s, char* buf, size_t len) {
  if (!s) return LVQ_EINVAL;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaGetLastError();
  lvq_status rc = LVQ_OK;
  std::string msg;
  if (e != cudaSuccess) {
    rc = LVQ_ECUDA;
    msg = cudaGetErrorString(e);
  } else {
    int32_t err = 0;
    if (cudaMemcpy(&err, s->ds.err, 4, cudaMemcpyDeviceToHost) == cudaSuccess && err) {
      rc = (lvq_status)err;
      msg = lvq_status_string(rc);
      cudaMemset(s->ds.err, 0, 4);
    } else {
      std::lock_guard<std::mutex> g(s->msg_mu);
      msg = s->last_msg;
    }
  }
  if (buf && len) {
    strncpy(buf, msg.c_str(), len - 1);
    buf[len - 1] = 0;
  }
  return rc;
}

}  // extern "C"
