/*
 * lvq.h -- C ABI of a B300 (sm_103a) library for Locally-adaptive Vector
 * Quantization search (Aguerrebere et al., "Locally-Adaptive Quantization for
 * Streaming Vector Search", arxiv 2402.02044).
 *
 * The library keeps LVQ-compressed vectors in a device-resident store and
 * scores batches of float32 queries against them:
 *   - encoding (Eq. 1-3 and Def. 1): centring by the nearest of M means,
 *     per-vector lower bound l and step D, B1-bit first-level codes and
 *     optional B2-bit residual codes on the grid Q_{B2,-D/2,D/2} (Sec. 2.2);
 *   - first-level scoring of 4-bit or 8-bit codes for the squared Euclidean
 *     distance or the inner product (Sec. 3.2), exhaustively or restricted to
 *     a candidate list, fused with top-k1 selection;
 *   - re-ranking of the k1 candidates with both levels (Sec. 2.2, App. C);
 *   - inserts into free slots and lazy deletes that are filtered out of
 *     every result (Sec. 2.1, App. A.2).
 *
 * Conventions for every entry point
 *   - Array arguments are DEVICE pointers owned by the caller unless the
 *     argument name ends in _host.  The library never frees them.
 *   - Work is enqueued on the given stream (NULL = legacy default stream) and
 *     the call returns without waiting for it.  Argument errors are returned
 *     at once and nothing is enqueued.  Errors found on the device (an id out
 *     of range, a full store) are recorded in the store and returned by the
 *     next call that synchronises (lvq_last_error, lvq_stats).
 *   - Calls that use one store must be ordered (one stream, or events): they
 *     share the store's scratch memory.
 *   - No C++ exception crosses this interface.
 *   - Results are sorted best first: ascending squared distance (LVQ_L2) or
 *     descending inner product (LVQ_IP); equal scores are ordered by
 *     ascending id.  A query with fewer than k live results is padded with
 *     id -1 and score +inf (LVQ_L2) or -inf (LVQ_IP).
 *   - Ids are slot indices in [0, capacity).
 */
#ifndef LVQ_H
#define LVQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL selects the legacy default stream. */
typedef struct CUstream_st *lvq_stream_t;

typedef enum {
  LVQ_OK = 0,
  LVQ_EINVAL = 1,    /* bad argument (null pointer, size or option out of range) */
  LVQ_ENOMEM = 2,    /* device allocation failed */
  LVQ_EFULL = 3,     /* an insert needed more free slots than the store had */
  LVQ_ENOTFOUND = 4, /* lvq_export was given an id that is not live */
  LVQ_ECUDA = 5,     /* a CUDA call failed (launch error, sticky device fault) */
  LVQ_ETIMEOUT = 6,  /* a bounded device wait gave up */
  LVQ_EBUSY = 7      /* reserved */
} lvq_status;

typedef enum { LVQ_L2 = 0, LVQ_IP = 1 } lvq_metric;

/* Arithmetic of the first-level scan <q, c>:
 *   LVQ_FP32      plain float32 on CUDA cores;
 *   LVQ_FP16_MMA  q rounded to float16, codes exact in float16, products
 *                 accumulated in float32 on the tcgen05 tensor cores;
 *   LVQ_INT16     q rounded to 16-bit integers (scale max|q| / 32767 per
 *                 query), exact integer products with the codes (dp4a) on
 *                 CUDA cores; batches of at most 4 queries, else LVQ_EINVAL;
 *   LVQ_AUTO      the library's choice for the batch size: LVQ_INT16 for 1
 *                 to 4 queries, the tensor cores above that. */
typedef enum { LVQ_FP32 = 0, LVQ_FP16_MMA = 1, LVQ_AUTO = 2, LVQ_INT16 = 3 } lvq_precision;

/* lvq_config.flags */
enum {
  /* The residual level on the App. C listing's signed grid (step D / 2^B2,
   * codes round(r / step) half to even, clipped to [-2^(B2-1), 2^(B2-1)-1],
   * stored as int8) instead of the text's Q_{B2,-D/2,D/2} (Sec. 2.2). */
  LVQ_FLAG_LISTING_RESIDUAL = 1
};

typedef struct {
  int32_t d;        /* dimensionality, 1 .. 4096 */
  int32_t bits1;    /* first-level bits B1: 2 .. 8 (Sec. 3.3 explores B1 and
                       B2); B1 <= 4 is stored in 4-bit containers, B1 >= 5
                       in bytes, and every scan reads those containers */
  int32_t bits2;    /* residual bits B2: 0 (LVQ-B1) or 2 .. 8 (LVQ-B1xB2),
                       stored in bytes */
  int32_t n_means;  /* M centring means, 1 .. 256 (M = 1 is plain LVQ) */
  int32_t metric;   /* lvq_metric */
  int32_t flags;    /* LVQ_FLAG_* ; other bits must be 0 */
  int64_t capacity; /* number of slots, 1 .. 2^31 - 1 */
} lvq_config;

typedef struct lvq_store lvq_store; /* opaque; owns all of its device memory */

/* Tile shapes of the scan kernels (chosen by the autotuner).  A field set to
 * 0 means "library default". */
typedef struct {
  int32_t mma_n;      /* queries per tcgen05 tile: 16, 32, 64 or 128 */
  int32_t mma_ctas;   /* persistent CTAs of the tensor-core scan (0 = one per SM) */
  int32_t fp32_q;     /* queries per CTA of the float32 scan: 1, 2, 4, 8 or 16 */
  int32_t fp32_splits;
  /* Failure detection of the tensor-core scan: polls of each pipeline wait
   * (a copy, an MMA or a partner role) before the scan gives up, records
   * LVQ_ETIMEOUT in the store (lvq_last_error) and ends its CTAs; the
   * results of that call are then undefined.  0 = the default, 2^24 polls
   * (seconds).  The waits for a CTA's own copies and MMAs in flight before
   * it exits always use the default, so no copy or MMA outlives the call. */
  int32_t wait_polls;
} lvq_tuning;

/* Create an empty store on the current CUDA device.
 * means_host: n_means x d float32 centring means, row-major, HOST memory,
 *   copied (Sec. 2.2: the sample mean; Def. 1: M centres).
 * out: receives the store handle.
 * Errors: LVQ_EINVAL for a bad config, LVQ_ENOMEM, LVQ_ECUDA. */
lvq_status lvq_create(const lvq_config *cfg, const float *means_host, lvq_store **out);

/* Free the store and all of its device memory (a view: its scratch memory
 * only).  Synchronises the device.  Destroy a store's views before it. */
lvq_status lvq_destroy(lvq_store *store);

/* A second handle on the same store: it shares the vectors, slots and
 * counters of `base` but has its own scratch memory, tile shapes and timing,
 * so searches through different views may run concurrently on different
 * streams.  Updates through any handle act on the shared store. */
lvq_status lvq_store_view(const lvq_store *base, lvq_store **out);

/* Encode n vectors without touching the store (Eq. 1-3, Def. 1, Sec. 2.2).
 * x: n x d float32, row-major.
 * codes1: n x d uint8, one first-level code per byte, in [0, 2^B1 - 1].
 * codes2: n x d uint8 residual codes in [0, 2^B2 - 1] (the listing's signed
 *   grid: int8 bytes in [-2^(B2-1), 2^(B2-1) - 1]), or NULL (required when
 *   bits2 > 0, ignored when bits2 = 0).
 * lower, step: n float32 each, l(x) and D of the vector.
 * mean_id: n uint8, index of the centring mean.
 * Every float32 step is rounded separately (no fused multiply-add):
 *   y = x - mu*, l = min y, D = (max y - l)/(2^B1 - 1),
 *   c = clamp(floor(fl(1/D') * (y - l) + 1/2)), D' = D or 1 when D = 0,
 *   r = y - (D c + l), c2 likewise with l2 = -D/2, D2 = D/(2^B2 - 1) (or on
 *   the listing's signed grid, LVQ_FLAG_LISTING_RESIDUAL). */
lvq_status lvq_encode(const lvq_store *store, const float *x, int64_t n, uint8_t *codes1,
                      uint8_t *codes2, float *lower, float *step, uint8_t *mean_id,
                      lvq_stream_t stream);

/* Insert n vectors (Sec. 2.1: X_t = X_{t-1} + {x}).  They are encoded on the
 * device into the n lowest-numbered free slots, in increasing slot order, and
 * become visible to searches that follow on the stream.
 * x: n x d float32.  out_ids: n int64, the slots taken.
 * All or nothing: when fewer than n slots are free nothing is inserted,
 * out_ids is filled with -1 and LVQ_EFULL is recorded (sticky). */
lvq_status lvq_insert(lvq_store *store, const float *x, int64_t n, int64_t *out_ids,
                      lvq_stream_t stream);

/* Deferred insert: like lvq_insert (same slot choice, encoding and errors)
 * but the slots stay invisible to searches, and unavailable to other inserts,
 * until lvq_publish.  A serving loop encodes new vectors while searches run
 * and publishes them between batches. */
lvq_status lvq_insert_deferred(lvq_store *store, const float *x, int64_t n, int64_t *out_ids,
                               lvq_stream_t stream);

/* Make slots written by lvq_insert_deferred visible.  ids: n int64; ids that
 * are out of range or not pending are ignored. */
lvq_status lvq_publish(lvq_store *store, const int64_t *ids, int64_t n, lvq_stream_t stream);

/* Delete slots (Sec. 2.1: X_t = X_{t-1} - {x}; lazy, App. A.2): from the
 * stream position of the call on, the slots are excluded from every result
 * and are free for later inserts.  Ids that are out of range, already free
 * or repeated are ignored.
 * ids: n int64.  out_n_deleted: 1 int64, receives the number freed. */
lvq_status lvq_delete(lvq_store *store, const int64_t *ids, int64_t n, int64_t *out_n_deleted,
                      lvq_stream_t stream);

/* Delete and hold (Sec. 2.1, lazy deletion of App. A.2): like lvq_delete,
 * but a slot that was live also stays unavailable to inserts until
 * lvq_release, so a search that still runs on an earlier visibility snapshot
 * (lvq_view_set_live) keeps reading the vector it sees there.
 * ids: n int64.  out_n_deleted: 1 int64 (device), receives the number of
 * live slots deleted. */
lvq_status lvq_delete_hold(lvq_store *store, const int64_t *ids, int64_t n, int64_t *out_n_deleted,
                           lvq_stream_t stream);

/* Free slots held by lvq_delete_hold: every slot among ids that is not live
 * and is reserved becomes free for inserts.  Pass only ids the caller held: a
 * slot written by lvq_insert_deferred and not yet published is also reserved
 * and not live, and would be freed too.  Ids out of range are ignored. */
lvq_status lvq_release(lvq_store *store, const int64_t *ids, int64_t n, lvq_stream_t stream);

/* Visibility snapshots.  The store's visibility is a bitmap of
 * ceil(capacity / 32) uint32 words (bit s % 32 of word s / 32 set: slot s is
 * live).  lvq_live_words returns that word count (host int64).
 * lvq_snapshot_live copies the current bitmap to dst (device, that many
 * words, caller-owned) in stream order.  lvq_view_set_live makes every
 * search through `view` (a handle from lvq_store_view) use the bitmap at
 * `live` (device, caller-owned, kept alive while searches use it) instead of
 * the store's; NULL restores the store's.  Updates through any handle act on
 * the store's own bitmap, never on a snapshot.  A search on a snapshot sees
 * exactly the slots live when it was taken, provided none of them has been
 * reused since (delete with lvq_delete_hold; release only after the last
 * search on the snapshot).  Returns LVQ_EINVAL for a handle that is not a
 * view. */
lvq_status lvq_live_words(const lvq_store *store, int64_t *out_words);
lvq_status lvq_snapshot_live(const lvq_store *store, uint32_t *dst, lvq_stream_t stream);
lvq_status lvq_view_set_live(lvq_store *view, const uint32_t *live);

/* M-LVQ centre update (Sec. 3.2, multi-means LVQ; re-encoding a centre's
 * vectors after an update is what makes M-LVQ suited to streaming data):
 * replace centre m by new_mean and re-encode every live slot tagged with m
 * against it, from the slot's float32 two-level reconstruction
 *   y = fl(fl(D c) + l) [+ fl(fl(D2 c2) + l2)],  x = fl(mu_m + y),
 * with the same per-vector encoding as lvq_insert; the tag stays m.  Other
 * slots are untouched.
 * new_mean: d float32 (device).  out_count: host int64, receives the number
 * of slots re-encoded.  Synchronises the stream once (to size the work);
 * no search or update of this store may run concurrently.  m outside
 * [0, n_means) returns LVQ_EINVAL. */
lvq_status lvq_update_mean(lvq_store *store, int32_t m, const float *new_mean, int64_t *out_count,
                           lvq_stream_t stream);

/* Greedy beam search over a caller-given graph (Alg. 1): per query a
 * search list of at most L nodes ordered by first-level score, seeded with
 * the start nodes; the best node not yet expanded is expanded (its live,
 * unseen out-neighbours are scored with the first level in float32) until
 * every listed node is expanded or max_expand expansions were made; the k1
 * best listed nodes are then re-ranked with both levels to k (k1 = 0 or a
 * store without a second level: the k best by first level).
 * graph: n_graph x R int32 out-neighbour ids (device; -1 = no edge; ids
 *   >= n_graph or deleted are skipped).  starts: n_starts int64 (device),
 *   1 <= n_starts <= L.  L: 1 .. 1024, >= k and k1.  max_expand: 0 = 4 L.
 * Outputs as in lvq_search_exhaustive.  LVQ_EINVAL when the seen-set of
 * (n_starts + R max_expand) ids does not fit in shared memory. */
lvq_status lvq_search_graph(const lvq_store *store, const float *q, int64_t nq, const int32_t *graph,
                            int64_t n_graph, int32_t R, const int64_t *starts, int32_t n_starts, int32_t L,
                            int32_t max_expand, int32_t k1, int32_t k, int64_t *out_ids, float *out_scores,
                            lvq_stream_t stream);

/* Exhaustive search over all live slots (Sec. 3.2 scoring, App. C re-rank).
 * q: nq x d float32 queries.
 * k1: first-level candidates per query, 1 .. 512; 0 (or a store without a
 *   second level) returns the k best first-level results directly.
 * k: results per query, 1 .. 512 and <= k1 when k1 > 0.
 * precision: lvq_precision of the first-level scan.
 * out_ids: nq x k int64; out_scores: nq x k float32.  Scores are the
 *   two-level distance / inner product when re-ranked, else first level. */
lvq_status lvq_search_exhaustive(const lvq_store *store, const float *q, int64_t nq, int32_t k1,
                                 int32_t k, int32_t precision, int64_t *out_ids,
                                 float *out_scores, lvq_stream_t stream);

/* lvq_search_exhaustive at LVQ_INT16 for 1 to 4 queries, with no device
 * memory allocated by the call.  The paper has no counterpart: it is a
 * systems entry point for callers that must not allocate on the call path,
 * because cudaMalloc/cudaFree there can synchronise the device and stall for
 * milliseconds (a latency-bound serving thread) or fail once the process has
 * given the rest of device memory to stores (lvq_search_exhaustive grows the
 * store's scratch on demand).
 * Scratch: a 4 MiB file-scope __device__ array of the library, one per
 *   device, whose address is looked up (cudaGetSymbolAddress) on the first
 *   call on each device; make that first call before any stream capture.
 *   Nothing in it needs to start at zero.  Calls whose device work can
 *   overlap (other streams, other stores on the same device) race on it:
 *   issue them in order on one stream.
 * Arguments and outputs as in lvq_search_exhaustive; nq outside 1 .. 4, a
 * store or k1 the integer scan does not take, or a plan larger than the
 * array return LVQ_EINVAL with a message (lvq_last_error). */
lvq_status lvq_search_exhaustive_static(const lvq_store *store, const float *q, int64_t nq, int32_t k1,
                                        int32_t k, int64_t *out_ids, float *out_scores,
                                        lvq_stream_t stream);

/* First stage alone: the k1 best live slots of each query by first-level
 * score, sorted, with their first-level scores (nq x k1 each). */
lvq_status lvq_search_first_level(const lvq_store *store, const float *q, int64_t nq, int32_t k1,
                                  int32_t precision, int64_t *out_ids, float *out_scores,
                                  lvq_stream_t stream);

/* ID-gather form: the search restricted to each query's candidate list, the
 * frontier-scoring step of greedy graph search (Alg. 1).  Float32 scoring.
 * cand: nq x n_cand int64 slot ids; -1, out-of-range, deleted and repeated
 *   ids are skipped.  n_cand: 1 .. 65536.  k1, k, outputs as in
 *   lvq_search_exhaustive. */
lvq_status lvq_search_candidates(const lvq_store *store, const float *q, int64_t nq,
                                 const int64_t *cand, int32_t n_cand, int32_t k1, int32_t k,
                                 int64_t *out_ids, float *out_scores, lvq_stream_t stream);

/* Re-rank given candidates with both levels (Sec. 2.2, App. C), float32.
 * ids: nq x k1 int64 (-1, out-of-range, deleted and repeated ids skipped).
 * k <= k1 <= 4096.  Outputs nq x k.  Needs a store with a residual level. */
lvq_status lvq_rerank(const lvq_store *store, const float *q, int64_t nq, const int64_t *ids,
                      int32_t k1, int32_t k, int64_t *out_ids, float *out_scores,
                      lvq_stream_t stream);

/* Read stored records back in the lvq_encode layout (one code per byte).
 * ids: n int64 live slots.  codes2 may be NULL.  A slot that is not live
 * yields zeros and records LVQ_ENOTFOUND (sticky). */
lvq_status lvq_export(const lvq_store *store, const int64_t *ids, int64_t n, uint8_t *codes1,
                      uint8_t *codes2, float *lower, float *step, uint8_t *mean_id,
                      lvq_stream_t stream);

/* Synchronise the stream, then report the number of live slots (host int64)
 * and return the first recorded device error (LVQ_OK if none; clears it). */
lvq_status lvq_stats(const lvq_store *store, int64_t *n_live_host, lvq_stream_t stream);

/* Pre-size the store's scratch memory for calls with up to max_nq queries,
 * k1 <= max_k1 and n_cand <= max_cand, so that later calls allocate nothing
 * (needed before capturing them in a CUDA graph). */
lvq_status lvq_reserve(lvq_store *store, int64_t max_nq, int32_t max_k1, int32_t max_cand);

/* Set / read the scan tile shapes (lvq_tuning). */
lvq_status lvq_set_tuning(lvq_store *store, const lvq_tuning *tuning);
lvq_status lvq_get_tuning(const lvq_store *store, lvq_tuning *tuning);

/* Per-kernel timing of the store's own launches, for benchmarks.  While
 * enabled, every kernel launch of a call on this store is bracketed by CUDA
 * events recorded on the call's stream.  lvq_profile_read synchronises the
 * device and returns, per kind (lvq_kernel_kind), the summed elapsed
 * milliseconds and the launch count since the last read, then resets them.
 * ms and launches: host arrays of n_kinds entries (n_kinds <= LVQ_KERNEL_KINDS). */
typedef enum {
  LVQ_K_PREP = 0,       /* query preparation (sums, norms, <q, mu_m>, rounding) */
  LVQ_K_SCAN_FP32 = 1,  /* float32 first-level scan */
  LVQ_K_SCAN_MMA = 2,   /* tcgen05 first-level scan */
  LVQ_K_MERGE = 3,      /* per-query merge of split lists (+ re-rank) */
  LVQ_K_GATHER = 4,     /* ID-gather search */
  LVQ_K_RERANK = 5,     /* lvq_rerank */
  LVQ_K_INSERT = 6,     /* slot allocation, encoding, publication */
  LVQ_K_DELETE = 7,     /* deletes */
  LVQ_K_SCAN_SMALL = 8,  /* small-batch integer first-level scan */
  LVQ_KERNEL_KINDS = 9
} lvq_kernel_kind;
lvq_status lvq_profile_enable(lvq_store *store, int32_t on);
lvq_status lvq_profile_read(lvq_store *store, double *ms, int64_t *launches, int32_t n_kinds);

/* Synchronise the device, copy the last error message (NUL-terminated, at
 * most len bytes) and return the first recorded error, clearing it. */
lvq_status lvq_last_error(const lvq_store *store, char *buf, size_t len);

/* Human-readable name of a status code (static storage). */
const char *lvq_status_string(lvq_status status);

#ifdef __cplusplus
}
#endif

#endif /* LVQ_H */
