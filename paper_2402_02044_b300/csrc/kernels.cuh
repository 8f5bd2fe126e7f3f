// Launchers of the LVQ kernels (called by the C ABI in lvq_api.cu).
#pragma once

#include <cuda.h>

#include "lvq_internal.cuh"

namespace lvq {

struct EncodeOut {
  // plain layout (lvq_encode); unused when slots != nullptr
  uint8_t* codes1 = nullptr;
  uint8_t* codes2 = nullptr;
  float* lower = nullptr;
  float* step = nullptr;
  uint8_t* mean_id = nullptr;
  // store layout (lvq_insert): vector i goes to slot slots[i]
  const int64_t* slots = nullptr;
  const int32_t* abort_flag = nullptr;  // set when the insert was abandoned
  int force_mean = -1;                  // >= 0: every vector takes this centre (no assignment)
};

cudaError_t launch_encode(const DeviceStore& st, const float* x, int64_t n, const EncodeOut& out,
                          cudaStream_t stream);
size_t alloc_scratch_bytes(int64_t capacity);
// M-LVQ local re-encode: the live slots below n_rows tagged with mean m go to
// list[0 .. *count) (count: one int64 that must start at zero)
cudaError_t launch_select_mean(const DeviceStore& st, int64_t n_rows, int m, int64_t* list,
                               unsigned long long* count, cudaStream_t stream);
// float32 reconstruction of slots list[0..n) with centre mu (d floats): x[i]
cudaError_t launch_reconstruct(const DeviceStore& st, const int64_t* list, int64_t n, const float* mu, float* x,
                               cudaStream_t stream);
cudaError_t launch_alloc_slots(const DeviceStore& st, int64_t n, int64_t* out_ids, int32_t* scratch,
                               int32_t* abort_flag, cudaStream_t stream);
cudaError_t launch_publish(const DeviceStore& st, const int64_t* ids, int64_t n, const int32_t* abort_flag,
                           int64_t* n_live, bool deferred, cudaStream_t stream);
cudaError_t launch_publish_reserved(const DeviceStore& st, const int64_t* ids, int64_t n, int64_t* n_live,
                                    cudaStream_t stream);
cudaError_t launch_delete(const DeviceStore& st, const int64_t* ids, int64_t n, int64_t* out_n,
                          unsigned long long* count, int64_t* n_live, cudaStream_t stream, bool hold);
cudaError_t launch_release(const DeviceStore& st, const int64_t* ids, int64_t n, cudaStream_t stream);
cudaError_t launch_export(const DeviceStore& st, const int64_t* ids, int64_t n, uint8_t* codes1,
                          uint8_t* codes2, float* lower, float* step, uint8_t* mean_id, cudaStream_t stream);

// ---- query preparation ------------------------------------------------------
// Per query: qsum = sum_j q_j, qnorm = ||q||^2, cm[m] = <q, mu_m> (float32),
// and q rounded to float16 into a zero-padded [nq_pad][kq] matrix.
// For the tensor-core scan (q16 != null) the float16 copy of dim j is scaled
// by 1/16 when B1 = 4 and j % 8 is 2, 3, 6 or 7 (those codes reach the tensor
// cores as 1024 + 16c, the others as 1024 + c); q16sum = sum of the stored
// float16 values, so that <q16, c> = acc - 1024 * q16sum.
struct QueryPrep {
  float* qsum;      // [nq]
  float* qnorm;     // [nq]
  float* cm;        // [nq][M]
  uint16_t* q16;    // [nq_pad][kq] (may be null)
  float* q16sum;    // [nq] (with q16)
  int64_t nq_pad;
  int kq;
};
cudaError_t launch_prep_queries(const DeviceStore& st, const float* q, int64_t nq, const QueryPrep& p,
                                cudaStream_t stream);

// ---- first-level scans ------------------------------------------------------
// Both scans write, for every (query, split), the split's k1 best keys in no
// particular order (kNoKey padded) to partial[(q * splits + split) * k1 + i].
struct ScanPlan {
  int splits;           // database splits
  int64_t n_rows;       // rows scanned: [0, n_rows)
  int k1;
  uint64_t* partial;    // [nq][splits][k1]
  uint64_t* cand;       // per-CTA candidate buffers
  int grid;             // persistent CTAs
  int* counts = nullptr;  // [nq][splits] valid keys per list (null: lists padded with kNoKey)
  uint64_t* gthr = nullptr;  // [nq] per-query bound shared by the CTAs of the tensor-core scan
  // tensor-core scan: [nq][splits][best_j] lowest keys of disjoint row sets
  // (rows of one segment, id mod best_j); best_j = 0 leaves them out
  uint64_t* seg_best = nullptr;
  int best_j = 0;
  uint32_t wait_polls = 0;   // polls of each pipeline wait of the tensor-core scan (0: the default)
};
constexpr int kMaxMergeLists = 1024;  // lists per query when counts are given

int fp32_scan_grid(const DeviceStore& st, int qb, int sm_count);
size_t fp32_scan_cand_bytes(int grid, int qb, int k1);
cudaError_t launch_scan_fp32(const DeviceStore& st, const float* q, int64_t nq, const QueryPrep& p,
                             int qb, const ScanPlan& plan, cudaStream_t stream);

// tcgen05 scan (scan_mma.cu)
size_t mma_scan_cand_bytes(int grid, int n_tile, int k1);
cudaError_t launch_scan_mma(const DeviceStore& st, int64_t nq, const QueryPrep& p, int n_tile,
                            const ScanPlan& plan, cudaStream_t stream);
bool mma_supported(const DeviceStore& st);
// TMA map of codes1 read in boxes of 128 rows x box_bytes (64: 64-byte
// swizzle, 128: 128-byte swizzle)
cudaError_t encode_code_map(const DeviceStore& st, CUtensorMap* cm, int box_bytes);
int mma_tile_limit(const DeviceStore& st);   // largest query tile whose queries fit in shared memory
// database segments per query tile: groups x segments is a multiple of grid
int mma_segments(int grid, int64_t groups, int64_t ntiles);   // segments per query tile in the partial lists

// small-batch integer scan (scan_small.cu): queries quantised to 16-bit
// integers (hi and lo bytes), codes as bytes, dp4a dot products on CUDA cores
constexpr int kSmallMaxQ = 4;
bool small_supported(const DeviceStore& st, int64_t nq, int k1);
size_t small_scratch_bytes(const DeviceStore& st, int64_t nq);
// rounds the queries to 16-bit integers into scratch (small_scratch_bytes)
cudaError_t launch_small_prep(const DeviceStore& st, const float* q, int64_t nq, void* scratch, cudaStream_t stream);
cudaError_t launch_scan_small(const DeviceStore& st, int64_t nq, const QueryPrep& p, const void* scratch,
                              const ScanPlan& plan, cudaStream_t stream);
// persistent CTAs of the small-batch scan: one per SM, at most one per tile
int small_grid(const DeviceStore& st, int64_t n_rows, int64_t nq, int k1, int sm_count);

// ---- greedy beam search over a graph (graph.cu) --------------------------------
// slots of the seen-set (power of two, at most half full) and shared memory
int beam_set_slots(int n_starts, int R, int max_expand);
size_t beam_smem(const DeviceStore& st, int L, int R, int H);
// first-level keys of the k1 best listed nodes per query into keys[nq][k1]
// (kNoKey pads) and their ids into ids[nq][k1] (-1 pads)
cudaError_t launch_beam(const DeviceStore& st, const float* q, int64_t nq, const int32_t* graph, int64_t n_graph,
                        int R, const int64_t* starts, int n_starts, int L, int max_expand, int k1, uint64_t* keys,
                        int64_t* ids, cudaStream_t stream);
cudaError_t launch_keys_to_results(const uint64_t* keys, int64_t nq, int k1, int k, int metric, int64_t* out_ids,
                                  float* out_scores, cudaStream_t stream);

// ---- selection and re-ranking ----------------------------------------------
// Merge the per-split lists of each query into its k1 best, then either write
// the k best (first level) or re-rank the k1 with both levels and write k.
cudaError_t launch_merge_rerank(const DeviceStore& st, const float* q, int64_t nq, const QueryPrep& p,
                                const uint64_t* partial, int splits, int k1, int k, bool rerank,
                                int64_t* out_ids, float* out_scores, cudaStream_t stream,
                                const int* counts = nullptr, int sm_count = 0);
cudaError_t launch_rerank(const DeviceStore& st, const float* q, int64_t nq, const QueryPrep& p,
                          const int64_t* ids, int k1, int k, int64_t* out_ids, float* out_scores,
                          cudaStream_t stream);
// Geometry of the ID-gather kernel's row ring: R rows per batch (32 / R lanes
// a row), slot stride (bytes), slot size, P slots per warp, dynamic shared
// memory in bytes.
struct GatherGeom {
  int R, stride, slot_bytes, P;
  size_t smem;
};
constexpr int kGatherSlotBudget = 13312;
constexpr size_t kGatherSmemBudget = 226 * 1024;
GatherGeom gather_geom(int row1, int d, int k);
cudaError_t launch_gather(const DeviceStore& st, const float* q, int64_t nq, const QueryPrep& p,
                          const int64_t* cand, int n_cand, int k, int64_t* out_ids, float* out_scores,
                          cudaStream_t stream);

}  // namespace lvq
