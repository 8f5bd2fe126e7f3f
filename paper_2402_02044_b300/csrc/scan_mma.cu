// tcgen05 tensor-core first-level scan (placeholder until the kernel lands).
#include "kernels.cuh"

namespace lvq {

bool mma_supported(const DeviceStore&) { return false; }
size_t mma_scan_cand_bytes(int, int, int) { return 0; }
cudaError_t launch_scan_mma(const DeviceStore&, int64_t, const QueryPrep&, int, const ScanPlan&, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace lvq
