// BF16 tensor-core distance pass for k-means (placeholder until it lands).
#include "mr_internal.h"
namespace mrgb {
bool km_tc_supported(uint32_t, uint32_t) { return false; }
cudaError_t launch_kmeans_tc_assign(const float*, uint32_t, uint32_t, const float*, uint32_t, KmBuffers&,
                                    const DevInfo&, cudaStream_t, uint64_t*) {
  return cudaErrorNotSupported;
}
}  // namespace mrgb
