// Persistent batched launch (placeholder).
#include "mr_internal.h"
namespace mrgb {
uint64_t batch_tiles_for(uint32_t, uint64_t) { return 1; }
cudaError_t launch_batch(const BatchJob*, uint32_t, uint64_t, unsigned long long*, const DevInfo&, cudaStream_t) {
  return cudaErrorNotSupported;
}
}  // namespace mrgb
