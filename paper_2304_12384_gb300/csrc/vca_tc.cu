// Tensor-core form of the analyzer (placeholder until the tcgen05 kernel lands).
#include "vca_internal.h"

namespace vca {

bool tc_supported(const Geometry&) { return false; }

cudaError_t launch_tc(const Geometry&, const FramePlanes&, int, const DeviceTables&, float*, int16_t* const[3],
                      cudaStream_t, int64_t*) {
  return cudaErrorNotSupported;
}

}  // namespace vca
