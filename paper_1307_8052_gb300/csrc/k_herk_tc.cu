// Tensor-core (tcgen05) grouped Hermitian rank-k update: placeholder until the
// split-bfloat16 kernel lands; the host rejects the BF16 modes meanwhile.
#include "rpa_internal.h"

namespace rpa {
size_t herk_tc_scratch_bytes(int64_t, int, int, int) { return 0; }
cudaError_t launch_herk_tc(const float2*, int64_t, int, const float*, int, int, double2*, void*, size_t,
                           cudaStream_t) {
  return cudaErrorNotSupported;
}
}  // namespace rpa
