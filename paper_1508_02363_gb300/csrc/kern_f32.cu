// FP32 (complex64) instantiations: the inner Krylov solve of the mixed-precision path.
#include "kern_impl.cuh"

namespace dbar {
DBAR_INSTANTIATE(float, float)
}  // namespace dbar
