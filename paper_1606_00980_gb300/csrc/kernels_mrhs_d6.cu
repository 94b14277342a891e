// The multi-RHS solvers instantiated for D = 6.
#include "mrhs_impl.cuh"

namespace bfmri {
BFMRI_MRHS_INSTANTIATE(6)
}  // namespace bfmri
