// The multi-RHS solvers instantiated for D = 7, 8.
#include "mrhs_impl.cuh"

namespace bfmri {
BFMRI_MRHS_INSTANTIATE(7)
BFMRI_MRHS_INSTANTIATE(8)
}  // namespace bfmri
