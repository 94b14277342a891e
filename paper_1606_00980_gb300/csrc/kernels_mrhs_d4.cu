// The multi-RHS solvers instantiated for D = 4, 5.
#include "mrhs_impl.cuh"

namespace bfmri {
BFMRI_MRHS_INSTANTIATE(4)
BFMRI_MRHS_INSTANTIATE(5)
}  // namespace bfmri
