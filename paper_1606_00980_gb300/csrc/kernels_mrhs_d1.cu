// The multi-RHS solvers instantiated for D = 1, 2, 3.
#include "mrhs_impl.cuh"

namespace bfmri {
BFMRI_MRHS_INSTANTIATE(1)
BFMRI_MRHS_INSTANTIATE(2)
BFMRI_MRHS_INSTANTIATE(3)
}  // namespace bfmri
