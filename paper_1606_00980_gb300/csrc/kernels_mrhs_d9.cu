// The multi-RHS solvers instantiated for D = 9, 10.
#include "mrhs_impl.cuh"

namespace bfmri {
BFMRI_MRHS_INSTANTIATE(9)
BFMRI_MRHS_INSTANTIATE(10)
}  // namespace bfmri
