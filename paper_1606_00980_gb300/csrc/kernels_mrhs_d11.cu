// The multi-RHS solvers instantiated for D = 11, 12.
#include "mrhs_impl.cuh"

namespace bfmri {
BFMRI_MRHS_INSTANTIATE(11)
BFMRI_MRHS_INSTANTIATE(12)
}  // namespace bfmri
