// The persistent PCG solvers instantiated for D = 4, 5.
#include "pcg_impl.cuh"

namespace bfmri {
BFMRI_PCG_INSTANTIATE(4)
BFMRI_PCG_INSTANTIATE(5)
}  // namespace bfmri
