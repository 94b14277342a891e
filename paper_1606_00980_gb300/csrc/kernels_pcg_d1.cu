// The persistent PCG solvers instantiated for D = 1, 2, 3.
#include "pcg_impl.cuh"

namespace bfmri {
BFMRI_PCG_INSTANTIATE(1)
BFMRI_PCG_INSTANTIATE(2)
BFMRI_PCG_INSTANTIATE(3)
}  // namespace bfmri
