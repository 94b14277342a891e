// The persistent PCG solvers instantiated for D = 9, 10, 11, 12.
#include "pcg_impl.cuh"

namespace bfmri {
BFMRI_PCG_INSTANTIATE(9)
BFMRI_PCG_INSTANTIATE(10)
BFMRI_PCG_INSTANTIATE(11)
BFMRI_PCG_INSTANTIATE(12)
}  // namespace bfmri
