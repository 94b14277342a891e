// The persistent PCG solvers instantiated for D = 7, 8.
#include "pcg_impl.cuh"

namespace bfmri {
BFMRI_PCG_INSTANTIATE(7)
BFMRI_PCG_INSTANTIATE(8)
}  // namespace bfmri
