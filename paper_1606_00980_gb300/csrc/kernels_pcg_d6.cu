// The persistent PCG solvers instantiated for D = 6.
#include "pcg_impl.cuh"

namespace bfmri {
BFMRI_PCG_INSTANTIATE(6)
}  // namespace bfmri
