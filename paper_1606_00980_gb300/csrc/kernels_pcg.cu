// Dispatch of the persistent PCG solvers by the block dimension D. The kernels and their
// launchers are in pcg_impl.cuh; kernels_pcg_d*.cu instantiate them for groups of D, so that
// the solvers compile as several parallel jobs.
#include "pcg.cuh"

namespace bfmri {

namespace pcg_detail {
template <int D>
cudaError_t launch_d(const PcgArgs& a, cudaStream_t stream, int* grid_out);
template <int D>
int max_grid_d();
template <int D>
cudaError_t precond_apply_d(const PcgArgs& a, cudaStream_t stream);
}  // namespace pcg_detail

int resident_voxels_per_cta(int N, int sm_cap) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int grid = (sm_cap > 0 && sm_cap < nsm) ? sm_cap : nsm;
  if ((N + 63) / 64 < grid) grid = (N + 63) / 64;
  if (grid < 1) grid = 1;
  return (N + grid - 1) / grid;
}

#define BFMRI_PCG_CASES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12)

cudaError_t launch_precond_apply(int D, const PcgArgs& a, cudaStream_t stream) {
  switch (D) {
#define CASE(d) case d: return pcg_detail::precond_apply_d<d>(a, stream);
    BFMRI_PCG_CASES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_pcg(int D, const PcgArgs& a, cudaStream_t stream, int* grid_out) {
  switch (D) {
#define CASE(d) case d: return pcg_detail::launch_d<d>(a, stream, grid_out);
    BFMRI_PCG_CASES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

int pcg_max_grid(int D) {
  switch (D) {
#define CASE(d) case d: return pcg_detail::max_grid_d<d>();
    BFMRI_PCG_CASES(CASE)
#undef CASE
    default: return 0;
  }
}

}  // namespace bfmri
