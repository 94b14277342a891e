// Multi-right-hand-side PCG (one matrix, S right-hand sides) in one cooperative launch.
// Used by the log-determinant / trace probes and by the spatial-VB step, whose N_s samples
// all solve with the one matrix B~_SVB and so can share its preconditioner (Section 3.3).
//
// Work decomposition: the grid's warps are split into S x C units (right-hand side r, voxel
// chunk c); lanes of a warp take consecutive voxels of the chunk, so every vector access is
// coalesced, and each unit produces one row of partial sums. At each reducing barrier the CTA
// that arrives last sums the rows of every right-hand side in a fixed order and advances its
// CG scalars (Chronopoulos-Gear recurrence, as in the single solve), records the CG
// coefficients (alpha_j, beta_j) of the first run for Lanczos quadrature, and marks converged
// right-hand sides, which then stop moving. Converged right-hand sides are confirmed with the
// true residual b - B~ x before they are released.
// The kernels and launchers are in mrhs_impl.cuh, instantiated for groups of D in
// kernels_mrhs_d*.cu; this file dispatches by D and holds the probe kernels.
#include "mrhs.cuh"

namespace bfmri {

namespace mrhs_detail {
template <int D>
cudaError_t launch_d(const MrhsArgs& a, cudaStream_t stream, int* units_out);
template <int D>
int max_units_d(int S);
}  // namespace mrhs_detail

#define BFMRI_MRHS_CASES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12)

cudaError_t launch_mrhs(int D, const MrhsArgs& a, cudaStream_t stream, int* units_out) {
  switch (D) {
#define CASE(d) case d: return mrhs_detail::launch_d<d>(a, stream, units_out);
    BFMRI_MRHS_CASES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

int mrhs_max_units(int D, int S) {
  switch (D) {
#define CASE(d) case d: return mrhs_detail::max_units_d<d>(S);
    BFMRI_MRHS_CASES(CASE)
#undef CASE
    default: return 0;
  }
}

}  // namespace bfmri

// ---------------------------------------------------------------------------------------
// Probe right-hand sides, log det of the preconditioner, and trace terms.
// ---------------------------------------------------------------------------------------
namespace bfmri {

// element (i, k, n) of a probe vector in the layout of ProbeArgs.tile
__device__ __forceinline__ size_t probe_idx(const ProbeArgs& a, int D, int i, int k, int n) {
  if (a.tile > 1)
    return (size_t)(i / a.tile) * ((size_t)D * a.ld * a.tile) + ((size_t)k * a.ld + n) * a.tile + (i % a.tile);
  return (size_t)i * a.vs + (size_t)k * a.ld + n;
}

// b_i = L v_i (v_i Rademacher, site lattice-linear * 4 + 3, stream i), x_i = 0.
template <int D, typename T>
__global__ void k_probe_rhs(ProbeArgs a) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (n >= a.N) return;
  Rng g = a.rng;
  g.c3 = (a.rng.c3 & 0xFF000000u) | ((uint32_t)i & 0xFFFFFFu);
  double v[D], bv[D];
  site_rademacher<D>(g, (uint32_t)a.lin[n] * 4u + 3u, v);
  if (a.mfac64) {
    double L[ntri(D)];
#pragma unroll
    for (int e = 0; e < ntri(D); ++e) L[e] = a.mfac64[(size_t)e * a.ld + n];
    lower_mul_invdiag<D>(L, v, bv);
  } else {
#pragma unroll
    for (int k = 0; k < D; ++k) bv[k] = v[k];
  }
  T* b = static_cast<T*>(a.b);
  T* x = static_cast<T*>(a.x);
#pragma unroll
  for (int k = 0; k < D; ++k) {
    b[probe_idx(a, D, i, k, n)] = (T)bv[k];
    x[probe_idx(a, D, i, k, n)] = T(0);
  }
}

// per-voxel log det of the preconditioner block: 2 sum_k log L_kk (stored inverted)
template <int D>
__global__ void k_logdet_m(ProbeArgs a, double* out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.N) return;
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) s -= 2.0 * log(a.mfac64[(size_t)tri(k, k) * a.ld + n]);
  out[n] = s;
}

// Trace terms t_{i,k} = sum_n (L^-T v_i)_{n,k} (D_w y_{i,k})_n with y_i = B~^-1 L v_i, whose
// mean over probes estimates tr(D_w^(k) B~^-1) (cyclic invariance: E[L^-T v v' L'] = I).
// Per-CTA partials [grid.x][S][D] in a fixed order.
template <int D, typename T>
__global__ void k_probe_traces(ProbeArgs a, double* part) {
  __shared__ double sh[128][D];
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  double c[D];
#pragma unroll
  for (int k = 0; k < D; ++k) c[k] = 0.0;
  if (n < a.N) {
    Rng g = a.rng;
    g.c3 = (a.rng.c3 & 0xFF000000u) | ((uint32_t)i & 0xFFFFFFu);
    double v[D], t[D];
    site_rademacher<D>(g, (uint32_t)a.lin[n] * 4u + 3u, v);
    if (a.mfac64) {
      double L[ntri(D)];
#pragma unroll
      for (int e = 0; e < ntri(D); ++e) L[e] = a.mfac64[(size_t)e * a.ld + n];
      // solve L' t = v (L lower, inverted diagonal)
#pragma unroll
      for (int r = D - 1; r >= 0; --r) {
        double acc = v[r];
#pragma unroll
        for (int j = r + 1; j < D; ++j) acc -= L[tri(j, r)] * t[j];
        t[r] = acc * L[tri(r, r)];
      }
    } else {
#pragma unroll
      for (int k = 0; k < D; ++k) t[k] = v[k];
    }
    const T* y = static_cast<const T*>(a.x);
    double yn[D], sum[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      yn[k] = (double)y[probe_idx(a, D, i, k, n)];
      sum[k] = 0.0;
    }
    double deg = 0.0;
    for (int d = 0; d < a.ndir; ++d) {
      const int m = a.nbr[(size_t)d * a.ld + n];
      if (m >= 0) {
        const double cd = a.cw[d >> 1];
        deg += cd;
#pragma unroll
        for (int k = 0; k < D; ++k) sum[k] += cd * (double)y[probe_idx(a, D, i, k, m)];
      }
    }
#pragma unroll
    for (int k = 0; k < D; ++k) c[k] = t[k] * (deg * yn[k] - sum[k]);
  }
#pragma unroll
  for (int k = 0; k < D; ++k) sh[threadIdx.x][k] = c[k];
  __syncthreads();
  for (int off = 64; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) {
#pragma unroll
      for (int k = 0; k < D; ++k) sh[threadIdx.x][k] += sh[threadIdx.x + off][k];
    }
    __syncthreads();
  }
  if (threadIdx.x < D) part[((size_t)blockIdx.x * a.S + i) * D + threadIdx.x] = sh[0][threadIdx.x];
}

template <int D>
static cudaError_t probe_launch_d(const ProbeArgs& a, int what, double* out, cudaStream_t s) {
  const dim3 grid((a.N + 127) / 128, a.S);
  if (what == 0) {
    if (a.f32) k_probe_rhs<D, float><<<grid, 128, 0, s>>>(a);
    else k_probe_rhs<D, double><<<grid, 128, 0, s>>>(a);
  } else if (what == 1) {
    k_logdet_m<D><<<(a.N + 127) / 128, 128, 0, s>>>(a, out);
  } else {
    if (a.f32) k_probe_traces<D, float><<<grid, 128, 0, s>>>(a, out);
    else k_probe_traces<D, double><<<grid, 128, 0, s>>>(a, out);
  }
  return cudaGetLastError();
}

// out[c] = sum over g of in[g * C + c], one CTA per column, each thread summing the rows
// t, t + 256, ... in order and the CTA combining its threads in a fixed tree: deterministic.
__global__ void __launch_bounds__(256) k_sum_columns(const double* __restrict__ in, int G, int C,
                                                      double* __restrict__ out) {
  __shared__ double sh[256];
  const int c = blockIdx.x;
  double acc = 0.0;
  for (int g = threadIdx.x; g < G; g += 256) acc += in[(size_t)g * C + c];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = sh[0];
}

cudaError_t launch_sum_columns(const double* in, int G, int C, double* out, cudaStream_t s) {
  if (C < 1) return cudaSuccess;
  k_sum_columns<<<C, 256, 0, s>>>(in, G, C, out);
  return cudaGetLastError();
}

cudaError_t launch_probe(int D, const ProbeArgs& a, int what, double* out, cudaStream_t s) {
  switch (D) {
#define CASE(d) case d: return probe_launch_d<d>(a, what, out, s);
    BFMRI_MRHS_CASES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bfmri
