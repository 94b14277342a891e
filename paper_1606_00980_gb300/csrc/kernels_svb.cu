// Spatial variational Bayes (Section 3.3; Appendix B, Eq. NFVBw and NFVBbB): the expectations
// over W and A are Monte Carlo averages over N_s samples paired by index (Eq. MC approx).
//  * E[c c'] of the whitening coefficients c = (1, -a) over the A samples turns the
//    statistics into the averaged W system (the W blocks are quadratic in a);
//  * the lagged residual Gram averaged over the W samples gives the averaged A system;
//  * the N_s perturbed right-hand sides use the same random numbers at every iteration
//    (stream = sample index, fixed draw counter), so previous samples are good warm starts;
//  * E[lambda_n] and the per-regressor quadratic forms average over the sample pairs.
#include "model.cuh"

namespace bfmri {

namespace {
constexpr int SVB_THREADS = 128;
}

__global__ void __launch_bounds__(SVB_THREADS) k_svb_cmom(SvbArgs a) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.g.N) return;
  const int P = a.P;
  const size_t ld = a.g.ld;
  double acc[PMAX + 1][PMAX + 1];
#pragma unroll
  for (int p = 0; p <= PMAX; ++p)
#pragma unroll
    for (int q = 0; q <= PMAX; ++q) acc[p][q] = 0.0;
  for (int j = 0; j < a.S; ++j) {
    double c[PMAX + 1];
    c[0] = 1.0;
#pragma unroll
    for (int p = 1; p <= PMAX; ++p) c[p] = p <= P ? -a.As[(size_t)j * P * ld + (size_t)(p - 1) * ld + n] : 0.0;
#pragma unroll
    for (int p = 0; p <= PMAX; ++p)
#pragma unroll
      for (int q = p; q <= PMAX; ++q) acc[p][q] += c[p] * c[q];
  }
  const double inv = 1.0 / (double)a.S;
#pragma unroll
  for (int p = 0; p <= PMAX; ++p)
#pragma unroll
    for (int q = p; q <= PMAX; ++q)
      if (q <= P) a.Cmom[(size_t)syy_index(p, q, P) * ld + n] = acc[p][q] * inv;
}

template <int K>
__global__ void __launch_bounds__(SVB_THREADS) k_svb_gram(SvbArgs a) {
  extern __shared__ double shQ[];
  const int P = a.P;
  load_quad_weights(a.Sxx, K, P, shQ);
  __syncthreads();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.g.N) return;
  const size_t ld = a.g.ld;
  double acc[PMAX + 1][PMAX + 1];
#pragma unroll
  for (int p = 0; p <= PMAX; ++p)
#pragma unroll
    for (int q = 0; q <= PMAX; ++q) acc[p][q] = 0.0;
  for (int j = 0; j < a.S; ++j) {
    double w[K], G[PMAX + 1][PMAX + 1];
#pragma unroll
    for (int k = 0; k < K; ++k) w[k] = a.Ws[(size_t)j * K * ld + (size_t)k * ld + n];
    lagged_gram<K>(a.stats, shQ, w, P, ld, n, G);
#pragma unroll
    for (int p = 0; p <= PMAX; ++p)
#pragma unroll
      for (int q = p; q <= PMAX; ++q) acc[p][q] += G[p][q];
  }
  const double inv = 1.0 / (double)a.S;
#pragma unroll
  for (int p = 0; p <= PMAX; ++p)
#pragma unroll
    for (int q = p; q <= PMAX; ++q)
      if (q <= P) a.Gin[(size_t)syy_index(p, q, P) * ld + n] = acc[p][q] * inv;
}

// rhs_j = bmean + L z2_j + sum_k sqrt(s_k) (G'z1_j)_k with stream j (Algorithm 2).
template <int D>
__global__ void __launch_bounds__(SVB_THREADS) k_svb_rhs(SvbArgs a) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (n >= a.g.N) return;
  const size_t ld = a.g.ld;
  Rng g = a.rng;
  g.c3 = (a.rng.c3 & 0xFF000000u) | ((uint32_t)j & 0xFFFFFFu);
  double L[ntri(D)], z[D], Lz[D], rhs[D], sq[D];
#pragma unroll
  for (int e = 0; e < ntri(D); ++e) L[e] = __ldg(a.ldata + (size_t)e * ld + n);
  const int lin = a.g.lin[n];
  site_normals<D>(g, (uint32_t)lin * 4u + 3u, z);
  lower_mul_invdiag<D>(L, z, Lz);
#pragma unroll
  for (int k = 0; k < D; ++k) {
    rhs[k] = __ldg(a.bmean + (size_t)k * ld + n) + Lz[k];
    sq[k] = sqrt(a.scale[k]);
  }
  if (a.spatial) add_edge_noise<D>(a.g, g, n, lin, sq, rhs);
#pragma unroll
  for (int k = 0; k < D; ++k) a.rhs[(size_t)j * a.vs + (size_t)k * ld + n] = rhs[k];
}

// E[lambda_n] = u~2 / (1/u1 + mean_j RSS_n(W^(j), A^(j)) / 2)
template <int K>
__global__ void __launch_bounds__(SVB_THREADS) k_svb_lambda(SvbArgs a) {
  extern __shared__ double shQ[];
  const int P = a.P;
  load_quad_weights(a.Sxx, K, P, shQ);
  __syncthreads();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.g.N) return;
  const size_t ld = a.g.ld;
  double sum = 0.0;
  for (int j = 0; j < a.S; ++j) {
    double w[K], G[PMAX + 1][PMAX + 1], c[PMAX + 1];
#pragma unroll
    for (int k = 0; k < K; ++k) w[k] = a.Ws[(size_t)j * K * ld + (size_t)k * ld + n];
    lagged_gram<K>(a.stats, shQ, w, P, ld, n, G);
    c[0] = 1.0;
#pragma unroll
    for (int p = 1; p <= PMAX; ++p) c[p] = p <= P ? -a.As[(size_t)j * P * ld + (size_t)(p - 1) * ld + n] : 0.0;
    double rss = 0.0;
#pragma unroll
    for (int p = 0; p <= PMAX; ++p)
#pragma unroll
      for (int q = 0; q <= PMAX; ++q)
        if (p <= P && q <= P) rss += c[p] * c[q] * G[p][q];
    sum += rss;
  }
  const double shape = 0.5 * (double)(a.T - P) + a.u2;
  a.lam[n] = shape / (1.0 / a.u1 + 0.5 * sum / (double)a.S);
}

// per-CTA partial sums of sum_j sum_edges (v_j,i - v_j,m)^2 for each component
template <int D>
__global__ void __launch_bounds__(SVB_THREADS) k_svb_quad(SvbArgs a, const double* V) {
  __shared__ double sh[SVB_THREADS][D];
  double acc[D];
#pragma unroll
  for (int k = 0; k < D; ++k) acc[k] = 0.0;
  const size_t ld = a.g.ld;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < a.g.N; n += gridDim.x * blockDim.x) {
    for (int d = 0; d < a.g.ndir / 2; ++d) {
      const int m = __ldg(a.g.nbr + (size_t)(2 * d + 1) * ld + n);
      if (m < 0) continue;
      const double c = a.g.cw[d];
      for (int j = 0; j < a.S; ++j) {
        const double* v = V + (size_t)j * D * ld;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const double df = v[(size_t)k * ld + n] - v[(size_t)k * ld + m];
          acc[k] += c * df * df;
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < D; ++k) sh[threadIdx.x][k] = acc[k];
  __syncthreads();
  for (int off = SVB_THREADS / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off)
#pragma unroll
      for (int k = 0; k < D; ++k) sh[threadIdx.x][k] += sh[threadIdx.x + off][k];
    __syncthreads();
  }
  if ((int)threadIdx.x < D) a.part[(size_t)blockIdx.x * D + threadIdx.x] = sh[0][threadIdx.x];
}

#define BFMRI_SVB_CASES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12)

template <int D>
static cudaError_t svb_d(int what, const SvbArgs& a, cudaStream_t s, int* grid_out) {
  const int blocks = (a.g.N + SVB_THREADS - 1) / SVB_THREADS;
  const size_t shm = quad_weight_doubles(D, a.P) * sizeof(double);
  switch (what) {
    case 1:
      if (cudaError_t e = raise_smem_limit((const void*)k_svb_gram<D>, shm)) return e;
      k_svb_gram<D><<<blocks, SVB_THREADS, shm, s>>>(a);
      break;
    case 2:
      k_svb_rhs<D><<<dim3(blocks, a.S), SVB_THREADS, 0, s>>>(a);
      break;
    case 3:
      if (cudaError_t e = raise_smem_limit((const void*)k_svb_lambda<D>, shm)) return e;
      k_svb_lambda<D><<<blocks, SVB_THREADS, shm, s>>>(a);
      break;
    case 4:
    case 5: {
      const int grid = blocks < 1024 ? (blocks < 1 ? 1 : blocks) : 1024;
      if (grid_out) *grid_out = grid;
      k_svb_quad<D><<<grid, SVB_THREADS, 0, s>>>(a, what == 4 ? a.Ws : a.As);
      break;
    }
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_svb(int what, int D, const SvbArgs& a, cudaStream_t s, int* grid_out) {
  if (a.g.N <= 0) return cudaSuccess;
  if (what == 0) {
    k_svb_cmom<<<(a.g.N + SVB_THREADS - 1) / SVB_THREADS, SVB_THREADS, 0, s>>>(a);
    return cudaGetLastError();
  }
  switch (D) {
#define CASE(d) case d: return svb_d<d>(what, a, s, grid_out);
    BFMRI_SVB_CASES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bfmri
