// Host interface of the per-voxel model kernels: sufficient statistics, assembly of the W and
// A full conditionals with the Algorithm 2 perturbation, and the Gamma full conditionals.
#pragma once

#include <vector>

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "device_common.cuh"

namespace bfmri {

constexpr int PMAX = 4;   // largest AR order
constexpr int KMAX = 12;  // largest number of regressors

// Layout of the per-voxel statistics record (planes of length ld):
//   Syy[p][q] (p <= q)      plane syy_index(p, q)
//   Sxy[p][q][k]            plane n_syy(P) + (p (P+1) + q) K + k
__host__ __device__ inline int n_syy(int P) { return (P + 1) * (P + 2) / 2; }
__host__ __device__ inline int syy_index(int p, int q, int P) {
  // row-major over p of the upper triangle p <= q
  return p * (P + 1) - p * (p - 1) / 2 + (q - p);
}
__host__ __device__ inline int n_stats(int K, int P) { return n_syy(P) + K * (P + 1) * (P + 1); }
__host__ __device__ inline size_t sxy_plane(int p, int q, int k, int K, int P) {
  return (size_t)(n_syy(P) + (p * (P + 1) + q) * K + k);
}

struct Geometry {
  int N;
  size_t ld;
  int ndir;           // 4 or 6
  const int* nbr;     // [6][ld]
  const int* lin;     // [ld] lattice-linear index of each voxel
  int stride[3];      // lattice-linear strides of +x, +y, +z
  double cw[3];       // edge weights of the x, y, z directions (weighted graph Laplacian;
                      // 1, 1, 1 is the UGL prior); neighbour slot d has weight cw[d / 2]
  const unsigned short* ce;   // [3][ld] BF16 factors of the edge from each voxel along +x, +y,
                              // +z (a general diagonal C: C_e = cw[d] * factor), or null (all 1)
};

// the FP64 value of a BF16 number (its bits are the high half of an FP32)
__device__ __forceinline__ double bf16_value(unsigned short b) {
  return (double)__uint_as_float((unsigned)b << 16);
}

// weight of the edge between voxel n and its in-mask neighbour m in slot d (-x, +x, -y, +y,
// -z, +z): the edge's factor is stored at its lower voxel, n for +d and m for -d
__device__ __forceinline__ double slot_weight(const Geometry& g, int n, int d, int m) {
  double c = g.cw[d >> 1];
  if (g.ce) c *= bf16_value(__ldg(g.ce + (size_t)(d >> 1) * g.ld + ((d & 1) ? n : m)));
  return c;
}

// ---------------------------------------------------------------------------------------
// Algorithm 2 perturbation for one voxel: rhs += sum_k sqrt(s_k) (G' z1_k)_n over the
// voxel's edges. Edge (i, i + stride_d) carries +z at i and -z at its upper endpoint; its
// normals come from site lattice-linear(i) * 4 + d.
// ---------------------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ void add_edge_noise(const Geometry& g, const Rng& rng, int n, int lin,
                                               const double* sq, double* rhs) {
  double z[D];
  for (int d = 0; d < g.ndir / 2; ++d) {
    const int mf = __ldg(g.nbr + (size_t)(2 * d + 1) * g.ld + n);
    if (mf >= 0) {
      site_normals<D>(rng, (uint32_t)lin * 4u + (uint32_t)d, z);
      const double c = sqrt(slot_weight(g, n, 2 * d + 1, mf));
#pragma unroll
      for (int k = 0; k < D; ++k) rhs[k] += c * sq[k] * z[k];
    }
    const int mb = __ldg(g.nbr + (size_t)(2 * d) * g.ld + n);
    if (mb >= 0) {
      site_normals<D>(rng, (uint32_t)(lin - g.stride[d]) * 4u + (uint32_t)d, z);
      const double c = sqrt(slot_weight(g, n, 2 * d, mb));
#pragma unroll
      for (int k = 0; k < D; ++k) rhs[k] -= c * sq[k] * z[k];
    }
  }
}

// The same sum from pre-generated edge terms E[d][k][n] = sqrt(s_k) z1_k of the edge from
// voxel n in direction +d (launch_edge_noise): + own forward edges, - backward neighbours'.
template <int D>
__device__ __forceinline__ void add_edge_terms(const Geometry& g, const double* __restrict__ E,
                                               int n, double* rhs) {
  for (int d = 0; d < g.ndir / 2; ++d) {
    if (__ldg(g.nbr + (size_t)(2 * d + 1) * g.ld + n) >= 0) {
#pragma unroll
      for (int k = 0; k < D; ++k) rhs[k] += __ldg(E + ((size_t)d * D + k) * g.ld + n);
    }
    const int m = __ldg(g.nbr + (size_t)(2 * d) * g.ld + n);
    if (m >= 0) {
#pragma unroll
      for (int k = 0; k < D; ++k) rhs[k] -= __ldg(E + ((size_t)d * D + k) * g.ld + m);
    }
  }
}

// weighted degree: sum of the edge weights of the in-mask neighbours
__device__ __forceinline__ double degree(const Geometry& g, int n) {
  double deg = 0.0;
  for (int d = 0; d < g.ndir; ++d) {
    const int m = __ldg(g.nbr + (size_t)d * g.ld + n);
    if (m >= 0) deg += slot_weight(g, n, d, m);
  }
  return deg;
}

// weighted degree along one direction (slots 2d and 2d + 1)
__device__ __forceinline__ double degree_dir(const Geometry& g, int n, int d) {
  double deg = 0.0;
  for (int s = 2 * d; s <= 2 * d + 1; ++s) {
    const int m = __ldg(g.nbr + (size_t)s * g.ld + n);
    if (m >= 0) deg += slot_weight(g, n, s, m);
  }
  return deg;
}

// diagonal of L'L at voxel n (L the weighted graph Laplacian): deg_n^2 + sum of the squared
// weights of the voxel's edges (column n of L holds deg_n and -c at each neighbour)
__device__ __forceinline__ double ltl_diagonal(const Geometry& g, int n) {
  double deg = 0.0, c2 = 0.0;
  for (int d = 0; d < g.ndir; ++d) {
    if (__ldg(g.nbr + (size_t)d * g.ld + n) >= 0) {
      const double c = g.cw[d >> 1];
      deg += c;
      c2 += c * c;
    }
  }
  return deg * deg + c2;
}

// Quadratic-form weights of the lagged X products for the lag pairs p <= q, filled by the
// whole CTA (the caller synchronises before use): Q[syy_index(p, q)][tri(i, j)] is
// Sxx[p][q][i][i] on the diagonal and Sxx[p][q][i][j] + Sxx[p][q][j][i] below it, so that
// w' Sxx[p][q] w = sum_e Q[e] w_i w_j: K(K+1)/2 multiply-adds per pair instead of K^2 + K.
__host__ __device__ inline size_t quad_weight_doubles(int K, int P) {
  return (size_t)n_syy(P) * (size_t)(K * (K + 1) / 2);
}

__device__ inline void load_quad_weights(const double* Sxx, int K, int P, double* Q) {
  const int nt = K * (K + 1) / 2, total = n_syy(P) * nt;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int pq = idx / nt, e = idx % nt;
    int p = 0, q = 0;
    for (int pp = 0; pp <= P; ++pp)
      for (int qq = pp; qq <= P; ++qq)
        if (syy_index(pp, qq, P) == pq) {
          p = pp;
          q = qq;
        }
    int i = 0;
    while ((i + 1) * (i + 2) / 2 <= e) ++i;
    const int j = e - i * (i + 1) / 2;
    const double* S = Sxx + (size_t)(p * (P + 1) + q) * K * K;
    Q[idx] = i == j ? S[i * K + i] : S[i * K + j] + S[j * K + i];
  }
}

// Lagged residual Gram G[p][q] = (L^p e)'(L^q e) of e = y - X w (symmetric; PMAX-padded with
// zeros), from the statistics record and the quadratic-form weights Q.
template <int K>
__device__ __forceinline__ void lagged_gram(const double* __restrict__ stats, const double* Q,
                                            const double* w, int P, size_t ld, int n,
                                            double G[PMAX + 1][PMAX + 1]) {
  double ww[ntri(K)];
#pragma unroll
  for (int i = 0; i < K; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) ww[tri(i, j)] = w[i] * w[j];
#pragma unroll
  for (int p = 0; p <= PMAX; ++p) {
#pragma unroll
    for (int q = p; q <= PMAX; ++q) {
      double g = 0.0;
      if (q <= P) {
        double t1 = 0.0, t2 = 0.0, quad = 0.0;
        const double* Qpq = Q + (size_t)syy_index(p, q, P) * ntri(K);
#pragma unroll
        for (int k = 0; k < K; ++k) {
          t1 += w[k] * __ldg(stats + (size_t)(n_syy(P) + (q * (P + 1) + p) * K + k) * ld + n);
          t2 += w[k] * __ldg(stats + (size_t)(n_syy(P) + (p * (P + 1) + q) * K + k) * ld + n);
        }
#pragma unroll
        for (int e = 0; e < ntri(K); ++e) quad += Qpq[e] * ww[e];
        g = __ldg(stats + (size_t)syy_index(p, q, P) * ld + n) - t1 - t2 + quad;
      }
      G[p][q] = g;
      G[q][p] = g;
    }
  }
}

// Spatial-VB kernels (kernels_svb.cu).
struct SvbArgs {
  Geometry g;
  int K, P, T, S;
  const double* stats;
  const double* Sxx;
  const double* Ws;     // [S][K][ld] W samples
  const double* As;     // [S][P][ld] A samples
  double* Cmom;         // [n_syy(P)][ld]
  double* Gin;          // [n_syy(P)][ld]
  const double* bmean;  // [D][ld]
  const double* ldata;  // [ntri(D)][ld]
  const double* scale;  // [D]
  int spatial;          // A system: 1 with the beta D_a prior
  double* rhs;          // [S][D][ld]
  size_t vs;            // stride between samples of rhs
  Rng rng;              // the sample index is the stream
  double u1, u2;
  double* lam;          // out: E[lambda]
  double* part;         // [grid][D] quadratic-form partials
};
// what: 0 Cmom, 1 Gin, 2 perturbed rhs (dimension D), 3 E[lambda], 4 Q partials of W (D = K),
// 5 Q partials of A (D = P). Returns the grid used for what 4/5 in *grid_out.
cudaError_t launch_svb(int what, int D, const SvbArgs& a, cudaStream_t s, int* grid_out);

struct StatsArgs {
  int N, T, K, P;
  size_t ld;
  const void* Y;      // T x N row-major (float or double)
  int y_is_f64;
  const double* X;    // T x K column-major
  double* stats;      // [n_stats][ld]
};
cudaError_t launch_stats(const StatsArgs& a, cudaStream_t s);

// Statistics of FP32 series on the tensor cores (exact digit products, see
// kernels_stats_tc.cu): P <= 3, K <= 16.
struct StatsTcArgs {
  int N, T, K, P;
  size_t ld;
  const float* Y;           // T x N row-major
  const double* X;          // T x K column-major (terms outside the common window)
  const uint16_t* xdig;     // [ceil(K/8)][I][Tpad][8] BF16 digits of X
  const int* xexp;          // [K] column exponents of X
  double* stats;            // [n_stats][ld]
  int I, Tpad, groups, sm_cap;
  int* err;                 // nonzero: a tensor-core pipeline wait gave up
};
cudaError_t launch_stats_tc(const StatsTcArgs& a, cudaStream_t s);
// whether the tensor-core statistics apply (and the number of X digits I that fits)
bool stats_tc_supported(int T, int K, int P, int* I_out);
void stats_tc_digits(const double* X, int T, int K, int P, int I, std::vector<uint16_t>& dig,
                     std::vector<int>& exps, int& Tpad);
size_t stats_tc_smem_bytes(int T, int K, int P, int I);

// W system: blocks Bd_n = lambda_n X~'X~ + eps I, b_w, block-Jacobi factor of
// Bd_n + diag(alpha) deg_n, and the perturbed right-hand side of Algorithm 2.
struct AssembleArgs {
  Geometry g;
  int K, P;
  const double* stats;
  const double* Sxx;    // [(P+1)^2][K][K] voxel-independent lagged X products
  const double* W;      // [K][ld]
  const double* A;      // [P][ld]
  const double* lam;    // [ld]
  const double* scale;  // alpha [K] (W system) or beta [P] (A system)
  double eps;
  int spatial;          // A system: 1 = beta D_a prior, 0 = independent voxels
  int perturb;          // 1: rhs = perturbed b; 0: rhs = b_w (mean system)
  int precond;          // 1: write block-Jacobi factor
  int g_only;           // A system: compute only the Gram G (for lambda)
  Rng rng;
  // outputs
  double* blocks;       // [ntri(D)][ld]
  double* mfac;         // [ntri(D)][ld]
  float* blocks32;      // [ntri(D)][ld] FP32 copies for the mixed-precision solver (or null)
  float* mfac32;
  double* rhs;          // [D][ld]
  double* bmean;        // [D][ld] (may be null)
  double* G;            // A system: [n_syy(P)][ld] lagged residual Gram (for lambda)
  double* x_direct;     // A system, independent prior: if set, the draw is written here
  int* bad_voxel;       // min index of a voxel whose block failed Cholesky (init INT_MAX)
  // spatial VB
  const double* Cmom;   // W system: [n_syy(P)][ld] E[c_p c_q] over A samples, replaces c c'
  const double* Gin;    // A system: [n_syy(P)][ld] lagged residual Gram averaged over W samples
  double* ldata;        // [ntri(D)][ld] Cholesky factor of the data block (or null)
  const double* edge;   // [3][D][ld] pre-generated edge terms (launch_edge_noise), or null;
                        // with ltl, [D][ld] prior terms of the perturbation (launch_ltl_noise)
  int ltl;              // W system under the L'L prior: D_w = L'L in the preconditioner's
                        // diagonal; the perturbation's prior part is read from edge (required)
  const double* scale3 = nullptr;  // W system under the anisotropic prior: [3][K] alpha_{d,k}, the
                        // preconditioner's diagonal sum_d alpha_{d,k} deg_d (edge required)
};

// E[d][k][n] = sqrt(scale_k) z1_k for the edge from voxel n in direction +d (zero when absent):
// each edge's normals are generated once instead of by both of its endpoints.
// Device draw counter of captured sweeps: set it, or advance it by one (one-thread kernels).
cudaError_t launch_set_counter(uint32_t* p, uint32_t v, cudaStream_t s);
cudaError_t launch_advance_counter(uint32_t* p, cudaStream_t s);
// With scale3 ([3][D], the anisotropic prior) the edge of direction d carries sqrt(scale3[d][k]).
cudaError_t launch_edge_noise(const Geometry& g, int D, const double* scale, Rng rng, double* E,
                              cudaStream_t s, const double* scale3 = nullptr);
cudaError_t launch_assemble_w(const AssembleArgs& a, cudaStream_t s);
// The L'L prior's part of the perturbation: E[k][n] = sqrt(scale_k) (L z1_k)_n with z1_k one
// normal per voxel (site lattice-linear * 4 + 0, lane k); uses E[D .. 2D) as scratch.
cudaError_t launch_ltl_noise(const Geometry& g, int D, const double* scale, Rng rng, double* E,
                             cudaStream_t s);
cudaError_t launch_assemble_a(const AssembleArgs& a, cudaStream_t s);

// lambda_n ~ Ga(1/(1/u1 + RSS_n/2), (T-P)/2 + u2) from the Gram of launch_assemble_a.
struct LambdaArgs {
  Geometry g;
  int P, T;
  double u1, u2;
  const double* G;
  const double* A;
  double* lam;
  Rng rng;
  int* exhausted;
};
cudaError_t launch_lambda(const LambdaArgs& a, cudaStream_t s);

// alpha / beta: Q_k = sum over edges (v_i - v_j)^2, then Ga(1/(Q_k/2 + 1/prior1), N/2 + prior2).
struct HyperArgs {
  Geometry g;
  int D;
  const double* V;      // [D][ld]
  double* part;         // [grid][D] partials (grid = hyper_grid(N))
  double prior1, prior2;
  double* out;          // [D], or null: only the quadratic forms are written to Q_out
  double* Q_out;        // [D] (may be null)
  Rng rng;
  int* exhausted;
  int ltl;              // quadratic forms |L v_k|^2 of the L'L prior instead of the edge sums
  int dirs = 0;         // per-direction edge sums Q_out[d][k] (3 x D; part holds grid x 3D),
                        // no draw
};
cudaError_t launch_hyper(const HyperArgs& a, cudaStream_t s);
int hyper_grid(int N);

// y = B~ x (inspection).
struct ApplyArgs {
  Geometry g;
  int D;
  const double* blocks;
  const double* scale;
  const double* x;
  double* y;
  double* t;            // [D][ld] scratch for L x under the L'L prior, or null (graph Laplacian)
  const double* scale3 = nullptr;  // [3][D] per-direction scales of the anisotropic prior, or null
};
cudaError_t launch_apply(const ApplyArgs& a, cudaStream_t s);

// ---------------------------------------------------------------------------------------
// Anisotropic prior (alpha_{d,k} per direction d and regressor k): the exchange step
// (Murray, Ghahramani & MacKay 2006) for the alphas.
// ---------------------------------------------------------------------------------------
struct AnisoArgs {
  int K;
  int nd;               // directions of the lattice (2 or 3)
  double step;          // log-normal random-walk step
  double q1, q2;        // Ga(scale q1, shape q2) prior of every alpha_{d,k}
  double* alpha3;       // [3][K] current values (updated on acceptance)
  double* prop3;        // [3][K] proposal
  const double* Q;      // [3][K] direction edge sums of W
  const double* Qp;     // [3][K] direction edge sums of the auxiliary field
  double* log_a;        // [K] log acceptance ratio of the last step
  long long* accepted;  // [K] accepted proposals (cumulative)
  Rng rng;              // tag TAG_ALPHA_PROP: normals (sub 0, 1), uniform (sub 2)
  // the ray move alpha -> lam alpha before the exchange step
  int N, parts;         // voxels and connected parts of the voxel graph
  double* lam;          // [K] the last lam
  Rng rng_scale;        // tag TAG_ALPHA: the Gamma draw of lam (site k)
  int* exhausted;       // Gamma attempts exhausted (counted)
};
// lam_k ~ Ga(shape nd q2 + (N - parts)/2, rate sum_d alpha_d (1/q1 + Q_d/2)); alpha3 *= lam_k
// in the lattice's directions (Q: the direction edge sums of W)
cudaError_t launch_aniso_scale(const AnisoArgs& a, cudaStream_t s);
// prop3 = alpha3 exp(step eps) in the lattice's directions (the others copied)
cudaError_t launch_aniso_propose(const AnisoArgs& a, cudaStream_t s);
// log a from Q, Qp; alpha3 = prop3 where log u < log a
cudaError_t launch_aniso_accept(const AnisoArgs& a, cudaStream_t s);
// The auxiliary system L(prop3) x = sum_d sqrt(prop3_d) G_d' C_d^(1/2) z: blocks = 0, Jacobi
// factor diag(sum_d prop3[d][k] deg_d) (1 where a voxel has no neighbour), rhs = the edge
// terms E (launch_edge_noise with scale3 = prop3), x = 0.
cudaError_t launch_aux_system(const Geometry& g, int D, const double* prop3, const double* E,
                              double* blocks, double* mfac, double* rhs, double* x, cudaStream_t s);

}  // namespace bfmri
