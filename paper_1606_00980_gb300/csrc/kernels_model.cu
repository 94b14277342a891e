// Per-voxel model kernels: sufficient statistics (Appendix A, Eq. log-like), assembly of the
// W and A full conditionals (Eq. full cond W temporal, Eq. fullcondTempA) fused with the
// Algorithm 2 perturbation and the block-Jacobi factorisation, and the Gamma full
// conditionals of lambda, alpha, beta (Eq. fullcondTemplambda, fullcondTempa, fullcondTempbeta).
#include <climits>

#include "model.cuh"

namespace bfmri {

namespace {

constexpr int STATS_THREADS = 128;
constexpr int VOX_THREADS = 128;
constexpr int HYPER_THREADS = 256;

}  // namespace

// ---------------------------------------------------------------------------------------
// Sufficient statistics, direct form (short series, T < 2P). Thread (n, p): for lag p it
// accumulates, over t = P+1..T (1-based), Syy[p][q] (q >= p) and Sxy[p][q][k] for all q, k.
// X is staged in shared memory (row-major T x K); a register window holds y_t .. y_{t-P}.
// ---------------------------------------------------------------------------------------
template <int K, typename TY>
__global__ void __launch_bounds__(STATS_THREADS) k_stats_direct(StatsArgs a) {
  extern __shared__ double shX[];
  const int T = a.T, P = a.P, N = a.N;
  for (int i = threadIdx.x; i < T * K; i += blockDim.x) {
    const int t = i / K, k = i - t * K;
    shX[i] = a.X[t + (size_t)T * k];
  }
  __syncthreads();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (n >= N) return;
  const TY* Y = static_cast<const TY*>(a.Y);
  double axy[PMAX + 1][K];
  double ayy[PMAX + 1];
  double yw[PMAX + 1];
#pragma unroll
  for (int q = 0; q <= PMAX; ++q) {
    ayy[q] = 0.0;
    yw[q] = 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) axy[q][k] = 0.0;
  }
#pragma unroll
  for (int j = 0; j <= PMAX; ++j)
    if (j <= P) yw[j] = (double)Y[(size_t)(P - j) * N + n];
  for (int t = P; t < T; ++t) {
    if (t > P) {
#pragma unroll
      for (int j = PMAX; j > 0; --j) yw[j] = yw[j - 1];
      yw[0] = (double)Y[(size_t)t * N + n];
    }
    const double v = (double)Y[(size_t)(t - p) * N + n];
#pragma unroll
    for (int q = 0; q <= PMAX; ++q) {
      if (q <= P) {
        ayy[q] += v * yw[q];
        const double* xr = shX + (size_t)(t - q) * K;
#pragma unroll
        for (int k = 0; k < K; ++k) axy[q][k] += v * xr[k];
      }
    }
  }
  const size_t ld = a.ld;
#pragma unroll
  for (int q = 0; q <= PMAX; ++q) {
    if (q <= P) {
      if (q >= p) a.stats[(size_t)syy_index(p, q, P) * ld + n] = ayy[q];
#pragma unroll
      for (int k = 0; k < K; ++k) a.stats[sxy_plane(p, q, k, K, P) * ld + n] = axy[q][k];
    }
  }
}

// ---------------------------------------------------------------------------------------
// W system. Bd_n = lambda_n sum_pq c_p c_q Sxx[p][q] + eps I, b_n = lambda_n sum_pq c_p c_q
// Sxy[p][q] with c = (1, -a_n); perturbed rhs = b_n + L_n z2_n + sum_k sqrt(alpha_k) (G'z1_k)_n
// with L_n = chol(Bd_n); preconditioner factor chol(Bd_n + diag(alpha) deg_n).
// ---------------------------------------------------------------------------------------
// The weights c_p c_q (and the SVB moments) are symmetric in (p, q) and Sxx[q][p] =
// Sxx[p][q]', so the block needs only the pairs p <= q: shT[syy_index(p, q)] holds the packed
// lower triangle of Sxx[p][p], or of Sxx[p][q] + Sxx[p][q]' for p < q ((P+1)(P+2)/2 packed
// matrices instead of (P+1)^2 full ones).
template <int K>
__global__ void __launch_bounds__(VOX_THREADS) k_assemble_w(AssembleArgs a) {
  extern __shared__ double shT[];
  const int P = a.P;
  const int nT = n_syy(P) * ntri(K);
  for (int idx = threadIdx.x; idx < nT; idx += blockDim.x) {
    const int pq = idx / ntri(K), e = idx % ntri(K);
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
    const double* S = a.Sxx + (size_t)(p * (P + 1) + q) * K * K;
    shT[idx] = p == q ? S[i * K + j] : S[i * K + j] + S[j * K + i];
  }
  __syncthreads();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.g.N) return;
  const size_t ld = a.g.ld;
  double c[PMAX + 1];
  c[0] = 1.0;
#pragma unroll
  for (int p = 1; p <= PMAX; ++p) c[p] = (p <= P) ? -a.A[(size_t)(p - 1) * ld + n] : 0.0;
  double B[ntri(K)], bw[K];
#pragma unroll
  for (int e = 0; e < ntri(K); ++e) B[e] = 0.0;
#pragma unroll
  for (int k = 0; k < K; ++k) bw[k] = 0.0;
#pragma unroll
  for (int p = 0; p <= PMAX; ++p) {
#pragma unroll
    for (int q = 0; q <= PMAX; ++q) {
      if (p <= P && q <= P) {
        const double cpq = a.Cmom ? __ldg(a.Cmom + (size_t)syy_index(p < q ? p : q, p < q ? q : p, P) * ld + n)
                                  : c[p] * c[q];
        if (p <= q) {
          const double* T = shT + (size_t)syy_index(p, q, P) * ntri(K);
#pragma unroll
          for (int e = 0; e < ntri(K); ++e) B[e] += cpq * T[e];
        }
#pragma unroll
        for (int k = 0; k < K; ++k) bw[k] += cpq * __ldg(a.stats + sxy_plane(p, q, k, K, P) * ld + n);
      }
    }
  }
  const double lam = a.lam[n];
#pragma unroll
  for (int e = 0; e < ntri(K); ++e) B[e] *= lam;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    B[tri(k, k)] += a.eps;
    bw[k] *= lam;
  }
  store_packed<K>(a.blocks, ld, n, B);
  if (a.blocks32) {
#pragma unroll
    for (int e = 0; e < ntri(K); ++e) a.blocks32[(size_t)e * ld + n] = (float)B[e];
  }
  if (a.bmean) {
#pragma unroll
    for (int k = 0; k < K; ++k) a.bmean[k * ld + n] = bw[k];
  }
  double rhs[K];
#pragma unroll
  for (int k = 0; k < K; ++k) rhs[k] = bw[k];
  double L[ntri(K)], Ld[K];
#pragma unroll
  for (int e = 0; e < ntri(K); ++e) L[e] = B[e];
  bool ok = chol_packed_invdiag<K>(L, Ld);
  if (a.ldata) store_packed<K>(a.ldata, ld, n, L);
  if (a.perturb) {
    const int lin = a.g.lin[n];
    double z[K], Lz[K];
    site_normals<K>(a.rng, (uint32_t)lin * 4u + 3u, z);
    lower_mul_diag<K>(L, Ld, z, Lz);
#pragma unroll
    for (int k = 0; k < K; ++k) rhs[k] += Lz[k];
    if (a.ltl) {
#pragma unroll
      for (int k = 0; k < K; ++k) rhs[k] += __ldg(a.edge + (size_t)k * ld + n);
    } else if (a.edge) {
      add_edge_terms<K>(a.g, a.edge, n, rhs);
    } else {
      double sq[K];
#pragma unroll
      for (int k = 0; k < K; ++k) sq[k] = sqrt(a.scale[k]);
      add_edge_noise<K>(a.g, a.rng, n, lin, sq, rhs);
    }
  }
#pragma unroll
  for (int k = 0; k < K; ++k) a.rhs[k * ld + n] = rhs[k];
  if (a.precond) {
    if (a.scale3) {
      double dd[3];
      for (int d = 0; d < 3; ++d) dd[d] = d < a.g.ndir / 2 ? degree_dir(a.g, n, d) : 0.0;
#pragma unroll
      for (int k = 0; k < K; ++k)
        B[tri(k, k)] += __ldg(a.scale3 + k) * dd[0] + __ldg(a.scale3 + K + k) * dd[1] +
                        __ldg(a.scale3 + 2 * K + k) * dd[2];
    } else {
      const double deg = a.ltl ? ltl_diagonal(a.g, n) : degree(a.g, n);
#pragma unroll
      for (int k = 0; k < K; ++k) B[tri(k, k)] += a.scale[k] * deg;
    }
    ok = chol_packed_invdiag<K>(B) && ok;
    store_packed<K>(a.mfac, ld, n, B);
    if (a.mfac32) {
#pragma unroll
      for (int e = 0; e < ntri(K); ++e) a.mfac32[(size_t)e * ld + n] = (float)B[e];
    }
  }
  if (!ok) atomicMin(a.bad_voxel, n);
}

// ---------------------------------------------------------------------------------------
// A system and the lagged residual Gram. With e = y - X w_n:
//   G[p][q] = (L^p e)'(L^q e) = Syy[p][q] - w.Sxy[q][p] - w.Sxy[p][q] + w' Sxx[p][q] w,
// the block lambda_n G[1:,1:], the right-hand side lambda_n G[1:,0] (Eq. fullcondTempA),
// perturbed with beta (spatial prior) or drawn per voxel directly (independent prior).
// The P x P matrices are embedded in PMAX x PMAX with identity padding.
// ---------------------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(VOX_THREADS) k_assemble_a(AssembleArgs a) {
  extern __shared__ double shQ[];
  const int P = a.P;
  load_quad_weights(a.Sxx, K, P, shQ);
  __syncthreads();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.g.N) return;
  const size_t ld = a.g.ld;
  double w[K];
#pragma unroll
  for (int k = 0; k < K; ++k) w[k] = a.Gin ? 0.0 : a.W[(size_t)k * ld + n];
  double Gm[PMAX + 1][PMAX + 1];
  if (!a.Gin) lagged_gram<K>(a.stats, shQ, w, P, ld, n, Gm);
#pragma unroll
  for (int p = 0; p <= PMAX; ++p) {
#pragma unroll
    for (int q = p; q <= PMAX; ++q) {
      if (q <= P && a.Gin) {
        Gm[p][q] = Gm[q][p] = __ldg(a.Gin + (size_t)syy_index(p, q, P) * ld + n);
      } else if (q <= P) {
        a.G[(size_t)syy_index(p, q, P) * ld + n] = Gm[p][q];
      } else {
        Gm[p][q] = Gm[q][p] = 0.0;
      }
    }
  }
  if (P == 0 || a.g_only) return;
  const double lam = a.lam[n];
  constexpr int PM = PMAX;
  double J[ntri(PM)], rhs[PM];
#pragma unroll
  for (int i = 0; i < PM; ++i) {
    rhs[i] = (i < P) ? lam * Gm[i + 1][0] : 0.0;
#pragma unroll
    for (int j = 0; j <= i; ++j)
      J[tri(i, j)] = (i < P) ? lam * Gm[i + 1][j + 1] : (i == j ? 1.0 : 0.0);
  }
  if (a.bmean) {
#pragma unroll
    for (int i = 0; i < PM; ++i)
      if (i < P) a.bmean[i * ld + n] = rhs[i];
  }
  double L[ntri(PM)];
#pragma unroll
  for (int e = 0; e < ntri(PM); ++e) L[e] = J[e];
  double Ld[PM];
  bool ok = chol_packed_invdiag<PM>(L, Ld);
  if (a.ldata) {
#pragma unroll
    for (int e = 0; e < ntri(PM); ++e)
      if (e < ntri(P)) a.ldata[(size_t)e * ld + n] = L[e];
  }
  const int lin = a.g.lin[n];
  if (a.perturb) {
    double z[PM], Lz[PM];
    site_normals<PM>(a.rng, (uint32_t)lin * 4u + 3u, z);
#pragma unroll
    for (int i = 0; i < PM; ++i)
      if (i >= P) z[i] = 0.0;
    lower_mul_diag<PM>(L, Ld, z, Lz);
#pragma unroll
    for (int i = 0; i < PM; ++i) rhs[i] += (i < P) ? Lz[i] : 0.0;
    if (a.spatial) {
      if (a.edge) {
        // terms generated for dimension P; the padded components stay zero
        double part[PM];
#pragma unroll
        for (int i = 0; i < PM; ++i) part[i] = 0.0;
        if (P == 1) add_edge_terms<1>(a.g, a.edge, n, part);
        else if (P == 2) add_edge_terms<2>(a.g, a.edge, n, part);
        else if (P == 3) add_edge_terms<3>(a.g, a.edge, n, part);
        else add_edge_terms<4>(a.g, a.edge, n, part);
#pragma unroll
        for (int i = 0; i < PM; ++i) rhs[i] += part[i];
      } else {
        double sq[PM];
#pragma unroll
        for (int i = 0; i < PM; ++i) sq[i] = (i < P) ? sqrt(a.scale[i]) : 0.0;
        add_edge_noise<PM>(a.g, a.rng, n, lin, sq, rhs);
      }
    }
  }
  if (a.x_direct) {
    // independent voxels: the draw is J^-1 rhs
    double x[PM];
    chol_solve_invdiag<PM>(L, rhs, x);
#pragma unroll
    for (int i = 0; i < PM; ++i)
      if (i < P) a.x_direct[i * ld + n] = x[i];
  }
  if (a.rhs) {
#pragma unroll
    for (int e = 0; e < ntri(PM); ++e)
      if (e < ntri(P)) {
        a.blocks[(size_t)e * ld + n] = J[e];
        if (a.blocks32) a.blocks32[(size_t)e * ld + n] = (float)J[e];
      }
#pragma unroll
    for (int i = 0; i < PM; ++i)
      if (i < P) a.rhs[i * ld + n] = rhs[i];
    if (a.precond) {
      const double deg = a.spatial ? degree(a.g, n) : 0.0;
#pragma unroll
      for (int i = 0; i < PM; ++i)
        if (i < P) J[tri(i, i)] += a.scale[i] * deg;
      ok = chol_packed_invdiag<PM>(J) && ok;
#pragma unroll
      for (int e = 0; e < ntri(PM); ++e)
        if (e < ntri(P)) {
          a.mfac[(size_t)e * ld + n] = J[e];
          if (a.mfac32) a.mfac32[(size_t)e * ld + n] = (float)J[e];
        }
    }
  }
  if (!ok) atomicMin(a.bad_voxel, n);
}

// ---------------------------------------------------------------------------------------
// The L'L prior: t = f .* (L v) for D planes (L the weighted graph Laplacian, symmetric, so
// L' v = L v), f_k = 1 or sqrt(scale_k); and the per-voxel normals z1 of its perturbation.
// ---------------------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(VOX_THREADS) k_laplacian(Geometry g, const double* v, double* t,
                                                           const double* scale) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.N) return;
  const size_t ld = g.ld;
  double sum[D], deg = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) sum[k] = 0.0;
  for (int d = 0; d < g.ndir; ++d) {
    const int m = __ldg(g.nbr + (size_t)d * ld + n);
    if (m >= 0) {
      const double c = g.cw[d >> 1];
      deg += c;
#pragma unroll
      for (int k = 0; k < D; ++k) sum[k] += c * v[(size_t)k * ld + m];
    }
  }
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const double f = scale ? sqrt(__ldg(scale + k)) : 1.0;
    t[(size_t)k * ld + n] = f * (deg * v[(size_t)k * ld + n] - sum[k]);
  }
}

template <int D>
__global__ void __launch_bounds__(VOX_THREADS) k_voxel_normals(Geometry g, Rng rng, double* Z) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.N) return;
  double z[D];
  site_normals<D>(rng, (uint32_t)g.lin[n] * 4u + 0u, z);
#pragma unroll
  for (int k = 0; k < D; ++k) Z[(size_t)k * g.ld + n] = z[k];
}

// alpha under the L'L prior: Q_k = sum_n ((L v_k)_n)^2, the same two-level reduction as
// k_quadform
template <int D>
__global__ void __launch_bounds__(HYPER_THREADS) k_quadform_ltl(HyperArgs a) {
  __shared__ double sh[HYPER_THREADS / 32][D];
  double acc[D];
#pragma unroll
  for (int k = 0; k < D; ++k) acc[k] = 0.0;
  const size_t ld = a.g.ld;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < a.g.N; n += gridDim.x * blockDim.x) {
    double sum[D], deg = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) sum[k] = 0.0;
    for (int d = 0; d < a.g.ndir; ++d) {
      const int m = __ldg(a.g.nbr + (size_t)d * ld + n);
      if (m >= 0) {
        const double c = a.g.cw[d >> 1];
        deg += c;
#pragma unroll
        for (int k = 0; k < D; ++k) sum[k] += c * a.V[(size_t)k * ld + m];
      }
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const double l = deg * a.V[(size_t)k * ld + n] - sum[k];
      acc[k] += l * l;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < D; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
    if (lane == 0) sh[warp][k] = acc[k];
  }
  __syncthreads();
  if (threadIdx.x < D) {
    double s = 0.0;
    for (int w = 0; w < HYPER_THREADS / 32; ++w) s += sh[w][threadIdx.x];
    a.part[(size_t)blockIdx.x * D + threadIdx.x] = s;
  }
}

// ---------------------------------------------------------------------------------------
// Edge terms of the perturbation, generated once per edge.
// ---------------------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(VOX_THREADS) k_edge_noise(Geometry g, const double* scale, Rng rng,
                                                            double* E, const double* scale3) {
  // sqrt(scale_k c_d) once per CTA (c_d: the edge weight of direction d; scale3[d][k] in
  // place of scale_k under the anisotropic prior)
  __shared__ double sq[3][D];
  if (threadIdx.x < 3 * D)
    sq[threadIdx.x / D][threadIdx.x % D] =
        sqrt((scale3 ? scale3[threadIdx.x] : scale[threadIdx.x % D]) * g.cw[threadIdx.x / D]);
  __syncthreads();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.N) return;
  const uint32_t lin = (uint32_t)g.lin[n];
  for (int d = 0; d < g.ndir / 2; ++d) {
    double z[D];
    const bool has = __ldg(g.nbr + (size_t)(2 * d + 1) * g.ld + n) >= 0;
    if (has) site_normals<D>(rng, lin * 4u + (uint32_t)d, z);
    // the edge's own factor of C (stored at its lower voxel n)
    const double f = g.ce ? sqrt(bf16_value(__ldg(g.ce + (size_t)d * g.ld + n))) : 1.0;
#pragma unroll
    for (int k = 0; k < D; ++k) E[((size_t)d * D + k) * g.ld + n] = has ? f * sq[d][k] * z[k] : 0.0;
  }
}

// ---------------------------------------------------------------------------------------
// lambda: RSS_n = c' G c with c = (1, -a_n) (the bracket of Eq. fullcondTemplambda).
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(VOX_THREADS) k_lambda(LambdaArgs a) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.g.N) return;
  const int P = a.P;
  const size_t ld = a.g.ld;
  double c[PMAX + 1];
  c[0] = 1.0;
#pragma unroll
  for (int p = 1; p <= PMAX; ++p) c[p] = (p <= P) ? -a.A[(size_t)(p - 1) * ld + n] : 0.0;
  double rss = 0.0;
#pragma unroll
  for (int p = 0; p <= PMAX; ++p) {
#pragma unroll
    for (int q = 0; q <= PMAX; ++q) {
      if (p <= P && q <= P) {
        const int pp = p < q ? p : q, qq = p < q ? q : p;
        rss += c[p] * c[q] * a.G[(size_t)syy_index(pp, qq, P) * ld + n];
      }
    }
  }
  const double shape = 0.5 * (double)(a.T - P) + a.u2;
  const double scale = 1.0 / (1.0 / a.u1 + 0.5 * rss);
  int ex = 0;
  a.lam[n] = gamma_draw(a.rng, (uint32_t)a.g.lin[n] * 4u + 3u, shape, scale, &ex);
  if (ex) atomicAdd(a.exhausted, 1);
}

// ---------------------------------------------------------------------------------------
// alpha / beta: deterministic two-level reduction of Q_k = sum_edges (v_i - v_j)^2.
// ---------------------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(HYPER_THREADS) k_quadform(HyperArgs a) {
  __shared__ double sh[HYPER_THREADS / 32][D];
  double acc[D];
#pragma unroll
  for (int k = 0; k < D; ++k) acc[k] = 0.0;
  const size_t ld = a.g.ld;
  const int nfwd = a.g.ndir / 2;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < a.g.N; n += gridDim.x * blockDim.x) {
    // the forward neighbours' indices, then all their values, in two rounds of loads
    int m[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) m[d] = d < nfwd ? __ldg(a.g.nbr + (size_t)(2 * d + 1) * ld + n) : -1;
    double v[D], vn[3][D];
#pragma unroll
    for (int k = 0; k < D; ++k) v[k] = a.V[(size_t)k * ld + n];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int k = 0; k < D; ++k) vn[d][k] = a.V[(size_t)k * ld + (m[d] >= 0 ? m[d] : n)];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (m[d] >= 0) {
        const double c = slot_weight(a.g, n, 2 * d + 1, m[d]);
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const double df = v[k] - vn[d][k];
          acc[k] += c * df * df;
        }
      }
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < D; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
    if (lane == 0) sh[warp][k] = acc[k];
  }
  __syncthreads();
  if (threadIdx.x < D) {
    double s = 0.0;
    for (int w = 0; w < HYPER_THREADS / 32; ++w) s += sh[w][threadIdx.x];
    a.part[(size_t)blockIdx.x * D + threadIdx.x] = s;
  }
}

// One warp per dimension k: the lanes add the CTA partials b = lane, lane + 32, ... and a
// butterfly combines them (a fixed order, so Q does not depend on timing).
__global__ void k_hyper_draw(HyperArgs a, int nblocks) {
  const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (k >= a.D) return;
  double Q = 0.0;
  for (int b = lane; b < nblocks; b += 32) Q += a.part[(size_t)b * a.D + k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) Q += __shfl_xor_sync(0xffffffffu, Q, o);
  if (lane != 0) return;
  if (a.Q_out) a.Q_out[k] = Q;
  if (!a.out) return;   // quadratic forms only
  const double scale = 1.0 / (0.5 * Q + 1.0 / a.prior1);
  const double shape = 0.5 * (double)a.g.N + a.prior2;
  int ex = 0;
  a.out[k] = gamma_draw(a.rng, (uint32_t)k, shape, scale, &ex);
  if (ex) atomicAdd(a.exhausted, 1);
}

// Per-direction edge sums Q[d][k] = sum over the direction-d edges of C_e (v_i - v_j)^2, with
// the partials of CTA b at part[(b * 3 + d) * D + k].
template <int D>
__global__ void __launch_bounds__(HYPER_THREADS) k_quadform_dirs(HyperArgs a) {
  __shared__ double sh[HYPER_THREADS / 32][3][D];
  double acc[3][D];
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int k = 0; k < D; ++k) acc[d][k] = 0.0;
  const size_t ld = a.g.ld;
  const int nfwd = a.g.ndir / 2;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < a.g.N; n += gridDim.x * blockDim.x) {
    double v[D];
#pragma unroll
    for (int k = 0; k < D; ++k) v[k] = a.V[(size_t)k * ld + n];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int m = d < nfwd ? __ldg(a.g.nbr + (size_t)(2 * d + 1) * ld + n) : -1;
      if (m >= 0) {
        const double c = slot_weight(a.g, n, 2 * d + 1, m);
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const double df = v[k] - a.V[(size_t)k * ld + m];
          acc[d][k] += c * df * df;
        }
      }
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int k = 0; k < D; ++k) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[d][k] += __shfl_down_sync(0xffffffffu, acc[d][k], o);
      if (lane == 0) sh[warp][d][k] = acc[d][k];
    }
  __syncthreads();
  for (int j = threadIdx.x; j < 3 * D; j += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < HYPER_THREADS / 32; ++w) s += sh[w][j / D][j % D];
    a.part[(size_t)blockIdx.x * 3 * D + j] = s;
  }
}

// Q_out[j] for j = d D + k: each warp adds the CTA partials of its j's in a fixed order.
__global__ void k_quad_dirs_sum(HyperArgs a, int nblocks) {
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = threadIdx.x >> 5; j < 3 * a.D; j += nw) {
    double Q = 0.0;
    for (int b = lane; b < nblocks; b += 32) Q += a.part[(size_t)b * 3 * a.D + j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) Q += __shfl_xor_sync(0xffffffffu, Q, o);
    if (lane == 0) a.Q_out[j] = Q;
  }
}

// ---------------------------------------------------------------------------------------
// Anisotropic prior: the exchange step's proposal and acceptance, one thread per k.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void aniso_eps(const AnisoArgs& a, int k, double* eps) {
  site_normals<3>(a.rng, (uint32_t)k, eps);
}

__global__ void k_aniso_scale(AnisoArgs a) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.K) return;
  double rate = 0.0;
  for (int d = 0; d < a.nd; ++d) rate += a.alpha3[d * a.K + k] * (1.0 / a.q1 + 0.5 * a.Q[d * a.K + k]);
  const double shape = a.nd * a.q2 + 0.5 * (double)(a.N - a.parts);
  int ex = 0;
  const double lam = gamma_draw(a.rng_scale, (uint32_t)k, shape, 1.0 / rate, &ex);
  if (ex) atomicAdd(a.exhausted, 1);
  a.lam[k] = lam;
  for (int d = 0; d < a.nd; ++d) a.alpha3[d * a.K + k] *= lam;
}

__global__ void k_aniso_propose(AnisoArgs a) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.K) return;
  double eps[3];
  aniso_eps(a, k, eps);
  for (int d = 0; d < 3; ++d) {
    const double t = a.alpha3[d * a.K + k];
    a.prop3[d * a.K + k] = d < a.nd ? t * exp(a.step * eps[d]) : t;
  }
}

__global__ void k_aniso_accept(AnisoArgs a) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.K) return;
  double eps[3];
  aniso_eps(a, k, eps);
  double la = 0.0;
  for (int d = 0; d < a.nd; ++d) {
    const int j = d * a.K + k;
    const double dt = a.prop3[j] - a.alpha3[j];
    la += -0.5 * dt * (a.Q[j] - a.Qp[j]) + a.q2 * (a.step * eps[d]) - dt / a.q1;
  }
  const uint4 w = a.rng.call((uint32_t)k, 2u);
  const double u = (u53(w.x, w.y) + 1.0) * 0x1.0p-53;
  a.log_a[k] = la;
  if (log(u) < la) {
    for (int d = 0; d < a.nd; ++d) a.alpha3[d * a.K + k] = a.prop3[d * a.K + k];
    a.accepted[k] += 1;
  }
}

template <int D>
__global__ void __launch_bounds__(VOX_THREADS) k_aux_system(Geometry g, const double* prop3, const double* E,
                                                            double* blocks, double* mfac, double* rhs,
                                                            double* x) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.N) return;
  const size_t ld = g.ld;
  double dd[3];
  for (int d = 0; d < 3; ++d) dd[d] = d < g.ndir / 2 ? degree_dir(g, n, d) : 0.0;
  double r[D];
#pragma unroll
  for (int k = 0; k < D; ++k) r[k] = 0.0;
  add_edge_terms<D>(g, E, n, r);
#pragma unroll
  for (int i = 0; i < D; ++i) {
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      blocks[(size_t)tri(i, j) * ld + n] = 0.0;
      mfac[(size_t)tri(i, j) * ld + n] = 0.0;
    }
    const double m = __ldg(prop3 + i) * dd[0] + __ldg(prop3 + D + i) * dd[1] + __ldg(prop3 + 2 * D + i) * dd[2];
    // inverted diagonal of the Cholesky factor of diag(m)
    mfac[(size_t)tri(i, i) * ld + n] = m > 0.0 ? 1.0 / sqrt(m) : 1.0;
    rhs[(size_t)i * ld + n] = r[i];
    x[(size_t)i * ld + n] = 0.0;
  }
}

// ---------------------------------------------------------------------------------------
// y = B~ x for inspection.
// ---------------------------------------------------------------------------------------
template <int D>
__global__ void k_apply(ApplyArgs a) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.g.N) return;
  const size_t ld = a.g.ld;
  double xn[D], y[D], B[ntri(D)];
#pragma unroll
  for (int k = 0; k < D; ++k) xn[k] = a.x[(size_t)k * ld + n];
  load_packed<D>(a.blocks, ld, n, B);
  sym_mul<D>(B, xn, y);
  double sum[D];
#pragma unroll
  for (int k = 0; k < D; ++k) sum[k] = 0.0;
  double deg = 0.0;
  // the prior part: scale .* (L x), or scale .* (L (L x)) with t = L x under the L'L prior
  const double* V = a.t ? a.t : a.x;
  for (int d = 0; d < a.g.ndir; ++d) {
    const int m = a.g.nbr[(size_t)d * ld + n];
    if (m >= 0) {
      const double c = slot_weight(a.g, n, d, m);
      if (a.scale3) {
        // anisotropic prior: sum over the slots of scale3[d][k] c (x_n - x_m)
#pragma unroll
        for (int k = 0; k < D; ++k)
          sum[k] += a.scale3[(d >> 1) * D + k] * c * (V[(size_t)k * ld + n] - V[(size_t)k * ld + m]);
      } else {
        deg += c;
#pragma unroll
        for (int k = 0; k < D; ++k) sum[k] += c * V[(size_t)k * ld + m];
      }
    }
  }
  if (a.scale3) {
#pragma unroll
    for (int k = 0; k < D; ++k) a.y[(size_t)k * ld + n] = y[k] + sum[k];
    return;
  }
#pragma unroll
  for (int k = 0; k < D; ++k)
    a.y[(size_t)k * ld + n] = y[k] + a.scale[k] * (deg * V[(size_t)k * ld + n] - sum[k]);
}

// ---------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------
#define BFMRI_K_CASES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12)

// ---------------------------------------------------------------------------------------
// Sufficient statistics, lag-difference form (T >= 2P). With s = t - p (0-based times),
//   Sxy[p][q][k] = sum_{s = P-p}^{T-1-p} y_s x_{s+d,k},   d = p - q,
//   Syy[p][q]    = sum_{s = P-q}^{T-1-q} y_s y_{s+e},     e = q - p >= 0,
// so every pair with the same lag difference shares the sum over the common window
// s = P .. T-1-P; each pair adds its own P boundary terms (s below P and above T-1-P).
// Thread (n, d) handles the lag difference d = p - q in [-P, P]: K + 1 products per time
// step instead of (P+1)(K+1), then the boundary terms of its pairs. X is staged in shared
// memory (row-major T x K).
// ---------------------------------------------------------------------------------------
template <int K, typename TY>
__global__ void __launch_bounds__(STATS_THREADS) k_stats(StatsArgs a) {
  extern __shared__ double shX[];
  const int T = a.T, P = a.P, N = a.N;
  for (int i = threadIdx.x; i < T * K; i += blockDim.x) {
    const int t = i / K, k = i - t * K;
    shX[i] = a.X[t + (size_t)T * k];
  }
  __syncthreads();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int d = (int)blockIdx.y - P;   // p - q
  if (n >= N) return;
  const TY* Y = static_cast<const TY*>(a.Y);
  auto y = [&](int t) { return (double)Y[(size_t)t * N + n]; };
  const int e = -d;                    // q - p, for the Syy pairs of this thread (e >= 0)
  double c[K], cyy = 0.0;
#pragma unroll
  for (int k = 0; k < K; ++k) c[k] = 0.0;
  for (int t = P; t <= T - 1 - P; ++t) {
    const double ys = y(t);
    const double* xr = shX + (size_t)(t + d) * K;
#pragma unroll
    for (int k = 0; k < K; ++k) c[k] += ys * xr[k];
    if (e >= 0) cyy += ys * y(t + e);
  }
  const size_t ld = a.ld;
  // Sxy pairs (p, q = p - d)
  for (int p = d > 0 ? d : 0; p <= P && p - d <= P; ++p) {
    const int q = p - d;
    double v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = c[k];
    for (int t = P - p; t <= P - 1; ++t) {
      const double ys = y(t);
      const double* xr = shX + (size_t)(t + d) * K;
#pragma unroll
      for (int k = 0; k < K; ++k) v[k] += ys * xr[k];
    }
    for (int t = T - P; t <= T - 1 - p; ++t) {
      const double ys = y(t);
      const double* xr = shX + (size_t)(t + d) * K;
#pragma unroll
      for (int k = 0; k < K; ++k) v[k] += ys * xr[k];
    }
#pragma unroll
    for (int k = 0; k < K; ++k) a.stats[sxy_plane(p, q, k, K, P) * ld + n] = v[k];
  }
  // Syy pairs (p, q = p + e), p <= q
  if (e >= 0) {
    for (int q = e; q <= P; ++q) {
      const int p = q - e;
      double v = cyy;
      for (int t = P - q; t <= P - 1; ++t) v += y(t) * y(t + e);
      for (int t = T - P; t <= T - 1 - q; ++t) v += y(t) * y(t + e);
      a.stats[(size_t)syy_index(p, q, P) * ld + n] = v;
    }
  }
}

template <int K>
static cudaError_t stats_k(const StatsArgs& a, cudaStream_t s) {
  const size_t shm = (size_t)a.T * K * sizeof(double);
  const unsigned gx = (unsigned)((a.N + STATS_THREADS - 1) / STATS_THREADS);
  const bool lagdiff = a.T >= 2 * a.P;
  const dim3 grid(gx, lagdiff ? 2 * a.P + 1 : a.P + 1);
  const void* kern = lagdiff ? (a.y_is_f64 ? (const void*)k_stats<K, double> : (const void*)k_stats<K, float>)
                             : (a.y_is_f64 ? (const void*)k_stats_direct<K, double>
                                           : (const void*)k_stats_direct<K, float>);
  cudaError_t e = raise_smem_limit(kern, shm);
  if (e != cudaSuccess) return e;
  if (lagdiff) {
    if (a.y_is_f64) k_stats<K, double><<<grid, STATS_THREADS, shm, s>>>(a);
    else k_stats<K, float><<<grid, STATS_THREADS, shm, s>>>(a);
  } else {
    if (a.y_is_f64) k_stats_direct<K, double><<<grid, STATS_THREADS, shm, s>>>(a);
    else k_stats_direct<K, float><<<grid, STATS_THREADS, shm, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_stats(const StatsArgs& a, cudaStream_t s) {
  if (a.N <= 0) return cudaSuccess;
  switch (a.K) {
#define CASE(k) case k: return stats_k<k>(a, s);
    BFMRI_K_CASES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

template <int K>
static cudaError_t assemble_w_k(const AssembleArgs& a, cudaStream_t s) {
  const size_t shm = (size_t)n_syy(a.P) * ntri(K) * sizeof(double);
  cudaError_t e = raise_smem_limit((const void*)k_assemble_w<K>, shm);
  if (e != cudaSuccess) return e;
  k_assemble_w<K><<<(a.g.N + VOX_THREADS - 1) / VOX_THREADS, VOX_THREADS, shm, s>>>(a);
  return cudaGetLastError();
}

template <int K>
static cudaError_t assemble_a_k(const AssembleArgs& a, cudaStream_t s) {
  const size_t shm = quad_weight_doubles(K, a.P) * sizeof(double);
  cudaError_t e = raise_smem_limit((const void*)k_assemble_a<K>, shm);
  if (e != cudaSuccess) return e;
  k_assemble_a<K><<<(a.g.N + VOX_THREADS - 1) / VOX_THREADS, VOX_THREADS, shm, s>>>(a);
  return cudaGetLastError();
}

__global__ void k_set_counter(uint32_t* p, uint32_t v) { *p = v; }
__global__ void k_advance_counter(uint32_t* p) { *p += 1u; }

cudaError_t launch_set_counter(uint32_t* p, uint32_t v, cudaStream_t s) {
  k_set_counter<<<1, 1, 0, s>>>(p, v);
  return cudaGetLastError();
}

cudaError_t launch_advance_counter(uint32_t* p, cudaStream_t s) {
  k_advance_counter<<<1, 1, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_assemble_w(const AssembleArgs& a, cudaStream_t s) {
  if (a.g.N <= 0) return cudaSuccess;
  switch (a.K) {
#define CASE(k) case k: return assemble_w_k<k>(a, s);
    BFMRI_K_CASES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_assemble_a(const AssembleArgs& a, cudaStream_t s) {
  if (a.g.N <= 0) return cudaSuccess;
  switch (a.K) {
#define CASE(k) case k: return assemble_a_k<k>(a, s);
    BFMRI_K_CASES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_lambda(const LambdaArgs& a, cudaStream_t s) {
  if (a.g.N <= 0) return cudaSuccess;
  k_lambda<<<(a.g.N + VOX_THREADS - 1) / VOX_THREADS, VOX_THREADS, 0, s>>>(a);
  return cudaGetLastError();
}

template <int D>
static cudaError_t edge_d(const Geometry& g, const double* scale, Rng rng, double* E, cudaStream_t s,
                          const double* scale3) {
  k_edge_noise<D><<<(g.N + VOX_THREADS - 1) / VOX_THREADS, VOX_THREADS, 0, s>>>(g, scale, rng, E, scale3);
  return cudaGetLastError();
}

cudaError_t launch_edge_noise(const Geometry& g, int D, const double* scale, Rng rng, double* E,
                              cudaStream_t s, const double* scale3) {
  if (g.N <= 0) return cudaSuccess;
  switch (D) {
#define CASE(k) case k: return edge_d<k>(g, scale, rng, E, s, scale3);
    BFMRI_K_CASES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

int hyper_grid(int N) {
  int g = (N + HYPER_THREADS - 1) / HYPER_THREADS;
  return g < 1 ? 1 : (g > 1024 ? 1024 : g);
}

template <int D>
static cudaError_t hyper_d(const HyperArgs& a, cudaStream_t s) {
  const int grid = hyper_grid(a.g.N);
  if (a.dirs) {
    k_quadform_dirs<D><<<grid, HYPER_THREADS, 0, s>>>(a);
    k_quad_dirs_sum<<<1, 32 * (3 * D < 32 ? 3 * D : 32), 0, s>>>(a, grid);
    return cudaGetLastError();
  }
  if (a.ltl) k_quadform_ltl<D><<<grid, HYPER_THREADS, 0, s>>>(a);
  else k_quadform<D><<<grid, HYPER_THREADS, 0, s>>>(a);
  k_hyper_draw<<<1, 32 * D, 0, s>>>(a, grid);
  return cudaGetLastError();
}

cudaError_t launch_hyper(const HyperArgs& a, cudaStream_t s) {
  switch (a.D) {
#define CASE(k) case k: return hyper_d<k>(a, s);
    BFMRI_K_CASES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

template <int D>
static cudaError_t apply_d(const ApplyArgs& a, cudaStream_t s) {
  const int grid = (a.g.N + VOX_THREADS - 1) / VOX_THREADS;
  if (a.t) k_laplacian<D><<<grid, VOX_THREADS, 0, s>>>(a.g, a.x, a.t, nullptr);
  k_apply<D><<<grid, VOX_THREADS, 0, s>>>(a);
  return cudaGetLastError();
}

template <int D>
static cudaError_t ltl_noise_d(const Geometry& g, const double* scale, Rng rng, double* E,
                               cudaStream_t s) {
  const int grid = (g.N + VOX_THREADS - 1) / VOX_THREADS;
  double* Z = E + (size_t)D * g.ld;
  k_voxel_normals<D><<<grid, VOX_THREADS, 0, s>>>(g, rng, Z);
  k_laplacian<D><<<grid, VOX_THREADS, 0, s>>>(g, Z, E, scale);
  return cudaGetLastError();
}

cudaError_t launch_ltl_noise(const Geometry& g, int D, const double* scale, Rng rng, double* E,
                             cudaStream_t s) {
  if (g.N <= 0) return cudaSuccess;
  switch (D) {
#define CASE(k) case k: return ltl_noise_d<k>(g, scale, rng, E, s);
    BFMRI_K_CASES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_aniso_scale(const AnisoArgs& a, cudaStream_t s) {
  if (a.K <= 0) return cudaSuccess;
  k_aniso_scale<<<1, 32, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_aniso_propose(const AnisoArgs& a, cudaStream_t s) {
  if (a.K <= 0) return cudaSuccess;
  k_aniso_propose<<<1, 32, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_aniso_accept(const AnisoArgs& a, cudaStream_t s) {
  if (a.K <= 0) return cudaSuccess;
  k_aniso_accept<<<1, 32, 0, s>>>(a);
  return cudaGetLastError();
}

template <int D>
static cudaError_t aux_d(const Geometry& g, const double* prop3, const double* E, double* blocks,
                         double* mfac, double* rhs, double* x, cudaStream_t s) {
  k_aux_system<D><<<(g.N + VOX_THREADS - 1) / VOX_THREADS, VOX_THREADS, 0, s>>>(g, prop3, E, blocks, mfac,
                                                                                rhs, x);
  return cudaGetLastError();
}

cudaError_t launch_aux_system(const Geometry& g, int D, const double* prop3, const double* E,
                              double* blocks, double* mfac, double* rhs, double* x, cudaStream_t s) {
  if (g.N <= 0) return cudaSuccess;
  switch (D) {
#define CASE(k) case k: return aux_d<k>(g, prop3, E, blocks, mfac, rhs, x, s);
    BFMRI_K_CASES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_apply(const ApplyArgs& a, cudaStream_t s) {
  if (a.g.N <= 0) return cudaSuccess;
  switch (a.D) {
#define CASE(k) case k: return apply_d<k>(a, s);
    BFMRI_K_CASES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bfmri
