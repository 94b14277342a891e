// Posterior summaries on the device.
//  * Chain accumulators (Section 3.2, Eq. MCMCPPM and Eq. MCMCjointPPM): per voxel and
//    contrast the number of Gibbs samples with c'W_.,n > gamma, per contrast the number of
//    samples in which every voxel of a set exceeds gamma, and shifted sample moments of W.
//  * SVB summaries (Section 3.3): moments of the N_s samples of q(W) and the Gaussian
//    contrast PPM with those moments.
//  * The unnormalised log joint posterior (Appendix A, Eq. UnnormalisedJointPosterior).
// Every kernel streams its planes once with one thread per voxel (coalesced along the
// voxel index); the reductions run in a fixed order, so results do not depend on timing.
#include <cmath>

#include "summary.cuh"

namespace bfmri {
namespace {

constexpr int SUM_THREADS = 256;
constexpr int S2_CHUNK = 36;   // packed second moments updated per load/store round
constexpr int LJ_THREADS = 128;   // ~240 registers a thread: two CTAs per SM

#define SUM_K_CASES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12)

// c'w over k = 0..K-1 in order with one rounding per product and per sum (never contracted
// into a fused multiply-add), so that the decision c'w > gamma is the same in any IEEE FP64
// evaluation of this order.
template <int K>
__device__ __forceinline__ double contrast_value(const double* c, const double* w) {
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < K; ++k) s = __dadd_rn(s, __dmul_rn(c[k], w[k]));
  return s;
}

template <int K>
__global__ void __launch_bounds__(SUM_THREADS) k_chain_accumulate(ChainSumArgs a) {
  __shared__ double shC[MAX_CONTRASTS * K];
  __shared__ double shg[MAX_CONTRASTS];
  __shared__ unsigned int sh_fail;
  __shared__ int sh_last;
  for (int i = threadIdx.x; i < a.nc * K; i += blockDim.x) shC[i] = a.C[i];
  for (int i = threadIdx.x; i < a.nc; i += blockDim.x) shg[i] = a.gamma[i];
  if (threadIdx.x == 0) sh_fail = 0u;
  __syncthreads();
  const size_t ld = a.g.ld;
  unsigned int fail = 0u;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < a.g.N; n += gridDim.x * blockDim.x) {
    // loads first, then the arithmetic, then the stores: the planes are distinct, but a store
    // between two loads would serialise them behind possible aliasing. S2 goes in chunks of
    // S2_CHUNK entries and the counts in groups of 4 contrasts to bound the registers.
    double w[K], d[K], s1[K], t[S2_CHUNK];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      w[k] = a.W[(size_t)k * ld + n];
      d[k] = a.ref[(size_t)k * ld + n];
      s1[k] = a.S1[(size_t)k * ld + n];
    }
#pragma unroll
    for (int e = 0; e < S2_CHUNK; ++e)
      if (e < ntri(K)) t[e] = a.S2[(size_t)e * ld + n];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      d[k] = w[k] - d[k];
      s1[k] += d[k];
      a.S1[(size_t)k * ld + n] = s1[k];
    }
#pragma unroll
    for (int e0 = 0; e0 < ntri(K); e0 += S2_CHUNK) {
      if (e0 > 0) {
#pragma unroll
        for (int e = 0; e < S2_CHUNK; ++e)
          if (e0 + e < ntri(K)) t[e] = a.S2[(size_t)(e0 + e) * ld + n];
      }
#pragma unroll
      for (int i = 0; i < K; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
          const int e = tri(i, j) - e0;
          if (e >= 0 && e < S2_CHUNK) t[e] += d[i] * d[j];
        }
#pragma unroll
      for (int e = 0; e < S2_CHUNK; ++e)
        if (e0 + e < ntri(K)) a.S2[(size_t)(e0 + e) * ld + n] = t[e];
    }
    const bool in_set = a.in_set && a.in_set[n];
    for (int c0 = 0; c0 < a.nc; c0 += 4) {
      int cnt[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) cnt[u] = c0 + u < a.nc ? a.count[(size_t)(c0 + u) * ld + n] : 0;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (c0 + u < a.nc) {
          const bool above = contrast_value<K>(shC + (c0 + u) * K, w) > shg[c0 + u];
          cnt[u] += above ? 1 : 0;
          if (in_set && !above) fail |= 1u << (c0 + u);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (c0 + u < a.nc) a.count[(size_t)(c0 + u) * ld + n] = cnt[u];
    }
  }
  // joint set: OR of the failures of this CTA, then of the grid; the last CTA to arrive books
  // the sample for every contrast whose set saw no failure and clears the scratch words
  fail = __reduce_or_sync(0xffffffffu, fail);
  if ((threadIdx.x & 31) == 0 && fail) atomicOr(&sh_fail, fail);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (sh_fail) atomicOr(a.fail, sh_fail);
    __threadfence();
    const unsigned int t = atomicAdd(a.ticket, 1u);
    sh_last = t == gridDim.x - 1 ? 1 : 0;
  }
  __syncthreads();
  if (sh_last && threadIdx.x == 0) {
    __threadfence();
    const unsigned int f = atomicExch(a.fail, 0u);
    if (a.in_set) {
      for (int c = 0; c < a.nc; ++c)
        if (!((f >> c) & 1u)) a.joint[c] += 1ull;
    } else {
      for (int c = 0; c < a.nc; ++c) a.joint[c] += 1ull;   // the empty set: always satisfied
    }
    atomicExch(a.ticket, 0u);
  }
}

template <int K>
__global__ void __launch_bounds__(SUM_THREADS) k_chain_finalize(ChainFinalArgs a) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.g.N) return;
  const size_t ld = a.g.ld;
  // FP64 division is a long instruction sequence on this part: the moments multiply by
  // reciprocals; the PPMs keep the exact quotient count / n
  const double nn = (double)a.n, rn = 1.0 / nn, rn1 = a.n >= 2 ? 1.0 / (nn - 1.0) : 0.0;
  double s1[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    s1[k] = a.S1[(size_t)k * ld + n];
    a.mean[(size_t)k * ld + n] = a.ref[(size_t)k * ld + n] + s1[k] * rn;
  }
#pragma unroll
  for (int i = 0; i < K; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      const size_t o = (size_t)tri(i, j) * ld + n;
      a.cov[o] = (a.S2[o] - s1[i] * s1[j] * rn) * rn1;
    }
  for (int c = 0; c < a.nc; ++c) a.ppm[(size_t)c * ld + n] = (double)a.count[(size_t)c * ld + n] / nn;
}

// Samples are taken SVB_UNROLL at a time with all their loads issued before the arithmetic,
// so that each thread keeps SVB_UNROLL * K loads in flight.
constexpr int SVB_THREADS = 128;
constexpr int SVB_UNROLL = 4;

template <int K>
__global__ void __launch_bounds__(SVB_THREADS) k_svb_summary(SvbSumArgs a) {
  __shared__ double shC[MAX_CONTRASTS * K];
  __shared__ double shg[MAX_CONTRASTS];
  for (int i = threadIdx.x; i < a.nc * K; i += blockDim.x) shC[i] = a.C[i];
  for (int i = threadIdx.x; i < a.nc; i += blockDim.x) shg[i] = a.gamma[i];
  __syncthreads();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.g.N) return;
  const size_t ld = a.g.ld, vs = (size_t)K * ld;
  const double* __restrict__ Wn = a.Ws + n;
  double x0[K], s1[K], s2[ntri(K)];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    x0[k] = __ldg(Wn + (size_t)k * ld);
    s1[k] = 0.0;
  }
#pragma unroll
  for (int e = 0; e < ntri(K); ++e) s2[e] = 0.0;
  auto add = [&](const double* d) {
#pragma unroll
    for (int k = 0; k < K; ++k) s1[k] += d[k];
#pragma unroll
    for (int i = 0; i < K; ++i)
#pragma unroll
      for (int jj = 0; jj <= i; ++jj) s2[tri(i, jj)] += d[i] * d[jj];
  };
  int j = 1;
  for (; j + SVB_UNROLL <= a.S; j += SVB_UNROLL) {
    double v[SVB_UNROLL][K];
#pragma unroll
    for (int u = 0; u < SVB_UNROLL; ++u)
#pragma unroll
      for (int k = 0; k < K; ++k) v[u][k] = __ldg(Wn + (size_t)(j + u) * vs + (size_t)k * ld);
#pragma unroll
    for (int u = 0; u < SVB_UNROLL; ++u) {
#pragma unroll
      for (int k = 0; k < K; ++k) v[u][k] -= x0[k];
      add(v[u]);
    }
  }
  for (; j < a.S; ++j) {
    double d[K];
#pragma unroll
    for (int k = 0; k < K; ++k) d[k] = __ldg(Wn + (size_t)j * vs + (size_t)k * ld) - x0[k];
    add(d);
  }
  const double S = (double)a.S;
  double mu[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    mu[k] = x0[k] + s1[k] / S;
    a.mean[(size_t)k * ld + n] = mu[k];
  }
#pragma unroll
  for (int i = 0; i < K; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      s2[tri(i, j)] = a.S >= 2 ? (s2[tri(i, j)] - s1[i] * s1[j] / S) / (S - 1.0) : 0.0;
      a.cov[(size_t)tri(i, j) * ld + n] = s2[tri(i, j)];
    }
  for (int c = 0; c < a.nc; ++c) {
    const double* cc = shC + c * K;
    double m = 0.0, v = 0.0;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      m += cc[i] * mu[i];
      double row = 0.0;
#pragma unroll
      for (int j = 0; j < K; ++j) row += s2[i >= j ? tri(i, j) : tri(j, i)] * cc[j];
      v += cc[i] * row;
    }
    a.ppm[(size_t)c * ld + n] = v > 0.0 ? 0.5 * erfc((shg[c] - m) / sqrt(2.0 * v)) : (m > shg[c] ? 1.0 : 0.0);
  }
}

template <int K>
__global__ void __launch_bounds__(LJ_THREADS) k_log_joint_voxels(LogJointArgs a) {
  extern __shared__ double shQ[];
  __shared__ double shred[LJ_THREADS / 32][2];
  load_quad_weights(a.Sxx, K, a.P, shQ);
  __syncthreads();
  const size_t ld = a.g.ld;
  const int P = a.P;
  double ll = 0.0, lp = 0.0;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < a.g.N; n += gridDim.x * blockDim.x) {
    double w[K];
#pragma unroll
    for (int k = 0; k < K; ++k) w[k] = a.W[(size_t)k * ld + n];
    double G[PMAX + 1][PMAX + 1];
    lagged_gram<K>(a.stats, shQ, w, P, ld, n, G);
    double c[PMAX + 1];
    c[0] = 1.0;
#pragma unroll
    for (int p = 1; p <= PMAX; ++p) c[p] = p <= P ? -a.A[(size_t)(p - 1) * ld + n] : 0.0;
    double rss = 0.0;
#pragma unroll
    for (int p = 0; p <= PMAX; ++p)
#pragma unroll
      for (int q = 0; q <= PMAX; ++q) rss += c[p] * c[q] * G[p][q];
    const double lam = a.lam[n], loglam = log(lam);
    ll += 0.5 * (double)(a.T - P) * loglam - 0.5 * lam * rss;
    lp += (a.u2 - 1.0) * loglam - lam / a.u1;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ll += __shfl_down_sync(0xffffffffu, ll, o);
    lp += __shfl_down_sync(0xffffffffu, lp, o);
  }
  if ((threadIdx.x & 31) == 0) {
    shred[threadIdx.x >> 5][0] = ll;
    shred[threadIdx.x >> 5][1] = lp;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double s = 0.0;
    for (int i = 0; i < LJ_THREADS / 32; ++i) s += shred[i][threadIdx.x];
    a.part[(size_t)blockIdx.x * 2 + threadIdx.x] = s;
  }
}

// Warp i (i = 0, 1) adds column i of the CTA sums with its lanes striding over the CTAs and
// a butterfly (a fixed order); thread 0 then adds the hyperparameter terms.
__global__ void k_log_joint_final(LogJointArgs a, int nblocks) {
  __shared__ double sh[2];
  const int col = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (col < 2) {
    double v = 0.0;
    for (int b = lane; b < nblocks; b += 32) v += a.part[(size_t)b * 2 + col];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[col] = v;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double ll = sh[0], lp = sh[1];
  const double halfN = 0.5 * (double)a.g.N;
  double wp = 0.0, ap = 0.0, alp = 0.0, bep = 0.0;
  for (int k = 0; k < a.K; ++k) {
    const double al = a.alpha[k], lg = log(al);
    wp += halfN * lg - 0.5 * al * a.Qw[k];
    alp += (a.q2 - 1.0) * lg - al / a.q1;
  }
  if (a.spatial && a.P > 0) {
    for (int p = 0; p < a.P; ++p) {
      const double be = a.beta[p], lg = log(be);
      ap += halfN * lg - 0.5 * be * a.Qa[p];
      bep += (a.r2 - 1.0) * lg - be / a.r1;
    }
  }
  a.terms[0] = ll;
  a.terms[1] = wp;
  a.terms[2] = ap;
  a.terms[3] = lp;
  a.terms[4] = alp;
  a.terms[5] = bep;
  a.terms[6] = ll + wp + ap + lp + alp + bep;
}

int sum_grid(int N) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int need = (N + SUM_THREADS - 1) / SUM_THREADS;
  const int cap = 4 * (nsm > 0 ? nsm : 1);
  return need < 1 ? 1 : (need < cap ? need : cap);
}

template <int K>
cudaError_t chain_acc_k(const ChainSumArgs& a, cudaStream_t s) {
  k_chain_accumulate<K><<<sum_grid(a.g.N), SUM_THREADS, 0, s>>>(a);
  return cudaGetLastError();
}

template <int K>
cudaError_t chain_fin_k(const ChainFinalArgs& a, cudaStream_t s) {
  k_chain_finalize<K><<<(a.g.N + SUM_THREADS - 1) / SUM_THREADS, SUM_THREADS, 0, s>>>(a);
  return cudaGetLastError();
}

template <int K>
cudaError_t svb_sum_k(const SvbSumArgs& a, cudaStream_t s) {
  k_svb_summary<K><<<(a.g.N + SVB_THREADS - 1) / SVB_THREADS, SVB_THREADS, 0, s>>>(a);
  return cudaGetLastError();
}

template <int K>
cudaError_t log_joint_k(const LogJointArgs& a, cudaStream_t s) {
  const size_t shm = quad_weight_doubles(K, a.P) * sizeof(double);
  if (cudaError_t e = raise_smem_limit((const void*)k_log_joint_voxels<K>, shm)) return e;
  const int grid = log_joint_grid(a.g.N);
  k_log_joint_voxels<K><<<grid, LJ_THREADS, shm, s>>>(a);
  k_log_joint_final<<<1, 64, 0, s>>>(a, grid);
  return cudaGetLastError();
}

}  // namespace

// one wave of two CTAs per SM, voxels strided over the grid
int log_joint_grid(int N) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int need = (N + LJ_THREADS - 1) / LJ_THREADS;
  const int cap = 2 * (nsm > 0 ? nsm : 1);
  return need < 1 ? 1 : (need < cap ? need : cap);
}

cudaError_t launch_chain_accumulate(const ChainSumArgs& a, cudaStream_t s) {
  if (a.g.N <= 0 || a.nc < 0 || a.nc > MAX_CONTRASTS) return cudaErrorInvalidValue;
  switch (a.K) {
#define CASE(k) case k: return chain_acc_k<k>(a, s);
    SUM_K_CASES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_chain_finalize(const ChainFinalArgs& a, cudaStream_t s) {
  if (a.g.N <= 0 || a.n <= 0) return cudaErrorInvalidValue;
  switch (a.K) {
#define CASE(k) case k: return chain_fin_k<k>(a, s);
    SUM_K_CASES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_svb_summary(const SvbSumArgs& a, cudaStream_t s) {
  if (a.g.N <= 0 || a.S <= 0 || a.nc < 0 || a.nc > MAX_CONTRASTS) return cudaErrorInvalidValue;
  switch (a.K) {
#define CASE(k) case k: return svb_sum_k<k>(a, s);
    SUM_K_CASES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_log_joint(const LogJointArgs& a, cudaStream_t s) {
  if (a.g.N <= 0) return cudaErrorInvalidValue;
  switch (a.K) {
#define CASE(k) case k: return log_joint_k<k>(a, s);
    SUM_K_CASES(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bfmri
