// Host interface of the posterior-summary kernels (kernels_summary.cu): chain accumulators
// for contrast PPMs and sample moments, SVB sample moments with Gaussian contrast PPMs, and
// the per-voxel part of the unnormalised log joint posterior.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "model.cuh"

namespace bfmri {

constexpr int MAX_CONTRASTS = 16;

// One Gibbs sample W (after a sweep) added to the chain accumulators, per voxel n:
//   S1[k] += d_k, S2[tri(i, j)] += d_i d_j with d = W_.,n - ref_.,n (moments shifted by a
//   reference sample, so that the covariance keeps its digits when the mean is large),
//   count[c] += (c'W_.,n > gamma_c)                                      (Eq. MCMCPPM),
// and, over the voxels flagged in in_set, joint[c] += 1 when every one of them exceeds
// gamma_c (Eq. MCMCjointPPM; the last CTA to finish books the sample).
struct ChainSumArgs {
  Geometry g;
  int K, nc;
  const double* W;          // [K][ld]
  const double* ref;        // [K][ld]
  const double* C;          // [nc][K] contrasts
  const double* gamma;      // [nc]
  const uint8_t* in_set;    // [ld] joint-set flags, or null (no joint set)
  double* S1;               // [K][ld]
  double* S2;               // [ntri(K)][ld]
  int* count;               // [nc][ld]
  unsigned long long* joint;  // [nc]
  unsigned int* fail;       // scratch word, zero between launches
  unsigned int* ticket;     // scratch word, zero between launches
};
cudaError_t launch_chain_accumulate(const ChainSumArgs& a, cudaStream_t s);

// mean = ref + S1 / n, cov = (S2 - S1 S1' / n) / (n - 1) (0 when n < 2), ppm = count / n.
struct ChainFinalArgs {
  Geometry g;
  int K, nc;
  long long n;
  const double* ref;
  const double* S1;
  const double* S2;
  const int* count;
  double* mean;             // [K][ld]
  double* cov;              // [ntri(K)][ld]
  double* ppm;              // [nc][ld]
};
cudaError_t launch_chain_finalize(const ChainFinalArgs& a, cudaStream_t s);

// Moments of S samples Ws[j][k][n] (shifted by sample 0) and, per contrast, the Gaussian tail
// P(c'W_.,n > gamma) = erfc((gamma - c'mu) / sqrt(2 c'Sigma c)) / 2 (indicator when the
// variance is 0).
struct SvbSumArgs {
  Geometry g;
  int K, S, nc;
  const double* Ws;         // [S][K][ld]
  const double* C;          // [nc][K]
  const double* gamma;      // [nc]
  double* mean;             // [K][ld]
  double* cov;              // [ntri(K)][ld]
  double* ppm;              // [nc][ld]
};
cudaError_t launch_svb_summary(const SvbSumArgs& a, cudaStream_t s);

// Log joint posterior: per-voxel likelihood and lambda-prior terms, summed per CTA
//   l_n = (T - P)/2 log lambda_n - lambda_n RSS_n / 2,  p_n = (u2 - 1) log lambda_n - lambda_n / u1
// with RSS_n = c' G_n c, c = (1, -a_n) and G_n the lagged residual Gram of W_.,n; then a
// one-warp kernel adds the CTA sums in order with the alpha / beta terms from the quadratic
// forms Q (launch_hyper with out = null): terms[0..6] = loglik, W prior, A prior,
// lambda prior, alpha prior, beta prior, total.
struct LogJointArgs {
  Geometry g;
  int K, P, T;
  int spatial;              // 1: the A prior and beta terms are included
  const double* stats;
  const double* Sxx;
  const double* W;
  const double* A;
  const double* lam;
  const double* alpha;
  const double* beta;
  const double* Qw;         // [K]
  const double* Qa;         // [P]
  double u1, u2, q1, q2, r1, r2;
  double* part;             // [grid][2]
  double* terms;            // [7]
};
cudaError_t launch_log_joint(const LogJointArgs& a, cudaStream_t s);
int log_joint_grid(int N);

}  // namespace bfmri
