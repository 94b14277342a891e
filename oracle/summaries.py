"""Posterior summaries of the sampler's output (test infrastructure only, like the whole
package: nothing in the product path may import it).

chain_summary -- Section 3.2, Eq. MCMCPPM and Eq. MCMCjointPPM: the marginal PPM of a contrast
                 c in voxel n is the fraction of Gibbs samples with c'W_.,n > gamma; the
                 joint PPM of a voxel set E is the fraction of samples in which every voxel
                 of E exceeds gamma. Also the sample mean and covariance of W_.,n.
svb_summary   -- Section 3.3: marginal and contrast PPMs of q(W) from the sample mean and
                 the per-voxel sample covariance of the N_s SVB samples (the Gaussian tail
                 probability of c'W_.,n with those moments).
log_joint     -- Appendix A, Eq. UnnormalisedJointPosterior: log of the unnormalised joint
                 posterior as the sum of the likelihood (Eq. log-like without its constant),
                 the UGL priors of W and A (Eq. UnnormalisedWPrior) and the Gamma
                 hyperpriors of lambda, alpha, beta.

Readings (the paper is silent on them):
* the contrast value c'W_.,n is accumulated over k = 0..K-1 in that order with one rounding
  per product and per sum (no fused multiply-add), so that a CUDA path doing the same takes
  every threshold decision identically;
* a joint PPM over the empty set is 1 (every sample satisfies the empty conjunction);
* sample covariances divide by S - 1 (S >= 2; zero for S = 1);
* the Gaussian PPM of a contrast with zero sample variance is the indicator c'mu > gamma;
* Ga(b, c) has scale b and shape c, so log Ga(x; b, c) = (c - 1) log x - x / b + const;
* under the independent AR prior (no spatial prior on A) the A-prior and beta terms are 0.
"""
from __future__ import annotations

import math

import numpy as np

from . import model
from .lattice import Lattice


def contrast_values(C, W):
    """c_i' W_.,n for every contrast i and voxel n, summed over k in order, one rounding per
    product and per addition. C: (n_c, K); W: (K, N). Returns (n_c, N)."""
    C = np.asarray(C, dtype=np.float64)
    n_c, K = C.shape
    out = np.zeros((n_c, W.shape[1]))
    for i in range(n_c):
        s = np.zeros(W.shape[1])
        for k in range(K):
            s = s + C[i, k] * W[k]
        out[i] = s
    return out


def sample_moments(samples):
    """Sample mean (K, N) and covariance (N, K, K) with divisor S - 1, two-pass."""
    S = len(samples)
    K, N = samples[0].shape
    mean = np.zeros((K, N))
    for Wj in samples:
        mean += Wj
    mean /= S
    cov = np.zeros((N, K, K))
    if S >= 2:
        for Wj in samples:
            d = Wj - mean
            cov += np.einsum("in,jn->nij", d, d)
        cov /= S - 1
    return mean, cov


def chain_summary(samples, C, gamma, E=None):
    """Eq. MCMCPPM / Eq. MCMCjointPPM over the Gibbs samples W^(1..S) (each K x N).

    Returns dict(n=S, mean, cov, count (n_c, N) exceedance counts, ppm = count / S,
    joint_count (n_c,), joint_ppm). E: voxel indices (compact order) of the joint set."""
    S = len(samples)
    gamma = np.asarray(gamma, dtype=np.float64)
    n_c = len(gamma)
    N = samples[0].shape[1]
    E = np.asarray([] if E is None else E, dtype=np.int64)
    count = np.zeros((n_c, N), dtype=np.int64)
    joint = np.zeros(n_c, dtype=np.int64)
    for Wj in samples:
        v = contrast_values(C, Wj)
        above = v > gamma[:, None]
        count += above
        for i in range(n_c):
            if all(above[i, n] for n in E):
                joint[i] += 1
    mean, cov = sample_moments(samples)
    return dict(n=S, mean=mean, cov=cov, count=count, ppm=count / S, joint_count=joint,
                joint_ppm=joint / S)


def svb_summary(samples, C, gamma):
    """Section 3.3: moments of the N_s samples of q(W) and, per voxel and contrast,
    P(c'W_.,n > gamma) for c'W_.,n ~ N(c'mu_n, c' Sigma_n c) with the sample moments."""
    mean, cov = sample_moments(samples)
    C = np.asarray(C, dtype=np.float64)
    gamma = np.asarray(gamma, dtype=np.float64)
    N = mean.shape[1]
    ppm = np.zeros((len(gamma), N))
    for i in range(len(gamma)):
        c = C[i]
        for n in range(N):
            m = float(c @ mean[:, n])
            v = float(c @ cov[n] @ c)
            if v > 0.0:
                ppm[i, n] = 0.5 * math.erfc((gamma[i] - m) / math.sqrt(2.0 * v))
            else:
                ppm[i, n] = 1.0 if m > gamma[i] else 0.0
    return dict(mean=mean, cov=cov, ppm=ppm)


def log_joint(lat: Lattice, Y, X, state, T, priors=model.PRIORS, spatial_ar=True, prior="ugl"):
    """Eq. UnnormalisedJointPosterior at state = dict(W, A, lam, alpha, beta).

    loglik      = sum_n [(T - P)/2 log lambda_n - lambda_n RSS_n / 2]   (Eq. log-like; RSS
                  from the residual time series)
    W prior     = sum_k [N/2 log alpha_k - alpha_k W_k D_w W_k' / 2]      (Eq. UnnormalisedWPrior)
    A prior     = sum_p [N/2 log beta_p - beta_p A_p D_a A_p' / 2]        (D_a = D_w)
    lambda, alpha, beta priors: Gamma log densities without their constants.
    prior = "ltl": D_w = L'L in the W prior (W_k D_w W_k' = |L W_k'|^2); its normaliser scales
    with alpha_k as that of L, so the N/2 log alpha_k term is the same.
    Returns dict of the six terms and their total."""
    W, A = state["W"], state["A"]
    lam = np.asarray(state["lam"], dtype=np.float64)
    alpha = np.asarray(state["alpha"], dtype=np.float64)
    beta = np.asarray(state.get("beta", np.zeros(0)), dtype=np.float64)
    P, N = A.shape
    rss = model.rss_direct(Y, X, W, A)
    terms = {}
    terms["loglik"] = float(np.sum(0.5 * (T - P) * np.log(lam) - 0.5 * lam * rss))
    Qw = model.quad_forms_ltl(lat, W) if prior == "ltl" else model.quad_forms_laplacian(lat, W)
    terms["W_prior"] = float(np.sum(0.5 * N * np.log(alpha) - 0.5 * alpha * Qw))
    sp_a = spatial_ar and P > 0
    if sp_a:
        Qa = model.quad_forms_laplacian(lat, A)
        terms["A_prior"] = float(np.sum(0.5 * N * np.log(beta) - 0.5 * beta * Qa))
    else:
        terms["A_prior"] = 0.0
    u1, u2 = priors["u1"], priors["u2"]
    q1, q2 = priors["q1"], priors["q2"]
    r1, r2 = priors["r1"], priors["r2"]
    terms["lambda_prior"] = float(np.sum((u2 - 1.0) * np.log(lam) - lam / u1))
    terms["alpha_prior"] = float(np.sum((q2 - 1.0) * np.log(alpha) - alpha / q1))
    terms["beta_prior"] = float(np.sum((r2 - 1.0) * np.log(beta) - beta / r1)) if sp_a else 0.0
    terms["total"] = sum(terms[k] for k in ("loglik", "W_prior", "A_prior", "lambda_prior",
                                            "alpha_prior", "beta_prior"))
    return terms
