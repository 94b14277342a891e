"""One Gibbs sweep (Section 3.2) composed from the full conditionals of Appendix A, with every
Gaussian draw made by Algorithm 2's perturbation and an EXACT solve in place of PCG.

Reading of the paper used here (the paper leaves the sweep order and start values open):
order W -> A -> lambda -> alpha -> beta; the prior on A is beta_p D_a with D_a = D_w
("spatial") or absent ("independent", beta unused); start values are the prior means
(Appendix C, trick 2) with A = 0 and W = 0.

Random numbers: every draw of sweep s uses Philox counter s with its own purpose tag
(oracle.philox), so a GPU sweep and an oracle sweep from the same state see the same
normals and uniforms.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import linalg, model, philox
from .lattice import Lattice


def default_state(K, P, N, priors=model.PRIORS):
    return dict(W=np.zeros((K, N)), A=np.zeros((P, N)),
                lam=np.full(N, priors["u1"] * priors["u2"]),
                alpha=np.full(K, priors["q1"] * priors["q2"]),
                beta=np.full(P, priors["r1"] * priors["r2"]))


def draw_gmrf(lat: Lattice, blocks, rhs, scale, seed, counter, tag, stream=0, prior="ugl"):
    """Algorithm 2 with an exact solve: b = rhs + sum_k sqrt(s_k) G'z1_k + H'L_data H z2
    (L' z1_k in place of G'z1_k for the L'L prior), then w = B~^-1 b. Returns (draw as
    (dim, N), conditional mean as (dim, N))."""
    N, K, _ = blocks.shape
    B = model.precision(lat, blocks, scale, prior)
    pert, _, _ = model.perturbation(lat, blocks, scale, seed, counter, tag, stream, prior)
    b_mean = model.kmajor(rhs)
    lu = linalg.factor(B)
    x = lu.solve(b_mean + pert)
    mu = lu.solve(b_mean)
    return x.reshape(K, N), mu.reshape(K, N)


def sample_W(lat, Y, X, state, seed, counter, eps=0.0, stream=0, prior="ugl"):
    Bd, bw = model.w_blocks_direct(Y, X, state["A"], state["lam"], eps)
    return draw_gmrf(lat, Bd, bw, state["alpha"], seed, counter, philox.TAG_W, stream, prior)[0]


def sample_A(lat, Y, X, state, seed, counter, spatial=True, stream=0):
    P = state["A"].shape[0]
    Ja, ba = model.a_blocks_direct(Y, X, state["W"], state["lam"], P)
    scale = state["beta"] if spatial else np.zeros(P)
    return draw_gmrf(lat, Ja, ba, scale, seed, counter, philox.TAG_A, stream)[0]


def sample_lambda(lat, Y, X, state, seed, counter, priors=model.PRIORS, stream=0):
    T = Y.shape[0]
    P = state["A"].shape[0]
    rss = model.rss_direct(Y, X, state["W"], state["A"])
    scale, shape = model.lambda_params(rss, T, P, priors["u1"], priors["u2"])
    lam, _ = philox.gamma(seed, lat.lin * 4 + 3, shape, scale, counter, philox.TAG_LAMBDA, stream)
    return lam


def sample_alpha(lat, state, seed, counter, priors=model.PRIORS, stream=0, prior="ugl", step=None):
    """Gamma full conditional of alpha_k (Eq. fullcondTempa); for the anisotropic prior the
    ray move and the exchange step (aniso_alpha_step) with log-normal step size `step`
    (default 1/sqrt(N))."""
    if prior == "aniso":
        return aniso_alpha_step(lat, state, seed, counter, 1.0 / np.sqrt(lat.N) if step is None else step,
                                priors, stream)[0]
    Q = (model.quad_forms_ltl if prior == "ltl" else model.quad_forms_edges)(lat, state["W"])
    scale, shape = model.alpha_params(Q, lat.N, priors["q1"], priors["q2"])
    a, _ = philox.gamma(seed, np.arange(len(Q)), shape, scale, counter, philox.TAG_ALPHA, stream)
    return a


# ----------------------------------------------------------------------------------------
# Anisotropic prior (Discussion): W_k has prior precision sum_d alpha_{d,k} L_d with
# alpha_{x,k}, alpha_{y,k}, alpha_{z,k} random. The paper leaves its inference open because
# the prior's determinant no longer factors out of the alpha's. The step below is the
# exchange algorithm of Murray, Ghahramani & MacKay (UAI 2006), which needs no determinant:
# for each k,
#   1. propose theta'_d = theta_d exp(step eps_d) (eps_d standard normal, d in the lattice's
#      directions; the z weight of a 4-neighbourhood lattice stays as it is);
#   2. draw an auxiliary field w' exactly from the prior at theta' (the GMRF draw of
#      Algorithm 2 with no data term: L(theta') w' = sum_d sqrt(theta'_d) G_d' C_d^(1/2) z);
#   3. accept theta' with probability min(1, a),
#        log a = sum_d [ -(theta'_d - theta_d)(Q_d(w) - Q_d(w')) / 2
#                        + q2 (log theta'_d - log theta_d) - (theta'_d - theta_d) / q1 ],
#      Q_d the direction-d edge sums: the likelihood ratio of (w, w') swapped between the two
#      parameter values, with the normalising constants cancelling, times the Ga(q1, q2) prior
#      ratio and the log-normal proposal's ratio theta'_d / theta_d.
# The intrinsic prior is improper along the constants of each connected part of the graph;
# w' is drawn on the complement (where it is a proper Gaussian) and Q_d does not see the
# constants.
# Before the exchange step, the common scale of alpha_{.,k} gets an exact draw: the move
# alpha -> lam alpha with lam from the posterior restricted to that ray (generalised Gibbs
# with the multiplicative group, Liu & Sabatti, JASA 2000: density pi(lam alpha) lam^(nd - 1)
# in lam). As pdet L(lam alpha) = lam^(N - c) pdet L(alpha) (c connected parts), this is
#   lam ~ Ga(shape nd q2 + (N - c)/2, rate sum_d alpha_d (1/q1 + Q_d / 2)),
# so the slow random walk only has to move the ratios between the directions.
# ----------------------------------------------------------------------------------------

def null_projector(lat: Lattice):
    """J = sum_c 1_c 1_c' / |c| over the connected parts of the voxel graph (the null space of
    every L(theta) with theta > 0)."""
    from scipy.sparse.csgraph import connected_components
    E = lat.edges()
    adj = sp.csr_matrix((np.ones(len(E)), (E[:, 0], E[:, 1])), shape=(lat.N, lat.N))
    nc, lab = connected_components(adj, directed=False)
    ind = sp.csr_matrix((np.ones(lat.N), (np.arange(lat.N), lab)), shape=(lat.N, nc))
    sizes = np.bincount(lab, minlength=nc).astype(np.float64)
    return (ind @ sp.diags(1.0 / sizes) @ ind.T).tocsr()


def aux_rhs(lat: Lattice, theta_k, z_k):
    """sum_d sqrt(theta_k[d]) G_d' C_d^(1/2) z_k for one k (z_k: one value per edge in edges()
    order): Algorithm 2's prior term, the auxiliary draw's right-hand side."""
    E = lat.edges()
    return lat.Gw().T @ (np.sqrt(np.asarray(theta_k, dtype=np.float64)[E[:, 2]]) * z_k)


def aux_solve(lat: Lattice, theta_k, z_k, J=None, Ls=None):
    """L(theta_k)^+ aux_rhs(theta_k, z_k) for one k. The right-hand side is orthogonal to the
    range of J, so (L + J) x = b gives x = L^+ b."""
    J = null_projector(lat) if J is None else J
    Ls = model.direction_laplacians(lat) if Ls is None else Ls
    theta_k = np.asarray(theta_k, dtype=np.float64)
    b = aux_rhs(lat, theta_k, z_k)
    return linalg.exact_solve(sum(theta_k[d] * Ls[d] for d in range(3)) + J, b)


def aux_prior_draw(lat: Lattice, theta, seed, counter, stream=0):
    """Step 2 for all k: aux_solve with z[e, k] the normal of edge e (site lattice-linear(i) * 4
    + d, lane k, TAG_ALPHA_AUX). Returns (K, N)."""
    theta = np.asarray(theta, dtype=np.float64)
    K = theta.shape[0]
    E = lat.edges()
    z = philox.normals(seed, lat.lin[E[:, 0]] * 4 + E[:, 2], K, counter, philox.TAG_ALPHA_AUX, stream)
    J = null_projector(lat)
    Ls = model.direction_laplacians(lat)
    return np.stack([aux_solve(lat, theta[k], z[:, k], J, Ls) for k in range(K)])


def n_parts(lat: Lattice):
    """Number of connected parts of the voxel graph."""
    from scipy.sparse.csgraph import connected_components
    E = lat.edges()
    adj = sp.csr_matrix((np.ones(len(E)), (E[:, 0], E[:, 1])), shape=(lat.N, lat.N))
    return connected_components(adj, directed=False)[0]


def scale_move_params(theta, Q, N, nparts, nd, priors=model.PRIORS):
    """(shape, rate) of lam per k for the ray move (theta, Q: K x 3)."""
    theta = np.asarray(theta, dtype=np.float64)
    shape = nd * priors["q2"] + 0.5 * (N - nparts)
    rate = np.sum(theta[:, :nd] * (1.0 / priors["q1"] + 0.5 * np.asarray(Q)[:, :nd]), axis=1)
    return shape, rate


def scale_move_alpha(lat, state, seed, counter, priors=model.PRIORS, stream=0):
    """The ray move for every k: returns (alpha' (K x 3), lam (K,)); lam from Philox tag
    TAG_ALPHA (site k), the Gamma generator of the graph-Laplacian alpha step."""
    theta = np.asarray(state["alpha"], dtype=np.float64)
    nd = lat.neighbourhood // 2
    Q = model.quad_forms_dirs(lat, state["W"])
    shape, rate = scale_move_params(theta, Q, lat.N, n_parts(lat), nd, priors)
    lam, _ = philox.gamma(seed, np.arange(theta.shape[0]), shape, 1.0 / rate, counter,
                          philox.TAG_ALPHA, stream)
    out = theta.copy()
    out[:, :nd] *= lam[:, None]
    return out, lam


def aniso_alpha_step(lat, state, seed, counter, step, priors=model.PRIORS, stream=0):
    """The anisotropic prior's alpha update: the ray move, then the exchange step from its
    result. Returns (alpha', accepted, details incl. lam and the scaled alphas)."""
    scaled, lam = scale_move_alpha(lat, state, seed, counter, priors, stream)
    new, acc, d = exchange_alpha(lat, dict(state, alpha=scaled), seed, counter, step, priors, stream)
    d.update(lam=lam, scaled=scaled)
    return new, acc, d


def exchange_log_ratio(theta, theta_p, Q, Qp, step_eps, nd, priors=model.PRIORS):
    """log a of step 3 per k (theta, theta_p, Q, Qp: K x 3; step_eps = log theta_p - log theta)."""
    dt = (theta_p - theta)[:, :nd]
    return np.sum(-0.5 * dt * (Q - Qp)[:, :nd] + priors["q2"] * step_eps[:, :nd] - dt / priors["q1"], axis=1)


def exchange_alpha(lat, state, seed, counter, step, priors=model.PRIORS, stream=0):
    """One exchange step for every k. state["alpha"] is K x 3. Returns (alpha', accepted (K,),
    details: proposal, eps, Q, Q', log a, u)."""
    theta = np.asarray(state["alpha"], dtype=np.float64)
    K = theta.shape[0]
    nd = lat.neighbourhood // 2
    eps = philox.normals(seed, np.arange(K), 3, counter, philox.TAG_ALPHA_PROP, stream)
    se = step * eps
    se[:, nd:] = 0.0
    theta_p = theta * np.exp(se)
    theta_p[:, nd:] = theta[:, nd:]
    wp = aux_prior_draw(lat, theta_p, seed, counter, stream)
    Q = model.quad_forms_dirs(lat, state["W"])
    Qp = model.quad_forms_dirs(lat, wp)
    la = exchange_log_ratio(theta, theta_p, Q, Qp, se, nd, priors)
    u = philox.uniform_open(seed, np.arange(K), 2, counter, philox.TAG_ALPHA_PROP, stream)
    acc = np.log(u) < la
    new = np.where(acc[:, None], theta_p, theta)
    return new, acc, dict(proposal=theta_p, eps=eps, Q=Q, Qp=Qp, log_a=la, u=u, aux=wp)


def sample_beta(lat, state, seed, counter, priors=model.PRIORS, stream=0):
    Q = model.quad_forms_edges(lat, state["A"])
    scale, shape = model.alpha_params(Q, lat.N, priors["r1"], priors["r2"])
    b, _ = philox.gamma(seed, np.arange(len(Q)), shape, scale, counter, philox.TAG_BETA, stream)
    return b


def gibbs_sweep(lat, Y, X, state, seed, counter, eps=0.0, spatial_ar=True,
                priors=model.PRIORS, stream=0, prior="ugl", step=None):
    """W -> A -> lambda -> alpha -> beta, each conditioned on the newest values (prior: the W
    prior, "ugl", "ltl" or "aniso"; A keeps the graph Laplacian)."""
    s = {k: np.array(v, copy=True) for k, v in state.items()}
    s["W"] = sample_W(lat, Y, X, s, seed, counter, eps, stream, prior)
    if s["A"].shape[0] > 0:
        s["A"] = sample_A(lat, Y, X, s, seed, counter, spatial_ar, stream)
    s["lam"] = sample_lambda(lat, Y, X, s, seed, counter, priors, stream)
    s["alpha"] = sample_alpha(lat, s, seed, counter, priors, stream, prior, step)
    if s["A"].shape[0] > 0 and spatial_ar:
        s["beta"] = sample_beta(lat, s, seed, counter, priors, stream)
    return s


# ----------------------------------------------------------------------------------------
# Spatial VB (Section 3.3; Appendix B, Eq. NFVBw / NFVBbB; Appendix C tricks)
# ----------------------------------------------------------------------------------------
# One SVB iteration, in the order W -> A -> lambda -> alpha -> beta. Expectations over W and A
# are Monte Carlo averages over N_s samples paired by index j (Eq. MC approx); the samples are
# drawn with Algorithm 2 from the averaged systems with the SAME random numbers at every
# iteration (stream j, a fixed draw counter), warm-started from the previous samples (the
# oracle solves exactly, so warm starts do not change its results).

def svb_w_system(Y, X, A_samples, lam_bar, eps=0.0):
    """B~_SVB blocks and b_SVB: the averages over j of the W-system blocks and right-hand
    sides evaluated at A^(j) with lambda replaced by its mean (Eq. NFVBbB)."""
    Bs, bs = zip(*[model.w_blocks_direct(Y, X, A, lam_bar, eps) for A in A_samples])
    return np.mean(Bs, axis=0), np.mean(bs, axis=0)


def svb_a_system(Y, X, W_samples, lam_bar, P):
    Js, bs = zip(*[model.a_blocks_direct(Y, X, W, lam_bar, P) for W in W_samples])
    return np.mean(Js, axis=0), np.mean(bs, axis=0)


def svb_draw(lat, blocks, rhs, scale, seed, counter, tag, n_samples):
    return [draw_gmrf(lat, blocks, rhs, scale, seed, counter, tag, stream=j)[0]
            for j in range(n_samples)]


def svb_lambda_mean(Y, X, W_samples, A_samples, priors=model.PRIORS):
    """E[lambda_n] = u~1n u~2 with 1/u~1n = 1/u1 + mean_j RSS_n(W^(j), A^(j)) / 2."""
    T = Y.shape[0]
    P = A_samples[0].shape[0]
    rss = np.mean([model.rss_direct(Y, X, W, A) for W, A in zip(W_samples, A_samples)], axis=0)
    scale, shape = model.lambda_params(rss, T, P, priors["u1"], priors["u2"])
    return scale * shape


def svb_hyper_mean(lat, samples, prior1, prior2):
    """E[alpha_k] = q~1k q~2 with 1/q~1k = mean_j W_k^(j) D W_k^(j)' / 2 + 1/q1
    (Eq. NFVB-alpha-parameters with Eq. MC approx); the same form for beta."""
    Q = np.mean([model.quad_forms_edges(lat, V) for V in samples], axis=0)
    scale, shape = model.alpha_params(Q, lat.N, prior1, prior2)
    return scale * shape, Q


def svb_extrapolate(history, proposal):
    """Appendix C, trick 1 (pinned branch by branch to values worked by hand from the rule
    the appendix states; the paper prints no iterate values). history
    holds the values used at iterations j-2 and j-1, proposal is the VB value at j. Fit a
    parabola through the three points; if its vertex lies after j use the vertex value, else
    step 20 times the last change; keep within a factor 5 of the proposal; fall back to the
    proposal when the prediction is not positive."""
    a2, a1 = history
    a0 = proposal
    # parabola through (-2, a2), (-1, a1), (0, a0): y = c x^2 + d x + a0
    c = 0.5 * (a2 - 2.0 * a1 + a0)
    d = 0.5 * (a2 - 4.0 * a1 + 3.0 * a0)
    pred = np.where((c != 0.0) & (-d / np.where(c != 0.0, 2.0 * c, 1.0) > 0.0),
                    a0 - d * d / np.where(c != 0.0, 4.0 * c, 1.0), a1 + 20.0 * (a0 - a1))
    pred = np.where(pred > 0.0, pred, a0)
    return np.clip(pred, a0 / 5.0, 5.0 * a0)


def svb_step(lat, Y, X, state, W_samples, A_samples, seed, counter, eps=0.0, spatial_ar=True,
             priors=model.PRIORS):
    """One SVB iteration without the Appendix C extrapolation; returns the new means and
    samples. state holds lam (E[lambda]), alpha (E[alpha]), beta (E[beta])."""
    Ns = len(W_samples)
    P = A_samples[0].shape[0]
    Bd, bw = svb_w_system(Y, X, A_samples, state["lam"], eps)
    Wn = svb_draw(lat, Bd, bw, state["alpha"], seed, counter, philox.TAG_W, Ns)
    An = list(A_samples)
    if P > 0:
        Ja, ba = svb_a_system(Y, X, Wn, state["lam"], P)
        scale = state["beta"] if spatial_ar else np.zeros(P)
        An = svb_draw(lat, Ja, ba, scale, seed, counter, philox.TAG_A, Ns)
    lam = svb_lambda_mean(Y, X, Wn, An, priors)
    alpha, QW = svb_hyper_mean(lat, Wn, priors["q1"], priors["q2"])
    beta = state["beta"]
    if P > 0 and spatial_ar:
        beta, _ = svb_hyper_mean(lat, An, priors["r1"], priors["r2"])
    return dict(lam=lam, alpha=alpha, beta=beta, QW=QW), Wn, An
