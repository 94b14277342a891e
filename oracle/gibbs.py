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

from . import linalg, model, philox
from .lattice import Lattice


def default_state(K, P, N, priors=model.PRIORS):
    return dict(W=np.zeros((K, N)), A=np.zeros((P, N)),
                lam=np.full(N, priors["u1"] * priors["u2"]),
                alpha=np.full(K, priors["q1"] * priors["q2"]),
                beta=np.full(P, priors["r1"] * priors["r2"]))


def draw_gmrf(lat: Lattice, blocks, rhs, scale, seed, counter, tag, stream=0):
    """Algorithm 2 with an exact solve: b = rhs + sum_k sqrt(s_k) G'z1_k + H'L_data H z2,
    then w = B~^-1 b. Returns (draw as (dim, N), conditional mean as (dim, N))."""
    N, K, _ = blocks.shape
    B = model.precision(lat, blocks, scale)
    pert, _, _ = model.perturbation(lat, blocks, scale, seed, counter, tag, stream)
    b_mean = model.kmajor(rhs)
    lu = linalg.factor(B)
    x = lu.solve(b_mean + pert)
    mu = lu.solve(b_mean)
    return x.reshape(K, N), mu.reshape(K, N)


def sample_W(lat, Y, X, state, seed, counter, eps=0.0, stream=0):
    Bd, bw = model.w_blocks_direct(Y, X, state["A"], state["lam"], eps)
    return draw_gmrf(lat, Bd, bw, state["alpha"], seed, counter, philox.TAG_W, stream)[0]


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


def sample_alpha(lat, state, seed, counter, priors=model.PRIORS, stream=0):
    Q = model.quad_forms_edges(lat, state["W"])
    scale, shape = model.alpha_params(Q, lat.N, priors["q1"], priors["q2"])
    a, _ = philox.gamma(seed, np.arange(len(Q)), shape, scale, counter, philox.TAG_ALPHA, stream)
    return a


def sample_beta(lat, state, seed, counter, priors=model.PRIORS, stream=0):
    Q = model.quad_forms_edges(lat, state["A"])
    scale, shape = model.alpha_params(Q, lat.N, priors["r1"], priors["r2"])
    b, _ = philox.gamma(seed, np.arange(len(Q)), shape, scale, counter, philox.TAG_BETA, stream)
    return b


def gibbs_sweep(lat, Y, X, state, seed, counter, eps=0.0, spatial_ar=True,
                priors=model.PRIORS, stream=0):
    """W -> A -> lambda -> alpha -> beta, each conditioned on the newest values."""
    s = {k: np.array(v, copy=True) for k, v in state.items()}
    s["W"] = sample_W(lat, Y, X, s, seed, counter, eps, stream)
    if s["A"].shape[0] > 0:
        s["A"] = sample_A(lat, Y, X, s, seed, counter, spatial_ar, stream)
    s["lam"] = sample_lambda(lat, Y, X, s, seed, counter, priors, stream)
    s["alpha"] = sample_alpha(lat, s, seed, counter, priors, stream)
    if s["A"].shape[0] > 0 and spatial_ar:
        s["beta"] = sample_beta(lat, s, seed, counter, priors, stream)
    return s
