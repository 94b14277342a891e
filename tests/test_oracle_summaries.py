"""Pins for the oracle's posterior summaries (CPU only).

Each pin compares the oracle with something other than itself: numpy's mean and covariance,
scipy's normal and Gamma densities, samples built so that every count is known in closed
form, exact invariants (complementary contrasts, one-voxel joint sets, monotonicity in the
threshold), Monte Carlo limits, and a time-domain evaluation of the likelihood with scipy's
normal density.
"""
import math

import numpy as np
import pytest
import scipy.stats as st

from oracle import model, summaries
from oracle.lattice import Lattice
from paper_1606_00980_gb300 import synth


def random_samples(S, K, N, seed, scale=1.0, shift=0.0):
    rng = np.random.default_rng(seed)
    return [shift + scale * rng.standard_normal((K, N)) for _ in range(S)]


def test_moments_match_numpy():
    xs = random_samples(9, 4, 7, 1, scale=0.3, shift=100.0)
    mean, cov = summaries.sample_moments(xs)
    stack = np.stack(xs)                             # (S, K, N)
    assert np.allclose(mean, stack.mean(axis=0), rtol=1e-14, atol=0)
    for n in range(7):
        assert np.allclose(cov[n], np.cov(stack[:, :, n].T, ddof=1), rtol=1e-11, atol=1e-13)
    _, c1 = summaries.sample_moments(xs[:1])
    assert np.all(c1 == 0.0)


def test_counts_in_closed_form():
    """W^(j)[0, n] = j + n/10 and W^(j)[1, n] = -j: for c = (1, 0), gamma = 2.5 the count is
    #{j < S : j + n/10 > 2.5}; for c = (1, 1), c'W = n/10 never exceeds 0.5. The joint count
    over all voxels is #{j : j > 2.5}."""
    S, N = 7, 5
    xs = [np.stack([j + np.arange(N) / 10.0, -float(j) * np.ones(N)]) for j in range(S)]
    C = np.array([[1.0, 0.0], [1.0, 1.0]])
    g = np.array([2.5, 0.5])
    r = summaries.chain_summary(xs, C, g, E=np.arange(N))
    want0 = np.array([sum(1 for j in range(S) if j + n / 10.0 > 2.5) for n in range(N)])
    assert np.array_equal(r["count"][0], want0)
    assert np.array_equal(r["count"][1], np.zeros(N, dtype=np.int64))
    assert r["joint_count"][0] == S - 3 and r["joint_count"][1] == 0
    assert np.allclose(r["ppm"][0], want0 / S, rtol=0, atol=0)


def test_ppm_invariants():
    xs = random_samples(50, 3, 11, 2)
    rng = np.random.default_rng(3)
    C = rng.standard_normal((3, 3))
    g = rng.standard_normal(3) * 0.3
    r = summaries.chain_summary(xs, C, g, E=[4])
    neg = summaries.chain_summary(xs, -C, -g, E=[4])
    # continuous samples: no ties, so P(c'w > g) + P(-c'w > -g) = 1
    assert np.allclose(r["ppm"] + neg["ppm"], 1.0, rtol=0, atol=1e-15)
    # a one-voxel joint set is that voxel's marginal PPM
    assert np.array_equal(r["joint_count"], r["count"][:, 4])
    # joint over a larger set is at most the smallest marginal; the empty set gives 1
    big = summaries.chain_summary(xs, C, g, E=[1, 4, 7, 9])
    assert np.all(big["joint_count"] <= r["count"][:, [1, 4, 7, 9]].min(axis=1))
    empty = summaries.chain_summary(xs, C, g, E=[])
    assert np.all(empty["joint_ppm"] == 1.0)
    # thresholds at -inf / +inf, and monotone in gamma
    lo = summaries.chain_summary(xs, C, np.full(3, -np.inf))
    hi = summaries.chain_summary(xs, C, np.full(3, np.inf))
    assert np.all(lo["ppm"] == 1.0) and np.all(hi["ppm"] == 0.0)
    up = summaries.chain_summary(xs, C, g + 0.2)
    assert np.all(up["count"] <= r["count"])


def test_contrast_values_round_like_sequential_products():
    """c'w summed in k order with one rounding per operation: equal to a Python float loop
    (which rounds every product and every sum) bit for bit."""
    rng = np.random.default_rng(4)
    C = rng.standard_normal((2, 5))
    W = rng.standard_normal((5, 6)) * 50.0
    v = summaries.contrast_values(C, W)
    for i in range(2):
        for n in range(6):
            s = 0.0
            for k in range(5):
                s = s + float(C[i, k]) * float(W[k, n])
            assert v[i, n] == s


def test_svb_ppm_is_the_normal_tail_of_the_sample_moments():
    xs = random_samples(12, 3, 8, 5, scale=0.5, shift=1.0)
    C = np.array([[1.0, 0.0, 0.0], [0.5, -1.0, 0.25]])
    g = np.array([1.1, -0.2])
    r = summaries.svb_summary(xs, C, g)
    mean, cov = summaries.sample_moments(xs)
    for i in range(2):
        for n in range(8):
            m = C[i] @ mean[:, n]
            sd = math.sqrt(C[i] @ cov[n] @ C[i])
            assert abs(r["ppm"][i, n] - st.norm.sf((g[i] - m) / sd)) <= 1e-14
    # zero variance: the indicator
    same = [np.ones((3, 4))] * 5
    z = summaries.svb_summary(same, C, np.array([0.9, 2.0]))
    assert np.all(z["ppm"][0] == 1.0) and np.all(z["ppm"][1] == 0.0)


def test_svb_ppm_converges_to_the_true_gaussian_tail():
    """Samples from a known N(mu, Sigma): the moment-based PPM approaches the exact tail
    probability (statistical pin: within 5 standard errors of the plug-in estimate)."""
    rng = np.random.default_rng(6)
    K, N, S = 2, 3, 20000
    mu = np.array([[0.3, -0.1, 1.0], [0.0, 0.5, -0.4]])
    L = np.array([[1.0, 0.0], [0.6, 0.8]])
    xs = [mu + L @ rng.standard_normal((K, N)) for _ in range(S)]
    c = np.array([[1.0, 1.0]])
    r = summaries.svb_summary(xs, c, np.array([0.2]))
    Sig = L @ L.T
    sd = math.sqrt(c[0] @ Sig @ c[0])
    for n in range(N):
        exact = st.norm.sf((0.2 - c[0] @ mu[:, n]) / sd)
        assert abs(r["ppm"][0, n] - exact) <= 5 * 0.4 / math.sqrt(S)


def tiny(dims, K, P, T, seed):
    nx, ny, nz = dims
    mask = np.ones((nz, ny, nx), np.uint8)
    w = synth.make_workload("tiny", dims, mask, T=T, K=K, P=P, neighbourhood=6, seed=seed,
                            ar_mean=(0.3, 0.1, 0.05)[:max(P, 1)], drift=False, n_blobs=1)
    return w, Lattice(w.mask, 6)


def state_of(w, rng):
    return dict(W=w.W_true + 0.1 * rng.standard_normal((w.K, w.N)),
                A=w.A_true + 0.02 * rng.standard_normal((w.P, w.N)),
                lam=rng.uniform(0.5, 2.0, w.N), alpha=rng.uniform(0.2, 3.0, w.K),
                beta=rng.uniform(1.0, 20.0, w.P))


def log_joint_scipy(lat, w, s, priors, spatial_ar, prior="ugl"):
    """The same density from normalised library densities: AR(P) innovations in the time
    domain with scipy's normal density, scipy's Gamma densities, and the GMRF term summed
    over the lattice edges. Differs from the oracle by a constant only."""
    Y, X, T, P, N = w.Y, w.X, w.T, w.P, w.N
    ll = 0.0
    for n in range(N):
        e = Y[:, n] - X @ s["W"][:, n]
        for t in range(P, T):
            innov = e[t] - sum(s["A"][p - 1, n] * e[t - p] for p in range(1, P + 1))
            ll += st.norm.logpdf(innov, scale=1.0 / math.sqrt(s["lam"][n]))
    E = lat.edges()

    def gmrf(V, prec, ltl=False):
        tot = 0.0
        for k in range(V.shape[0]):
            if ltl:
                # |L v|^2 with (L v)_i = sum over the edges at i of (v_i - v_j)
                lv = np.zeros(N)
                for i, j, _ in E:
                    lv[i] += V[k, i] - V[k, j]
                    lv[j] += V[k, j] - V[k, i]
                q = float(lv @ lv)
            else:
                q = sum((V[k, i] - V[k, j]) ** 2 for i, j, _ in E)
            tot += 0.5 * N * math.log(prec[k]) - 0.5 * prec[k] * q
        return tot
    out = ll + gmrf(s["W"], s["alpha"], prior == "ltl")
    out += st.gamma.logpdf(s["lam"], a=priors["u2"], scale=priors["u1"]).sum()
    out += st.gamma.logpdf(s["alpha"], a=priors["q2"], scale=priors["q1"]).sum()
    if spatial_ar and P > 0:
        out += gmrf(s["A"], s["beta"])
        out += st.gamma.logpdf(s["beta"], a=priors["r2"], scale=priors["r1"]).sum()
    return out


@pytest.mark.parametrize("prior", ["ugl", "ltl"])
@pytest.mark.parametrize("P,spatial", [(0, True), (2, True), (2, False)])
def test_log_joint_differences_match_library_densities(P, spatial, prior):
    """Ratios of the unnormalised joint posterior (the quantity the paper uses it for) equal
    those of fully normalised scipy densities: any dropped term, sign or factor would show
    up in the difference of two states."""
    w, lat = tiny((3, 3, 2), K=3, P=P, T=25, seed=7 + P)
    rng = np.random.default_rng(11)
    s1, s2 = state_of(w, rng), state_of(w, rng)
    o1 = summaries.log_joint(lat, w.Y, w.X, s1, w.T, spatial_ar=spatial, prior=prior)
    o2 = summaries.log_joint(lat, w.Y, w.X, s2, w.T, spatial_ar=spatial, prior=prior)
    r1 = log_joint_scipy(lat, w, s1, model.PRIORS, spatial, prior)
    r2 = log_joint_scipy(lat, w, s2, model.PRIORS, spatial, prior)
    assert abs((o1["total"] - o2["total"]) - (r1 - r2)) <= 1e-9 * max(1.0, abs(r1 - r2))
    # the parts change with the parameters they name only
    s3 = dict(s1, alpha=s1["alpha"] * 1.5)
    o3 = summaries.log_joint(lat, w.Y, w.X, s3, w.T, spatial_ar=spatial, prior=prior)
    for key in ("loglik", "A_prior", "lambda_prior", "beta_prior"):
        assert o3[key] == o1[key]
    assert o3["W_prior"] != o1["W_prior"] and o3["alpha_prior"] != o1["alpha_prior"]
