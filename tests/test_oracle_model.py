"""Pins for the oracle's full conditionals, perturbation and exact solves (CPU only).

Each pin compares the oracle against something other than itself: a brute-force
evaluation of the log posterior from the raw time series, numpy's least squares, dense
inversion / eigendecomposition, the algebraic covariance of the perturbation, or Monte
Carlo moments.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import gibbs, linalg, model, philox
from oracle.lattice import Lattice
from paper_1606_00980_gb300 import synth


def tiny(dims=(3, 3, 1), K=3, P=1, T=30, nb=4, seed=0, mask=None):
    nx, ny, nz = dims
    if mask is None:
        mask = np.ones((nz, ny, nx), np.uint8)
    w = synth.make_workload("tiny", dims, mask, T=T, K=K, P=P, neighbourhood=nb, seed=seed,
                            ar_mean=(0.3, 0.1, 0.05)[:max(P, 1)], drift=(K >= 4), n_blobs=1)
    return w, Lattice(w.mask, nb)


def random_state(w, rng):
    N, K, P = w.N, w.K, w.P
    return dict(W=w.W_true + 0.1 * rng.standard_normal((K, N)),
                A=w.A_true + 0.02 * rng.standard_normal((P, N)),
                lam=rng.uniform(0.5, 2.0, N), alpha=rng.uniform(0.1, 3.0, K),
                beta=rng.uniform(1.0, 20.0, P))


@pytest.mark.parametrize("P", [0, 1, 3])
def test_stats_expansion_equals_direct_whitening(P):
    """The sufficient-statistics expansion of Appendix A equals the direct whitened
    products of the time series (W block, A block, RSS)."""
    w, lat = tiny(dims=(4, 3, 2), K=4, P=P, T=50, nb=6)
    rng = np.random.default_rng(1)
    s = random_state(w, rng)
    st = model.sufficient_stats(w.Y, w.X, P)
    Bd1, b1 = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"], 1e-3)
    Bd2, b2 = model.w_blocks_from_stats(st, s["A"], s["lam"], 1e-3)
    assert np.max(np.abs(Bd1 - Bd2)) <= 1e-12 * np.max(np.abs(Bd1))
    assert np.max(np.abs(b1 - b2)) <= 1e-12 * np.max(np.abs(b1))
    r1 = model.rss_direct(w.Y, w.X, s["W"], s["A"])
    r2 = model.rss_from_stats(st, s["W"], s["A"])
    yy = np.max(st["Syy"][:, 0, 0])
    assert np.max(np.abs(r1 - r2)) <= 1e-13 * yy
    if P > 0:
        J1, a1 = model.a_blocks_direct(w.Y, w.X, s["W"], s["lam"], P)
        J2, a2 = model.a_blocks_from_stats(st, s["W"], s["lam"])
        assert np.max(np.abs(J1 - J2)) <= 1e-13 * yy
        assert np.max(np.abs(a1 - a2)) <= 1e-13 * yy


def test_P0_reduces_to_iid_model():
    """P = 0: block lambda X'X and right-hand side lambda X'y over the full time range
    (Eq. fullcondiidW), RSS = ||y - X w||^2 (Eq. fullcondiidlambda), shape T/2 + u2."""
    w, lat = tiny(K=3, P=0, T=25)
    rng = np.random.default_rng(2)
    lam = rng.uniform(0.5, 2, w.N)
    Bd, bw = model.w_blocks_direct(w.Y, w.X, np.zeros((0, w.N)), lam)
    for n in range(w.N):
        assert np.allclose(Bd[n], lam[n] * w.X.T @ w.X, rtol=1e-14, atol=0)
        assert np.allclose(bw[n], lam[n] * w.X.T @ w.Y[:, n], rtol=1e-14, atol=0)
    W = rng.standard_normal((3, w.N))
    rss = model.rss_direct(w.Y, w.X, W, np.zeros((0, w.N)))
    assert np.allclose(rss, ((w.Y - w.X @ W) ** 2).sum(axis=0), rtol=1e-13)
    scale, shape = model.lambda_params(rss, w.T, 0, 10.0, 0.1)
    assert shape == w.T / 2 + 0.1


@pytest.mark.parametrize("dims,nb,K,P", [((3, 3, 1), 4, 3, 1), ((4, 4, 4), 6, 6, 3)])
def test_precision_is_hessian_of_log_posterior(dims, nb, K, P):
    """B~ and b_w are the Hessian and linear term of minus the log full conditional of W,
    evaluated by brute force from the time series and the edge differences:
        f(w) = 1/2 sum_n lambda_n ||y~_n - X~_n w_n||^2 + 1/2 sum_k alpha_k sum_edges (dw)^2
             = f(0) - b_w'w + 1/2 w'B~w           (Eq. full cond W temporal, Eq. Wk prior)."""
    w, lat = tiny(dims=dims, K=K, P=P, T=40, nb=nb)
    rng = np.random.default_rng(3)
    s = random_state(w, rng)
    Bd, bw = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"])
    B = model.precision(lat, Bd, s["alpha"])
    b = model.kmajor(bw)
    E = lat.edges()

    def f(vec):
        Wm = vec.reshape(K, w.N)
        tot = 0.0
        for n in range(w.N):
            yt, Xt = model.whiten(w.Y[:, n], w.X, s["A"][:, n])
            r = yt - Xt @ Wm[:, n]
            tot += 0.5 * s["lam"][n] * r @ r
        d = Wm[:, E[:, 0]] - Wm[:, E[:, 1]]
        return tot + 0.5 * np.sum(s["alpha"][:, None] * d * d)

    f0 = f(np.zeros(K * w.N))
    for _ in range(3):
        v = rng.standard_normal(K * w.N)
        lhs = f(v) - f0
        rhs = -b @ v + 0.5 * v @ (B @ v)
        assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(lhs))
    # symmetric, positive definite
    Bdn = B.toarray()
    assert np.array_equal(Bdn, Bdn.T)
    assert np.linalg.eigvalsh(Bdn).min() > 0


@pytest.mark.parametrize("dims,nb,K", [((3, 3, 1), 4, 3), ((4, 4, 4), 6, 6)])
def test_exact_solve_matches_dense_inverse(dims, nb, K):
    """Sparse-LU mean and draw vs the dense inverse on a 3x3 slice and a 4x4x4 cube."""
    w, lat = tiny(dims=dims, K=K, P=1, T=40, nb=nb)
    s = random_state(w, np.random.default_rng(4))
    Bd, bw = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"], 1e-6)
    x, mu = gibbs.draw_gmrf(lat, Bd, bw, s["alpha"], seed=11, counter=5, tag=philox.TAG_W)
    B = model.precision(lat, Bd, s["alpha"]).toarray()
    Binv = np.linalg.inv(B)
    pert, _, _ = model.perturbation(lat, Bd, s["alpha"], 11, 5, philox.TAG_W)
    mu_d = Binv @ model.kmajor(bw)
    x_d = Binv @ (model.kmajor(bw) + pert)
    assert np.linalg.norm(mu.ravel() - mu_d) <= 1e-12 * np.linalg.norm(mu_d)
    assert np.linalg.norm(x.ravel() - x_d) <= 1e-12 * np.linalg.norm(x_d)


@pytest.mark.parametrize("dims,nb,K", [((3, 3, 1), 4, 2), ((4, 3, 2), 6, 3)])
def test_perturbation_covariance_is_precision(dims, nb, K):
    """Algorithm 2 is exact because the perturbation M z has covariance M M' = B~:
    sum_k alpha_k G'G (= alpha (x) D_w) plus H' L_data L_data' H (= the data blocks)."""
    w, lat = tiny(dims=dims, K=K, P=1, T=30, nb=nb)
    s = random_state(w, np.random.default_rng(5))
    Bd, _ = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"])
    M = model.perturbation_matrix(lat, Bd, s["alpha"]).toarray()
    B = model.precision(lat, Bd, s["alpha"]).toarray()
    assert np.max(np.abs(M @ M.T - B)) <= 1e-12 * np.max(np.abs(B))
    # and perturbation() is that map applied to its own normals
    pert, z1, z2 = model.perturbation(lat, Bd, s["alpha"], 3, 9, philox.TAG_W, 2)
    z = np.concatenate([model.kmajor(z1), model.kmajor(z2)])
    assert np.allclose(M @ z, pert, rtol=0, atol=1e-12 * np.abs(pert).max())


def test_isolated_voxels_reduce_to_least_squares():
    """Voxels with no neighbours decouple: the conditional mean is per-voxel GLS, i.e. the
    least-squares fit of the whitened series (numpy lstsq), whatever alpha is."""
    mask = (np.indices((3, 3, 3)).sum(axis=0) % 2).astype(np.uint8)
    w, lat = tiny(dims=(3, 3, 3), K=3, P=2, T=40, nb=6, mask=mask)
    s = random_state(w, np.random.default_rng(6))
    Bd, bw = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"])
    _, mu = gibbs.draw_gmrf(lat, Bd, bw, np.array([5.0, 0.1, 100.0]), 1, 1, philox.TAG_W)
    for n in range(w.N):
        yt, Xt = model.whiten(w.Y[:, n], w.X, s["A"][:, n])
        ref = np.linalg.lstsq(Xt, yt, rcond=None)[0]
        assert np.allclose(mu[:, n], ref, rtol=1e-10, atol=1e-12)


def test_large_alpha_makes_coefficients_constant():
    """alpha -> infinity: W_k is constant over the connected mask (the UGL penalises any
    difference between neighbours), and equals the pooled GLS estimate."""
    w, lat = tiny(dims=(4, 4, 1), K=2, P=0, T=30, nb=4)
    lam = np.ones(w.N)
    Bd, bw = model.w_blocks_direct(w.Y, w.X, np.zeros((0, w.N)), lam)
    _, mu = gibbs.draw_gmrf(lat, Bd, bw, np.array([1e9, 1e9]), 1, 1, philox.TAG_W)
    pooled = np.linalg.solve(Bd.sum(axis=0), bw.sum(axis=0))
    assert np.allclose(mu, pooled[:, None], rtol=1e-5, atol=1e-6)


def test_monte_carlo_moments_of_draws():
    """Draws w = B~^-1 (b_w + M z) with Philox normals: sample mean -> B~^-1 b_w and sample
    covariance -> B~^-1 within 5 standard errors (3x3 slice, K = 2)."""
    w, lat = tiny(dims=(3, 3, 1), K=2, P=0, T=30, nb=4)
    lam = np.full(w.N, 0.01)
    Bd, bw = model.w_blocks_direct(w.Y, w.X, np.zeros((0, w.N)), lam)
    alpha = np.array([0.7, 2.0])
    B = model.precision(lat, Bd, alpha).toarray()
    Binv = np.linalg.inv(B)
    M = model.perturbation_matrix(lat, Bd, alpha).toarray()
    n_draw = 20000
    E = lat.edges()
    sites_e = lat.lin[E[:, 0]] * 4 + E[:, 2]
    # normals for many draw counters at once: draw r uses counter r
    cnt = np.arange(n_draw)[None, :]
    def lanes(sites):
        out = []
        for j in range(1):
            z0, z1 = philox.normal_pair(philox.philox4x32_10(
                np.asarray(sites, np.uint64)[:, None], j, cnt, philox.c3_of(philox.TAG_W, 0), 17, 0))
            out += [z0, z1]
        return out                  # lane k -> (n_sites, n_draw)
    z1 = lanes(sites_e)
    z2 = lanes(lat.lin * 4 + 3)
    Z = np.concatenate([z1[0], z1[1], z2[0], z2[1]], axis=0)   # regressor-major blocks
    X = Binv @ (model.kmajor(bw)[:, None] + M @ Z)
    mean = X.mean(axis=1)
    mu = Binv @ model.kmajor(bw)
    sd = np.sqrt(np.diag(Binv))
    assert np.all(np.abs(mean - mu) < 5 * sd / np.sqrt(n_draw))
    C = np.cov(X)
    se = np.sqrt((Binv ** 2 + np.outer(np.diag(Binv), np.diag(Binv))) / n_draw)
    assert np.all(np.abs(C - Binv) < 5 * se + 1e-15)


def test_quad_forms_edges_equal_laplacian():
    w, lat = tiny(dims=(5, 4, 3), K=3, P=0, T=10, nb=6)
    V = np.random.default_rng(7).standard_normal((3, w.N))
    q1 = model.quad_forms_edges(lat, V)
    q2 = model.quad_forms_laplacian(lat, V)
    assert np.allclose(q1, q2, rtol=1e-13)


def test_logdet_and_slq():
    """log det from LU = dense Cholesky = sum of log eigenvalues; Lanczos quadrature of
    z' log(B) z is exact at m = n; Hutchinson mean within 4 sigma of the exact log det."""
    w, lat = tiny(dims=(4, 3, 2), K=2, P=1, T=30, nb=6)
    s = random_state(w, np.random.default_rng(8))
    Bd, _ = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"])
    B = model.precision(lat, Bd, s["alpha"])
    Bd_ = B.toarray()
    ev = np.linalg.eigvalsh(Bd_)
    ld = np.sum(np.log(ev))
    assert abs(linalg.logdet_sparse(B) - ld) <= 1e-10 * abs(ld)
    assert abs(linalg.logdet_dense(B) - ld) <= 1e-10 * abs(ld)
    n = Bd_.shape[0]
    Z = philox.rademacher(3, np.arange(n), 64, 0, philox.TAG_PROBE, 0)   # (n, 64)
    exact = linalg.logm_quadform_dense(Bd_, Z)
    z = Z[:, 0]
    v = linalg.slq_quadform(lambda x: B @ x, z, n)
    assert abs(v - exact[0]) <= 1e-8 * abs(exact[0])
    Lg = np.linalg.eigh(Bd_)
    logB = Lg[1] @ np.diag(np.log(Lg[0])) @ Lg[1].T
    sigma = np.sqrt(2 * (np.sum(logB ** 2) - np.sum(np.diag(logB) ** 2)) / Z.shape[1])
    assert abs(exact.mean() - ld) < 4 * sigma


def test_probe_estimators_are_unbiased_for_logdet_and_traces():
    """The oracle's probe terms: their mean over many probes approaches log det B~ - log det M
    (tr log C) and tr(D_w^(k) B~^-1) (exact dense values), within 5 standard errors."""
    from oracle import probes
    w, lat = tiny(dims=(3, 3, 2), K=2, P=1, T=30, nb=6)
    s = random_state(w, np.random.default_rng(9))
    Bd, _ = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"])
    V = probes.probe_vectors(lat, 2, 400, seed=5, counter=1)
    ldm, quad, tr, ldb = probes.exact_probe_terms(lat, Bd, s["alpha"], V)
    assert abs(quad.mean() - (ldb - ldm)) < 5 * quad.std() / np.sqrt(len(quad))
    exact = probes.exact_traces(lat, Bd, s["alpha"])
    se = tr.std(axis=0) / np.sqrt(len(tr))
    assert np.all(np.abs(tr.mean(axis=0) - exact) < 5 * se)
    # log det M from the factor equals the dense log det of the preconditioner
    M = model.precision(lat, probes.precond_blocks(lat, Bd, s["alpha"]), np.zeros(2))
    assert abs(ldm - np.linalg.slogdet(M.toarray())[1]) < 1e-10 * abs(ldm)


def test_svb_means_reduce_to_gibbs_parameters_for_one_sample():
    """With one sample the SVB expectations are the Gibbs full-conditional parameters at that
    sample: E[lambda] = scale * shape of Eq. fullcondTemplambda, E[alpha] likewise."""
    w, lat = tiny(dims=(4, 3, 2), K=2, P=1, T=30, nb=6)
    s = random_state(w, np.random.default_rng(11))
    lam = gibbs.svb_lambda_mean(w.Y, w.X, [s["W"]], [s["A"]])
    rss = model.rss_direct(w.Y, w.X, s["W"], s["A"])
    sc, sh = model.lambda_params(rss, w.T, 1, 10.0, 0.1)
    assert np.allclose(lam, sc * sh, rtol=1e-14)
    a, Q = gibbs.svb_hyper_mean(lat, [s["W"]], 10.0, 0.1)
    sc, sh = model.alpha_params(model.quad_forms_laplacian(lat, s["W"]), w.N, 10.0, 0.1)
    assert np.allclose(a, sc * sh, rtol=1e-12)


def test_svb_w_system_is_average_of_sample_systems():
    """Eq. NFVBbB: averaging the blocks over A samples equals using E[c c'] of the whitening
    coefficients c = (1, -a) in the sufficient-statistics expansion."""
    w, lat = tiny(dims=(3, 3, 2), K=3, P=2, T=40, nb=6)
    rng = np.random.default_rng(12)
    A_s = [w.A_true + 0.05 * rng.standard_normal(w.A_true.shape) for _ in range(4)]
    lam = rng.uniform(0.5, 2.0, w.N)
    Bd, bw = gibbs.svb_w_system(w.Y, w.X, A_s, lam)
    st = model.sufficient_stats(w.Y, w.X, 2)
    C = [np.concatenate([np.ones((1, w.N)), -A], axis=0) for A in A_s]
    Ecc = np.mean([np.einsum("pn,qn->npq", c, c) for c in C], axis=0)
    XtX = np.einsum("npq,pqij->nij", Ecc, st["Sxx"])
    Xty = np.einsum("npq,npqk->nk", Ecc, st["Sxy"])
    assert np.allclose(Bd, lam[:, None, None] * XtX, rtol=1e-11)
    assert np.allclose(bw, lam[:, None] * Xty, rtol=1e-11)


def test_svb_extrapolation_rules():
    """Appendix C trick 1, every branch at values worked by hand from the rule the appendix
    states: a parabola through the last three values (x = iteration - j); its vertex value
    when the vertex lies after j, maximum or minimum; otherwise a_{j-1} + 20 (a_j - a_{j-1});
    then no more than a factor 5 from the VB proposal a_j. A prediction that is not positive
    falls back to the proposal (the reading taken where the appendix says nothing)."""
    def ex(a2, a1, a0):
        return gibbs.svb_extrapolate((np.array([a2]), np.array([a1])), np.array([a0]))[0]
    # concave, vertex after j: -x^2/8 + x/8 + 1.75, vertex at x = 1/2 with value 57/32
    assert abs(ex(1.0, 1.5, 1.75) - 1.78125) <= 1e-15
    # convex, vertex after j: x^2/2 - x/2 + 1, vertex at x = 1/2 with value 7/8
    assert abs(ex(4.0, 2.0, 1.0) - 0.875) <= 1e-15
    # convex, vertex before j (x = -2/3): the 20x step 1.5 + 20 (0.1) = 3.5, inside [0.32, 8]
    assert abs(ex(2.0, 1.5, 1.6) - 3.5) <= 1e-12
    # a straight line has no vertex: 1.25 + 20 (0.25) = 6.25, inside [0.3, 7.5]
    assert ex(1.0, 1.25, 1.5) == 6.25
    # the 20x step limited to 5 a_j: 2 + 20 (1) = 22 -> 15
    assert ex(1.0, 2.0, 3.0) == 15.0
    # vertex before j (x = -1): 2.1 + 20 (-0.1) = 0.1 lifted to a_j / 5 = 0.4
    assert abs(ex(2.0, 2.1, 2.0) - 0.4) <= 1e-15
    # a negative prediction (2 + 20 (-1) = -18) falls back to the proposal
    assert ex(3.0, 2.0, 1.0) == 1.0


def test_paper_simulation_workloads_have_the_papers_shapes():
    """Appendix D's simulation: N = 1e3 / 1e4 / 1e5 centred boxes of the 53x63x46 block,
    K = 5, P = 1, T = 351, voxel means scaled to 100; the UGL-prior rows are centred and
    smoother (smaller neighbour differences) the larger their alpha."""
    w = synth.paper_simulation(1000, seed=3)
    assert w.N == 1000 and w.K == 5 and w.P == 1 and w.T == 351
    assert w.dims == (53, 63, 46) and int(w.mask.sum()) == 1000
    assert np.allclose(w.Y.mean(axis=0), 100.0)
    assert np.all(np.abs(w.A_true) <= 0.9)
    lat = Lattice(w.mask, 6)
    E = lat.edges()
    spread = [np.mean((w.W_true[k, E[:, 0]] - w.W_true[k, E[:, 1]]) ** 2) for k in range(4)]
    assert spread[0] > spread[1] > spread[2] > spread[3]
    # increments of the periodic UGL field have variance 1/(3 alpha) per direction on average
    f = synth.periodic_ugl_field((46, 63, 53), 0.5, np.random.default_rng(1))
    assert abs(f.mean()) < 1e-12
    d = np.concatenate([np.diff(f, axis=a).ravel() for a in range(3)])
    assert abs(np.var(d) * 0.5 * 3 - 1.0) < 0.15
    for N in (10000,):
        assert int(synth.paper_simulation(N, seed=4).mask.sum()) == N


WGL_WEIGHTS = (2.0, 0.5, 3.25)


def test_weighted_laplacian_equals_scaled_incidence_gram():
    """WGL (Discussion): D_w built from weighted adjacency equals G' C G, with C the edge
    weights of each edge's direction; equal weights c scale the UGL Laplacian by c; the
    perturbation uses C^(1/2) G; the edge quadratic forms carry the weights."""
    for nb in (6, 4):
        w, _ = tiny(dims=(4, 3, 3) if nb == 6 else (5, 4, 1), K=2, P=1, T=30, nb=nb)
        lat = Lattice(w.mask, nb, weights=WGL_WEIGHTS)
        G = lat.G()
        C = sp.diags(lat.edge_weights())
        assert np.array_equal((G.T @ C @ G).toarray(), lat.D().toarray())
        assert np.allclose((lat.Gw().T @ lat.Gw()).toarray(), lat.D().toarray(), rtol=0, atol=1e-14)
        ugl = Lattice(w.mask, nb)
        eq = Lattice(w.mask, nb, weights=(1.5, 1.5, 1.5))
        assert np.array_equal(eq.D().toarray(), 1.5 * ugl.D().toarray())
        V = np.random.default_rng(2).standard_normal((3, lat.N))
        assert np.allclose(model.quad_forms_edges(lat, V), model.quad_forms_laplacian(lat, V),
                           rtol=1e-13, atol=0)


@pytest.mark.parametrize("nb", [6, 4])
def test_weighted_perturbation_covariance_is_precision(nb):
    """Algorithm 2 under the WGL prior: M M' = B~ with the weighted Laplacian, so the draw is
    exact; and the weighted precision is SPD."""
    w, _ = tiny(dims=(3, 3, 2) if nb == 6 else (4, 3, 1), K=2, P=1, T=30, nb=nb)
    lat = Lattice(w.mask, nb, weights=WGL_WEIGHTS)
    s = random_state(w, np.random.default_rng(6))
    Bd, _ = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"])
    M = model.perturbation_matrix(lat, Bd, s["alpha"]).toarray()
    B = model.precision(lat, Bd, s["alpha"]).toarray()
    assert np.max(np.abs(M @ M.T - B)) <= 1e-12 * np.max(np.abs(B))
    assert np.linalg.eigvalsh(B).min() > 0


def innovations_by_loops(y, X, w, a):
    """eps_t = (y_t - x_t w) - sum_p a_p (y_{t-p} - x_{t-p} w) for t = P+1..T (1-based),
    written out term by term from Eq. likeliTemp's bracket (no lag helper, no whitening)."""
    T, P = len(y), len(a)
    out = []
    for t in range(P, T):                     # 0-based t = P..T-1
        e = y[t] - X[t] @ w
        for p in range(1, P + 1):
            e -= a[p - 1] * (y[t - p] - X[t - p] @ w)
        out.append(e)
    return np.array(out)


@pytest.mark.parametrize("dims,nb,K,P", [((3, 3, 1), 4, 3, 1), ((3, 3, 2), 6, 4, 3)])
def test_a_precision_is_hessian_of_log_posterior(dims, nb, K, P):
    """The A full conditional (Eq. fullcondTempA) with the spatial prior D_a = D_w: minus its
    log density, evaluated by brute force from the raw time series and the edge differences,
        g(a) = 1/2 sum_n lambda_n sum_t eps_t(a_n)^2 + 1/2 sum_p beta_p sum_edges (da_p)^2
             = g(0) - b_a'a + 1/2 a'B_a a,
    where B_a = blkdiag(a_blocks_direct) + diag(beta) (x) D_w and b_a its right-hand side. A
    sign or lag-index slip in a_blocks_direct changes the quadratic or the linear term."""
    w, lat = tiny(dims=dims, K=K, P=P, T=35, nb=nb)
    rng = np.random.default_rng(13)
    s = random_state(w, rng)
    Ja, ba = model.a_blocks_direct(w.Y, w.X, s["W"], s["lam"], P)
    B = model.precision(lat, Ja, s["beta"])
    b = model.kmajor(ba)
    E = lat.edges()

    def g(vec):
        Am = vec.reshape(P, w.N)
        tot = 0.0
        for n in range(w.N):
            e = innovations_by_loops(w.Y[:, n], w.X, s["W"][:, n], Am[:, n])
            tot += 0.5 * s["lam"][n] * e @ e
        d = Am[:, E[:, 0]] - Am[:, E[:, 1]]
        return tot + 0.5 * np.sum(s["beta"][:, None] * d * d)

    g0 = g(np.zeros(P * w.N))
    for _ in range(3):
        v = 0.3 * rng.standard_normal(P * w.N)
        lhs = g(v) - g0
        rhs = -b @ v + 0.5 * v @ (B @ v)
        assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(lhs))


@pytest.mark.parametrize("P", [1, 2, 3])
def test_lambda_conditional_matches_normalised_density(P):
    """Eq. fullcondTemplambda at P > 0: the normalised full conditional of lambda_n, computed
    by brute force on a grid as prod_t N(eps_t; 0, 1/lambda) times the Ga(scale u1, shape u2)
    prior density (eps_t written out from the raw series), equals the Gamma density with
    lambda_params' scale and shape ((T - P)/2 + u2): a wrong shape or a wrong RSS fails."""
    from scipy import stats
    w, lat = tiny(dims=(2, 2, 1), K=3, P=P, T=30, nb=4)
    rng = np.random.default_rng(20 + P)
    s = random_state(w, rng)
    u1, u2 = 10.0, 0.1
    rss = model.rss_direct(w.Y, w.X, s["W"], s["A"])
    scale, shape = model.lambda_params(rss, w.T, P, u1, u2)
    for n in range(w.N):
        e = innovations_by_loops(w.Y[:, n], w.X, s["W"][:, n], s["A"][:, n])
        mode = max((shape - 1.0) * scale[n], 1e-6)
        sd = np.sqrt(shape) * scale[n]
        lam = np.linspace(max(mode - 12 * sd, 1e-9), mode + 12 * sd, 20001)
        loglik = np.array([np.sum(stats.norm.logpdf(e, scale=1.0 / np.sqrt(l))) for l in lam])
        logp = loglik + stats.gamma.logpdf(lam, a=u2, scale=u1)
        dens = np.exp(logp - logp.max())
        dens /= np.trapezoid(dens, lam)
        ref = stats.gamma.pdf(lam, a=shape, scale=scale[n])
        assert np.max(np.abs(dens - ref)) <= 1e-6 * ref.max()


def test_lanczos_probe_terms_equal_dense_ones():
    """probes.probe_terms_lanczos (sparse, mid-size) reproduces the dense eigendecomposition
    form exact_probe_terms: per-probe v' log(C) v, the trace terms and both log dets."""
    from oracle import probes
    w, lat = tiny(dims=(4, 4, 3), K=3, P=1, T=30, nb=6)
    s = random_state(w, np.random.default_rng(31))
    Bd, _ = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"])
    V = probes.probe_vectors(lat, 3, 5, seed=9, counter=2)
    ldm, quad, tr, ldb = probes.exact_probe_terms(lat, Bd, s["alpha"], V)
    ldm2, quad2, tr2, ldb2 = probes.probe_terms_lanczos(lat, Bd, s["alpha"], V)
    assert abs(ldm2 - ldm) <= 1e-12 * abs(ldm)
    assert abs(ldb2 - ldb) <= 1e-10 * abs(ldb)
    assert np.max(np.abs(quad2 - quad)) <= 1e-10 * np.abs(quad).max()
    assert np.max(np.abs(tr2 - tr)) <= 1e-10 * np.abs(tr).max()


def test_fixed_step_probe_quadrature():
    """probes.probe_quadrature_m: with m = the dimension the Gauss quadrature is exact (the
    dense eigendecomposition's v' log(C) v); with m = 5 it is |v|^2 e1' log(Q' C Q) e1 for
    an orthonormal basis Q of the Krylov space span{v, C v, ..., C^4 v} whose first column is
    v / |v|, built here by a QR factorisation of the dense Krylov matrix."""
    from oracle import probes
    w, lat = tiny(dims=(4, 4, 3), K=3, P=1, T=30, nb=6)
    s = random_state(w, np.random.default_rng(32))
    Bd, _ = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"])
    v = probes.probe_vectors(lat, 3, 1, seed=9, counter=3)[0]
    _, quad, _, _ = probes.exact_probe_terms(lat, Bd, s["alpha"], [v])
    n = 3 * w.N
    assert abs(probes.probe_quadrature_m(lat, Bd, s["alpha"], v, n) - quad[0]) <= 1e-9 * abs(quad[0])
    Ls = probes.block_chol_factors(lat, Bd, s["alpha"])
    H = model.H_perm(w.N, 3)
    L = (H.T @ model.blkdiag(Ls) @ H).toarray()
    B = model.precision(lat, Bd, s["alpha"]).toarray()
    C = np.linalg.solve(L, np.linalg.solve(L, B).T).T          # L^-1 B L^-T (symmetric)
    vk = model.kmajor(v)
    Kry = np.stack([np.linalg.matrix_power(C, j) @ vk for j in range(5)], axis=1)
    Q, _ = np.linalg.qr(Kry)
    th, S = np.linalg.eigh(Q.T @ C @ Q)
    ref = float((vk @ vk) * np.sum(S[0, :] ** 2 * np.log(th)))
    got = probes.probe_quadrature_m(lat, Bd, s["alpha"], v, 5)
    assert abs(got - ref) <= 1e-9 * abs(ref)
    assert abs(got - quad[0]) > 1e-6 * abs(quad[0])           # 5 steps are not yet exact


def test_nested_dissection_order_and_factor():
    """linalg.nested_dissection is a permutation whose first split leaves no lattice edge
    between the two halves (only the separator plane touches both), and factor_nd solves
    B~ x = b like the dense inverse (6x5x4 block, K = 3) and gives its log det."""
    w, lat = tiny(dims=(6, 5, 4), K=3, P=1, T=30, nb=6)
    x, y, z = lat.coords()
    C = np.stack([x, y, z], 1)
    order = linalg.nested_dissection(C, leaf=8)
    assert np.array_equal(np.sort(order), np.arange(w.N))
    # first level: split across x (the longest extent) at the median plane
    mid = int(np.median(x))
    left, right = set(np.flatnonzero(x < mid)), set(np.flatnonzero(x > mid))
    for i, j, _ in lat.edges():
        assert not ((i in left and j in right) or (i in right and j in left))
    s = random_state(w, np.random.default_rng(41))
    Bd, bw = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"])
    B = model.precision(lat, Bd, s["alpha"])
    f = linalg.factor_nd(B, C, 3)
    b = model.kmajor(bw)
    xd = np.linalg.solve(B.toarray(), b)
    assert np.linalg.norm(f.solve(b) - xd) <= 1e-12 * np.linalg.norm(xd)
    assert abs(f.logdet() - np.linalg.slogdet(B.toarray())[1]) <= 1e-10 * abs(f.logdet())
