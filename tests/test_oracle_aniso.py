"""Pins of the oracle's anisotropic prior (Discussion: W_k with prior precision
G_w' C_k G_w, C_k = diag(alpha_x,k I, alpha_y,k I, alpha_z,k I), the alphas random) and of
its exchange step (Murray, Ghahramani & MacKay 2006; the paper leaves this inference open).

* the direction Laplacians L_d sum to the graph Laplacian entry by entry, and each one's
  quadratic form is the brute-force sum over the direction's coordinate pairs;
* the precision with alpha_{d,k} = alpha_k for every d is the graph-Laplacian one, and its
  prior part's quadratic form is the brute-force pair sum weighted per direction;
* Algorithm 2's perturbation has covariance exactly B~, and the vector form equals the
  matrix form applied to the same normals;
* the direction quadratic forms add up to the edge sums and match brute force;
* the auxiliary draw has covariance L(theta)^+ (numpy's pseudo-inverse) and no component
  along the constants of any connected part;
* log a equals the log of the density ratio the exchange algorithm accepts with, evaluated
  from brute-force quadratic forms and scipy's Gamma and log-normal densities;
* the ray move's Gamma density differs from the posterior along the ray, pi(lam alpha)
  lam^(nd - 1) with the exact pseudo-determinant from numpy's eigenvalues, by a constant in lam
  (on a connected lattice and on one of two parts);
* chains of exchange steps, alone and after the ray move, on a 20-voxel lattice reach the
  posterior mean of log alpha that a grid integration with the exact pseudo-determinant
  gives (this is what catches a dropped proposal Jacobian or an auxiliary draw that ignores
  the proposal).
"""
import numpy as np
import pytest

from oracle import gibbs, model, philox
from oracle.lattice import Lattice

W3 = (2.0, 0.5, 1.25)


def bf16_factors(shape, seed):
    return np.random.default_rng(seed).integers(4, 41, size=(3,) + shape) / 16.0


def lattice(dims, nb, factors=True, hole=True):
    nx, ny, nz = dims
    mask = np.ones((nz, ny, nx), np.uint8)
    if hole:
        mask[0, 1, 1] = 0
    f = bf16_factors((nz, ny, nx), 3) if factors else None
    return Lattice(mask, nb, weights=W3, edge_factors=f)


def pair_sums(lat, v):
    """Brute force: per direction d, sum over in-mask pairs (i, i + e_d) of C (v_i - v_j)^2."""
    x, y, z = lat.coords()
    pos = {(int(a), int(b), int(c)): i for i, (a, b, c) in enumerate(zip(x, y, z))}
    f = lat.edge_factors
    out = np.zeros(3)
    steps = [(1, 0, 0), (0, 1, 0), (0, 0, 1)][:lat.neighbourhood // 2]
    for (a, b, c), i in pos.items():
        for d, (dx, dy, dz) in enumerate(steps):
            j = pos.get((a + dx, b + dy, c + dz))
            if j is not None:
                cw = W3[d] * (f[d, lat.lin[i]] if f is not None else 1.0)
                out[d] += cw * (v[i] - v[j]) ** 2
    return out


CASES = [((5, 4, 3), 6), ((6, 5, 1), 4)]


@pytest.mark.parametrize("dims,nb", CASES)
def test_direction_laplacians_sum_and_pair_sums(dims, nb):
    lat = lattice(dims, nb)
    Ls = model.direction_laplacians(lat)
    assert np.array_equal(sum(L.toarray() for L in Ls), lat.D().toarray())
    v = np.random.default_rng(5).standard_normal(lat.N)
    bf = pair_sums(lat, v)
    for d in range(3):
        assert abs(v @ (Ls[d] @ v) - bf[d]) <= 1e-12 * max(bf.max(), 1.0)
    Q = model.quad_forms_dirs(lat, v[None])[0]
    assert np.allclose(Q, bf, rtol=1e-13, atol=0)
    assert abs(Q.sum() - model.quad_forms_edges(lat, v[None])[0]) <= 1e-12 * Q.sum()


@pytest.mark.parametrize("dims,nb", CASES)
def test_precision_special_case_and_quadratic_form(dims, nb):
    lat = lattice(dims, nb)
    K = 3
    rng = np.random.default_rng(6)
    blocks = np.einsum("nij,nkj->nik", *(2 * [rng.standard_normal((lat.N, K, K))])) + np.eye(K)
    a = rng.uniform(0.3, 3.0, K)
    iso = model.precision(lat, blocks, np.repeat(a[:, None], 3, axis=1), "aniso")
    ugl = model.precision(lat, blocks, a)
    assert np.max(np.abs((iso - ugl).toarray())) <= 1e-13 * np.abs(ugl.toarray()).max()
    theta = rng.uniform(0.2, 4.0, (K, 3))
    Pk = model.aniso_prior(lat, theta)
    X = rng.standard_normal((K, lat.N))
    got = X.reshape(-1) @ (Pk @ X.reshape(-1))
    ref = sum(theta[k] @ pair_sums(lat, X[k]) for k in range(K))
    assert abs(got - ref) <= 1e-12 * abs(ref)


@pytest.mark.parametrize("dims,nb", CASES)
def test_perturbation_covariance_and_vector_form(dims, nb):
    lat = lattice(dims, nb)
    K = 2
    rng = np.random.default_rng(7)
    blocks = np.einsum("nij,nkj->nik", *(2 * [rng.standard_normal((lat.N, K, K))])) + np.eye(K)
    theta = rng.uniform(0.2, 4.0, (K, 3))
    Pm = model.perturbation_matrix(lat, blocks, theta, "aniso")
    B = model.precision(lat, blocks, theta, "aniso").toarray()
    G = (Pm @ Pm.T).toarray()
    assert np.max(np.abs(G - B)) <= 1e-12 * np.abs(B).max()
    pert, z1, z2 = model.perturbation(lat, blocks, theta, 9, 4, philox.TAG_W, 0, "aniso")
    z = np.concatenate([z1.T.reshape(-1), model.kmajor(z2)])
    assert np.max(np.abs(Pm @ z - pert)) <= 1e-12 * np.abs(pert).max()


def test_auxiliary_draw_covariance_is_the_pseudo_inverse():
    # two connected parts: a 3 x 3 block and a 2 x 1 strip, 4-neighbourhood
    mask = np.zeros((1, 4, 6), np.uint8)
    mask[0, :3, :3] = 1
    mask[0, 0:2, 5] = 1
    lat = Lattice(mask, 4, weights=W3)
    theta = np.array([0.7, 2.5, 1.0])
    E = lat.edges()
    M = np.stack([gibbs.aux_solve(lat, theta, np.eye(len(E))[e]) for e in range(len(E))], axis=1)
    L = sum(theta[d] * Ld.toarray() for d, Ld in enumerate(model.direction_laplacians(lat)))
    ref = np.linalg.pinv(L)
    assert np.max(np.abs(M @ M.T - ref)) <= 1e-10 * np.abs(ref).max()
    w = gibbs.aux_prior_draw(lat, np.tile(theta, (2, 1)), 3, 1)
    big = np.flatnonzero(lat.coords()[0] < 3)
    assert np.all(np.abs(w[:, big].sum(axis=1)) <= 1e-12)
    assert np.all(np.abs(np.delete(w, big, axis=1).sum(axis=1)) <= 1e-12)


def test_log_ratio_is_the_exchange_density_ratio():
    stats = pytest.importorskip("scipy.stats")
    lat = lattice((5, 4, 3), 6)
    rng = np.random.default_rng(8)
    K, step = 3, 0.3
    theta = rng.uniform(0.3, 3.0, (K, 3))
    eps = rng.standard_normal((K, 3))
    tp = theta * np.exp(step * eps)
    W = rng.standard_normal((K, lat.N))
    Wp = rng.standard_normal((K, lat.N))
    la = gibbs.exchange_log_ratio(theta, tp, model.quad_forms_dirs(lat, W),
                                  model.quad_forms_dirs(lat, Wp), step * eps, 3)
    pr = model.PRIORS

    def logf(v, th):   # unnormalised log density of the anisotropic GMRF
        return -0.5 * th @ pair_sums(lat, v)

    for k in range(K):
        ref = (logf(W[k], tp[k]) + logf(Wp[k], theta[k]) - logf(W[k], theta[k]) - logf(Wp[k], tp[k])
               + stats.gamma.logpdf(tp[k], a=pr["q2"], scale=pr["q1"]).sum()
               - stats.gamma.logpdf(theta[k], a=pr["q2"], scale=pr["q1"]).sum()
               + stats.lognorm.logpdf(theta[k], s=step, scale=tp[k]).sum()
               - stats.lognorm.logpdf(tp[k], s=step, scale=theta[k]).sum())
        assert abs(la[k] - ref) <= 1e-9 * (1.0 + abs(ref))


def test_exchange_step_uses_its_random_numbers():
    lat = lattice((5, 4, 1), 4, hole=False)
    rng = np.random.default_rng(9)
    K = 4
    st = dict(W=rng.standard_normal((K, lat.N)), alpha=rng.uniform(0.5, 2.0, (K, 3)))
    new, acc, d = gibbs.exchange_alpha(lat, st, 21, 5, 0.4)
    eps = philox.normals(21, np.arange(K), 3, 5, philox.TAG_ALPHA_PROP, 0)
    assert np.array_equal(d["proposal"][:, :2], st["alpha"][:, :2] * np.exp(0.4 * eps[:, :2]))
    assert np.array_equal(d["proposal"][:, 2], st["alpha"][:, 2])      # no z edges in 2D
    assert np.array_equal(acc, np.log(d["u"]) < d["log_a"])
    assert np.array_equal(new[acc], d["proposal"][acc]) and np.array_equal(new[~acc], st["alpha"][~acc])


@pytest.mark.parametrize("two_parts", [False, True])
def test_ray_move_is_the_posterior_along_the_ray(two_parts):
    stats = pytest.importorskip("scipy.stats")
    if two_parts:
        mask = np.zeros((2, 4, 6), np.uint8)
        mask[:, :3, :3] = 1
        mask[:, 0:2, 5] = 1
        lat = Lattice(mask, 6, weights=W3)
    else:
        lat = lattice((5, 4, 3), 6)
    nd, c = 3, gibbs.n_parts(lat)
    assert c == (2 if two_parts else 1)
    rng = np.random.default_rng(10)
    theta = rng.uniform(0.3, 3.0, 3)
    w = rng.standard_normal(lat.N)
    Q = pair_sums(lat, w)
    Ls = [L.toarray() for L in model.direction_laplacians(lat)]
    pr = model.PRIORS
    shape, rate = gibbs.scale_move_params(theta[None], Q[None], lat.N, c, nd)
    diffs = []
    for lam in (0.3, 0.8, 1.0, 2.5, 7.0):
        t = lam * theta
        ev = np.linalg.eigvalsh(sum(t[d] * Ls[d] for d in range(3)))[c:]
        logpi = (stats.gamma.logpdf(t, a=pr["q2"], scale=pr["q1"]).sum() + 0.5 * np.sum(np.log(ev))
                 - 0.5 * t @ Q)
        diffs.append(logpi + (nd - 1) * np.log(lam) - stats.gamma.logpdf(lam, a=shape, scale=1.0 / rate[0]))
    assert np.ptp(diffs) <= 1e-9 * max(1.0, np.abs(diffs).max())


def test_ray_move_uses_its_random_numbers():
    lat = lattice((5, 4, 1), 4, hole=False)
    rng = np.random.default_rng(11)
    K = 3
    st = dict(W=rng.standard_normal((K, lat.N)), alpha=rng.uniform(0.5, 2.0, (K, 3)))
    out, lam = gibbs.scale_move_alpha(lat, st, 5, 2)
    shape, rate = gibbs.scale_move_params(st["alpha"], model.quad_forms_dirs(lat, st["W"]), lat.N, 1, 2)
    ref, _ = philox.gamma(5, np.arange(K), shape, 1.0 / rate, 2, philox.TAG_ALPHA, 0)
    assert np.array_equal(lam, ref)
    assert np.array_equal(out[:, :2], st["alpha"][:, :2] * lam[:, None])
    assert np.array_equal(out[:, 2], st["alpha"][:, 2])


def exact_posterior_mean_log(lat, w, priors, grid=160):
    """E[log alpha_x], E[log alpha_y] under p(alpha | w) for a connected 2D lattice and one
    field w: Ga(q1, q2) priors times pdet(L(alpha))^(1/2) exp(-Q(alpha) / 2), on a grid."""
    from scipy.stats import gamma
    Ls = [L.toarray() for L in model.direction_laplacians(lat)]
    Q = model.quad_forms_dirs(lat, w[None])[0]
    lg = np.linspace(-5.0, 4.0, grid)
    logp = np.empty((grid, grid))
    for i, tx in enumerate(np.exp(lg)):
        for j, ty in enumerate(np.exp(lg)):
            ev = np.linalg.eigvalsh(tx * Ls[0] + ty * Ls[1])[1:]       # one zero eigenvalue
            th = np.array([tx, ty])
            logp[i, j] = (0.5 * np.sum(np.log(ev)) - 0.5 * th @ Q[:2]
                          + np.sum(gamma.logpdf(th, a=priors["q2"], scale=priors["q1"])) + lg[i] + lg[j])
    p = np.exp(logp - logp.max())
    p /= p.sum()
    LX, LY = np.meshgrid(lg, lg, indexing="ij")
    return np.array([np.sum(p * LX), np.sum(p * LY)])


@pytest.mark.parametrize("kernel", ["exchange", "ray_then_exchange"])
def test_exchange_chain_reaches_the_exact_posterior(kernel):
    pytest.importorskip("scipy.stats")
    lat = Lattice(np.ones((1, 4, 5), np.uint8), 4)
    rng = np.random.default_rng(1)
    w = gibbs.aux_solve(lat, [0.5, 4.0, 1.0], rng.standard_normal(len(lat.edges())))
    ref = exact_posterior_mean_log(lat, w, model.PRIORS)
    K, steps, burn = 8, 1200, 200          # 8 independent chains on the same field
    st = dict(W=np.repeat(w[None], K, axis=0), alpha=np.ones((K, 3)))
    trace = []
    for c in range(steps):
        step = gibbs.exchange_alpha if kernel == "exchange" else gibbs.aniso_alpha_step
        st["alpha"], _, _ = step(lat, st, 11, c, 0.6)
        trace.append(np.log(st["alpha"][:, :2]))
    x = np.array(trace)[burn:]
    nb = 10
    bl = len(x) // nb
    bm = np.array([x[i * bl:(i + 1) * bl].mean(axis=0) for i in range(nb)]).reshape(-1, 2)
    se = bm.std(axis=0, ddof=1) / np.sqrt(len(bm))
    z = (x.mean(axis=(0, 1)) - ref) / se
    assert np.all(np.abs(z) <= 4.0), (x.mean(axis=(0, 1)), ref, se)
