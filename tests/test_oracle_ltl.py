"""Pins of the oracle's L'L prior (D_w = L'L, L the graph Laplacian; Section 2 names it as the
alternative to the UGL default), checked against brute force and the mathematics rather than
against the oracle's own sparse algebra.

* the stencil: an interior voxel's row of L'L has 25 nonzeros on the 6-neighbour lattice and
  13 on the 4-neighbour slice lattice, with the values a second difference gives (diagonal
  deg^2 + deg, -2 deg at face neighbours, 2 at in-plane diagonals, 1 two steps away);
* the precision is the Hessian of the brute-force log full conditional of W, whose prior
  term sums, voxel by voxel, the squared Laplacian (deg_n w_n - sum of the neighbours' w);
* Algorithm 2's perturbation with L' in place of G' has covariance exactly B~;
* the alpha quadratic form |L w|^2 equals the brute-force voxel sum, and is zero for a
  constant field (L'L shares L's null space).
"""
import numpy as np
import pytest

from oracle import model, philox
from oracle.lattice import Lattice
from paper_1606_00980_gb300 import synth


def tiny(dims, K=2, P=1, T=30, nb=6, seed=0, mask=None):
    nx, ny, nz = dims
    if mask is None:
        mask = np.ones((nz, ny, nx), np.uint8)
    w = synth.make_workload("tiny", dims, mask, T=T, K=K, P=P, neighbourhood=nb, seed=seed,
                            ar_mean=(0.3,), n_blobs=1)
    return w, Lattice(w.mask, nb)


def neighbours(lat):
    """Adjacency lists by explicit coordinate lookup (independent of the sparse builders)."""
    x, y, z = lat.coords()
    index = {(int(a), int(b), int(c)): i for i, (a, b, c) in enumerate(zip(x, y, z))}
    offs = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0)]
    if lat.neighbourhood == 6:
        offs += [(0, 0, 1), (0, 0, -1)]
    return [[index[(int(x[i]) + dx, int(y[i]) + dy, int(z[i]) + dz)]
             for dx, dy, dz in offs if (int(x[i]) + dx, int(y[i]) + dy, int(z[i]) + dz) in index]
            for i in range(lat.N)]


def lap_brute(nbrs, v):
    return np.array([len(nb) * v[i] - sum(v[j] for j in nb) for i, nb in enumerate(nbrs)])


@pytest.mark.parametrize("dims,nb,count", [((7, 7, 7), 6, 25), ((9, 9, 1), 4, 13)])
def test_stencil_width_and_values(dims, nb, count):
    w, lat = tiny(dims, nb=nb)
    D = model.prior_precision(lat, "ltl").toarray()
    nbrs = neighbours(lat)
    x, y, z = lat.coords()
    c = [i for i in range(lat.N) if x[i] == dims[0] // 2 and y[i] == dims[1] // 2 and z[i] == dims[2] // 2][0]
    row = D[c]
    assert np.count_nonzero(row) == count
    deg = len(nbrs[c])
    assert row[c] == deg * deg + deg
    for j in nbrs[c]:
        assert row[j] == -2 * deg
    # every entry equals the brute-force second difference sum_m L_cm L_mj
    e = np.zeros(lat.N)
    for j in range(lat.N):
        e[:] = 0.0
        e[j] = 1.0
        assert row[j] == lap_brute(nbrs, lap_brute(nbrs, e))[c]


@pytest.mark.parametrize("dims,nb", [((4, 3, 3), 6), ((5, 4, 1), 4)])
def test_ltl_precision_is_hessian_of_log_posterior(dims, nb):
    w, lat = tiny(dims, K=2, P=1, T=40, nb=nb)
    rng = np.random.default_rng(3)
    lam = rng.uniform(0.5, 2.0, w.N)
    alpha = rng.uniform(0.1, 3.0, w.K)
    A = w.A_true
    Bd, bw = model.w_blocks_direct(w.Y, w.X, A, lam)
    B = model.precision(lat, Bd, alpha, "ltl")
    b = model.kmajor(bw)
    nbrs = neighbours(lat)

    def f(vec):
        Wm = vec.reshape(w.K, w.N)
        tot = 0.0
        for n in range(w.N):
            yt, Xt = model.whiten(w.Y[:, n], w.X, A[:, n])
            r = yt - Xt @ Wm[:, n]
            tot += 0.5 * lam[n] * r @ r
        for k in range(w.K):
            tot += 0.5 * alpha[k] * np.sum(lap_brute(nbrs, Wm[k]) ** 2)
        return tot

    f0 = f(np.zeros(w.K * w.N))
    for _ in range(3):
        v = rng.standard_normal(w.K * w.N)
        lhs = f(v) - f0
        rhs = -b @ v + 0.5 * v @ (B @ v)
        assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(lhs))


@pytest.mark.parametrize("dims,nb", [((4, 3, 3), 6), ((5, 4, 1), 4)])
def test_ltl_perturbation_covariance_is_precision(dims, nb):
    w, lat = tiny(dims, K=2, P=1, T=30, nb=nb)
    rng = np.random.default_rng(5)
    lam = rng.uniform(0.5, 2.0, w.N)
    alpha = rng.uniform(0.1, 3.0, w.K)
    Bd, _ = model.w_blocks_direct(w.Y, w.X, w.A_true, lam)
    M = model.perturbation_matrix(lat, Bd, alpha, "ltl").toarray()
    B = model.precision(lat, Bd, alpha, "ltl").toarray()
    assert np.max(np.abs(M @ M.T - B)) <= 1e-12 * np.max(np.abs(B))
    pert, z1, z2 = model.perturbation(lat, Bd, alpha, 3, 9, philox.TAG_W, 0, "ltl")
    assert z1.shape == (w.N, w.K)          # one normal per voxel and regressor
    z = np.concatenate([model.kmajor(z1), model.kmajor(z2)])
    assert np.allclose(M @ z, pert, rtol=0, atol=1e-12 * np.abs(pert).max())
    # z1 of voxel n uses site lattice-linear(n) * 4 + 0
    assert np.array_equal(z1, philox.normals(3, lat.lin * 4 + 0, w.K, 9, philox.TAG_W, 0))


def test_ltl_quadratic_form():
    w, lat = tiny((5, 4, 3), K=3, nb=6)
    V = np.random.default_rng(7).standard_normal((3, w.N))
    nbrs = neighbours(lat)
    ref = np.array([np.sum(lap_brute(nbrs, V[k]) ** 2) for k in range(3)])
    assert np.allclose(model.quad_forms_ltl(lat, V), ref, rtol=1e-13)
    assert np.max(np.abs(model.quad_forms_ltl(lat, np.full((1, w.N), 2.5)))) <= 1e-20
