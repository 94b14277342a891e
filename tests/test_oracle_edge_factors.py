"""Pins of the oracle's per-edge weights (a general diagonal C in D_w = G_w' C G_w, the
Discussion's weighted graph Laplacian with C chosen per edge): C_ee = weights[d] times the
factor stored at the edge's lower site. Two independent constructions must agree and match
brute force:

* G_w' C G_w (from the edge list) equals D() (built by adjacency lookups), entry by entry;
* w' D w equals the brute-force sum over coordinate pairs of C_e (w_i - w_j)^2;
* Algorithm 2's perturbation (rows of G_w scaled by sqrt(C_ee)) has covariance exactly B~;
* the alpha quadratic form of the oracle (edge sums) equals w' D w.
"""
import numpy as np
import pytest

from oracle import model, philox
from oracle.lattice import Lattice
from paper_1606_00980_gb300 import synth


def factors(shape, seed):
    """BF16-representable positive factors (k / 16 for k = 4 .. 40)."""
    r = np.random.default_rng(seed)
    return r.integers(4, 41, size=(3,) + shape).astype(np.float64) / 16.0


@pytest.mark.parametrize("dims,nb", [((5, 4, 3), 6), ((6, 5, 1), 4)])
def test_incidence_gram_equals_lookup_laplacian_and_brute_force(dims, nb):
    nx, ny, nz = dims
    mask = np.ones((nz, ny, nx), np.uint8)
    mask[0, 1, 1] = 0
    f = factors((nz, ny, nx), 3)
    lat = Lattice(mask, nb, weights=(2.0, 0.5, 1.25), edge_factors=f)
    G = lat.G()
    C = lat.edge_weights()
    D1 = (G.T @ np_diag(C) @ G).toarray()
    D2 = lat.D().toarray()
    assert np.array_equal(D1, D2)
    v = np.random.default_rng(4).standard_normal(lat.N)
    x, y, z = lat.coords()
    pos = {(int(a), int(b), int(c)): i for i, (a, b, c) in enumerate(zip(x, y, z))}
    w3 = (2.0, 0.5, 1.25)
    brute = 0.0
    for (a, b, c), i in pos.items():
        for d, (dx, dy, dz) in enumerate([(1, 0, 0), (0, 1, 0), (0, 0, 1)][:3 if nb == 6 else 2]):
            j = pos.get((a + dx, b + dy, c + dz))
            if j is not None:
                brute += w3[d] * f[d, c, b, a] * (v[i] - v[j]) ** 2
    assert abs(v @ D2 @ v - brute) <= 1e-12 * abs(brute)
    assert abs(model.quad_forms_edges(lat, v[None])[0] - brute) <= 1e-12 * abs(brute)


def np_diag(c):
    import scipy.sparse as sp
    return sp.diags(c)


def test_perturbation_covariance_with_edge_factors():
    w = synth.small3d(seed=5, dims=(4, 4, 3), K=2, P=1, T=30)
    f = factors((3, 4, 4), 6)
    lat = Lattice(w.mask, 6, weights=(1.0, 2.0, 0.75), edge_factors=f)
    rng = np.random.default_rng(7)
    Bd, _ = model.w_blocks_direct(w.Y, w.X, w.A_true, rng.uniform(0.5, 2.0, w.N))
    alpha = rng.uniform(0.1, 3.0, w.K)
    M = model.perturbation_matrix(lat, Bd, alpha).toarray()
    B = model.precision(lat, Bd, alpha).toarray()
    assert np.max(np.abs(M @ M.T - B)) <= 1e-12 * np.max(np.abs(B))
    pert, z1, z2 = model.perturbation(lat, Bd, alpha, 3, 9, philox.TAG_W, 0)
    z = np.concatenate([model.kmajor(z1), model.kmajor(z2)])
    assert np.allclose(M @ z, pert, rtol=0, atol=1e-12 * np.abs(pert).max())
