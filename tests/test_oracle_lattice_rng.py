"""Pins for the oracle's lattice graph and random-number generators (CPU only)."""
import os

import numpy as np
import pytest
import scipy.stats as ss

from oracle import philox
from oracle.lattice import Lattice
from paper_1606_00980_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _masks():
    rng = np.random.default_rng(0)
    holes = synth.ellipsoid_mask(7, 6, 5, 3.5, 3.0, 2.5)
    holes[2, 3, 3] = 0
    holes[1, 2, 2] = 0
    checker = (np.indices((4, 4, 4)).sum(axis=0) % 2).astype(np.uint8)  # no face neighbours
    rand = (rng.random((5, 6, 7)) < 0.6).astype(np.uint8)
    return [(synth.circle_mask(9, 9, 4.0), 4), (holes, 6), (holes, 4), (checker, 6),
            (rand, 6), (np.ones((3, 4, 5), np.uint8), 6)]


@pytest.mark.parametrize("case", range(6))
def test_G_transpose_G_equals_laplacian(case):
    """D_w = G_w' G_w exactly (Section 3.1, Eq. 6-7), with D_w built from adjacency lookups."""
    mask, nb = _masks()[case]
    lat = Lattice(mask, nb)
    G = lat.G()
    D = lat.D()
    assert np.array_equal((G.T @ G).toarray(), D.toarray())
    assert np.all(np.asarray(D.sum(axis=1)).ravel() == 0)


def test_full_box_degrees_and_edge_count():
    """A full nx*ny*nz box: interior degree 6 (3D) / 4 (2D), edge count (nx-1)ny nz + ..."""
    nx, ny, nz = 5, 4, 3
    lat = Lattice(np.ones((nz, ny, nx), np.uint8), 6)
    assert len(lat.edges()) == (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1)
    deg = lat.D().diagonal()
    centre = lat.index_of[1 * nx * ny + 1 * nx + 2]
    assert deg[centre] == 6
    lat2 = Lattice(np.ones((nz, ny, nx), np.uint8), 4)
    assert lat2.D().diagonal()[centre] == 4
    assert len(lat2.edges()) == (nx - 1) * ny * nz + nx * (ny - 1) * nz


def test_checkerboard_has_no_edges():
    mask, nb = _masks()[3]
    lat = Lattice(mask, nb)
    assert len(lat.edges()) == 0 and lat.D().nnz == 0


def test_philox_known_answers():
    """Philox4x32-10 against the published known-answer vectors (tests/golden)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = philox.philox4x32_10(*[np.array([c]) for c in v[:4]], v[4], v[5])
        assert [int(o[0]) for o in out] == v[6:]


def test_normals_moments_and_ks():
    z = philox.normals(seed=123, sites=np.arange(50000), width=6, counter=7,
                       tag=philox.TAG_W, stream=3).ravel()
    n = len(z)
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    assert ss.kstest(z, "norm").pvalue > 1e-4
    # lanes are uncorrelated
    zz = philox.normals(123, np.arange(50000), 6, 7, philox.TAG_W, 3)
    c = np.corrcoef(zz.T)
    assert np.max(np.abs(c - np.eye(6))) < 5 / np.sqrt(50000)


def test_rademacher():
    r = philox.rademacher(9, np.arange(40000), 8, 1, philox.TAG_PROBE, 0)
    assert set(np.unique(r)) == {-1.0, 1.0}
    assert abs(r.mean()) < 5 / np.sqrt(r.size)


@pytest.mark.parametrize("shape,scale", [(0.5, 2.0), (1.5, 1.0), (75.1, 0.02), (25000.1, 1e-4)])
def test_gamma_moments_and_ks(shape, scale):
    """Marsaglia-Tsang draws: mean b c, variance b^2 c (Ga(b, c), Appendix B Eq. alphamean)."""
    n = 40000
    g, exhausted = philox.gamma(5, np.arange(n), shape, scale, 3, philox.TAG_LAMBDA, 1)
    assert exhausted == 0
    assert abs(g.mean() - shape * scale) < 5 * np.sqrt(shape * scale ** 2 / n)
    v = shape * scale ** 2
    assert abs(g.var() - v) < 6 * v * np.sqrt(2.0 / n) * (1 + 3.0 / shape)
    assert ss.kstest(g, ss.gamma(a=shape, scale=scale).cdf).pvalue > 1e-4


def test_prior_means_from_section2():
    vals = dict(l.split() for l in open(os.path.join(GOLDEN, "priors_section2.txt"))
                if l.strip() and not l.startswith("#"))
    from oracle.model import PRIORS
    for k, v in vals.items():
        assert PRIORS[k] == float(v)
    assert PRIORS["q1"] * PRIORS["q2"] == 1.0 and PRIORS["r1"] * PRIORS["r2"] == 1000.0
