"""Pins of the oracle's aggregation multigrid preconditioner (CPU only): the Galerkin coarse
operator against the coarse graph Laplacian built directly from the fine edges, the single
level against the red-black SSOR preconditioner with omega = 1, the V-cycle's symmetry and
its spectrum bound 0 < eig(M^-1 B~) <= 1, and PCG with it against the direct solve."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import model, multigrid, precond
from oracle.lattice import Lattice


def problem(seed, mask, nb, K=2, weights=(1.0, 1.0, 1.0), data=1.0, scale_range=(0.3, 2.0)):
    rng = np.random.default_rng(seed)
    lat = Lattice(mask, nb, weights=weights)
    N = lat.N
    G = rng.standard_normal((N, K, K))
    blocks = data * (np.einsum("nij,nkj->nik", G, G) + 0.5 * np.eye(K)[None])
    scale = rng.uniform(*scale_range, K)
    return lat, blocks, scale


def ellipsoid(nx, ny, nz):
    z, y, x = np.indices((nz, ny, nx))
    r = (((x - (nx - 1) / 2) / (nx / 2)) ** 2 + ((y - (ny - 1) / 2) / (ny / 2)) ** 2
         + ((z - (nz - 1) / 2) / (nz / 2)) ** 2)
    return (r <= 1.0).astype(np.uint8)


@pytest.mark.parametrize("nb,weights", [(6, (1.0, 1.0, 1.0)), (6, (2.0, 0.5, 3.25)),
                                        (4, (1.0, 1.0, 1.0))])
def test_galerkin_operator_is_coarse_blocks_plus_coarse_laplacian(nb, weights):
    mask = ellipsoid(7, 6, 5) if nb == 6 else ellipsoid(9, 7, 1)
    lat, blocks, scale = problem(3, mask, nb, K=3, weights=weights)
    levels = multigrid.hierarchy(lat, blocks, scale, n_min=1, max_levels=2)
    fine, coarse = levels
    cc, agg = multigrid.aggregate(fine.coords, nb == 4)
    nc = len(cc)
    assert np.array_equal(cc, coarse.coords)
    Bc = np.zeros((nc, 3, 3))
    np.add.at(Bc, agg, blocks)
    Dc = multigrid.coarse_laplacian(cc, agg, lat)
    H = model.H_perm(nc, 3)
    want = H.T @ model.blkdiag(Bc) @ H + sp.kron(sp.diags(scale), Dc)
    assert abs(coarse.A - want).max() <= 1e-12 * abs(want).max()


@pytest.mark.parametrize("nb", [6, 4])
def test_single_level_is_ssor_with_omega_one(nb):
    mask = ellipsoid(6, 5, 4) if nb == 6 else ellipsoid(8, 7, 1)
    lat, blocks, scale = problem(5, mask, nb)
    level = multigrid.hierarchy(lat, blocks, scale, n_min=10 ** 9)[0]
    v = np.random.default_rng(1).standard_normal((lat.N, 2))
    z = multigrid.symmetric_gs(level, model.kmajor(v))
    zs = precond.ssor_apply(lat, blocks, scale, v, 1.0)
    assert np.allclose(model.from_kmajor(z, 2).T, zs, rtol=0, atol=1e-12 * np.abs(zs).max())


@pytest.mark.parametrize("coarse_steps", [None, 1, 3])
@pytest.mark.parametrize("nb", [6, 4])
def test_vcycle_is_symmetric_with_spectrum_in_zero_one(nb, coarse_steps):
    """Exact coarsest solve or a few symmetric Gauss-Seidel steps there: either way the cycle
    is symmetric and 0 < eig(M^-1 B~) <= 1."""
    mask = np.ones((4, 6, 6), np.uint8) if nb == 6 else np.ones((1, 9, 8), np.uint8)
    if nb == 6:
        mask[1, 2, 3] = mask[3, 0, 0] = 0
    lat, blocks, scale = problem(7, mask, nb, data=0.05, scale_range=(1.0, 20.0))
    levels = multigrid.hierarchy(lat, blocks, scale, n_min=8)
    assert len(levels) >= 3
    A = levels[0].A.toarray()
    n = A.shape[0]
    Minv = np.stack([multigrid.vcycle(levels, e, coarse_steps=coarse_steps) for e in np.eye(n)],
                    axis=1)
    assert np.max(np.abs(Minv - Minv.T)) <= 1e-10 * np.max(np.abs(Minv))
    ev = np.linalg.eigvals(Minv @ A)
    assert np.max(np.abs(ev.imag)) <= 1e-8
    assert ev.real.min() > 0 and ev.real.max() <= 1 + 1e-10


def test_pcg_with_vcycle_reaches_the_direct_solve_in_fewer_iterations():
    """A stiff prior (large scale, weak data) on a 16x16x10 ellipsoid: PCG with the V-cycle
    converges to the direct solve and needs fewer iterations than symmetric Gauss-Seidel."""
    lat, blocks, scale = problem(11, ellipsoid(16, 16, 10), 6, data=0.01,
                                 scale_range=(5.0, 50.0))
    levels = multigrid.hierarchy(lat, blocks, scale, n_min=16)
    A = levels[0].A
    b = np.random.default_rng(2).standard_normal(A.shape[0])
    x_direct = spla.spsolve(A.tocsc(), b)
    x_mg, it_mg = multigrid.pcg(A, b, lambda r: multigrid.vcycle(levels, r), tol=1e-10)
    x_gs, it_gs = multigrid.pcg(A, b, lambda r: multigrid.symmetric_gs(levels[0], r), tol=1e-10)
    x_m2, it_m2 = multigrid.pcg(A, b, lambda r: multigrid.vcycle(levels[:3], r, coarse_steps=2),
                                tol=1e-10)
    assert np.linalg.norm(x_mg - x_direct) <= 1e-8 * np.linalg.norm(x_direct)
    assert np.linalg.norm(x_gs - x_direct) <= 1e-8 * np.linalg.norm(x_direct)
    assert np.linalg.norm(x_m2 - x_direct) <= 1e-8 * np.linalg.norm(x_direct)
    assert it_mg < it_gs / 2, (it_mg, it_gs)
    assert it_m2 < it_gs / 2, (it_m2, it_gs)


def test_three_level_cycle_with_smoothed_coarsest_equals_its_definition():
    """The three-level cycle the GPU runs (two coarsenings, two symmetric Gauss-Seidel steps
    on the coarsest level), written out as explicit matrices: with S_l(c) the colour-c
    half-sweep x <- x + E_c D^-1 E_c' (b - A x), the cycle equals the composition of the
    pre-sweeps, the Galerkin coarse correction and the post-sweeps, applied to unit vectors."""
    lat, blocks, scale = problem(19, ellipsoid(8, 8, 6), 6, K=2, data=0.2)
    levels = multigrid.hierarchy(lat, blocks, scale, n_min=1, max_levels=3)
    assert len(levels) == 3

    def half(L, c):
        A = L.A.toarray()
        Dinv = np.linalg.inv(L.diag_blocks())
        E = np.zeros_like(A)
        for v in np.flatnonzero(L.colour() == c):
            idx = L.block_index([v])[0]
            E[np.ix_(idx, idx)] = Dinv[v]
        # x_new = x + E (b - A x) = (I - E A) x + E b
        return np.eye(A.shape[0]) - E @ A, E

    def smoother(L, colours):
        n = L.A.shape[0]
        T, C = np.eye(n), np.zeros((n, n))
        for c in colours:
            G, E = half(L, c)
            T, C = G @ T, G @ C + E
        return T, C          # x = T x0 + C b

    def cycle(l):
        L = levels[l]
        n = L.A.shape[0]
        if l == len(levels) - 1:
            return smoother(L, (0, 1, 0, 1, 0))[1]
        A = L.A.toarray()
        _, Cpre = smoother(L, (0, 1))
        Tpost, Cpost = smoother(L, (1, 0))
        P = L.P.toarray()
        Mc = cycle(l + 1)
        x1 = Cpre                                   # after the pre-sweeps from zero
        x2 = x1 + P @ Mc @ P.T @ (np.eye(n) - A @ x1)
        return Tpost @ x2 + Cpost

    Minv = cycle(0)
    n = levels[0].A.shape[0]
    got = np.stack([multigrid.vcycle(levels, e, coarse_steps=2) for e in np.eye(n)], axis=1)
    assert np.max(np.abs(got - Minv)) <= 1e-12 * np.max(np.abs(Minv))
