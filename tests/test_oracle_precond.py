"""Pins of the oracle's preconditioners (CPU only): the red-black symmetric SOR operator in
factored form against the voxel-by-voxel forward/backward SOR sweeps (brute force, tiny
lattices), its SPD-ness and the SSOR bound 0 < eig(M^-1 B~) <= 1, the reduction to
block-Jacobi without couplings, the two-colouring of the lattice, the red-black reduced
(Schur) system, and CG on its split-preconditioned form against block-Jacobi PCG."""
import numpy as np
import pytest

from oracle import model, precond
from oracle.lattice import Lattice


def small_problem(seed, D=2, neighbourhood=6):
    rng = np.random.default_rng(seed)
    if neighbourhood == 6:
        mask = np.ones((3, 3, 4), np.uint8)
        mask[1, 1, 1] = 0
        mask[2, 0, 3] = 0
    else:
        mask = np.ones((1, 4, 5), np.uint8)
        mask[0, 2, 2] = 0
    lat = Lattice(mask, neighbourhood)
    N = lat.N
    G = rng.standard_normal((N, D, D))
    blocks = np.einsum("nij,nkj->nik", G, G) + 0.5 * np.eye(D)[None]
    scale = rng.uniform(0.3, 2.0, D)
    v = rng.standard_normal((N, D))
    return lat, blocks, scale, v


@pytest.mark.parametrize("omega", [0.7, 1.0, 1.3])
@pytest.mark.parametrize("neighbourhood", [6, 4])
def test_factored_form_equals_sor_sweeps(omega, neighbourhood):
    lat, blocks, scale, v = small_problem(3, neighbourhood=neighbourhood)
    z = precond.ssor_apply(lat, blocks, scale, v, omega)
    zs = precond.ssor_apply_sweeps(lat, blocks, scale, v, omega)
    assert np.max(np.abs(z - zs)) <= 1e-12 * np.max(np.abs(zs))


@pytest.mark.parametrize("omega", [0.7, 1.0, 1.3])
def test_ssor_is_spd_and_bounds_the_spectrum(omega):
    lat, blocks, scale, v = small_problem(5, D=3)
    M = precond.ssor_matrix(lat, blocks, scale, omega)
    assert np.max(np.abs(M - M.T)) <= 1e-12 * np.max(np.abs(M))
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0
    B = model.precision(lat, blocks, scale).toarray()
    ev = np.linalg.eigvals(np.linalg.solve(M, B)).real
    assert ev.min() > 0 and ev.max() <= 1 + 1e-10


def test_apply_inverts_matrix_form():
    lat, blocks, scale, _ = small_problem(7, D=3)
    v = np.random.default_rng(2).standard_normal((lat.N, 3))
    M = precond.ssor_matrix(lat, blocks, scale, 1.2)
    z = precond.ssor_apply(lat, blocks, scale, v, 1.2)
    vz = model.from_kmajor(M @ model.kmajor(z), 3).T
    assert np.max(np.abs(vz - v)) <= 1e-11 * np.max(np.abs(v))


def test_without_couplings_sgs_is_block_jacobi():
    lat, blocks, _, v = small_problem(9)
    z = precond.ssor_apply(lat, blocks, np.zeros(2), v, 1.0)
    zb = np.stack([np.linalg.solve(blocks[n], v[n]) for n in range(lat.N)])
    assert np.max(np.abs(z - zb)) <= 1e-13 * np.max(np.abs(zb))


@pytest.mark.parametrize("neighbourhood", [6, 4])
def test_every_edge_joins_two_colours(neighbourhood):
    lat, _, _, _ = small_problem(1, neighbourhood=neighbourhood)
    c = precond.colours(lat)
    E = lat.edges()
    assert np.all(c[E[:, 0]] != c[E[:, 1]])
    assert 0 < c.sum() < lat.N


def test_schur_solve_equals_the_direct_solve():
    """Block elimination of the red voxels is exact: the reduced solve reproduces the
    direct sparse solve of B~ x = b."""
    import scipy.sparse.linalg as spla
    for nb, K in [(6, 3), (4, 2)]:
        lat, blocks, scale, b = small_problem(5 + nb, D=K, neighbourhood=nb)
        x = precond.schur_solve(lat, blocks, scale, b)
        B = model.precision(lat, blocks, scale).tocsc()
        xd = model.from_kmajor(spla.spsolve(B, model.kmajor(b)), K).T
        assert np.linalg.norm(x - xd) <= 1e-12 * np.linalg.norm(xd)


def test_ssor_omega1_spectrum_is_one_and_the_reduced_spectrum():
    """With red-black ordering and omega = 1, M^-1 B~ has the eigenvalue 1 once per red
    unknown and otherwise the eigenvalues of Dg_b^-1 S: PCG with symmetric Gauss-Seidel is
    CG on the reduced system preconditioned by its block diagonal (same Krylov spaces, so
    the same iteration counts up to the red component of the start residual)."""
    lat, blocks, scale, _ = small_problem(9, D=2, neighbourhood=6)
    M = precond.ssor_matrix(lat, blocks, scale, omega=1.0)
    B = model.precision(lat, blocks, scale).toarray()
    ev = np.sort(np.linalg.eigvals(np.linalg.solve(M, B)).real)
    S, _, _, nr = precond.schur_system(lat, blocks, scale, np.zeros((lat.N, 2)))
    order, Dg, _, _ = precond.split(lat, blocks, scale)
    Db = Dg.toarray()[nr:, nr:]
    evs = np.linalg.eigvals(np.linalg.solve(Db, S.toarray())).real
    want = np.sort(np.concatenate([np.ones(nr), evs]))
    assert np.allclose(ev, want, rtol=0, atol=1e-10)


@pytest.mark.parametrize("omega", [0.8, 1.0])
def test_weighted_factored_form_equals_sor_sweeps(omega):
    """Under the WGL prior (edge weights per direction) the SSOR operator in factored form
    still equals one forward and one backward SOR sweep voxel by voxel."""
    lat, blocks, scale, v = small_problem(13, D=2, neighbourhood=6)
    lat = Lattice(lat.mask, 6, weights=(2.0, 0.5, 3.25))
    a = precond.ssor_apply(lat, blocks, scale, v, omega)
    b = precond.ssor_apply_sweeps(lat, blocks, scale, v, omega)
    assert np.allclose(a, b, rtol=1e-12, atol=1e-12)


def test_split_preconditioned_cg_has_the_iterates_of_block_jacobi_pcg():
    """CG without a preconditioner on L_b^-1 S L_b^-T (Dg_b = L_b L_b', the black voxels'
    diagonal blocks) produces, mapped back by x_b = L_b^-T x^, the iterates of CG on S
    preconditioned by Dg_b, and its residual maps back by r = L_b r^. So a solver on the
    split form may stop on |L_b r^| with the iteration counts of the preconditioned one."""
    lat, blocks, scale, _ = small_problem(17, D=3, neighbourhood=6)
    rng = np.random.default_rng(4)
    b = rng.standard_normal((lat.N, 3))
    S, bhat, _, nr = precond.schur_system(lat, blocks, scale, b)
    S = S.toarray()
    _, Dg, _, _ = precond.split(lat, blocks, scale)
    Db = Dg.toarray()[nr:, nr:]
    Lb = np.linalg.cholesky(Db)
    Li = np.linalg.inv(Lb)
    Sh = Li @ S @ Li.T
    n = len(bhat)
    x = np.zeros(n)
    r = bhat.copy()
    z = np.linalg.solve(Db, r)
    p = z.copy()
    rz = r @ z
    xh = np.zeros(n)
    rh = Li @ bhat
    ph = rh.copy()
    rr = rh @ rh
    for _ in range(8):
        q = S @ p
        a = rz / (p @ q)
        x, r = x + a * p, r - a * q
        z = np.linalg.solve(Db, r)
        rz2 = r @ z
        p, rz = z + rz2 / rz * p, rz2
        qh = Sh @ ph
        ah = rr / (ph @ qh)
        xh, rh = xh + ah * ph, rh - ah * qh
        rr2 = rh @ rh
        ph, rr = rh + rr2 / rr * ph, rr2
        assert np.allclose(Li.T @ xh, x, rtol=0, atol=1e-10 * np.abs(x).max())
        assert np.allclose(Lb @ rh, r, rtol=0, atol=1e-10 * np.abs(bhat).max())
