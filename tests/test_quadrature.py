"""Host Lanczos quadrature of the library (CPU only) against numpy's symmetric eigensolver."""
import numpy as np
import pytest

from oracle import linalg


@pytest.fixture(scope="module")
def lib():
    from paper_1606_00980_gb300 import build
    build.build()
    from paper_1606_00980_gb300 import bfmri
    return bfmri


def cg_coefficients(A, b, Minv, m):
    """Plain preconditioned CG from x = 0, returning its step and direction coefficients."""
    r = b.copy()
    z = Minv @ r
    p = z.copy()
    rz = r @ z
    al, be = [], []
    for _ in range(m):
        q = A @ p
        a = rz / (p @ q)
        r = r - a * q
        z = Minv @ r
        rz_new = r @ z
        al.append(a)
        be.append(rz_new / rz)
        p = z + be[-1] * p
        rz = rz_new
    return np.array(al), np.array(be)


@pytest.mark.parametrize("n", [1, 2, 7, 30])
def test_quadrature_matches_dense_eigen_of_T(lib, n):
    rng = np.random.default_rng(n)
    al = rng.uniform(0.1, 2.0, n)
    be = rng.uniform(0.01, 1.5, n)
    T = np.diag(1 / al + np.concatenate([[0.0], be[:-1] / al[:-1]]))
    off = np.sqrt(be[:-1]) / al[:-1]
    T += np.diag(off, 1) + np.diag(off, -1)
    lam, Q = np.linalg.eigh(T)
    ref = float(np.sum(Q[0] ** 2 * np.log(lam)))
    got = lib.lanczos_log_quadrature(al, be[:-1] if n > 1 else np.zeros(0))
    assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref))


def test_quadrature_is_exact_at_full_lanczos_run(lib):
    """Preconditioned CG on A with M = L L' and right-hand side L v is Lanczos on
    C = L^-1 A L^-T from v: after n steps the quadrature equals v' log(C) v / ||v||^2."""
    rng = np.random.default_rng(3)
    n = 24
    G = rng.standard_normal((n, n))
    A = G @ G.T + n * np.eye(n)
    Mdiag = np.diag(A) * rng.uniform(0.8, 1.2, n)
    L = np.diag(np.sqrt(Mdiag))
    v = rng.choice([-1.0, 1.0], n)
    al, be = cg_coefficients(A, L @ v, np.diag(1 / Mdiag), n)
    got = lib.lanczos_log_quadrature(al, be[:-1]) * (v @ v)
    C = np.linalg.inv(L) @ A @ np.linalg.inv(L).T
    ref = linalg.logm_quadform_dense(C, v[:, None])[0]
    assert abs(got - ref) <= 1e-9 * abs(ref)
