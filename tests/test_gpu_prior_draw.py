"""Draws from the UGL prior alone through the library (needs a GB300).

The paper simulates its task rows of W and its AR row from the UGL prior by running the
W and A draws with no data term from a zero start (Appendix D); the benchmark's simulation
study does the same with lambda = 1e-200. Without data, Algorithm 2 solves
alpha G'G w = sqrt(alpha) G'z1, whose right-hand side lies in the range of G', and the edge
increments G w of one row are a draw of the increments of the
intrinsic GMRF: alpha |G w|^2 = |Pi z1|^2 with Pi the projector onto the range of G, a
chi-square with N - 1 degrees of freedom (one connected component). Checked on a block
lattice for every row, within five standard deviations. A preconditioned solve may add a
constant (the null space of G'G) to w, which the increments do not see; the paper notes that
the draws have a mean close to zero, checked loosely against the row's spread.
"""
import numpy as np
import pytest

from oracle.lattice import Lattice

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precond", ["reduced", "bj"])
def test_prior_draw_with_no_data_term(precond):
    from paper_1606_00980_gb300 import bfmri
    from paper_1606_00980_gb300.bfmri import Model
    nx, ny, nz = 24, 20, 18
    n = nx * ny * nz
    alphas = np.array([1e-4, 5e-4, 2e-3, 1e-2])
    beta = 10.0
    K, P, T = len(alphas), 1, 8
    rng = np.random.default_rng(5)
    pc = bfmri.PRECOND_RB_REDUCED if precond == "reduced" else bfmri.PRECOND_BLOCK_JACOBI
    m = Model((nx, ny, nz, 6), np.ones((nz, ny, nx), np.uint8), rng.standard_normal((T, K)),
              rng.standard_normal((T, n)), K, P, delta=1e-10, seed=17, max_iter=20000,
              precond=pc)
    m.precompute_stats()
    m.set_state(W=np.zeros((K, n)), A=np.zeros((P, n)), lam=np.full(n, 1e-200), alpha=alphas,
                beta=np.array([beta]))
    W, info = m.sample_W(counter=1)
    A, ia = m.sample_A(counter=2)
    m.close()
    assert info.rel_residual <= 1e-10 and ia.rel_residual <= 1e-10
    E = Lattice(np.ones((nz, ny, nx), np.uint8), 6).edges()
    dof = n - 1
    for row, prec in list(zip(W, alphas)) + [(A[0], beta)]:
        assert abs(row.mean()) <= row.std()
        q = prec * np.sum((row[E[:, 0]] - row[E[:, 1]]) ** 2)
        assert abs(q - dof) <= 5 * np.sqrt(2 * dof), (prec, q, dof)
