"""Geometric aggregation multigrid as a PCG preconditioner for B~ (test infrastructure).

The paper preconditions PCG with an incomplete Cholesky factor (Section 3.1). This module
defines a multigrid V-cycle replacement on the same in-mask voxel lattice, from textbook
definitions (aggregation multigrid with Galerkin coarse operators):

* aggregation: fine voxel (x, y, z) belongs to coarse voxel (x // 2, y // 2, z // 2), or
  (x // 2, y // 2, z) for slice-wise 2D lattices (4-neighbour prior); a coarse voxel exists
  when any of its fine voxels is in the mask. P is the piecewise-constant prolongation:
  P[(k, n), (k, agg(n))] = 1 for every regressor k (regressor-major order of B~);
* coarse operator A_c = P' A P (Galerkin). For B~ = H' blkdiag(B_n) H + diag(scale) (x) D_w
  this keeps the same structure: the coarse block is the sum of the fine data blocks, and
  the coarse GMRF part is diag(scale) (x) D_c with D_c the weighted Laplacian of the coarse
  graph (weight = the summed edge weights of the fine edges that join two aggregates);
* smoothing: symmetric red-black block Gauss-Seidel (one forward sweep red then black before
  the coarse correction, one backward sweep black then red after it). Every coarse coupling
  joins face-adjacent aggregates, so the parity of the coarse coordinates two-colours every
  level;
* coarsest level: exact sparse solve, or a fixed number of symmetric red-black block
  Gauss-Seidel steps from zero (the form the GPU runs: it keeps the cycle SPD).

The V-cycle with pre- and post-smoothing mirrored and an exact coarsest solve is a symmetric
positive definite preconditioner M, with the eigenvalues of M^-1 A in (0, 1]. With a single
level and no coarse correction it is one symmetric red-black Gauss-Seidel step, i.e. the
red-black SSOR preconditioner with omega = 1 (``precond.ssor_apply``).

Everything works on explicit scipy sparse matrices in the regressor-major order of
``model.precision``; the arrays are small enough for the tests only.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import model
from .lattice import Lattice


@dataclass
class Level:
    A: sp.csr_matrix          # operator of this level, regressor-major (K blocks of n)
    coords: np.ndarray        # (n, 3) integer (x, y, z) of each voxel of this level
    K: int
    P: sp.csr_matrix | None = None   # prolongation to this level from the next coarser one
    lu: object = None                # exact factor on the coarsest level

    @property
    def n(self):
        return self.coords.shape[0]

    def colour(self):
        return self.coords.sum(axis=1) % 2

    def block_index(self, voxels):
        """Row indices of the K components of the given voxels, shape (len(voxels), K)."""
        return np.arange(self.K)[None, :] * self.n + np.asarray(voxels)[:, None]

    def diag_blocks(self):
        """The K x K diagonal block of every voxel, (n, K, K)."""
        idx = self.block_index(np.arange(self.n))
        A = self.A
        out = np.empty((self.n, self.K, self.K))
        for i in range(self.K):
            for j in range(self.K):
                out[:, i, j] = np.asarray(A[idx[:, i], idx[:, j]]).ravel()
        return out


def aggregate(coords, two_d):
    """Coarse coordinates and the aggregate index of every voxel (2x2x2, or 2x2 in-slice)."""
    c = coords.copy()
    c[:, 0] //= 2
    c[:, 1] //= 2
    if not two_d:
        c[:, 2] //= 2
    uniq, agg = np.unique(c, axis=0, return_inverse=True)
    return uniq, agg.ravel()


def prolongation(agg, n_coarse, K):
    n = len(agg)
    P1 = sp.csr_matrix((np.ones(n), (np.arange(n), agg)), shape=(n, n_coarse))
    return sp.kron(sp.identity(K, format="csr"), P1, format="csr")


def hierarchy(lat: Lattice, blocks, scale, n_min=64, max_levels=10, min_coarse=0):
    """Levels from the fine B~ down to at most n_min voxels (Galerkin coarse operators); a
    coarser level is only added while it has at least min_coarse voxels."""
    N, K, _ = blocks.shape
    x, y, z = lat.coords()
    coords = np.stack([x, y, z], axis=1).astype(np.int64)
    two_d = lat.neighbourhood == 4
    levels = [Level(model.precision(lat, blocks, scale).tocsr(), coords, K)]
    while levels[-1].n > n_min and len(levels) < max_levels:
        fine = levels[-1]
        cc, agg = aggregate(fine.coords, two_d)
        if len(cc) == fine.n or len(cc) < min_coarse:
            break
        fine.P = prolongation(agg, len(cc), K)
        Ac = (fine.P.T @ fine.A @ fine.P).tocsr()
        levels.append(Level(Ac, cc, K))
    levels[-1].lu = spla.splu(levels[-1].A.tocsc())
    return levels


def block_gs(level: Level, b, x, colours):
    """Block Gauss-Seidel half-sweeps over the given colours in order: the voxels of one
    colour are updated together (no couplings inside a colour) from the current residual."""
    D = level.diag_blocks()
    Dinv = np.linalg.inv(D)
    col = level.colour()
    x = x.copy()
    for c in colours:
        vox = np.flatnonzero(col == c)
        idx = level.block_index(vox)
        r = b - level.A @ x
        x[idx] += np.einsum("nij,nj->ni", Dinv[vox], r[idx])
    return x


def vcycle(levels, b, l=0, coarse_steps=None):
    """z = M^-1 b for the V-cycle preconditioner starting at level l (regressor-major).
    The coarsest level is solved exactly (coarse_steps None) or approximated by that many
    symmetric red-black block Gauss-Seidel steps from zero (half-sweeps red, black, red,
    ..., red: 2 coarse_steps + 1 of them), which keeps the cycle symmetric positive
    definite."""
    L = levels[l]
    if l == len(levels) - 1:
        if coarse_steps is None:
            return L.lu.solve(b)
        return block_gs(L, b, np.zeros_like(b), (0,) + (1, 0) * coarse_steps)
    x = block_gs(L, b, np.zeros_like(b), (0, 1))          # red, then black
    r = b - L.A @ x
    x = x + L.P @ vcycle(levels, L.P.T @ r, l + 1, coarse_steps)
    return block_gs(L, b, x, (1, 0))                      # black, then red


def symmetric_gs(level: Level, b):
    """One symmetric red-black block Gauss-Seidel step from zero (no coarse correction)."""
    return block_gs(level, b, np.zeros_like(b), (0, 1, 0))


def coarse_laplacian(coords_c, agg, lat: Lattice):
    """The weighted coarse-graph Laplacian built directly from the fine edges: every fine edge
    (i, j) joining two different aggregates adds its weight C_ee to the
    coupling of the two aggregates (for the Galerkin pin)."""
    E = lat.edges()
    w = lat.edge_weights()
    a, b = agg[E[:, 0]], agg[E[:, 1]]
    keep = a != b
    nc = len(coords_c)
    W = sp.csr_matrix((w[keep], (a[keep], b[keep])), shape=(nc, nc))
    W = W + W.T
    deg = np.asarray(W.sum(axis=1)).ravel()
    return (sp.diags(deg) - W).tocsr()


def pcg(A, b, M, x0=None, tol=1e-10, max_iter=500):
    """Plain preconditioned CG; returns (x, iterations) at ||b - A x|| <= tol ||b||."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A @ x
    nb = np.linalg.norm(b)
    if np.linalg.norm(r) <= tol * nb:
        return x, 0
    z = M(r)
    p = z.copy()
    rz = r @ z
    for it in range(1, max_iter + 1):
        q = A @ p
        a = rz / (p @ q)
        x += a * p
        r -= a * q
        if np.linalg.norm(r) <= tol * nb:
            return x, it
        z = M(r)
        rz2 = r @ z
        p = z + (rz2 / rz) * p
        rz = rz2
    return x, max_iter
