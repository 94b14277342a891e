"""Preconditioners of the PCG solve, written from their definitions (test infrastructure).

The paper preconditions its PCG with an incomplete Cholesky factor (Section 3.1); the GPU
path replaces it. Two replacements are defined here, on the precision B~ = Dg + L + U
split into its voxel-block diagonal Dg (block n: B_n + diag(scale) deg_n, the data block
plus the GMRF diagonal) and its strictly lower and upper block parts L, U = L' taken in
red-black order: every voxel with x + y + z even ("red") before every odd ("black") one.
On the face-neighbour lattice every coupling joins a red and a black voxel, so L holds
exactly the black-row / red-column couplings.

  block-Jacobi       M = Dg
  symmetric SOR      M(omega) = (Dg + omega L) Dg^-1 (Dg + omega U) / (omega (2 - omega))
                              = (Dg / omega + L) (Dg / omega)^-1 (Dg / omega + U) / (2 - omega),
                     0 < omega < 2; omega = 1 is symmetric Gauss-Seidel.

``ssor_apply`` solves with the explicit factors above (sparse solves of the two block
triangular factors in the red-black ordering); ``ssor_apply_sweeps`` is the same operator
written as what it is, a forward then a backward SOR sweep, voxel by voxel, from a zero
start: its pin needs no matrix algebra (pure Python loops, tiny inputs only).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import model
from .lattice import Lattice


def colours(lat: Lattice):
    """0 for red voxels (x + y + z even), 1 for black."""
    x, y, z = lat.coords()
    return ((x + y + z) % 2).astype(np.int64)


def redblack_order(lat: Lattice, D):
    """Permutation (as an index array into the regressor-major vector) that lists the D
    components of every red voxel, then those of every black voxel (voxel-major inside
    each colour)."""
    col = colours(lat)
    vox = np.concatenate([np.flatnonzero(col == 0), np.flatnonzero(col == 1)])
    N = lat.N
    return (np.arange(D)[None, :] * N + vox[:, None]).reshape(-1)


def split(lat: Lattice, blocks, scale):
    """(order, Dg, L, U) of B~ in red-black order; Dg, L, U sparse."""
    N, D, _ = blocks.shape
    order = redblack_order(lat, D)
    B = model.precision(lat, blocks, scale).tocsr()[order][:, order].tocoo()
    vox = order % N
    same = vox[B.row] == vox[B.col]
    Dg = sp.csr_matrix((B.data[same], (B.row[same], B.col[same])), shape=B.shape)
    low = (~same) & (B.row > B.col)
    up = (~same) & (B.row < B.col)
    L = sp.csr_matrix((B.data[low], (B.row[low], B.col[low])), shape=B.shape)
    U = sp.csr_matrix((B.data[up], (B.row[up], B.col[up])), shape=B.shape)
    return order, Dg, L, U


def ssor_matrix(lat: Lattice, blocks, scale, omega=1.0):
    """M(omega) as a dense matrix in the regressor-major order of B~ (small problems)."""
    order, Dg, L, U = split(lat, blocks, scale)
    Dw = (Dg / omega).toarray()
    M = (Dw + L.toarray()) @ np.linalg.inv(Dw) @ (Dw + U.toarray()) / (2.0 - omega)
    n = len(order)
    out = np.empty((n, n))
    out[np.ix_(order, order)] = M
    return out


def ssor_apply(lat: Lattice, blocks, scale, v_nk, omega=1.0):
    """z = M(omega)^-1 v, with v and z as (N, D) voxel rows."""
    N, D, _ = blocks.shape
    order, Dg, L, U = split(lat, blocks, scale)
    vr = model.kmajor(v_nk)[order]
    Dw = (Dg / omega).tocsr()
    # block triangular systems (dense D x D diagonal blocks): general sparse solves
    y = spla.spsolve((Dw + L).tocsc(), vr)
    t = Dw @ y
    z = spla.spsolve((Dw + U).tocsc(), t) * (2.0 - omega)
    out = np.empty(N * D)
    out[order] = z
    return model.from_kmajor(out, D).T.copy()


def ssor_apply_sweeps(lat: Lattice, blocks, scale, v_nk, omega=1.0):
    """The same z = M(omega)^-1 v as one symmetric SOR iteration for B~ z = v from z = 0,
    voxel by voxel: a forward sweep over the voxels in red-black order, then a backward
    sweep in the reverse order. Each voxel update solves its own D x D diagonal block for
    the residual left by its neighbours' current values and relaxes by omega."""
    N, D, _ = blocks.shape
    col = colours(lat)
    diag = blocks + lat.degree()[:, None, None] * np.diag(scale)[None]
    nbrs = [[] for _ in range(N)]
    for (i, j, d), c in zip(lat.edges(), lat.edge_weights()):
        nbrs[i].append((j, c))
        nbrs[j].append((i, c))
    v = np.asarray(v_nk, dtype=float)
    z = np.zeros((N, D))
    order = [n for n in range(N) if col[n] == 0] + [n for n in range(N) if col[n] == 1]

    def relax(n):
        # off-diagonal coupling of voxels n, m in component k is -scale_k c_e (edge weight)
        r = v[n] + sum(scale * c * z[m] for m, c in nbrs[n])
        z[n] = (1.0 - omega) * z[n] + omega * np.linalg.solve(diag[n], r)

    for n in order:
        relax(n)
    for n in reversed(order):
        relax(n)
    return z


def schur_system(lat: Lattice, blocks, scale, b_nk):
    """The red-black reduced system. Eliminating the red voxels from B~ x = b (their rows
    read Dg_r x_r + U x_b = b_r, with Dg_r block diagonal) leaves for the black voxels
        S x_b = b^_b,   S = Dg_b - L Dg_r^-1 U,   b^_b = b_b - L Dg_r^-1 b_r,
    after which x_r = Dg_r^-1 (b_r - U x_b). Returns (S, b^_b, recover, n_red) with S and
    b^ in the red-black order restricted to the black block and recover(x_b) -> x as
    (N, D) voxel rows."""
    N, D, _ = blocks.shape
    order, Dg, L, U = split(lat, blocks, scale)
    nr = int((colours(lat) == 0).sum()) * D
    Dg = Dg.tocsr()
    Dr = Dg[:nr, :nr].tocsc()
    Db = Dg[nr:, nr:]
    Lbr = L.tocsr()[nr:, :nr]
    Urb = U.tocsr()[:nr, nr:]
    b = model.kmajor(np.asarray(b_nk, dtype=float))[order]
    br, bb = b[:nr], b[nr:]
    DrinvU = spla.spsolve(Dr, Urb.tocsc())
    DrinvU = sp.csr_matrix(DrinvU) if not sp.issparse(DrinvU) else DrinvU.tocsr()
    S = (Db - Lbr @ DrinvU).tocsr()
    bhat = bb - Lbr @ spla.spsolve(Dr, br)

    def recover(xb):
        xr = spla.spsolve(Dr, br - Urb @ xb)
        out = np.empty(N * D)
        out[order] = np.concatenate([xr, xb])
        return model.from_kmajor(out, D).T.copy()

    return S, bhat, recover, nr


def schur_solve(lat: Lattice, blocks, scale, b_nk):
    """x = B~^-1 b through the reduced system: exact sparse solve of S x_b = b^_b, then the
    red voxels from their own rows."""
    S, bhat, recover, _ = schur_system(lat, blocks, scale, b_nk)
    return recover(spla.spsolve(S.tocsc(), bhat))
