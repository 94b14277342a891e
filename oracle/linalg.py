"""Exact solves, log-determinants and Lanczos quadrature for the oracle.

* Exact solves of B~ x = b replace PCG (Algorithm 2, step 7) by a sparse LU factorisation
  (SuperLU, a library primitive); the conditional mean B~^-1 b_w and a draw B~^-1 b under
  the same perturbation then follow exactly (Section 3.1: PCG approximates this solution
  to relative residual delta).
* log det B~ from the same factorisation; a dense Cholesky / eigen path for small sizes.
* Stochastic Lanczos quadrature (Ubaru, Chen & Saad 2017): for a probe z, z' f(C) z is
  approximated by ||z||^2 e1' f(T_m) e1 with T_m the Lanczos tridiagonal of C started at
  z / ||z||. Lanczos here keeps full reorthogonalisation, so at m = n it is exact. The paper
  names the log-determinant as future work (Discussion); this is the plain definition.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def exact_solve(B, b):
    lu = spla.splu(sp.csc_matrix(B))
    return lu.solve(np.asarray(b, dtype=np.float64))


def factor(B):
    """Sparse LU factorisation object with .solve(b)."""
    return spla.splu(sp.csc_matrix(B))


def logdet_sparse(B):
    """log det of an SPD sparse matrix from its LU factors: sum log |U_ii| (L is unit)."""
    lu = spla.splu(sp.csc_matrix(B))
    return float(np.sum(np.log(np.abs(lu.U.diagonal()))))


def logdet_dense(B):
    Bd = B.toarray() if sp.issparse(B) else np.asarray(B)
    L = np.linalg.cholesky(Bd)
    return 2.0 * float(np.sum(np.log(np.diag(L))))


def logm_quadform_dense(C, Z):
    """z' log(C) z for each column z of Z, via a dense symmetric eigendecomposition."""
    lam, V = np.linalg.eigh(C)
    proj = V.T @ Z
    return np.einsum("ij,i,ij->j", proj, np.log(lam), proj)


def lanczos(matvec, z, m):
    """m steps of Lanczos with full reorthogonalisation; returns the (m, m) tridiagonal
    (fewer rows if an invariant subspace is found first)."""
    n = len(z)
    Q = np.zeros((n, m + 1), order="F")       # columns contiguous for the reorthogonalisation
    a = np.zeros(m)
    b = np.zeros(m)
    Q[:, 0] = z / np.linalg.norm(z)
    k = m
    for j in range(m):
        w = matvec(Q[:, j])
        a[j] = Q[:, j] @ w
        w = w - a[j] * Q[:, j] - (b[j - 1] * Q[:, j - 1] if j > 0 else 0.0)
        w = w - Q[:, :j + 1] @ (Q[:, :j + 1].T @ w)
        w = w - Q[:, :j + 1] @ (Q[:, :j + 1].T @ w)
        b[j] = np.linalg.norm(w)
        if b[j] <= 1e-14 * max(1.0, abs(a[j])):
            k = j + 1
            break
        Q[:, j + 1] = w / b[j]
    T = np.diag(a[:k]) + np.diag(b[:k - 1], 1) + np.diag(b[:k - 1], -1)
    return T


def slq_quadform(matvec, z, m, f=np.log):
    """||z||^2 e1' f(T_m) e1 (Gauss quadrature for z' f(C) z)."""
    T = lanczos(matvec, z, m)
    theta, S = np.linalg.eigh(T)
    return float((z @ z) * np.sum(S[0, :] ** 2 * f(theta)))


def nested_dissection(coords, leaf=64):
    """Geometric nested-dissection order of lattice points (recursive plane bisection): the
    points of a box are split by the median plane across its longest extent; the two halves
    are ordered first (recursively) and the separating plane last. With face-neighbour
    couplings only, no point of one half couples to the other, so a Cholesky or LU factor in
    this order fills in only within the halves and against their separators (George 1973).
    coords: (n, 3) integer coordinates; returns a permutation of range(n)."""
    coords = np.asarray(coords)
    out = []

    def rec(idx):
        if len(idx) <= leaf:
            out.extend(idx.tolist())
            return
        c = coords[idx]
        ext = c.max(axis=0) - c.min(axis=0)
        ax = int(np.argmax(ext))
        if ext[ax] == 0:
            out.extend(idx.tolist())
            return
        mid = int(np.median(c[:, ax]))
        if mid == c[:, ax].min():
            mid += 1
        left, sep, right = idx[c[:, ax] < mid], idx[c[:, ax] == mid], idx[c[:, ax] > mid]
        rec(left)
        rec(right)
        out.extend(sep.tolist())

    rec(np.arange(len(coords)))
    return np.array(out, dtype=np.int64)


def factor_nd(B, coords, D):
    """Sparse LU of B~ (k-major unknowns, D per voxel) in nested-dissection order of the
    voxels, each voxel's D unknowns together, with diagonal pivots (B~ is SPD: its LU with
    diagonal pivots is its Cholesky factorisation up to the diagonal scaling). Returns an
    object with .solve(b) in the original order."""
    N = len(coords)
    order = nested_dissection(coords)
    perm = (np.arange(D)[None, :] * N + order[:, None]).reshape(-1)
    Bp = sp.csc_matrix(B)[perm][:, perm]
    lu = spla.splu(sp.csc_matrix(Bp), permc_spec="NATURAL", diag_pivot_thresh=0.0,
                   options=dict(SymmetricMode=True))

    class _Solver:
        def solve(self, b):
            b = np.asarray(b, dtype=np.float64)
            x = np.empty_like(b)
            x[perm] = lu.solve(b[perm])
            return x

        def logdet(self):
            return float(np.sum(np.log(np.abs(lu.U.diagonal()))))

        nnz = lu.L.nnz + lu.U.nnz

    return _Solver()
