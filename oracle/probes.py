"""Log-determinant and trace probes of the full-conditional precision, written out plainly.

The paper names the log-determinant of B~ as future work (Discussion: model evidence and a
collapsed alpha); the trace tr(D_w Cov(W_k)) is the term the SVB alpha update needs
(Eq. quad-form-expectation). With the block-Jacobi preconditioner M = L L'
(M_n = B_n + diag(scale) deg_n per voxel, L_n its lower Cholesky factor):

  log det B~ = log det M + tr log C,   C = L^-1 B~ L^-T,
  tr log C   estimated by the mean over Rademacher probes v_i of v_i' log(C) v_i,
  tr(D^(k) B~^-1) estimated by the mean of (L^-T v_i)' D^(k) B~^-1 L v_i  (E[v v'] = I).

Everything here is dense linear algebra on explicit matrices (small problems only); the
probe vectors come from the same counter-based generator as the CUDA path.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import model, philox
from .lattice import Lattice


def precond_blocks(lat: Lattice, blocks, scale):
    deg = lat.D().diagonal()
    N, D, _ = blocks.shape
    return blocks + deg[:, None, None] * np.diag(scale)[None]


def probe_vectors(lat: Lattice, D, n_probes, seed, counter):
    """v_i as (N, D) arrays: lane k of site lattice-linear * 4 + 3, stream i."""
    return [philox.rademacher(seed, lat.lin * 4 + 3, D, counter, philox.TAG_PROBE, i)
            for i in range(n_probes)]


def exact_probe_terms(lat: Lattice, blocks, scale, V):
    """(log det M, [v_i' log(C) v_i], [[(L^-T v_i)' D (B~^-1 L v_i)]_k], log det B~)."""
    N, D, _ = blocks.shape
    Mb = precond_blocks(lat, blocks, scale)
    Ls = np.stack([np.linalg.cholesky(Mb[n]) for n in range(N)])
    logdet_m = 2.0 * np.sum(np.log(np.stack([np.diag(L) for L in Ls])))
    H = model.H_perm(N, D)
    L = (H.T @ sp.block_diag([sp.csr_matrix(x) for x in Ls], format="csr") @ H).toarray()
    B = model.precision(lat, blocks, scale).toarray()
    Linv = np.linalg.inv(L)
    C = Linv @ B @ Linv.T
    lam, Q = np.linalg.eigh(C)
    Dw = lat.D().toarray()
    quad, traces = [], []
    for v in V:
        vk = model.kmajor(v)
        pr = Q.T @ vk
        quad.append(float(np.sum(pr * pr * np.log(lam))))
        y = np.linalg.solve(B, L @ vk).reshape(D, N)
        t = np.linalg.solve(L.T, vk).reshape(D, N)
        traces.append([float(t[k] @ (Dw @ y[k])) for k in range(D)])
    logdet_b = float(np.linalg.slogdet(B)[1])
    return logdet_m, np.array(quad), np.array(traces), logdet_b


def exact_traces(lat: Lattice, blocks, scale):
    """tr(D_w^(k) B~^-1) for every component k (dense inverse)."""
    N, D, _ = blocks.shape
    Binv = np.linalg.inv(model.precision(lat, blocks, scale).toarray())
    Dw = lat.D().toarray()
    return np.array([np.trace(Dw @ Binv[k * N:(k + 1) * N, k * N:(k + 1) * N]) for k in range(D)])


def block_chol_factors(lat: Lattice, blocks, scale):
    """Per-voxel lower Cholesky factors L_n of the block-Jacobi blocks M_n (N, D, D)."""
    return np.linalg.cholesky(precond_blocks(lat, blocks, scale))


def probe_quadrature_m(lat: Lattice, blocks, scale, v, m):
    """v' log(C) v by the m-point Gauss quadrature of an m-step Lanczos run on
    C = L^-1 B~ L^-T (M = L L' the block-Jacobi preconditioner), with sparse operators only,
    at any size. Preconditioned CG on B~ started from zero with right-hand side L v builds the
    tridiagonal of this Lanczos run step by step, so with m the iterations of a probe solve
    this is the value that solve's CG coefficients define."""
    from . import linalg
    N, D, _ = blocks.shape
    Linv = np.linalg.inv(block_chol_factors(lat, blocks, scale))
    B = model.precision(lat, blocks, scale).tocsr()

    def kmaj_apply(F, x, transpose=False):
        X = x.reshape(D, N).T
        Y = np.einsum("nji,nj->ni" if transpose else "nij,nj->ni", F, X)
        return Y.T.reshape(-1)

    vk = model.kmajor(v)
    return linalg.slq_quadform(lambda x: kmaj_apply(Linv, B @ kmaj_apply(Linv, x, transpose=True)),
                               vk, m)


def probe_terms_lanczos(lat: Lattice, blocks, scale, V, tol=1e-13, m_max=400):
    """Mid-size form of exact_probe_terms (same four results) with sparse operators only:
    v' log(C) v by Lanczos quadrature with full reorthogonalisation (linalg.lanczos), the
    number of steps grown until the value no longer changes (Gauss quadrature is exact at
    m = n, and converges long before that for these spectra); the trace terms by an exact
    sparse solve with B~; log det M and log det B~ from the factors."""
    from . import linalg
    N, D, _ = blocks.shape
    Ls = block_chol_factors(lat, blocks, scale)
    Linv = np.linalg.inv(Ls)
    logdet_m = 2.0 * float(np.sum(np.log(np.einsum("nii->ni", Ls))))
    B = model.precision(lat, blocks, scale).tocsc()
    lu = linalg.factor(B)

    def kmaj_apply(F, x, transpose=False):        # x in k-major order, F per-voxel (N, D, D)
        X = x.reshape(D, N).T
        Y = np.einsum("nji,nj->ni" if transpose else "nij,nj->ni", F, X)
        return Y.T.reshape(-1)

    def cmat(x):                                   # C x = L^-1 B~ L^-T x
        return kmaj_apply(Linv, B @ kmaj_apply(Linv, x, transpose=True))

    n = D * N
    Dw = lat.D()
    quad, traces = [], []
    for v in V:
        vk = model.kmajor(v)
        # the tridiagonal of the first m steps of a Lanczos run is that of an m-step run, so
        # the quadrature is read off for growing m until two successive values agree; the
        # run is repeated with twice the steps if it has not settled
        steps, val = 64, None
        while val is None:
            T = linalg.lanczos(cmat, vk, min(steps, n))
            prev = None
            for m in range(8, T.shape[0] + 8, 8):
                m = min(m, T.shape[0])
                theta, S = np.linalg.eigh(T[:m, :m])
                q = float((vk @ vk) * np.sum(S[0, :] ** 2 * np.log(theta)))
                if (prev is not None and abs(q - prev) <= tol * abs(q)) or m == n:
                    val = q
                    break
                prev = q
            if val is None and (steps >= m_max or T.shape[0] < min(steps, n)):
                raise RuntimeError("Lanczos quadrature did not settle")
            steps *= 2
        quad.append(val)
        y = lu.solve(kmaj_apply(Ls, vk)).reshape(D, N)
        t = kmaj_apply(Linv, vk, transpose=True).reshape(D, N)
        traces.append([float(t[k] @ (Dw @ y[k])) for k in range(D)])
    logdet_b = linalg.logdet_sparse(B)
    return logdet_m, np.array(quad), np.array(traces), logdet_b
