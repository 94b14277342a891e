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
