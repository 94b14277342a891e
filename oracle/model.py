"""Full conditionals of the spatial fMRI GLM with AR(P) noise (Appendix A, temporal noise model).

Notation: Y is T x N (voxel n = column n), X is T x K, W is K x N, A is P x N, lambda is N,
alpha is K, beta is P. Every sum over time runs over t = P+1..T (1-based): the paper
conditions on the first P time points (Eq. likeliTemp), and we read the i.i.d.-looking
terms of Eq. log-like (Y'Y, Y'X, X'X) with the same range so that they combine with the
AR terms; with P = 0 this is the full range of Appendix A's i.i.d. model.

Whitening: with c = (1, -a_1, ..., -a_P), the residual innovation of voxel n is
    eps_t = (y_t - x_t w) - sum_p a_p (y_{t-p} - x_{t-p} w) = sum_p c_p (y_{t-p} - x_{t-p} w),
which is Eq. likeliTemp's bracket. Expanding its square in w gives the W full conditional
(Eq. full cond W temporal): block lambda_n X~'X~, right-hand side lambda_n X~'y~ where
X~ = sum_p c_p L^p X and y~ = sum_p c_p L^p y; expanding it in a gives the A full
conditional (Eq. fullcondTempA) and its value at (w, a) gives the lambda full conditional
(Eq. fullcondTemplambda).

The paper's tensors B_n, R, D_n, S are contractions of the lagged cross-products
    Syy[p, q]    = sum_t y_{t-p} y_{t-q}
    Sxy[p, q, k] = sum_t y_{t-p} x_{t-q, k}
    Sxx[p, q]    = sum_t x_{t-p} x_{t-q}'          (K x K, voxel independent)
(p, q in 0..P), which is how sufficient_stats() stores them; the direct functions below
never use them and serve as their pin.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import philox
from .lattice import Lattice

# Hyperprior defaults (Section 2, last paragraph): q1 = u1 = 10, r1 = 10000, q2 = r2 = u2 = 0.1.
PRIORS = dict(q1=10.0, q2=0.1, u1=10.0, u2=0.1, r1=10000.0, r2=0.1)


def lag(v, p, P):
    """Rows t = P+1..T of L^p v (1-based), i.e. v[P-p : T-p] (0-based)."""
    T = v.shape[0]
    return v[P - p:T - p]


def ar_coeffs(a):
    """c = (1, -a_1, ..., -a_P)."""
    return np.concatenate([[1.0], -np.asarray(a, dtype=np.float64)])


# ----------------------------------------------------------------------------------------
# Direct (time-series) forms: the reference for everything built from statistics.
# ----------------------------------------------------------------------------------------

def whiten(y, X, a):
    """y~ = sum_p c_p L^p y and X~ = sum_p c_p L^p X over t = P+1..T (Eq. likeliTemp)."""
    P = len(a)
    c = ar_coeffs(a)
    yt = sum(c[p] * lag(y, p, P) for p in range(P + 1))
    Xt = sum(c[p] * lag(X, p, P) for p in range(P + 1))
    return yt, Xt


def w_blocks_direct(Y, X, A, lam, eps=0.0):
    """Per-voxel data block Bd_n = lambda_n X~'X~ + eps I and b_n = lambda_n X~'y~
    (Eq. full cond W temporal, the n-th blkdiag block and the n-th row of b_w)."""
    T, N = Y.shape
    K = X.shape[1]
    Bd = np.empty((N, K, K))
    bw = np.empty((N, K))
    for n in range(N):
        yt, Xt = whiten(Y[:, n], X, A[:, n])
        Bd[n] = lam[n] * (Xt.T @ Xt) + eps * np.eye(K)
        bw[n] = lam[n] * (Xt.T @ yt)
    return Bd, bw


def residual_lags(y, X, w, P):
    """Columns L^p (y - X w) for p = 0..P over t = P+1..T."""
    e = y - X @ w
    return np.stack([lag(e, p, P) for p in range(P + 1)], axis=1)


def a_blocks_direct(Y, X, W, lam, P):
    """A full conditional (Eq. fullcondTempA): with E = [L^1 e, ..., L^P e] and e = y - X w_n,
    the block is lambda_n E'E and the right-hand side lambda_n E'(L^0 e)."""
    N = Y.shape[1]
    Ja = np.empty((N, P, P))
    ba = np.empty((N, P))
    for n in range(N):
        E = residual_lags(Y[:, n], X, W[:, n], P)
        Ja[n] = lam[n] * (E[:, 1:].T @ E[:, 1:])
        ba[n] = lam[n] * (E[:, 1:].T @ E[:, 0])
    return Ja, ba


def rss_direct(Y, X, W, A):
    """Sum over t = P+1..T of the squared innovation eps_t (the bracket of
    Eq. fullcondTemplambda), computed from the residual time series without cancellation."""
    P, N = A.shape
    out = np.empty(N)
    for n in range(N):
        E = residual_lags(Y[:, n], X, W[:, n], P)
        eps = E @ ar_coeffs(A[:, n])
        out[n] = eps @ eps
    return out


# ----------------------------------------------------------------------------------------
# Sufficient statistics (Appendix A: "pre-computed outside the Gibbs algorithm").
# ----------------------------------------------------------------------------------------

def sufficient_stats(Y, X, P):
    """Lagged cross-products over t = P+1..T: Syy (N, P+1, P+1), Sxy (N, P+1, P+1, K) with
    Sxy[n, p, q, k] = sum_t y_{t-p, n} x_{t-q, k}, and Sxx (P+1, P+1, K, K)."""
    T, N = Y.shape
    K = X.shape[1]
    Ly = [lag(Y, p, P) for p in range(P + 1)]
    Lx = [lag(X, p, P) for p in range(P + 1)]
    Syy = np.empty((N, P + 1, P + 1))
    Sxy = np.empty((N, P + 1, P + 1, K))
    Sxx = np.empty((P + 1, P + 1, K, K))
    for p in range(P + 1):
        for q in range(P + 1):
            Syy[:, p, q] = np.einsum("tn,tn->n", Ly[p], Ly[q])
            Sxy[:, p, q, :] = Ly[p].T @ Lx[q]
            Sxx[p, q] = Lx[p].T @ Lx[q]
    return dict(Syy=Syy, Sxy=Sxy, Sxx=Sxx, P=P, T=T)


def w_blocks_from_stats(st, A, lam, eps=0.0):
    """X~'X~ = sum_pq c_p c_q Sxx[p, q] and X~'y~ = sum_pq c_p c_q Sxy[p, q] (the expansion of
    Eq. full cond W temporal in terms of R, S, B_n, D_n)."""
    Sxx, Sxy = st["Sxx"], st["Sxy"]
    P = st["P"]
    N = Sxy.shape[0]
    K = Sxx.shape[-1]
    C = np.concatenate([np.ones((1, N)), -A], axis=0)          # (P+1, N)
    XtX = np.einsum("pn,qn,pqij->nij", C, C, Sxx)
    Xty = np.einsum("pn,qn,npqk->nk", C, C, Sxy)
    return lam[:, None, None] * XtX + eps * np.eye(K)[None], lam[:, None] * Xty


def lagged_residual_gram(st, W):
    """G[n, p, q] = (L^p e)'(L^q e) with e = y - X w_n, from statistics:
    Syy[p,q] - w.Sxy[q,p] - w.Sxy[p,q] + w' Sxx[p,q] w   (note Sxy[p,q] = (L^q X)' L^p y)."""
    Syy, Sxy, Sxx = st["Syy"], st["Sxy"], st["Sxx"]
    t1 = np.einsum("kn,npqk->npq", W, Sxy)
    quad = np.einsum("kn,pqkl,ln->npq", W, Sxx, W)
    return Syy - t1 - np.transpose(t1, (0, 2, 1)) + quad


def a_blocks_from_stats(st, W, lam):
    G = lagged_residual_gram(st, W)
    return lam[:, None, None] * G[:, 1:, 1:], lam[:, None] * G[:, 1:, 0]


def rss_from_stats(st, W, A):
    G = lagged_residual_gram(st, W)
    N = G.shape[0]
    C = np.concatenate([np.ones((1, N)), -A], axis=0)
    return np.einsum("pn,npq,qn->n", C, G, C)


# ----------------------------------------------------------------------------------------
# Posterior precision in the paper's ordering (Eq. wr full conditional / full cond W temporal)
# ----------------------------------------------------------------------------------------

def H_perm(N, K):
    """H_w with vec(W) = H_w vec(W') for a K x N matrix W (Section 3.1, before Algorithm 2):
    vec(W) is voxel-major (index n K + k), vec(W') is regressor-major (index k N + n)."""
    rows = (np.arange(N)[None, :] * K + np.arange(K)[:, None]).reshape(-1)  # vec(W) index
    cols = (np.arange(K)[:, None] * N + np.arange(N)[None, :]).reshape(-1)  # vec(W') index
    return sp.csr_matrix((np.ones(N * K), (rows, cols)), shape=(N * K, N * K))


def blkdiag(blocks):
    return sp.block_diag([sp.csr_matrix(b) for b in blocks], format="csr")


def prior_precision(lat: Lattice, prior="ugl"):
    """The spatial precision D_w of Section 2: the (weighted) graph Laplacian L ("ugl", the
    SPM12 default the paper uses), or L'L ("ltl", the prior of Penny et al. 2005 that the
    paper mentions as an alternative: a 25-point stencil in 3D, 13-point in 2D)."""
    L = lat.D()
    if prior == "ugl":
        return L
    if prior == "ltl":
        return (L.T @ L).tocsr()
    raise ValueError(prior)


def direction_laplacians(lat: Lattice):
    """L_d = G_d' C_d G_d for d = x, y, z: the graph Laplacian of the direction-d edges alone,
    from the incidence matrix with the other directions' rows weighted 0 (sum_d L_d = D_w).
    The Discussion's anisotropic prior gives W_k the precision sum_d alpha_{d,k} L_d."""
    G = lat.G()
    e = lat.edges()
    c = lat.edge_weights()
    return [(G.T @ sp.diags(np.where(e[:, 2] == d, c, 0.0)) @ G).tocsr() for d in range(3)]


def aniso_prior(lat: Lattice, scale):
    """blockdiag_k(sum_d scale[k, d] L_d): the anisotropic prior precision of the Discussion
    (C_k = diag(alpha_x,k I, alpha_y,k I, alpha_z,k I) between G_w' and G_w)."""
    Ls = direction_laplacians(lat)
    scale = np.asarray(scale, dtype=np.float64)
    return sp.block_diag([sum(scale[k, d] * Ls[d] for d in range(3)) for k in range(scale.shape[0])],
                         format="csr")


def precision(lat: Lattice, blocks, scale, prior="ugl"):
    """B~ = H' blkdiag_n(blocks_n) H + diag(scale) (x) D_w  in regressor-major order; for the
    anisotropic prior ("aniso") scale is K x 3 and the prior part is aniso_prior()."""
    N, K, _ = blocks.shape
    H = H_perm(N, K)
    if prior == "aniso":
        return (H.T @ blkdiag(blocks) @ H + aniso_prior(lat, scale)).tocsr()
    return (H.T @ blkdiag(blocks) @ H + sp.kron(sp.diags(scale), prior_precision(lat, prior))).tocsr()


def kmajor(v_nk):
    """(N, K) voxel rows -> vec(V') regressor-major vector of length K N."""
    return np.ascontiguousarray(np.asarray(v_nk).T).reshape(-1)


def from_kmajor(v, K):
    return v.reshape(K, -1)


def perturbation(lat: Lattice, blocks, scale, seed, counter, tag, stream=0, prior="ugl"):
    """The random part of Algorithm 2's right-hand side,
        sum_k sqrt(scale_k) (G' z1_k)  +  H' L_data H z2        (regressor-major),
    with L_data the per-voxel lower Cholesky factor of the data block. z1[e, k] is the
    normal of edge e (site = lattice-linear(i) * 4 + d) and z2[n, k] that of voxel n
    (site = lattice-linear(n) * 4 + 3), lane k (oracle.philox.normals).
    For the L'L prior the square root of D_w = L'L is L' itself (N x N): z1[n, k] is then one
    normal per voxel (site = lattice-linear(n) * 4 + 0) and the first term sqrt(scale_k) L' z1_k,
    whose covariance is scale_k L'L. For the anisotropic prior (scale K x 3) edge e of
    direction d carries sqrt(scale[k, d]) on top of sqrt(C_ee): covariance sum_d scale[k, d] L_d."""
    N, K, _ = blocks.shape
    z2 = philox.normals(seed, lat.lin * 4 + 3, K, counter, tag, stream)
    if prior == "ltl":
        z1 = philox.normals(seed, lat.lin * 4 + 0, K, counter, tag, stream)
        Lt = lat.D().T.tocsr()
        part1 = np.concatenate([np.sqrt(scale[k]) * (Lt @ z1[:, k]) for k in range(K)])
    else:
        E = lat.edges()
        sites_e = lat.lin[E[:, 0]] * 4 + E[:, 2]
        z1 = philox.normals(seed, sites_e, K, counter, tag, stream)
        G = lat.Gw()
        if prior == "aniso":
            sq = np.sqrt(np.asarray(scale, dtype=np.float64)[:, E[:, 2]])   # (K, edges)
            part1 = np.concatenate([G.T @ (sq[k] * z1[:, k]) for k in range(K)])
        else:
            part1 = np.concatenate([np.sqrt(scale[k]) * (G.T @ z1[:, k]) for k in range(K)])
    Lz = np.stack([np.linalg.cholesky(blocks[n]) @ z2[n] for n in range(N)])  # (N, K)
    part2 = kmajor(Lz)
    return part1 + part2, z1, z2


def perturbation_matrix(lat: Lattice, blocks, scale, prior="ugl"):
    """The linear map (z1, z2) -> perturbation as an explicit matrix (for the covariance pin:
    its Gram matrix must equal B~ exactly, which is why Algorithm 2 samples correctly)."""
    N, K, _ = blocks.shape
    G = lat.D().T if prior == "ltl" else lat.Gw()
    if prior == "aniso":
        d = lat.edges()[:, 2]
        part1 = sp.block_diag([(G.T @ sp.diags(np.sqrt(np.asarray(scale[k], dtype=np.float64)[d]))).tocsr()
                               for k in range(K)], format="csr")
    else:
        part1 = sp.block_diag([sp.csr_matrix(np.sqrt(scale[k]) * G.T) for k in range(K)], format="csr")
    H = H_perm(N, K)
    L = blkdiag([np.linalg.cholesky(blocks[n]) for n in range(N)])
    part2 = H.T @ L @ H          # z2 indexed regressor-major here
    return sp.hstack([part1, part2]).tocsr()


# ----------------------------------------------------------------------------------------
# Gamma full conditionals (Appendix A): Ga(scale, shape)
# ----------------------------------------------------------------------------------------

def lambda_params(rss, T, P, u1, u2):
    """Eq. fullcondTemplambda: 1/u~1n = 1/u1 + RSS_n / 2, u~2 = (T - P)/2 + u2."""
    return 1.0 / (1.0 / u1 + 0.5 * rss), (T - P) / 2.0 + u2


def quad_forms_edges(lat: Lattice, V):
    """Q_k = V_k D V_k' as the weighted sum over edges of squared differences
    (D = G'CG, Eq. 6-7 and the Discussion's WGL form)."""
    E = lat.edges()
    diff = V[:, E[:, 0]] - V[:, E[:, 1]]
    return (lat.edge_weights()[None, :] * diff * diff).sum(axis=1)


def quad_forms_dirs(lat: Lattice, V):
    """Q[k, d] = sum over the direction-d edges of C_e (V_k,i - V_k,j)^2 (K x 3): the
    statistics of the anisotropic prior's alpha_{d,k}."""
    E = lat.edges()
    diff = V[:, E[:, 0]] - V[:, E[:, 1]]
    q = lat.edge_weights()[None, :] * diff * diff
    return np.stack([q[:, E[:, 2] == d].sum(axis=1) for d in range(3)], axis=1)


def quad_forms_ltl(lat: Lattice, V):
    """Q_k = V_k L'L V_k' = |L V_k'|^2 for the L'L prior."""
    L = lat.D()
    return np.array([float(np.sum((L @ V[k]) ** 2)) for k in range(V.shape[0])])


def quad_forms_laplacian(lat: Lattice, V):
    D = lat.D()
    return np.array([V[k] @ (D @ V[k]) for k in range(V.shape[0])])


def alpha_params(Q, N, q1, q2):
    """Eq. fullcondTempa: 1/q~1k = Q_k / 2 + 1/q1, q~2 = N/2 + q2 (same for beta with r1, r2,
    Eq. fullcondTempbeta)."""
    return 1.0 / (0.5 * Q + 1.0 / q1), N / 2.0 + q2
