"""Pins of the oracle's prior and of Algorithm 2 against closed forms (CPU only).

* With no data (B_data = eps I, eps -> 0) the UGL prior makes the increments of W_k along the
  edges of a tree independent with variance 1/alpha_k (Section 3.1, Eq. 6-7: G_w has full row
  rank on a tree, so G (G'G)^+ G' = I). On any graph the weighted increments sum to
  E[sum_e c_e (w_i - w_j)^2] = (N - #components) / alpha_k, the rank of the Laplacian, which
  is the expectation that the alpha full conditional's quadratic form Q_k is built on.
* Algorithm 1 (mean plus the Cholesky factor's back-substitution of fresh normals) and
  Algorithm 2 (perturbation + solve) draw from the same Gaussian: two-sample tests on
  projections of the two sets of draws.
"""
import numpy as np
import pytest
import scipy.sparse.csgraph as csg
import scipy.stats as ss

from oracle import gibbs, model, philox
from oracle.lattice import Lattice

EPS = 1e-9


def no_data_blocks(N, K):
    return np.broadcast_to(EPS * np.eye(K), (N, K, K)).copy()


def increment_covariance(lat, alpha, k):
    """Exact covariance of the edge increments (w_i - w_j) of component k under B~ with
    B_data = eps I: G_k-rows of the dense inverse of the oracle's precision."""
    K = len(alpha)
    B = model.precision(lat, no_data_blocks(lat.N, K), alpha).toarray()
    Sig = np.linalg.inv(B)[k * lat.N:(k + 1) * lat.N, k * lat.N:(k + 1) * lat.N]
    G = lat.G().toarray()
    return G @ Sig @ G.T


def test_increments_on_a_path_are_independent_with_variance_one_over_alpha():
    mask = np.ones((1, 1, 12), np.uint8)          # 12 voxels in a row: a path graph
    lat = Lattice(mask, 4)
    alpha = np.array([0.4, 2.5])
    for k in range(2):
        C = increment_covariance(lat, alpha, k)
        assert C.shape == (11, 11)
        assert np.allclose(C, np.eye(11) / alpha[k], rtol=0, atol=1e-6 / alpha[k])


@pytest.mark.parametrize("nb,weights", [(4, (1.0, 1.0, 1.0)), (6, (1.0, 1.0, 1.0)),
                                        (6, (2.0, 0.5, 3.25))])
def test_expected_weighted_edge_sum_is_rank_over_alpha(nb, weights):
    """sum_e c_e Var(w_i - w_j) = tr(C^(1/2) G Sigma G' C^(1/2)) -> (N - #components)/alpha,
    checked on a mask with a hole and a detached voxel (two connected components)."""
    if nb == 4:
        mask = np.ones((1, 5, 6), np.uint8)    # mask[z, y, x]
        mask[0, 2, 2] = mask[0, 2, 3] = 0      # a hole
        mask[0, 4, 4] = mask[0, 3, 5] = 0      # voxel (x=5, y=4) loses both neighbours
    else:
        mask = np.ones((3, 4, 4), np.uint8)
        mask[1, 1, 1] = mask[1, 2, 2] = 0      # holes
        mask[2, 3, 2] = mask[2, 2, 3] = mask[1, 3, 3] = 0   # voxel (3, 3, 2) is detached
    lat = Lattice(mask, nb, weights=weights)
    E = lat.edges()
    ncomp = csg.connected_components(abs(lat.D()) > 0, directed=False)[0]
    assert ncomp == 2
    alpha = np.array([0.7, 3.0])
    K = 2
    B = model.precision(lat, no_data_blocks(lat.N, K), alpha).toarray()
    Sig = np.linalg.inv(B)
    Gw = lat.Gw().toarray()
    for k in range(K):
        S = Sig[k * lat.N:(k + 1) * lat.N, k * lat.N:(k + 1) * lat.N]
        tr = np.trace(Gw @ S @ Gw.T)
        assert abs(tr * alpha[k] - (lat.N - ncomp)) <= 1e-6 * lat.N
    assert len(E) > 0


def test_prior_draws_have_the_expected_quadratic_form():
    """Monte Carlo through the oracle's Algorithm 2 draw with no data: the mean of
    Q_k = sum_e (w_i - w_j)^2 over draws is (N - 1)/alpha_k on a connected 4x4 slice, within
    5 standard errors (Q_k alpha_k is chi-square with N - 1 degrees of freedom as eps -> 0)."""
    mask = np.ones((1, 4, 4), np.uint8)
    lat = Lattice(mask, 4)
    alpha = np.array([0.5, 4.0])
    K, N = 2, lat.N
    blocks = no_data_blocks(N, K)
    zero = np.zeros((N, K))
    n = 400
    Q = np.empty((n, K))
    for c in range(n):
        w, _ = gibbs.draw_gmrf(lat, blocks, zero, alpha, 31, c, philox.TAG_W)
        Q[c] = model.quad_forms_edges(lat, w)
    dof = N - 1
    for k in range(K):
        m = Q[:, k].mean() * alpha[k]
        assert abs(m - dof) < 5 * np.sqrt(2.0 * dof / n)
        # and the full distribution: alpha Q is chi-square(N - 1)
        assert ss.kstest(Q[:, k] * alpha[k], ss.chi2(dof).cdf).pvalue > 1e-4


def test_algorithm_1_and_algorithm_2_draw_from_the_same_gaussian():
    """Algorithm 1: w = mu + L'^-1 z with B~ = L L' (dense Cholesky, numpy normals).
    Algorithm 2: the oracle's perturbation + exact solve (Philox normals). Two-sample KS on
    three fixed projections and on the squared Mahalanobis norm, plus matching means."""
    mask = np.ones((1, 3, 3), np.uint8)
    lat = Lattice(mask, 4)
    K, N = 2, lat.N
    rng = np.random.default_rng(8)
    G = rng.standard_normal((N, K, K))
    blocks = np.einsum("nij,nkj->nik", G, G) + 0.3 * np.eye(K)[None]
    rhs = rng.standard_normal((N, K))
    alpha = np.array([0.8, 1.7])
    B = model.precision(lat, blocks, alpha).toarray()
    mu = np.linalg.solve(B, model.kmajor(rhs))
    L = np.linalg.cholesky(B)
    n = 1500
    Z = rng.standard_normal((K * N, n))
    X1 = mu[:, None] + np.linalg.solve(L.T, Z)                      # Algorithm 1
    X2 = np.stack([gibbs.draw_gmrf(lat, blocks, rhs, alpha, 77, c, philox.TAG_W)[0].reshape(-1)
                   for c in range(n)], axis=1)                       # Algorithm 2
    P = rng.standard_normal((3, K * N))
    for p in P:
        assert ss.ks_2samp(p @ X1, p @ X2).pvalue > 1e-4
    m1 = np.einsum("in,ij,jn->n", X1 - mu[:, None], B, X1 - mu[:, None])
    m2 = np.einsum("in,ij,jn->n", X2 - mu[:, None], B, X2 - mu[:, None])
    assert ss.ks_2samp(m1, m2).pvalue > 1e-4
    assert ss.kstest(m2, ss.chi2(K * N).cdf).pvalue > 1e-4
    sd = np.sqrt(np.diag(np.linalg.inv(B)))
    assert np.all(np.abs(X2.mean(axis=1) - mu) < 5 * sd / np.sqrt(n))
