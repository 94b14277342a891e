"""Sufficient statistics of FP32 series on the tensor cores against the FP64 oracle (needs a
GB300).

The tensor-core kernel forms the common-window lagged products sum_s y_s x_{s+d,k} as exact
BF16 digit products (Appendix A's pre-computed sums; Ozaki-style splitting), the rest in
FP64. Each case compares it element by element with the oracle's statistics of the same
FP32-rounded series (1e-12 of the largest statistic, and 1e-12 of the largest Sxy for the
Sxy block alone) and with the FP64 CUDA-core kernel. The cases cover K = 1..12 (one and two
column groups of eight), P = 0..3, series shorter than one 16-step chunk and longer than one
512-step accumulation window, ragged voxel tiles, and series whose values span many powers
of two within one voxel.
"""
import numpy as np
import pytest

from oracle import model
from paper_1606_00980_gb300 import synth

pytestmark = pytest.mark.gpu


def ref_record(Y, X, P):
    st = model.sufficient_stats(np.asarray(Y, np.float64), X, P)
    iu = [(p, q) for p in range(P + 1) for q in range(p, P + 1)]
    syy = np.stack([st["Syy"][:, p, q] for p, q in iu], axis=1)
    return np.concatenate([syy, st["Sxy"].reshape(Y.shape[1], -1)], axis=1), syy.shape[1]


def stats_of(w, Y32, kernel):
    from paper_1606_00980_gb300.bfmri import Model
    nx, ny, nz = w.dims
    m = Model((nx, ny, nz, w.neighbourhood), w.mask, w.X, Y32, w.K, w.P, stats_kernel=kernel)
    m.precompute_stats()
    out = m.get_stats()
    m.close()
    return out


CASES = [  # (K, P, T, dims)
    (1, 0, 12, (5, 4, 3)),
    (3, 1, 40, (9, 8, 6)),
    (4, 2, 37, (11, 9, 7)),
    (6, 3, 300, (13, 11, 7)),
    (8, 3, 150, (12, 10, 6)),
    (9, 1, 60, (8, 7, 5)),
    (10, 3, 600, (10, 9, 6)),
    (12, 2, 560, (9, 7, 5)),
    (5, 3, 20, (7, 6, 4)),
]


@pytest.mark.parametrize("K,P,T,dims", CASES)
def test_tensor_core_stats_match_oracle(K, P, T, dims):
    from paper_1606_00980_gb300 import bfmri
    w = synth.small3d(seed=100 + K * 7 + P, dims=dims, K=K, P=P, T=T)
    Y32 = w.Y.astype(np.float32)
    ref, nsyy = ref_record(Y32, w.X, P)
    got = stats_of(w, Y32, bfmri.STATS_TENSOR)
    fp64 = stats_of(w, Y32, bfmri.STATS_FP64)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.abs(ref).max()
    sx, sx_ref = got[:, nsyy:], ref[:, nsyy:]
    assert np.max(np.abs(sx - sx_ref)) <= 1e-12 * np.abs(sx_ref).max()
    assert np.max(np.abs(got - fp64)) <= 2e-12 * np.abs(ref).max()


def test_tensor_core_stats_wide_dynamic_range():
    """Zero-mean series with rare spikes a million times larger: the small values sit 20
    binary orders below their voxel's largest value and are still represented exactly."""
    from paper_1606_00980_gb300 import bfmri
    w = synth.small3d(seed=5, dims=(10, 9, 6), K=6, P=3, T=200)
    rng = np.random.default_rng(3)
    Y = rng.standard_normal(w.Y.shape)
    spikes = rng.random(Y.shape) < 0.01
    Y[spikes] *= 1e6
    Y32 = Y.astype(np.float32)
    ref, nsyy = ref_record(Y32, w.X, w.P)
    got = stats_of(w, Y32, bfmri.STATS_TENSOR)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.abs(ref).max()
    # per voxel, against that voxel's own scale
    scale = np.abs(ref).max(axis=1, keepdims=True)
    assert np.max(np.abs(got - ref) / scale) <= 1e-11


def test_tensor_core_stats_reject_unsupported_shapes():
    from paper_1606_00980_gb300 import bfmri
    from paper_1606_00980_gb300.bfmri import Model
    w = synth.make_workload("p4", (6, 5, 4), np.ones((4, 5, 6), np.uint8), T=40, K=3, P=4,
                            neighbourhood=6, seed=6, ar_uniform=(0.02, 0.1))
    nx, ny, nz = w.dims
    m = Model((nx, ny, nz, w.neighbourhood), w.mask, w.X, w.Y.astype(np.float32), w.K, w.P,
              stats_kernel=bfmri.STATS_TENSOR)
    with pytest.raises(bfmri.BfmriError) as ei:
        m.precompute_stats()
    assert ei.value.status == -1
    m.close()
    w2 = synth.small3d(seed=7, dims=(6, 5, 4), K=3, P=2, T=40)
    m = Model((nx, ny, nz, w2.neighbourhood), w2.mask, w2.X, w2.Y, w2.K, w2.P,
              stats_kernel=bfmri.STATS_TENSOR)       # FP64 series
    with pytest.raises(bfmri.BfmriError):
        m.precompute_stats()
    m.close()


def test_serving_stats_shape_sampled():
    """The largest serving shape's statistics (T = 600, K = 10, P = 3) on 20k voxels with the
    voxel count not a multiple of the 128-voxel tile: a sample of voxels against the oracle."""
    from paper_1606_00980_gb300 import bfmri
    w = synth.request_workload(seed=9, N_target=20000, K=10, T=600, P=3)
    Y32 = w.Y.astype(np.float32)
    assert w.N % 128 != 0
    got = stats_of(w, Y32, bfmri.STATS_TENSOR)
    pick = np.random.default_rng(1).choice(w.N, 300, replace=False)
    pick = np.concatenate([pick, [w.N - 1, w.N - 2, 0]])
    ref, _ = ref_record(Y32[:, pick], w.X, w.P)
    assert np.max(np.abs(got[pick] - ref)) <= 1e-12 * np.abs(ref).max()
