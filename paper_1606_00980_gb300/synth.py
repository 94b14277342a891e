"""Seeded synthetic fMRI workloads shaped like the paper's slice-wise and whole-brain data.

This module simulates data FROM the generative model of Section 2 (Y = XW + E with
per-voxel AR(P) noise, Appendix A "temporal noise model"); it contains none of the
inference arithmetic (no full conditionals, no solver, no sampler). Both the CUDA path
and the FP64 oracle consume its outputs; neither is imported here.

Recipe (Appendix D gives the paper's own simulation shapes; the named workloads below
follow it with the sizes of the benchmark configurations):

* TR = 2 s. Task regressors are boxcars convolved with a double-gamma canonical HRF
  (gamma densities with shapes 6 and 16, unit scale, undershoot ratio 1/6), each column
  scaled to unit peak; an intercept column follows, and optionally a linear drift.
* True W: Gaussian blobs (sigma 3 voxels, amplitude 2) for the task regressors,
  intercept 100 (the SPM scaling to mean 100), drift 0.5.
* Noise: stationary AR(P) with innovation precision lambda (sigma = 1 unless stated),
  100 burn-in samples before the first kept time point.
* Masks: a centred circle (2D) or ellipsoid (3D); the realised voxel count is reported.

All randomness comes from numpy's PCG64 seeded by the caller, so a (name, seed) pair is
a fixed dataset.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TR = 2.0


@dataclass
class Workload:
    name: str
    dims: tuple            # (nx, ny, nz)
    neighbourhood: int     # 4 (2D slices) or 6 (3D)
    mask: np.ndarray       # uint8, shape (nz, ny, nx), x fastest in memory
    X: np.ndarray          # (T, K) float64
    Y: np.ndarray          # (T, N) float64, column n = in-mask voxel n in raster order
    P: int
    W_true: np.ndarray     # (K, N)
    A_true: np.ndarray     # (P, N)
    lambda_true: np.ndarray  # (N,)
    eps: float = 0.0       # ridge folded into the per-voxel data block
    delta: float = 1e-8    # PCG relative-residual tolerance
    meta: dict = field(default_factory=dict)

    @property
    def N(self):
        return self.Y.shape[1]

    @property
    def T(self):
        return self.X.shape[0]

    @property
    def K(self):
        return self.X.shape[1]


def canonical_hrf(tr=TR, length=32.0, dt=0.1):
    """Double-gamma HRF sampled at resolution dt (peak ~5-6 s, undershoot ~16 s)."""
    t = np.arange(0.0, length, dt)
    g1 = t ** 5 * np.exp(-t) / math.gamma(6)
    g2 = t ** 15 * np.exp(-t) / math.gamma(16)
    h = g1 - g2 / 6.0
    return h / h.sum()


def _convolve_boxcar(onsets, durations, T, tr=TR, dt=0.1):
    n_fine = int(round(T * tr / dt))
    box = np.zeros(n_fine)
    for on, du in zip(onsets, durations):
        a = int(round(on / dt))
        b = min(n_fine, int(round((on + du) / dt)))
        box[a:b] = 1.0
    h = canonical_hrf(tr, dt=dt)
    conv = np.convolve(box, h)[:n_fine]
    step = int(round(tr / dt))
    col = conv[::step][:T]
    peak = np.abs(col).max()
    return col / peak if peak > 0 else col


def ellipsoid_mask(nx, ny, nz, ax, ay, az):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cx, cy, cz = (nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0
    r = ((x - cx) / ax) ** 2 + ((y - cy) / ay) ** 2 + ((z - cz) / az) ** 2
    return (r <= 1.0).astype(np.uint8)


def circle_mask(nx, ny, radius):
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    cx, cy = (nx - 1) / 2.0, (ny - 1) / 2.0
    m = ((x - cx) ** 2 + (y - cy) ** 2 <= radius ** 2).astype(np.uint8)
    return m[None, :, :]


def _blobs(mask, n_blobs, rng, sigma=3.0, amplitude=2.0):
    nz, ny, nx = mask.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    inside = np.argwhere(mask > 0)
    field_ = np.zeros(mask.shape)
    for _ in range(n_blobs):
        cz, cy, cx = inside[rng.integers(len(inside))]
        d2 = (x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2
        field_ += amplitude * np.exp(-0.5 * d2 / sigma ** 2)
    return field_[mask > 0]


def simulate_ar_noise(a, lam, T, rng, burn=100):
    """AR(P) noise per voxel: e_t = sum_p a_p e_{t-p} + eps_t, eps_t ~ N(0, 1/lambda)."""
    P, N = a.shape
    sd = 1.0 / np.sqrt(lam)
    total = T + burn
    e = np.zeros((total, N))
    innov = rng.standard_normal((total, N)) * sd[None, :]
    for t in range(total):
        v = innov[t].copy()
        for p in range(1, P + 1):
            if t - p >= 0:
                v += a[p - 1] * e[t - p]
        e[t] = v
    return e[burn:]


def make_design(T, n_task, rng, block_range=(10.0, 30.0), drift=False, phases=None):
    cols = []
    total_s = T * TR
    for j in range(n_task):
        if phases is not None:
            period, offset = phases[j]
            onsets = np.arange(offset, total_s, period)
            durs = np.full(len(onsets), period / 2.0)
        else:
            onsets, durs, tcur = [], [], rng.uniform(0, 20)
            while tcur < total_s:
                d = rng.uniform(*block_range)
                onsets.append(tcur)
                durs.append(d)
                tcur += d + rng.uniform(*block_range)
        cols.append(_convolve_boxcar(onsets, durs, T))
    cols.append(np.ones(T))
    if drift:
        cols.append(np.linspace(-1.0, 1.0, T))
    return np.stack(cols, axis=1)


def make_workload(name, dims, mask, T, K, P, neighbourhood, seed, ar_mean=None,
                  ar_jitter=0.05, ar_uniform=None, eps=0.0, delta=1e-8, drift=False,
                  phases=None, n_blobs=3):
    rng = np.random.default_rng(seed)
    n_task = K - 1 - (1 if drift else 0)
    X = make_design(T, n_task, rng, drift=drift, phases=phases)
    N = int(mask.sum())
    W = np.zeros((K, N))
    for k in range(n_task):
        W[k] = _blobs(mask, n_blobs, rng)
    W[n_task] = 100.0
    if drift:
        W[n_task + 1] = 0.5
    A = np.zeros((P, N))
    if P > 0:
        # sum_p |a_p| < 1 is sufficient for stationarity; redraw the rare failures.
        todo = np.arange(N)
        for _ in range(50):
            if ar_uniform is not None:
                cand = rng.uniform(*ar_uniform, size=(P, len(todo)))
            else:
                cand = np.asarray(ar_mean[:P])[:, None] + rng.uniform(
                    -ar_jitter, ar_jitter, size=(P, len(todo)))
            ok = np.abs(cand).sum(axis=0) < 0.98
            A[:, todo[ok]] = cand[:, ok]
            todo = todo[~ok]
            if len(todo) == 0:
                break
    lam = np.ones(N)
    E = simulate_ar_noise(A, lam, T, rng)
    Y = X @ W + E
    return Workload(name=name, dims=dims, neighbourhood=neighbourhood, mask=mask, X=X,
                    Y=np.ascontiguousarray(Y), P=P, W_true=W, A_true=A, lambda_true=lam,
                    eps=eps, delta=delta, meta={"seed": seed, "N": N})


def slice2d(seed=1):
    """2D slice: 32x32 lattice, circular mask (~800 voxels), T=200, K=3 (two boxcars at
    different phases plus intercept), AR(1) with phi ~ U(0.1, 0.4), 4-neighbour prior,
    ridge 1e-6, PCG tolerance 1e-10."""
    mask = circle_mask(32, 32, 16.0)
    return make_workload("slice2d_32x32_K3_P1", (32, 32, 1), mask, T=200, K=3, P=1,
                         neighbourhood=4, seed=seed, ar_uniform=(0.1, 0.4), eps=1e-6,
                         delta=1e-10, phases=[(40.0, 0.0), (40.0, 10.0)])


def wholebrain3d(seed=2, K=6, dims=(64, 64, 33), axes=(28.5, 28.5, 14.7), T=300):
    """3D whole brain: 64x64x33 lattice, ellipsoid mask (~50k voxels), T=300, K=6
    (4 HRF blocks with random onsets, intercept, linear drift), AR(3), 6-neighbour."""
    nx, ny, nz = dims
    mask = ellipsoid_mask(nx, ny, nz, *axes)
    return make_workload(f"wholebrain3d_{nx}x{ny}x{nz}_K{K}_P3", dims, mask, T=T, K=K,
                         P=3, neighbourhood=6, seed=seed, ar_mean=(0.3, 0.1, 0.05),
                         drift=True, n_blobs=6)


def batch3d(seed=4):
    """Batched workload lattice: 96x96x60, ellipsoid (~250k voxels), K=8, AR(3), T=300."""
    return wholebrain3d(seed=seed, K=8, dims=(96, 96, 60), axes=(45.7, 45.7, 28.6), T=300)


def small3d(seed=7, dims=(8, 8, 6), K=3, P=2, T=40, axes=None, neighbourhood=6):
    """A few hundred voxels in 3D: the parity-test size (spans several CTAs and a ragged tail)."""
    nx, ny, nz = dims
    if axes is None:
        axes = (nx / 2.0, ny / 2.0, nz / 2.0)
    mask = ellipsoid_mask(nx, ny, nz, *axes)
    drift = K >= 4
    return make_workload(f"small3d_{nx}x{ny}x{nz}_K{K}_P{P}", dims, mask, T=T, K=K, P=P,
                         neighbourhood=neighbourhood, seed=seed,
                         ar_mean=(0.3, 0.1, 0.05)[:max(P, 1)], drift=drift, n_blobs=2)


def request_workload(seed, N_target, K, T, P):
    """One serving request: an ellipsoid mask with ~N_target voxels, aspect like the
    whole-brain lattice (z semi-axis about half of x/y)."""
    # ellipsoid volume 4/3 pi a a (a/2) = N  ->  a = (3 N / (2 pi))^(1/3)
    a = (3.0 * N_target / (2.0 * math.pi)) ** (1.0 / 3.0)
    nx = ny = int(math.ceil(2 * a + 2))
    nz = int(math.ceil(a + 2))
    mask = ellipsoid_mask(nx, ny, nz, a, a, a / 2.0)
    drift = K >= 4
    return make_workload(f"request_N{int(mask.sum())}_K{K}_T{T}_P{P}", (nx, ny, nz), mask,
                         T=T, K=K, P=P, neighbourhood=6, seed=seed,
                         ar_mean=(0.3, 0.1, 0.05)[:P], drift=drift, n_blobs=4)


def zslab(w: Workload, z0: int, z1: int) -> Workload:
    """The sub-workload of the mask's slices z0 <= z < z1 (same data, fewer voxels): the
    bounded sample on which the CPU oracle is timed."""
    mask = w.mask.copy()
    mask[:z0] = 0
    mask[z1:] = 0
    keep = mask.reshape(-1)[np.flatnonzero(w.mask.reshape(-1))] > 0
    return Workload(name=f"{w.name}_z{z0}-{z1}", dims=w.dims, neighbourhood=w.neighbourhood,
                    mask=mask, X=w.X, Y=np.ascontiguousarray(w.Y[:, keep]), P=w.P,
                    W_true=w.W_true[:, keep], A_true=w.A_true[:, keep],
                    lambda_true=w.lambda_true[keep], eps=w.eps, delta=w.delta,
                    meta=dict(w.meta, N=int(keep.sum()), parent_N=w.N))


# ---------------------------------------------------------------------------------------
# The paper's simulation study (Appendix D): K = 5 (four task regressors and an intercept),
# P = 1, T = 351, a 53 x 63 x 46 block of which centred boxes of 10x10x10, 25x20x20 and
# 50x50x40 voxels (N = 1e3, 1e4, 1e5) are analysed. Intercepts ~ N(900, 130^2) i.i.d.,
# 1/lambda_n = 100, alpha = (1e-4, 5e-4, 2e-3, 1e-2) for the task rows of W, beta_1 = 10 for
# A; Y is scaled per voxel to mean 100 (the SPM default). Stand-ins, since the paper's
# inputs are not available: the task regressors are synthetic boxcar designs convolved with
# the canonical HRF (not the face-repetition paradigm), and the UGL-prior rows of W and A are
# drawn on the periodic block by spectral sampling (white noise filtered by 1/sqrt(alpha times
# the periodic lattice Laplacian's eigenvalues, mean mode removed)) instead of by the
# paper's PCG draw from a zero start.
# ---------------------------------------------------------------------------------------
PAPER_SIM_BOXES = {1000: (10, 10, 10), 10000: (25, 20, 20), 100000: (50, 50, 40)}
PAPER_SIM_BLOCK = (53, 63, 46)
PAPER_SIM_ALPHA = (1e-4, 5e-4, 2e-3, 1e-2)


def periodic_ugl_field(shape_zyx, prec, rng):
    """A zero-mean field on the periodic lattice with precision prec times its graph
    Laplacian (eigenvalues sum_d 2 (1 - cos w_d)); the constant mode is set to zero."""
    nz, ny, nx = shape_zyx
    white = rng.standard_normal(shape_zyx)
    wz = 2.0 * np.pi * np.fft.fftfreq(nz)[:, None, None]
    wy = 2.0 * np.pi * np.fft.fftfreq(ny)[None, :, None]
    wx = 2.0 * np.pi * np.fft.fftfreq(nx)[None, None, :]
    eig = 2.0 * ((1 - np.cos(wx)) + (1 - np.cos(wy)) + (1 - np.cos(wz)))
    filt = np.zeros_like(eig)
    filt[eig > 0] = 1.0 / np.sqrt(prec * eig[eig > 0])
    return np.real(np.fft.ifftn(np.fft.fftn(white) * filt))


def paper_simulation(N=1000, seed=11, T=351, prior_rows=None):
    """The paper's simulated dataset of N voxels (1e3, 1e4 or 1e5): a centred box of the
    53 x 63 x 46 block, analysed on that block's lattice.

    The four task rows of W (alpha = 1e-4, 5e-4, 2e-3, 1e-2) and the AR row (beta = 10) are
    fields on the whole block drawn from the UGL prior. prior_rows, if given, is a callable
    (block_xyz, alphas, beta, seed) -> (W_rows [4][nx*ny*nz], A_row [nx*ny*nz]) in raster
    order that draws them (the benchmark passes the library's PCG from a zero start with no
    data term, as the paper's simulation does); without it they are periodic spectral draws
    (periodic_ugl_field), which need no solver. The AR row is clipped to [-0.9, 0.9] so that
    every voxel's AR(1) noise is stationary."""
    if N not in PAPER_SIM_BOXES:
        raise ValueError(f"N must be one of {sorted(PAPER_SIM_BOXES)}")
    rng = np.random.default_rng(seed)
    nx, ny, nz = PAPER_SIM_BLOCK
    bx, by, bz = PAPER_SIM_BOXES[N]
    mask = np.zeros((nz, ny, nx), np.uint8)
    x0, y0, z0 = (nx - bx) // 2, (ny - by) // 2, (nz - bz) // 2
    mask[z0:z0 + bz, y0:y0 + by, x0:x0 + bx] = 1
    inside = mask.reshape(-1) > 0
    K, P = 5, 1
    X = make_design(T, K - 1, rng)
    W = np.zeros((K, N))
    if prior_rows is None:
        for k, a in enumerate(PAPER_SIM_ALPHA):
            W[k] = periodic_ugl_field((nz, ny, nx), a, rng).reshape(-1)[inside]
        a_row = periodic_ugl_field((nz, ny, nx), 10.0, rng).reshape(-1)
    else:
        w_rows, a_row = prior_rows((nx, ny, nz), PAPER_SIM_ALPHA, 10.0, seed)
        for k in range(len(PAPER_SIM_ALPHA)):
            W[k] = np.asarray(w_rows[k]).reshape(-1)[inside]
        a_row = np.asarray(a_row).reshape(-1)
    W[K - 1] = rng.normal(900.0, 130.0, N)
    A = np.clip(a_row[inside], -0.9, 0.9)[None, :]
    lam = np.full(N, 0.01)
    E = simulate_ar_noise(A, lam, T, rng)
    Y = X @ W + E
    Y = Y * (100.0 / Y.mean(axis=0))[None, :]
    return Workload(name=f"paper_sim_N{N}_K5_P1_T{T}", dims=(nx, ny, nz), neighbourhood=6,
                    mask=mask, X=X, Y=np.ascontiguousarray(Y), P=P, W_true=W, A_true=A,
                    lambda_true=lam, eps=0.0, delta=1e-8,
                    meta={"seed": seed, "N": N, "box": (bx, by, bz), "block": (nx, ny, nz),
                          "prior_rows": "spectral" if prior_rows is None else "caller"})
