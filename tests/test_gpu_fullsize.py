"""The benchmark's workloads at their full sizes, in the launch configurations bench.py times
(needs a GB300).

Whole-brain headline workload (64x64x33 ellipsoid, N = 49,928, K = 6, P = 3, T = 300; FP64,
the reduced red-black solver, delta = 1e-8, 152 CTAs of 352 threads with lane pairs for
the W solve): the statistics at 300 sampled voxels against the oracle's statistics of those
voxels' series (FP64 series and, through the tensor-core kernel, FP32 series); each step of
a sweep from one known state, every draw against the oracle's version of the same step. The
W and A draws are checked by a property that holds at any size, their residual in the
oracle's own perturbed system: the oracle builds B~ and b = b_mean + perturbation from the
state (an exact sparse solve at 300k unknowns is out of reach of a test), and the GPU draw
must solve it to delta plus what the blocks' assembly error allows.

Batched-probe workload (96x96x60 ellipsoid, N = 250,176, K = 8; 64 FP32 probes to 1e-5,
the right-hand-side tile the autotuner picks): a sampled probe's quadrature against the
oracle's Lanczos quadrature with the same number of steps (Lanczos and CG build the same
tridiagonal), within the FP32 storage's 1e-3.
"""
import numpy as np
import pytest

from oracle import gibbs, model, philox, probes
from oracle.lattice import Lattice
from paper_1606_00980_gb300 import synth

pytestmark = pytest.mark.gpu

SEED = 2024   # the headline chain's seed


def state_for(w, rng):
    return dict(W=w.W_true + 0.2 * rng.standard_normal((w.K, w.N)),
                A=w.A_true + 0.02 * rng.standard_normal((w.P, w.N)),
                lam=rng.uniform(0.5, 2.0, w.N), alpha=rng.uniform(0.2, 3.0, w.K),
                beta=rng.uniform(2.0, 20.0, w.P))


@pytest.fixture(scope="module")
def wholebrain():
    w = synth.wholebrain3d()
    return w, Lattice(w.mask, w.neighbourhood), state_for(w, np.random.default_rng(12))


def headline_model(w, Y=None):
    from paper_1606_00980_gb300 import bfmri
    from paper_1606_00980_gb300.bfmri import Model
    nx, ny, nz = w.dims
    return Model((nx, ny, nz, w.neighbourhood), w.mask, w.X, w.Y if Y is None else Y, w.K, w.P,
                 eps=w.eps, delta=1e-8, seed=SEED, stream_id=0, precond=bfmri.PRECOND_RB_REDUCED)


@pytest.mark.parametrize("series", ["f64", "f32"])
def test_wholebrain_statistics_at_sampled_voxels(wholebrain, series):
    w, lat, _ = wholebrain
    Y = w.Y if series == "f64" else w.Y.astype(np.float32)
    m = headline_model(w, Y)
    m.precompute_stats()
    got = m.get_stats()
    m.close()
    idx = np.random.default_rng(5).choice(w.N, 300, replace=False)
    st = model.sufficient_stats(np.asarray(Y[:, idx], dtype=np.float64), w.X, w.P)
    P = w.P
    iu = [(p, q) for p in range(P + 1) for q in range(p, P + 1)]
    ref = np.concatenate([np.stack([st["Syy"][:, p, q] for p, q in iu], axis=1),
                          st["Sxy"].reshape(len(idx), -1)], axis=1)
    assert np.max(np.abs(got[idx] - ref)) <= 1e-12 * np.abs(ref).max()


def residual_in_oracle_system(lat, blocks, bmean, scale, tag, counter, x):
    """||B~ x - b|| / ||b|| in the oracle's system with b = b_mean + the perturbation."""
    pert, _, _ = model.perturbation(lat, blocks, scale, SEED, counter, tag)
    b = model.kmajor(bmean) + pert
    B = model.precision(lat, blocks, scale)
    r = B @ x.reshape(-1) - b
    return np.linalg.norm(r) / np.linalg.norm(b), np.linalg.norm(b)


def test_wholebrain_steps_in_the_bench_configuration(wholebrain):
    w, lat, s = wholebrain
    m = headline_model(w)
    m.precompute_stats()
    m.set_state(W=s["W"], A=s["A"], lam=s["lam"], alpha=s["alpha"], beta=s["beta"])
    W, iw = m.sample_W(counter=5)
    m.set_state(W=s["W"])
    A, ia = m.sample_A(counter=5)
    m.set_state(A=s["A"])
    lam = m.sample_lambda(counter=5)
    alpha = m.sample_alpha(counter=5)
    beta = m.sample_beta(counter=5)
    m.close()
    assert iw.rel_residual <= 1e-8 and ia.rel_residual <= 1e-8
    # W: per-entry assembly error of the blocks at most 1e-12 of the largest block entry
    Bd, bw = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"], w.eps)
    res, nb = residual_in_oracle_system(lat, Bd, bw, s["alpha"], philox.TAG_W, 5, W)
    e = 1e-12 * np.abs(Bd).max()
    assert res <= 1e-8 + (w.K * e * np.linalg.norm(W) + 1e-12 * nb) / nb, res
    # A: blocks are differences of lagged y'y products, accurate to 1e-12 of the largest
    # lambda-weighted y'y sum (per entry, also for the right-hand side)
    Ja, ba = model.a_blocks_direct(w.Y, w.X, s["W"], s["lam"], w.P)
    res, nb = residual_in_oracle_system(lat, Ja, ba, s["beta"], philox.TAG_A, 5, A)
    st = model.sufficient_stats(w.Y, w.X, w.P)
    e = 1e-12 * (s["lam"] * st["Syy"][:, 0, 0]).max()
    assert res <= 1e-8 + (w.P * e * np.linalg.norm(A) + e * np.sqrt(w.P * w.N)) / nb, res
    # lambda, alpha, beta from the known state: closed-form Gamma parameters, same draws
    assert np.max(np.abs(lam / gibbs.sample_lambda(lat, w.Y, w.X, s, SEED, 5) - 1)) <= 1e-10
    assert np.max(np.abs(alpha / gibbs.sample_alpha(lat, s, SEED, 5) - 1)) <= 1e-10
    assert np.max(np.abs(beta / gibbs.sample_beta(lat, s, SEED, 5) - 1)) <= 1e-10


def test_batched_probes_in_the_bench_configuration():
    from paper_1606_00980_gb300 import bfmri
    from paper_1606_00980_gb300.bfmri import Model
    w = synth.batch3d()
    lat = Lattice(w.mask, w.neighbourhood)
    s = state_for(w, np.random.default_rng(13))
    m = Model.from_workload(w, delta=1e-5, precision=bfmri.PREC_MIXED, seed=4242)
    m.precompute_stats()
    m.set_state(W=s["W"], A=s["A"], lam=s["lam"], alpha=s["alpha"], beta=s["beta"])
    res = m.logdet_probe(0, 64, 3000, counter=2, traces=False)
    tile, _ = m.probe_tuning()
    m.close()
    assert tile in (1, 2, 4)
    Bd, _ = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"], w.eps)
    for i in (37,):
        v = philox.rademacher(4242, lat.lin * 4 + 3, w.K, 2, philox.TAG_PROBE, i)
        q = probes.probe_quadrature_m(lat, Bd, s["alpha"], v, int(res["iterations"][i]))
        assert abs(res["per_probe"][i] - q) <= 1e-3 * abs(q), (i, res["per_probe"][i], q)
