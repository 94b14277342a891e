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


@pytest.mark.parametrize("precond", ["bj", "reduced"])
def test_wholebrain_anisotropic_prior_steps(wholebrain, precond):
    """The anisotropic prior on the whole-brain workload in the configurations the bench's
    prior_variants leg times (the register-resident block-Jacobi and reduced red-black
    kernels, delta 1e-8): the W
    draw's residual in the oracle's anisotropic system; for the alpha step the direction edge
    sums of W (1e-12), lam against the oracle's Gamma draw from those sums (1e-10), the
    proposal, the auxiliary field's residual in the oracle's L(theta') system (delta), its
    edge sums (1e-12), log a from the oracle's formula (1e-9 of its terms' size) and the
    decision wherever |log u - log a| exceeds that."""
    from paper_1606_00980_gb300 import bfmri
    from paper_1606_00980_gb300.bfmri import Model
    w, lat, s = wholebrain
    theta = np.random.default_rng(14).uniform(0.5, 3.0, (w.K, 3))
    nx, ny, nz = w.dims
    m = Model((nx, ny, nz, w.neighbourhood), w.mask, w.X, w.Y, w.K, w.P, eps=w.eps, delta=1e-8,
              seed=SEED, w_prior=bfmri.PRIOR_ANISO,
              precond=bfmri.PRECOND_BLOCK_JACOBI if precond == "bj" else bfmri.PRECOND_RB_REDUCED)
    m.precompute_stats()
    m.set_state(W=s["W"], A=s["A"], lam=s["lam"], beta=s["beta"])
    m.set_alpha_dirs(theta)
    W, iw = m.sample_W(counter=5)
    m.set_state(W=s["W"])
    m.sample_alpha(counter=6)
    a3, _ = m.get_alpha_dirs()
    ls = m.aniso_last_step()
    m.close()
    assert iw.rel_residual <= 1e-8
    Bd, bw = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"], w.eps)
    pert, _, _ = model.perturbation(lat, Bd, theta, SEED, 5, philox.TAG_W, 0, "aniso")
    b = model.kmajor(bw) + pert
    r = model.precision(lat, Bd, theta, "aniso") @ W.reshape(-1) - b
    nb = np.linalg.norm(b)
    e = 1e-12 * np.abs(Bd).max()
    assert np.linalg.norm(r) / nb <= 1e-8 + (w.K * e * np.linalg.norm(W) + 1e-12 * nb) / nb
    # the alpha step from (W, theta)
    Q = model.quad_forms_dirs(lat, s["W"])
    assert rel_max(ls["Q"], Q) <= 1e-12
    shape, rate = gibbs.scale_move_params(theta, Q, w.N, gibbs.n_parts(lat), 3)
    lam, _ = philox.gamma(SEED, np.arange(w.K), shape, 1.0 / rate, 6, philox.TAG_ALPHA, 0)
    assert np.max(np.abs(ls["lam"] / lam - 1)) <= 1e-10
    scaled = theta * ls["lam"][:, None]
    step = 1.0 / np.sqrt(w.N)
    eps = philox.normals(SEED, np.arange(w.K), 3, 6, philox.TAG_ALPHA_PROP, 0)
    prop = scaled * np.exp(step * eps)
    E = lat.edges()
    z = philox.normals(SEED, lat.lin[E[:, 0]] * 4 + E[:, 2], w.K, 6, philox.TAG_ALPHA_AUX, 0)
    Ls = model.direction_laplacians(lat)
    for k in range(w.K):
        bk = gibbs.aux_rhs(lat, prop[k], z[:, k])
        rk = sum(prop[k, d] * (Ls[d] @ ls["w_aux"][k]) for d in range(3)) - bk
        # delta, plus the proposal's difference from the GPU's (a common factor within lam's
        # 1e-10, which moves the residual by 1.5e-10 of |b|)
        assert np.linalg.norm(rk) <= (1e-8 + 1e-9) * np.linalg.norm(bk), k
    Qp = model.quad_forms_dirs(lat, ls["w_aux"])
    assert rel_max(ls["Q_aux"], Qp) <= 1e-12
    la = gibbs.exchange_log_ratio(scaled, prop, Q, Qp, step * eps, 3)
    size = np.sum(np.abs(0.5 * (prop - scaled) * (Q + Qp)), axis=1) + 1.0
    assert np.all(np.abs(ls["log_a"] - la) <= 1e-9 * size)
    u = philox.uniform_open(SEED, np.arange(w.K), 2, 6, philox.TAG_ALPHA_PROP, 0)
    for k in range(w.K):
        if abs(np.log(u[k]) - la[k]) > 1e-9 * size[k]:
            ref = prop[k] if np.log(u[k]) < la[k] else scaled[k]
            assert np.allclose(a3[k], ref, rtol=1e-10, atol=0), k


def rel_max(a, b):
    return np.max(np.abs(np.asarray(a) - b)) / np.max(np.abs(b))


def test_wholebrain_per_edge_factors_in_the_reduced_solver(wholebrain):
    """Per-edge BF16 factors on the whole-brain workload with the resident reduced solver (the
    bench's prior_variants configuration, delta 1e-8): the W draw's residual in the oracle's
    system on the lattice with the same factors, and alpha against the oracle's Gamma draw."""
    from paper_1606_00980_gb300 import bfmri
    w, _, s = wholebrain
    nx, ny, nz = w.dims
    f = np.random.default_rng(15).integers(8, 25, size=(3, nz, ny, nx)) / 16.0
    lat = Lattice(w.mask, w.neighbourhood, edge_factors=f)
    m = headline_model(w)
    m.set_edge_factors(f)
    m.precompute_stats()
    m.set_state(W=s["W"], A=s["A"], lam=s["lam"], alpha=s["alpha"], beta=s["beta"])
    W, iw = m.sample_W(counter=5)
    m.set_state(W=s["W"])
    alpha = m.sample_alpha(counter=5)
    m.close()
    assert iw.rel_residual <= 1e-8
    Bd, bw = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"], w.eps)
    res, nb = residual_in_oracle_system(lat, Bd, bw, s["alpha"], philox.TAG_W, 5, W)
    e = 1e-12 * np.abs(Bd).max()
    assert res <= 1e-8 + (w.K * e * np.linalg.norm(W) + 1e-12 * nb) / nb, res
    assert np.max(np.abs(alpha / gibbs.sample_alpha(lat, s, SEED, 5) - 1)) <= 1e-10
