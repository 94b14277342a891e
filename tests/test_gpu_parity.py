"""GPU path vs the FP64 oracle, element by element, through the C ABI (needs a GB300).

Tolerances (FP64 path): statistics, blocks and right-hand sides 1e-12 relative (same
arithmetic, different summation order); B~ x 1e-13; a W or A draw 1e-8 relative L2 against
the oracle's exact solve of the same perturbed system (PCG stopped at relative residual
1e-12, so the error is below kappa * 1e-12); lambda, alpha, beta 1e-10 relative.
"""
import numpy as np
import pytest

from oracle import gibbs, model, philox
from oracle.lattice import Lattice
from paper_1606_00980_gb300 import synth

pytestmark = pytest.mark.gpu

SEED = 1234


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def random_state(w, rng):
    N, K, P = w.N, w.K, w.P
    return dict(W=w.W_true + 0.2 * rng.standard_normal((K, N)),
                A=w.A_true + 0.02 * rng.standard_normal((P, N)),
                lam=rng.uniform(0.5, 2.0, N), alpha=rng.uniform(0.2, 3.0, K),
                beta=rng.uniform(2.0, 20.0, P))


def make(w, state=None, **opts):
    from paper_1606_00980_gb300.bfmri import Model
    opts.setdefault("delta", 1e-12)
    opts.setdefault("seed", SEED)
    m = Model.from_workload(w, **opts)
    m.precompute_stats()
    if state is not None:
        m.set_state(W=state["W"], A=state["A"], lam=state["lam"], alpha=state["alpha"],
                    beta=state["beta"] if w.P > 0 else None)
    return m


def workloads():
    holes = synth.ellipsoid_mask(9, 8, 6, 4.5, 4.0, 3.0)
    holes[3, 4, 4] = 0
    holes[2, 3, 2] = 0
    holes[0, :, :] = 0
    holes[5, 4, 4] = 1          # an isolated voxel on the top slice
    return {
        "small3d_K3_P2": synth.small3d(seed=11, dims=(8, 8, 6), K=3, P=2, T=40),
        "slab_K6_P3": synth.small3d(seed=12, dims=(13, 11, 7), K=6, P=3, T=60),
        "slice2d_K3_P1": synth.make_workload("slice", (17, 15, 1), synth.circle_mask(17, 15, 7.3),
                                             T=50, K=3, P=1, neighbourhood=4, seed=13,
                                             ar_uniform=(0.1, 0.4), eps=1e-6),
        "holes_K4_P1": synth.make_workload("holes", (9, 8, 6), holes, T=45, K=4, P=1,
                                           neighbourhood=6, seed=14, ar_mean=(0.3,), drift=True),
        "P0_K2": synth.make_workload("p0", (6, 5, 4), np.ones((4, 5, 6), np.uint8), T=30, K=2,
                                     P=0, neighbourhood=6, seed=15),
        "K10_P2": synth.small3d(seed=16, dims=(9, 8, 6), K=10, P=2, T=70),
    }


WL = workloads()


@pytest.fixture(scope="module", params=sorted(WL))
def case(request):
    w = WL[request.param]
    lat = Lattice(w.mask, w.neighbourhood)
    st = model.sufficient_stats(w.Y, w.X, w.P)
    state = random_state(w, np.random.default_rng(5))
    return w, lat, st, state


def test_stats(case):
    w, lat, st, _ = case
    m = make(w)
    got = m.get_stats()
    P, K = w.P, w.K
    iu = [(p, q) for p in range(P + 1) for q in range(p, P + 1)]
    ref = np.concatenate([np.stack([st["Syy"][:, p, q] for p, q in iu], axis=1),
                          st["Sxy"].reshape(w.N, -1)], axis=1)
    scale = np.abs(ref).max()
    assert np.max(np.abs(got - ref)) <= 1e-12 * scale
    m.close()


@pytest.mark.parametrize("which", [0, 1])
def test_system_and_perturbation(case, which):
    w, lat, st, s = case
    if which == 1 and w.P == 0:
        pytest.skip("no AR part")
    m = make(w, s)
    blocks, bmean, bpert = m.build_system(which, counter=21)
    if which == 0:
        Bd, bw = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"], w.eps)
        scale, tag = s["alpha"], philox.TAG_W
    else:
        Bd, bw = model.a_blocks_direct(w.Y, w.X, s["W"], s["lam"], w.P)
        scale, tag = s["beta"], philox.TAG_A
    if which == 0:
        tol_b, tol_r = 1e-12 * np.abs(Bd).max(), 1e-12 * np.abs(bw).max()
    else:
        # the A system is a difference of lagged y'y products (~T * 100^2 for fMRI-scaled
        # data) that cancel to the residual scale; bound the error by the summands' size
        yy = (s["lam"] * st["Syy"][:, 0, 0]).max()
        tol_b = tol_r = 1e-12 * yy
    assert np.max(np.abs(blocks - Bd)) <= tol_b
    assert np.max(np.abs(bmean - bw.T)) <= tol_r
    pert, _, _ = model.perturbation(lat, Bd, scale, SEED, 21, tag)
    ref = (model.kmajor(bw) + pert).reshape(bpert.shape)
    if which == 0:
        assert rel(bpert, ref) <= 1e-12
    else:
        assert np.max(np.abs(bpert - ref)) <= tol_r + 1e-12 * np.abs(ref).max()
    m.close()


@pytest.mark.parametrize("which", [0, 1])
def test_apply_precision(case, which):
    w, lat, st, s = case
    if which == 1 and w.P == 0:
        pytest.skip("no AR part")
    m = make(w, s)
    D = w.K if which == 0 else w.P
    x = np.random.default_rng(7).standard_normal((D, w.N))
    y = m.apply_precision(which, x)
    if which == 0:
        Bd, _ = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"], w.eps)
        B = model.precision(lat, Bd, s["alpha"])
    else:
        Bd, _ = model.a_blocks_direct(w.Y, w.X, s["W"], s["lam"], w.P)
        B = model.precision(lat, Bd, s["beta"])
    ref = (B @ x.reshape(-1)).reshape(D, w.N)
    if which == 0:
        assert rel(y, ref) <= 1e-13
    else:
        # cancellation-limited blocks (see test_system_and_perturbation)
        yy = (s["lam"] * st["Syy"][:, 0, 0]).max()
        assert np.max(np.abs(y - ref)) <= 1e-12 * yy * np.abs(x).max() * D + 1e-13 * np.abs(ref).max()
    m.close()


@pytest.mark.parametrize("variant", ["auto", "streaming"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sample_W_matches_exact_solve(case, variant, precision):
    """Both solver variants (register-resident and streaming) and both precisions reach the
    oracle's exact draw: FP64 and FP32-inner/FP64-refined solves to relative residual 1e-12."""
    from paper_1606_00980_gb300 import bfmri
    w, lat, st, s = case
    m = make(w, s, pcg_variant=bfmri.PCG_AUTO if variant == "auto" else bfmri.PCG_STREAMING,
             precision=bfmri.PREC_FP64 if precision == "fp64" else bfmri.PREC_MIXED)
    W, info = m.sample_W(counter=3)
    Bd, bw = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"], w.eps)
    ref, mu = gibbs.draw_gmrf(lat, Bd, bw, s["alpha"], SEED, 3, philox.TAG_W)
    assert info.rel_residual <= 1e-12
    assert rel(W, ref) <= 1e-8
    assert rel(W, mu) > 1e-4          # it is a draw, not the mean
    if precision == "mixed":
        assert info.refinements >= 1
    m.close()


def test_mixed_precision_at_delta_1e8(case):
    """Mixed precision stopped at the paper's delta = 1e-8: the draw is within 1e-5 (relative
    L2) of the FP64 oracle's exact draw."""
    from paper_1606_00980_gb300 import bfmri
    w, lat, st, s = case
    m = make(w, s, precision=bfmri.PREC_MIXED, delta=1e-8)
    W, info = m.sample_W(counter=8)
    Bd, bw = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"], w.eps)
    ref, _ = gibbs.draw_gmrf(lat, Bd, bw, s["alpha"], SEED, 8, philox.TAG_W)
    assert info.rel_residual <= 1e-8
    assert rel(W, ref) <= 1e-5
    m.close()


@pytest.mark.parametrize("spatial,variant", [(True, "auto"), (True, "streaming"), (False, "auto")])
def test_sample_A_matches_exact_solve(case, spatial, variant):
    w, lat, st, s = case
    if w.P == 0:
        pytest.skip("no AR part")
    from paper_1606_00980_gb300 import bfmri
    m = make(w, s, ar_prior=bfmri.AR_SPATIAL if spatial else bfmri.AR_INDEPENDENT,
             pcg_variant=bfmri.PCG_AUTO if variant == "auto" else bfmri.PCG_STREAMING)
    A, info = m.sample_A(counter=4)
    ref = gibbs.sample_A(lat, w.Y, w.X, s, SEED, 4, spatial=spatial)
    assert rel(A, ref) <= 1e-8
    m.close()


def test_sample_lambda_alpha_beta(case):
    w, lat, st, s = case
    m = make(w, s)
    lam = m.sample_lambda(counter=5)
    ref = gibbs.sample_lambda(lat, w.Y, w.X, s, SEED, 5)
    assert np.max(np.abs(lam / ref - 1)) <= 1e-10
    alpha = m.sample_alpha(counter=6)
    ref = gibbs.sample_alpha(lat, s, SEED, 6)
    assert np.max(np.abs(alpha / ref - 1)) <= 1e-10
    if w.P > 0:
        beta = m.sample_beta(counter=7)
        ref = gibbs.sample_beta(lat, s, SEED, 7)
        assert np.max(np.abs(beta / ref - 1)) <= 1e-10
    m.close()


def test_gibbs_sweep_single_step_parity(case):
    """One GPU sweep from a given state; the oracle replays each step from the GPU's own
    outputs of the previous steps (W -> A -> lambda -> alpha -> beta)."""
    w, lat, st, s = case
    m = make(w, s)
    info = m.gibbs_sweep(1, first_counter=9)
    g = m.get_state()
    Wr = gibbs.sample_W(lat, w.Y, w.X, s, SEED, 9, w.eps)
    assert rel(g["W"], Wr) <= 1e-8
    s1 = dict(s, W=g["W"])
    if w.P > 0:
        Ar = gibbs.sample_A(lat, w.Y, w.X, s1, SEED, 9, spatial=True)
        assert rel(g["A"], Ar) <= 1e-8
        s1["A"] = g["A"]
    lr = gibbs.sample_lambda(lat, w.Y, w.X, s1, SEED, 9)
    assert np.max(np.abs(g["lam"] / lr - 1)) <= 1e-10
    ar = gibbs.sample_alpha(lat, s1, SEED, 9)
    assert np.max(np.abs(g["alpha"] / ar - 1)) <= 1e-10
    if w.P > 0:
        br = gibbs.sample_beta(lat, s1, SEED, 9)
        assert np.max(np.abs(g["beta"] / br - 1)) <= 1e-10
    assert info.pcg_iterations_W > 0
    m.close()


@pytest.mark.parametrize("T,K,P", [(7, 1, 4), (8, 2, 4), (9, 3, 3)])
def test_stats_short_and_boundary_series(T, K, P):
    """Series shorter than 2P take the direct summation; T = 2P and T = 2P + 1 have an empty
    or one-step common window in the lag-difference form (all boundary terms)."""
    w = synth.make_workload("short", (5, 4, 3), np.ones((3, 4, 5), np.uint8), T=T, K=K, P=P,
                            neighbourhood=6, seed=17 + T, ar_uniform=(0.05, 0.2))
    m = make(w)
    got = m.get_stats()
    st = model.sufficient_stats(w.Y, w.X, P)
    iu = [(p, q) for p in range(P + 1) for q in range(p, P + 1)]
    ref = np.concatenate([np.stack([st["Syy"][:, p, q] for p, q in iu], axis=1),
                          st["Sxy"].reshape(w.N, -1)], axis=1)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.abs(ref).max()
    m.close()


def test_stats_from_float32_series():
    """Single-precision Y (the serving input format): statistics equal the FP64 oracle's for
    the same rounded values."""
    w = WL["slab_K6_P3"]
    from paper_1606_00980_gb300.bfmri import Model
    Y32 = w.Y.astype(np.float32)
    nx, ny, nz = w.dims
    m = Model((nx, ny, nz, w.neighbourhood), w.mask, w.X, Y32, w.K, w.P, seed=SEED)
    m.precompute_stats()
    got = m.get_stats()
    st = model.sufficient_stats(Y32.astype(np.float64), w.X, w.P)
    iu = [(p, q) for p in range(w.P + 1) for q in range(p, w.P + 1)]
    ref = np.concatenate([np.stack([st["Syy"][:, p, q] for p, q in iu], axis=1),
                          st["Sxy"].reshape(w.N, -1)], axis=1)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.abs(ref).max()
    m.close()


def test_sweeps_are_bitwise_reproducible():
    w = WL["slab_K6_P3"]
    outs = []
    for _ in range(2):
        m = make(w, delta=1e-10)
        m.gibbs_sweep(3, first_counter=100)
        outs.append(m.get_state())
        m.close()
    for k in outs[0]:
        assert np.array_equal(outs[0][k], outs[1][k])


@pytest.mark.parametrize("precision,lanes", [("fp64", 2), ("fp64", 1), ("mixed", 0)])
def test_reduced_red_black_solver_matches_exact_solve(case, precision, lanes):
    """PRECOND_RB_REDUCED on every parity workload (isolated voxels, holes, 2D slices, P = 0,
    K = 10): the pipelined reduced-system solvers where they apply (resident, D <= 6; FP64
    with lane pairs or one lane per voxel), the unpipelined ones for larger blocks, SSOR
    (omega = 1) in the streaming fallback; W and A draws reach the oracle's exact solve."""
    from paper_1606_00980_gb300 import bfmri
    w, lat, st, s = case
    m = make(w, s, precond=bfmri.PRECOND_RB_REDUCED, pcg_lanes=lanes,
             precision=bfmri.PREC_FP64 if precision == "fp64" else bfmri.PREC_MIXED)
    W, info = m.sample_W(counter=3)
    Bd, bw = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"], w.eps)
    ref, _ = gibbs.draw_gmrf(lat, Bd, bw, s["alpha"], SEED, 3, philox.TAG_W)
    assert info.rel_residual <= 1e-12
    assert rel(W, ref) <= 1e-8
    if w.P > 0:
        A, ia = m.sample_A(counter=4)
        Ar = gibbs.sample_A(lat, w.Y, w.X, dict(s, W=W), SEED, 4, spatial=True)
        assert ia.rel_residual <= 1e-12
        assert rel(A, Ar) <= 1e-8
    m.close()
