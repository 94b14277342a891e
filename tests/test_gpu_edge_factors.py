"""Per-edge weights of the spatial prior on the GPU (bfmri_set_edge_factors; needs a GB300).

The Discussion's weighted graph Laplacian puts a diagonal C between G_w' and G_w (Eq. 7);
with per-direction weights C has three values, here every edge has its own: the handle keeps
one BF16 factor per voxel and direction (the edge to the +d neighbour, stored at its lower
site) and multiplies it into the direction weight in the solvers' neighbour sums (resident
block-Jacobi and red-black reduced kernels with the voxel's slot weights in shared memory,
streaming block-Jacobi),
the block-Jacobi diagonal, the sqrt(C) G_w noise of Algorithm 2 and the alpha / beta edge
sums. Everything is checked against the oracle's lattice with the same factors (pinned in
tests/test_oracle_edge_factors.py) at the bars of the graph-Laplacian tests: B~ x 1e-13,
perturbed systems 1e-12, draws 1e-8 against the exact solve, alpha and beta 1e-10, a sweep
step by step; the captured sweep is bitwise the direct one. Factors that are not BF16 values
are rounded to the nearest one (ties to even), checked against PyTorch's own conversion.
"""
import numpy as np
import pytest

from block_bounds import apply_tolerance
from oracle import gibbs, model, philox
from oracle.lattice import Lattice
from paper_1606_00980_gb300 import synth

pytestmark = pytest.mark.gpu

SEED = 6262


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def state_for(w, rng):
    return dict(W=w.W_true + 0.2 * rng.standard_normal((w.K, w.N)),
                A=w.A_true + 0.02 * rng.standard_normal((w.P, w.N)),
                lam=rng.uniform(0.5, 2.0, w.N), alpha=rng.uniform(0.2, 3.0, w.K),
                beta=rng.uniform(2.0, 20.0, w.P))


def bf16_factors(w, seed):
    """BF16-representable positive factors k / 16, k = 4 .. 40, shape (3, nz, ny, nx)."""
    nx, ny, nz = w.dims
    return np.random.default_rng(seed).integers(4, 41, size=(3, nz, ny, nx)) / 16.0


CASES = {
    "small3d_K3_P2": (synth.small3d(seed=91, dims=(9, 8, 6), K=3, P=2, T=40), (1.0, 1.0, 1.0)),
    "weighted3d_K4_P1": (synth.small3d(seed=92, dims=(8, 7, 6), K=4, P=1, T=40), (2.0, 0.5, 3.25)),
    "slice2d_K3_P1": (synth.make_workload("slice", (15, 13, 1), synth.circle_mask(15, 13, 6.1),
                                          T=40, K=3, P=1, neighbourhood=4, seed=93,
                                          ar_uniform=(0.1, 0.4), eps=1e-6), (1.0, 1.0, 1.0)),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    w, cw = CASES[request.param]
    f = bf16_factors(w, 94)
    lat = Lattice(w.mask, w.neighbourhood, weights=cw, edge_factors=f)
    return w, cw, f, lat, state_for(w, np.random.default_rng(95))


def make(w, cw, f, state, **opts):
    from paper_1606_00980_gb300.bfmri import Model
    opts.setdefault("delta", 1e-12)
    opts.setdefault("precond", 1)
    m = Model.from_workload(w, seed=SEED, edge_weight=cw, **opts)
    m.set_edge_factors(f)
    m.precompute_stats()
    m.set_state(W=state["W"], A=state["A"], lam=state["lam"], alpha=state["alpha"],
                beta=state["beta"])
    return m


def test_precision_and_perturbed_systems(case):
    w, cw, f, lat, s = case
    m = make(w, cw, f, s)
    x = np.random.default_rng(1).standard_normal((w.K, w.N))
    y = m.apply_precision(0, x)
    _, _, bpert = m.build_system(0, counter=21)
    xa = np.random.default_rng(2).standard_normal((w.P, w.N))
    ya = m.apply_precision(1, xa)
    _, _, apert = m.build_system(1, counter=22)
    m.close()
    Bd, bw = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"], w.eps)
    B = model.precision(lat, Bd, s["alpha"])
    assert rel(y, (B @ x.reshape(-1)).reshape(w.K, w.N)) <= 1e-13
    pert, _, _ = model.perturbation(lat, Bd, s["alpha"], SEED, 21, philox.TAG_W)
    assert rel(bpert, (model.kmajor(bw) + pert).reshape(bpert.shape)) <= 1e-12
    Ja, ba = model.a_blocks_direct(w.Y, w.X, s["W"], s["lam"], w.P)
    # the A blocks are differences of lagged y'y products that cancel to the residual scale:
    # bound their error by the summands' size, as the graph-Laplacian parity tests do
    st = model.sufficient_stats(w.Y, w.X, w.P)
    yy = (s["lam"] * st["Syy"][:, 0, 0]).max()
    Ba = model.precision(lat, Ja, s["beta"])
    ref = (Ba @ xa.reshape(-1)).reshape(w.P, w.N)
    assert np.max(np.abs(ya - ref)) <= 1e-12 * yy * np.abs(xa).max() * w.P + 1e-13 * np.abs(ref).max()
    pa, _, _ = model.perturbation(lat, Ja, s["beta"], SEED, 22, philox.TAG_A)
    ref = (model.kmajor(ba) + pa).reshape(apert.shape)
    assert np.max(np.abs(apert - ref)) <= 1e-12 * yy + 1e-12 * np.abs(ref).max()


def test_block_jacobi_apply_uses_the_weighted_degree(case):
    w, cw, f, lat, s = case
    m = make(w, cw, f, s)
    x = np.random.default_rng(3).standard_normal((w.K, w.N))
    got = m.apply_preconditioner(0, x)
    m.close()
    Bd, _ = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"], w.eps)
    deg = lat.degree()
    Mb = Bd + s["alpha"][None, :, None] * np.eye(w.K)[None] * deg[:, None, None]
    ref = np.stack([np.linalg.solve(Mb[n], x[:, n]) for n in range(w.N)], axis=1)
    assert rel(got, ref) <= apply_tolerance(Bd, 1e-12 * np.abs(Bd).max())


@pytest.mark.parametrize("variant", ["auto", "streaming"])
@pytest.mark.parametrize("precond", ["none", "bj", "reduced"])
def test_draws_and_precisions(case, precond, variant):
    """The register-resident kernels (auto at these sizes: block-Jacobi, or CG on the red-black
    reduced system) and the streaming kernel (block-Jacobi on the same blocks for both), with
    and without a preconditioner."""
    from paper_1606_00980_gb300 import bfmri
    w, cw, f, lat, s = case
    pc = dict(none=bfmri.PRECOND_NONE, bj=bfmri.PRECOND_BLOCK_JACOBI, reduced=bfmri.PRECOND_RB_REDUCED)
    m = make(w, cw, f, s, precond=pc[precond],
             pcg_variant=bfmri.PCG_AUTO if variant == "auto" else bfmri.PCG_STREAMING)
    W, iw = m.sample_W(counter=3)
    m.set_state(W=s["W"])
    A, ia = m.sample_A(counter=3)
    m.set_state(A=s["A"])
    alpha = m.sample_alpha(counter=4)
    beta = m.sample_beta(counter=4)
    m.close()
    assert iw.rel_residual <= 1e-12 and ia.rel_residual <= 1e-12
    assert rel(W, gibbs.sample_W(lat, w.Y, w.X, s, SEED, 3, w.eps)) <= 1e-8
    assert rel(A, gibbs.sample_A(lat, w.Y, w.X, s, SEED, 3, spatial=True)) <= 1e-8
    assert np.max(np.abs(alpha / gibbs.sample_alpha(lat, s, SEED, 4) - 1)) <= 1e-10
    assert np.max(np.abs(beta / gibbs.sample_beta(lat, s, SEED, 4) - 1)) <= 1e-10


@pytest.mark.parametrize("precond", ["bj", "reduced"])
def test_sweep_step_by_step_and_captured(case, precond):
    from paper_1606_00980_gb300 import bfmri
    w, cw, f, lat, s = case
    pc = bfmri.PRECOND_BLOCK_JACOBI if precond == "bj" else bfmri.PRECOND_RB_REDUCED
    m = make(w, cw, f, s, precond=pc)
    m.gibbs_sweep(1, first_counter=9)
    g = m.get_state()
    m.close()
    assert rel(g["W"], gibbs.sample_W(lat, w.Y, w.X, s, SEED, 9, w.eps)) <= 1e-8
    s1 = dict(s, W=g["W"])
    assert rel(g["A"], gibbs.sample_A(lat, w.Y, w.X, s1, SEED, 9, spatial=True)) <= 1e-8
    s1["A"] = g["A"]
    assert np.max(np.abs(g["lam"] / gibbs.sample_lambda(lat, w.Y, w.X, s1, SEED, 9) - 1)) <= 1e-10
    s1["lam"] = g["lam"]
    assert np.max(np.abs(g["alpha"] / gibbs.sample_alpha(lat, s1, SEED, 9) - 1)) <= 1e-10
    assert np.max(np.abs(g["beta"] / gibbs.sample_beta(lat, s1, SEED, 9) - 1)) <= 1e-10
    runs = []
    for graph in (0, 1):
        mm = make(w, cw, f, s, use_graph=graph, delta=1e-10, precond=pc)
        mm.gibbs_sweep(3, first_counter=12)
        runs.append(mm.get_state())
        mm.close()
    for k in runs[0]:
        assert np.array_equal(runs[0][k], runs[1][k]), k


def test_factors_round_to_bf16_and_clear():
    torch = pytest.importorskip("torch")
    w, cw = CASES["weighted3d_K4_P1"]
    s = state_for(w, np.random.default_rng(96))
    nx, ny, nz = w.dims
    f = np.random.default_rng(97).uniform(0.3, 3.0, size=(3, nz, ny, nx)).astype(np.float32)
    fr = torch.from_numpy(f).to(torch.bfloat16).to(torch.float64).numpy()
    assert not np.array_equal(fr, f.astype(np.float64))
    m = make(w, cw, f, s)
    x = np.random.default_rng(4).standard_normal((w.K, w.N))
    y = m.apply_precision(0, x)
    m.set_edge_factors(None)
    y0 = m.apply_precision(0, x)
    m.close()
    Bd, _ = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"], w.eps)
    B = model.precision(Lattice(w.mask, w.neighbourhood, weights=cw, edge_factors=fr), Bd, s["alpha"])
    assert rel(y, (B @ x.reshape(-1)).reshape(w.K, w.N)) <= 1e-13
    B0 = model.precision(Lattice(w.mask, w.neighbourhood, weights=cw), Bd, s["alpha"])
    assert rel(y0, (B0 @ x.reshape(-1)).reshape(w.K, w.N)) <= 1e-13


def test_options_values_and_calls_that_do_not_take_factors():
    from paper_1606_00980_gb300 import bfmri
    from paper_1606_00980_gb300.bfmri import Model, gibbs_sweep_group
    w, cw = CASES["small3d_K3_P2"]
    f = bf16_factors(w, 98)
    for bad in (dict(precond=bfmri.PRECOND_SSOR), dict(precond=bfmri.PRECOND_MULTIGRID),
                dict(precision=bfmri.PREC_MIXED), dict(w_prior=bfmri.PRIOR_LTL)):
        m = Model.from_workload(w, **bad)
        with pytest.raises(bfmri.BfmriError) as ei:
            m.set_edge_factors(f)
        assert ei.value.status == -1
        m.close()
    s = state_for(w, np.random.default_rng(99))
    m = Model.from_workload(w, precond=1)
    z, y, x = np.argwhere(np.asarray(w.mask).reshape(f.shape[1:]) != 0)[0]
    for v in (0.0, -1.0, np.nan, np.inf):
        g = f.copy()
        g[1, z, y, x] = v
        with pytest.raises(bfmri.BfmriError) as ei:
            m.set_edge_factors(g)
        assert ei.value.status == -1
    m.close()
    ms = [make(w, cw, f, s), make(w, cw, f, s)]
    with pytest.raises(bfmri.BfmriError):
        gibbs_sweep_group(ms, 1, 0)
    with pytest.raises(bfmri.BfmriError):
        ms[0].logdet_probe(0, 4, 100, counter=1)
    with pytest.raises(bfmri.BfmriError):
        ms[0].spvb_step(4, 1)
    for m in ms:
        m.close()
    mr = make(w, cw, f, s, precond=bfmri.PRECOND_RB_REDUCED)
    with pytest.raises(bfmri.BfmriError):
        mr.apply_preconditioner(0, np.ones((w.K, w.N)))
    mr.close()


def test_log_joint_with_factors_matches_the_oracle():
    """Eq. UnnormalisedJointPosterior with per-edge factors: the W and A prior terms take the
    factors in their edge sums (their pseudo-determinant is a constant of the sampled
    parameters), at the summaries' bar of 1e-10 of the terms' size, from a known state and
    after two sweeps."""
    from oracle import summaries
    w, cw = CASES["small3d_K3_P2"]
    f = bf16_factors(w, 101)
    lat = Lattice(w.mask, w.neighbourhood, weights=cw, edge_factors=f)
    s = state_for(w, np.random.default_rng(102))
    m = make(w, cw, f, s)
    for sweep in range(3):
        if sweep:
            m.gibbs_sweep(1, sweep)
        got = m.log_joint()
        st = m.get_state()
        ref = summaries.log_joint(lat, w.Y, w.X, st, w.T)
        scale = sum(abs(ref[k]) for k in ("loglik", "W_prior", "A_prior", "lambda_prior",
                                           "alpha_prior", "beta_prior"))
        for key in ref:
            assert abs(got[key] - ref[key]) <= 1e-10 * scale, (key, got[key], ref[key])
    m.close()
