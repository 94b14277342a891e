"""The L'L prior of W on the GPU (options.w_prior = PRIOR_LTL; needs a GB300).

D_w = L'L with L the (weighted) graph Laplacian: Section 2 names it as the alternative to the
graph-Laplacian default. Its 25-point stencil (13 in 2D) reaches the neighbours' neighbours;
the GPU forms every product as t = L v over all voxels, a grid barrier, then L t, and the
Algorithm 2 perturbation's prior part as sqrt(alpha_k) L z1_k with one normal per voxel.
Everything is checked against the oracle's L'L prior (pinned in tests/test_oracle_ltl.py) at
the bars of the graph-Laplacian tests: B~ x 1e-13, perturbed systems 1e-12, the block-Jacobi
apply within the blocks' assembly bound, draws 1e-8 against the exact solve, alpha 1e-10, a
whole sweep step by step, on 3D and 2D lattices and with edge weights; the captured sweep is
bitwise the direct one.
"""
import numpy as np
import pytest

from block_bounds import apply_tolerance
from oracle import gibbs, model, philox, probes
from oracle.lattice import Lattice
from paper_1606_00980_gb300 import synth

pytestmark = pytest.mark.gpu

SEED = 5151


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def state_for(w, rng):
    return dict(W=w.W_true + 0.2 * rng.standard_normal((w.K, w.N)),
                A=w.A_true + 0.02 * rng.standard_normal((w.P, w.N)),
                lam=rng.uniform(0.5, 2.0, w.N), alpha=rng.uniform(0.2, 3.0, w.K),
                beta=rng.uniform(2.0, 20.0, w.P))


CASES = {
    "small3d_K3_P2": (synth.small3d(seed=81, dims=(9, 8, 6), K=3, P=2, T=40), (1.0, 1.0, 1.0)),
    "weighted3d_K4_P1": (synth.small3d(seed=82, dims=(8, 7, 6), K=4, P=1, T=40), (2.0, 0.5, 3.25)),
    "slice2d_K3_P1": (synth.make_workload("slice", (15, 13, 1), synth.circle_mask(15, 13, 6.1),
                                          T=40, K=3, P=1, neighbourhood=4, seed=83,
                                          ar_uniform=(0.1, 0.4), eps=1e-6), (1.0, 1.0, 1.0)),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    w, cw = CASES[request.param]
    lat = Lattice(w.mask, w.neighbourhood, weights=cw)
    return w, cw, lat, state_for(w, np.random.default_rng(90))


def make(w, cw, state, **opts):
    from paper_1606_00980_gb300 import bfmri
    from paper_1606_00980_gb300.bfmri import Model
    opts.setdefault("delta", 1e-12)
    m = Model.from_workload(w, seed=SEED, edge_weight=cw, w_prior=bfmri.PRIOR_LTL, **opts)
    m.precompute_stats()
    m.set_state(W=state["W"], A=state["A"], lam=state["lam"], alpha=state["alpha"],
                beta=state["beta"])
    return m


def test_precision_and_perturbed_system(case):
    w, cw, lat, s = case
    m = make(w, cw, s)
    x = np.random.default_rng(1).standard_normal((w.K, w.N))
    y = m.apply_precision(0, x)
    blocks, bmean, bpert = m.build_system(0, counter=21)
    m.close()
    Bd, bw = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"], w.eps)
    B = model.precision(lat, Bd, s["alpha"], "ltl")
    assert rel(y, (B @ x.reshape(-1)).reshape(w.K, w.N)) <= 1e-13
    pert, _, _ = model.perturbation(lat, Bd, s["alpha"], SEED, 21, philox.TAG_W, 0, "ltl")
    assert rel(bpert, (model.kmajor(bw) + pert).reshape(bpert.shape)) <= 1e-12


def test_block_jacobi_apply(case):
    w, cw, lat, s = case
    m = make(w, cw, s)
    x = np.random.default_rng(2).standard_normal((w.K, w.N))
    got = m.apply_preconditioner(0, x)
    m.close()
    Bd, _ = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"], w.eps)
    dl = model.prior_precision(lat, "ltl").diagonal()
    Mb = Bd + s["alpha"][None, :, None] * np.eye(w.K)[None] * dl[:, None, None]
    ref = np.stack([np.linalg.solve(Mb[n], x[:, n]) for n in range(w.N)], axis=1)
    assert rel(got, ref) <= apply_tolerance(Bd, 1e-12 * np.abs(Bd).max())


@pytest.mark.parametrize("variant", ["auto", "streaming"])
@pytest.mark.parametrize("precond", [0, 1])
def test_w_draw_and_alpha(case, precond, variant):
    """The register-resident block-Jacobi kernel (auto at these sizes: t = L v published, a grid
    barrier, then L t) and the streaming two-pass kernel, with and without block-Jacobi."""
    from paper_1606_00980_gb300 import bfmri
    w, cw, lat, s = case
    m = make(w, cw, s, precond=precond,
             pcg_variant=bfmri.PCG_AUTO if variant == "auto" else bfmri.PCG_STREAMING)
    W, info = m.sample_W(counter=3)
    m.set_state(W=s["W"])
    alpha = m.sample_alpha(counter=4)
    m.close()
    assert info.rel_residual <= 1e-12
    assert rel(W, gibbs.sample_W(lat, w.Y, w.X, s, SEED, 3, w.eps, prior="ltl")) <= 1e-8
    ref = gibbs.sample_alpha(lat, s, SEED, 4, prior="ltl")
    assert np.max(np.abs(alpha / ref - 1)) <= 1e-10


def test_sweep_step_by_step_and_captured(case):
    w, cw, lat, s = case
    m = make(w, cw, s)
    m.gibbs_sweep(1, first_counter=9)
    g = m.get_state()
    m.close()
    assert rel(g["W"], gibbs.sample_W(lat, w.Y, w.X, s, SEED, 9, w.eps, prior="ltl")) <= 1e-8
    s1 = dict(s, W=g["W"])
    # the A prior stays the graph Laplacian
    assert rel(g["A"], gibbs.sample_A(Lattice(w.mask, w.neighbourhood, weights=cw), w.Y, w.X, s1,
                                      SEED, 9, spatial=True)) <= 1e-8
    s1["A"] = g["A"]
    assert np.max(np.abs(g["lam"] / gibbs.sample_lambda(lat, w.Y, w.X, s1, SEED, 9) - 1)) <= 1e-10
    s1["lam"] = g["lam"]
    assert np.max(np.abs(g["alpha"] / gibbs.sample_alpha(lat, s1, SEED, 9, prior="ltl") - 1)) <= 1e-10
    assert np.max(np.abs(g["beta"] / gibbs.sample_beta(lat, s1, SEED, 9) - 1)) <= 1e-10
    runs = []
    for graph in (0, 1):
        mm = make(w, cw, s, use_graph=graph, delta=1e-10)
        mm.gibbs_sweep(3, first_counter=12)
        runs.append(mm.get_state())
        mm.close()
    for k in runs[0]:
        assert np.array_equal(runs[0][k], runs[1][k]), k


def test_options_and_calls_that_do_not_take_the_ltl_prior():
    from paper_1606_00980_gb300 import bfmri
    from paper_1606_00980_gb300.bfmri import Model, gibbs_sweep_group
    w, cw = CASES["small3d_K3_P2"]
    for bad in (dict(precond=bfmri.PRECOND_SSOR), dict(precond=bfmri.PRECOND_RB_REDUCED),
                dict(precision=bfmri.PREC_MIXED)):
        with pytest.raises(bfmri.BfmriError) as ei:
            Model.from_workload(w, w_prior=bfmri.PRIOR_LTL, **bad)
        assert ei.value.status == -1
    s = state_for(w, np.random.default_rng(91))
    ms = [make(w, cw, s), make(w, cw, s)]
    with pytest.raises(bfmri.BfmriError):
        gibbs_sweep_group(ms, 1, 0)
    with pytest.raises(bfmri.BfmriError):
        ms[0].logdet_probe(0, 4, 100, counter=1)
    with pytest.raises(bfmri.BfmriError):
        ms[0].spvb_step(4, 1)
    for m in ms:
        m.close()


def test_log_joint_matches_the_oracle(case):
    """Eq. UnnormalisedJointPosterior under the L'L prior (W prior term with |L w_k|^2, the A
    prior the graph Laplacian) at the summaries' bar of 1e-10 of the terms' size, from a known
    state and after two sweeps."""
    from oracle import summaries
    w, cw, lat, s = case
    m = make(w, cw, s)
    for sweep in range(3):
        if sweep:
            m.gibbs_sweep(1, sweep)
        got = m.log_joint()
        st = m.get_state()
        ref = summaries.log_joint(lat, w.Y, w.X, st, w.T, prior="ltl")
        scale = sum(abs(ref[k]) for k in ("loglik", "W_prior", "A_prior", "lambda_prior",
                                           "alpha_prior", "beta_prior"))
        for key in ref:
            assert abs(got[key] - ref[key]) <= 1e-10 * scale, (key, got[key], ref[key])
    m.close()
