"""The weighted graph-Laplacian (WGL) prior on the GPU (needs a GB300).

With options.edge_weight = (c_x, c_y, c_z), the prior precision is alpha_k G_w' C G_w
(Discussion; C the weight of each edge's direction) and Algorithm 2 scales every edge's noise
by sqrt(C). Everything built on the prior is checked against the oracle's weighted lattice at
the same bars as the UGL tests: systems and perturbations 1e-12, B~ x 1e-13, draws 1e-8
(every preconditioner and solver variant, FP64 and mixed), lambda / alpha / beta 1e-10, SVB
samples 1e-8, grouped chains 1e-8, log-det probes against the exact terms.
"""
import numpy as np
import pytest

from oracle import gibbs, model, philox, probes
from oracle.lattice import Lattice
from paper_1606_00980_gb300 import synth

pytestmark = pytest.mark.gpu

SEED = 4711
WEIGHTS = (2.0, 0.5, 3.25)


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def state_for(w, rng):
    return dict(W=w.W_true + 0.2 * rng.standard_normal((w.K, w.N)),
                A=w.A_true + 0.02 * rng.standard_normal((w.P, w.N)),
                lam=rng.uniform(0.5, 2.0, w.N), alpha=rng.uniform(0.2, 3.0, w.K),
                beta=rng.uniform(2.0, 20.0, w.P))


def make(w, state=None, **opts):
    from paper_1606_00980_gb300.bfmri import Model
    opts.setdefault("delta", 1e-12)
    opts.setdefault("seed", SEED)
    m = Model.from_workload(w, edge_weight=WEIGHTS, **opts)
    m.precompute_stats()
    if state is not None:
        m.set_state(W=state["W"], A=state["A"], lam=state["lam"], alpha=state["alpha"],
                    beta=state["beta"] if w.P > 0 else None)
    return m


WL = {
    "slab_K6_P3": synth.small3d(seed=61, dims=(13, 11, 7), K=6, P=3, T=60),
    "small3d_K3_P2": synth.small3d(seed=62, dims=(9, 8, 6), K=3, P=2, T=40),
    "slice2d_K3_P1": synth.make_workload("slice", (17, 15, 1), synth.circle_mask(17, 15, 7.3),
                                         T=50, K=3, P=1, neighbourhood=4, seed=63,
                                         ar_uniform=(0.1, 0.4), eps=1e-6),
}


@pytest.fixture(scope="module", params=sorted(WL))
def case(request):
    w = WL[request.param]
    lat = Lattice(w.mask, w.neighbourhood, weights=WEIGHTS)
    return w, lat, state_for(w, np.random.default_rng(5))


def test_system_perturbation_and_precision(case):
    w, lat, s = case
    m = make(w, s)
    blocks, bmean, bpert = m.build_system(0, counter=21)
    Bd, bw = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"], w.eps)
    pert, _, _ = model.perturbation(lat, Bd, s["alpha"], SEED, 21, philox.TAG_W)
    ref = (model.kmajor(bw) + pert).reshape(bpert.shape)
    assert rel(bpert, ref) <= 1e-12
    x = np.random.default_rng(7).standard_normal((w.K, w.N))
    y = m.apply_precision(0, x)
    B = model.precision(lat, Bd, s["alpha"])
    assert rel(y, (B @ x.reshape(-1)).reshape(w.K, w.N)) <= 1e-13
    m.close()


@pytest.mark.parametrize("precond", [1, 2, 3])
@pytest.mark.parametrize("variant", ["auto", "streaming"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_draws_match_exact_solve(case, precond, variant, precision):
    from paper_1606_00980_gb300 import bfmri
    w, lat, s = case
    m = make(w, s, precond=precond,
             pcg_variant=bfmri.PCG_AUTO if variant == "auto" else bfmri.PCG_STREAMING,
             precision=bfmri.PREC_FP64 if precision == "fp64" else bfmri.PREC_MIXED)
    W, info = m.sample_W(counter=3)
    Bd, bw = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"], w.eps)
    ref, _ = gibbs.draw_gmrf(lat, Bd, bw, s["alpha"], SEED, 3, philox.TAG_W)
    assert info.rel_residual <= 1e-12
    assert rel(W, ref) <= 1e-8
    if w.P > 0:
        A, ia = m.sample_A(counter=4)
        Ar = gibbs.sample_A(lat, w.Y, w.X, dict(s, W=W), SEED, 4, spatial=True)
        assert rel(A, Ar) <= 1e-8
    m.close()


def test_gibbs_sweep_single_step_parity(case):
    w, lat, s = case
    m = make(w, s, precond=3)
    m.gibbs_sweep(1, first_counter=9)
    g = m.get_state()
    assert rel(g["W"], gibbs.sample_W(lat, w.Y, w.X, s, SEED, 9, w.eps)) <= 1e-8
    s1 = dict(s, W=g["W"])
    if w.P > 0:
        assert rel(g["A"], gibbs.sample_A(lat, w.Y, w.X, s1, SEED, 9, spatial=True)) <= 1e-8
        s1["A"] = g["A"]
    lr = gibbs.sample_lambda(lat, w.Y, w.X, s1, SEED, 9)
    assert np.max(np.abs(g["lam"] / lr - 1)) <= 1e-10
    ar = gibbs.sample_alpha(lat, s1, SEED, 9)
    assert np.max(np.abs(g["alpha"] / ar - 1)) <= 1e-10
    if w.P > 0:
        br = gibbs.sample_beta(lat, s1, SEED, 9)
        assert np.max(np.abs(g["beta"] / br - 1)) <= 1e-10
    m.close()


@pytest.mark.parametrize("precond", [1, 3])
def test_grouped_chains_and_svb(case, precond):
    from paper_1606_00980_gb300.bfmri import gibbs_sweep_group
    w, lat, s = case
    seeds = [SEED, SEED + 1]
    ms = [make(w, s, seed=sd, precond=precond) for sd in seeds]
    gibbs_sweep_group(ms, 1, first_counter=9)
    for m, sd in zip(ms, seeds):
        assert rel(m.get_state()["W"], gibbs.sample_W(lat, w.Y, w.X, s, sd, 9, w.eps)) <= 1e-8
        m.close()
    m = make(w, s, precond=precond)
    Ns, c = 3, 11
    m.spvb_step(Ns, c, extrapolate=False)
    Bd, bw = gibbs.svb_w_system(w.Y, w.X, [s["A"]] * Ns, s["lam"], w.eps)
    Wo = gibbs.svb_draw(lat, Bd, bw, s["alpha"], SEED, c, philox.TAG_W, Ns)
    for j in range(Ns):
        assert rel(m.svb_sample(j)[0], Wo[j]) <= 1e-8
    m.close()


def test_logdet_probe_matches_exact_terms(case):
    w, lat, s = case
    m = make(w, s, precond=1)
    res = m.logdet_probe(0, 8, 2000, counter=6)
    Bd, _ = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"], w.eps)
    V = probes.probe_vectors(lat, w.K, 8, SEED, 6)
    ldm, quad, tr, ldb = probes.exact_probe_terms(lat, Bd, s["alpha"], V)
    assert np.max(np.abs(res["per_probe"] - quad) / np.abs(quad)) <= 1e-6
    assert np.allclose(res["traces"], tr.mean(axis=0), rtol=1e-8, atol=1e-8 * np.abs(tr).mean())
    m.close()


def test_unit_weights_are_the_ugl_prior_bitwise():
    """edge_weight = (1, 1, 1) reproduces the UGL handle bit for bit."""
    from paper_1606_00980_gb300.bfmri import Model
    w = WL["small3d_K3_P2"]
    a = Model.from_workload(w, seed=3, delta=1e-10, precond=3)
    b = Model.from_workload(w, seed=3, delta=1e-10, precond=3, edge_weight=(1.0, 1.0, 1.0))
    for m in (a, b):
        m.precompute_stats()
        m.gibbs_sweep(3, 0)
    sa, sb = a.get_state(), b.get_state()
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k
    a.close()
    b.close()
