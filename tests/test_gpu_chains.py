"""Independent chains advanced together (bfmri_gibbs_sweep_group): each chain's W and A
systems are solved by one multi-RHS launch with a matrix per chain. Per chain, one sweep
is checked step by step against the FP64 oracle replaying the chain's own outputs (the same
bar as the single-chain sweep: draws 1e-8 relative L2 against the exact solve of the same
perturbed system, lambda/alpha/beta 1e-10), and the grouped chains are checked against the
same chains advanced alone (same random numbers; the two solvers stop at the same relative
residual, so the states agree to the solver tolerance). Needs a GB300.
"""
import numpy as np
import pytest

from oracle import gibbs, model
from oracle.lattice import Lattice
from paper_1606_00980_gb300 import synth

pytestmark = pytest.mark.gpu

SEEDS = [101, 202, 303]


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def state_for(w, rng):
    N, K, P = w.N, w.K, w.P
    return dict(W=w.W_true + 0.2 * rng.standard_normal((K, N)),
                A=w.A_true + 0.02 * rng.standard_normal((P, N)),
                lam=rng.uniform(0.5, 2.0, N), alpha=rng.uniform(0.2, 3.0, K),
                beta=rng.uniform(2.0, 20.0, P))


def make(w, seed, state, **opts):
    from paper_1606_00980_gb300.bfmri import Model
    opts.setdefault("delta", 1e-12)
    m = Model.from_workload(w, seed=seed, **opts)
    m.precompute_stats()
    m.set_state(W=state["W"], A=state["A"], lam=state["lam"], alpha=state["alpha"],
                beta=state["beta"] if w.P > 0 else None)
    return m


WL = {
    "small3d_K3_P2": synth.small3d(seed=21, dims=(9, 8, 6), K=3, P=2, T=40),
    "slab_K6_P3": synth.small3d(seed=22, dims=(13, 11, 7), K=6, P=3, T=60),
    "P0_K2": synth.make_workload("p0", (6, 5, 4), np.ones((4, 5, 6), np.uint8), T=30, K=2,
                                 P=0, neighbourhood=6, seed=23),
}


# block-Jacobi, red-black SSOR and the red-black reduced system in the multi-RHS solves
PRECONDS = {"bj": dict(), "ssor": dict(precond=2), "ssor_w1.3": dict(precond=2, ssor_omega=1.3),
            "reduced": dict(precond=3)}


@pytest.mark.parametrize("pc", sorted(PRECONDS))
@pytest.mark.parametrize("name", sorted(WL))
def test_group_sweep_matches_oracle_per_chain(name, pc):
    from paper_1606_00980_gb300.bfmri import gibbs_sweep_group
    w = WL[name]
    lat = Lattice(w.mask, w.neighbourhood)
    states = [state_for(w, np.random.default_rng(40 + i)) for i in range(len(SEEDS))]
    models = [make(w, sd, st, **PRECONDS[pc]) for sd, st in zip(SEEDS, states)]
    infos = gibbs_sweep_group(models, 1, first_counter=9)
    for m, sd, s, inf in zip(models, SEEDS, states, infos):
        g = m.get_state()
        Wr = gibbs.sample_W(lat, w.Y, w.X, s, sd, 9, w.eps)
        assert rel(g["W"], Wr) <= 1e-8
        s1 = dict(s, W=g["W"])
        if w.P > 0:
            Ar = gibbs.sample_A(lat, w.Y, w.X, s1, sd, 9, spatial=True)
            assert rel(g["A"], Ar) <= 1e-8
            s1["A"] = g["A"]
        lr = gibbs.sample_lambda(lat, w.Y, w.X, s1, sd, 9)
        assert np.max(np.abs(g["lam"] / lr - 1)) <= 1e-10
        ar = gibbs.sample_alpha(lat, s1, sd, 9)
        assert np.max(np.abs(g["alpha"] / ar - 1)) <= 1e-10
        if w.P > 0:
            br = gibbs.sample_beta(lat, s1, sd, 9)
            assert np.max(np.abs(g["beta"] / br - 1)) <= 1e-10
        assert inf.sweeps == 1 and inf.pcg_iterations_W > 0
        assert (inf.pcg_iterations_A > 0) == (w.P > 0)
        assert inf.last_rel_residual_W <= 1e-12
    for m in models:
        m.close()


@pytest.mark.parametrize("pc", ["bj", "ssor", "reduced"])
def test_group_matches_chains_advanced_alone(pc):
    """Three sweeps at a tight tolerance (1e-10): grouped and lone chains agree to the
    solver tolerance, sweep after sweep (the later steps see the earlier draws)."""
    from paper_1606_00980_gb300.bfmri import gibbs_sweep_group
    w = WL["slab_K6_P3"]
    states = [state_for(w, np.random.default_rng(70 + i)) for i in range(len(SEEDS))]
    grouped = [make(w, sd, st, delta=1e-10, **PRECONDS[pc]) for sd, st in zip(SEEDS, states)]
    alone = [make(w, sd, st, delta=1e-10, **PRECONDS[pc]) for sd, st in zip(SEEDS, states)]
    gibbs_sweep_group(grouped, 3, first_counter=4)
    for m in alone:
        m.gibbs_sweep(3, first_counter=4)
    for a, b in zip(grouped, alone):
        ga, gb = a.get_state(), b.get_state()
        assert rel(ga["W"], gb["W"]) <= 1e-7
        assert rel(ga["A"], gb["A"]) <= 1e-7
        assert np.max(np.abs(ga["lam"] / gb["lam"] - 1)) <= 1e-6
        assert np.max(np.abs(ga["alpha"] / gb["alpha"] - 1)) <= 1e-6
        assert np.max(np.abs(ga["beta"] / gb["beta"] - 1)) <= 1e-6
    # the chains are distinct draws, not copies of one another
    assert rel(grouped[0].get_state()["W"], grouped[1].get_state()["W"]) > 1e-3
    for m in grouped + alone:
        m.close()


def test_group_independent_ar_prior_and_single_chain():
    from paper_1606_00980_gb300 import bfmri
    w = WL["small3d_K3_P2"]
    lat = Lattice(w.mask, w.neighbourhood)
    s = state_for(w, np.random.default_rng(3))
    m = make(w, 55, s, ar_prior=bfmri.AR_INDEPENDENT)
    (inf,) = bfmri.gibbs_sweep_group([m], 1, first_counter=2)
    g = m.get_state()
    assert rel(g["W"], gibbs.sample_W(lat, w.Y, w.X, s, 55, 2, w.eps)) <= 1e-8
    s1 = dict(s, W=g["W"])
    assert rel(g["A"], gibbs.sample_A(lat, w.Y, w.X, s1, 55, 2, spatial=False)) <= 1e-8
    assert inf.pcg_iterations_A == 0
    m.close()


def test_group_rejects_mismatched_chains():
    from paper_1606_00980_gb300 import bfmri
    w = WL["small3d_K3_P2"]
    s = state_for(w, np.random.default_rng(1))
    a = make(w, 1, s)
    b = make(w, 2, s)
    other = WL["slab_K6_P3"]
    c = make(other, 3, state_for(other, np.random.default_rng(2)))
    d = make(w, 4, s, precision=bfmri.PREC_MIXED)
    e = make(w, 5, s, precond=2)
    f = make(w, 6, s, precond=2, ssor_omega=1.2)
    for group in ([a, c], [a, a], [a, d], [a, e], [e, f]):
        with pytest.raises(bfmri.BfmriError) as ei:
            bfmri.gibbs_sweep_group(group, 1)
        assert ei.value.status == -1
    # the valid pair still runs after the rejected calls
    bfmri.gibbs_sweep_group([a, b], 1)
    for m in (a, b, c, d, e, f):
        m.close()


def test_group_sweep_graph_replays_the_direct_sweeps():
    """options.use_graph on the first chain: the group sweep is captured once as a CUDA graph
    (each chain's draws reading its device counter) and replayed per sweep, also by a second
    call; the chains' states are bitwise those of the same group advanced by direct launches,
    and a group over different lattices is captured as well."""
    from paper_1606_00980_gb300.bfmri import gibbs_sweep_group, load_library
    lib = load_library()
    for ws in ([WL["slab_K6_P3"]] * 3,
               [WL["small3d_K3_P2"], synth.small3d(seed=24, dims=(10, 7, 5), K=3, P=2, T=40)]):
        states = [state_for(w, np.random.default_rng(50 + i)) for i, w in enumerate(ws)]
        runs = []
        for graph in (0, 1):
            models = [make(w, sd, st, use_graph=graph, precond=3)
                      for w, sd, st in zip(ws, SEEDS, states)]
            gibbs_sweep_group(models, 2, first_counter=11)
            gibbs_sweep_group(models, 3, first_counter=13)
            if graph:
                msg = lib.bfmri_last_error(models[0].handle) or b""
                assert not msg.startswith(b"CUDA graph capture unavailable"), msg
            runs.append([m.get_state() for m in models])
            for m in models:
                m.close()
        for direct, replayed in zip(*runs):
            for k in direct:
                assert np.array_equal(direct[k], replayed[k]), k
