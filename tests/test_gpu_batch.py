"""One multi-RHS launch for chains of different subjects, and for chains beside log-det
probes (bfmri_gibbs_sweep_group over uneven masks, bfmri_gibbs_sweep_group_probes; needs a
GB300).

Subjects on different lattices (different box sizes, holes, voxel counts) advance together,
each right-hand side of the launch carrying its own lattice and the work units shared out in
proportion to the voxels; every chain's sweep is replayed by the FP64 oracle step by step
(draws 1e-8 relative L2 against the exact solve of the same perturbed system, lambda, alpha,
beta 1e-10). With probes in the same launch, every probe's Lanczos quadrature is compared
with the oracle's exact v' log(C) v (1e-6) and the estimate with log det M plus the probes'
mean, for a probe handle that is one of the chains and for one outside the group on its own
lattice.
"""
import numpy as np
import pytest

from oracle import gibbs, model, probes
from oracle.lattice import Lattice
from paper_1606_00980_gb300 import synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def subjects():
    holes = np.ones((5, 8, 10), np.uint8)
    holes[2, 3:5, 4:7] = 0
    return [synth.small3d(seed=61, dims=(9, 8, 6), K=3, P=2, T=40),
            synth.small3d(seed=62, dims=(12, 7, 5), K=3, P=2, T=44),
            synth.make_workload("holes", (10, 8, 5), holes, T=36, K=3, P=2, neighbourhood=6,
                                seed=63, ar_uniform=(0.1, 0.4))]


def state_for(w, rng):
    return dict(W=w.W_true + 0.2 * rng.standard_normal((w.K, w.N)),
                A=w.A_true + 0.02 * rng.standard_normal((w.P, w.N)),
                lam=rng.uniform(0.5, 2.0, w.N), alpha=rng.uniform(0.2, 3.0, w.K),
                beta=rng.uniform(2.0, 20.0, w.P))


def make(w, seed, state, **opts):
    from paper_1606_00980_gb300.bfmri import Model
    opts.setdefault("delta", 1e-12)
    m = Model.from_workload(w, seed=seed, **opts)
    m.precompute_stats()
    m.set_state(W=state["W"], A=state["A"], lam=state["lam"], alpha=state["alpha"],
                beta=state["beta"])
    return m


def check_chain(w, seed, s, g, counter):
    lat = Lattice(w.mask, w.neighbourhood)
    Wr = gibbs.sample_W(lat, w.Y, w.X, s, seed, counter, w.eps)
    assert rel(g["W"], Wr) <= 1e-8
    s1 = dict(s, W=g["W"])
    Ar = gibbs.sample_A(lat, w.Y, w.X, s1, seed, counter, spatial=True)
    assert rel(g["A"], Ar) <= 1e-8
    s1["A"] = g["A"]
    lr = gibbs.sample_lambda(lat, w.Y, w.X, s1, seed, counter)
    assert np.max(np.abs(g["lam"] / lr - 1)) <= 1e-10
    assert np.max(np.abs(g["alpha"] / gibbs.sample_alpha(lat, s1, seed, counter) - 1)) <= 1e-10
    assert np.max(np.abs(g["beta"] / gibbs.sample_beta(lat, s1, seed, counter) - 1)) <= 1e-10


@pytest.mark.parametrize("pc", ["bj", "ssor", "reduced"])
def test_group_over_different_lattices_matches_oracle(pc):
    from paper_1606_00980_gb300 import bfmri
    from paper_1606_00980_gb300.bfmri import gibbs_sweep_group
    opts = {"bj": dict(), "ssor": dict(precond=bfmri.PRECOND_SSOR),
            "reduced": dict(precond=bfmri.PRECOND_RB_REDUCED)}[pc]
    ws = subjects()
    assert len({w.N for w in ws}) == len(ws)          # uneven masks
    seeds = [501, 502, 503]
    states = [state_for(w, np.random.default_rng(70 + i)) for i, w in enumerate(ws)]
    models = [make(w, sd, st, **opts) for w, sd, st in zip(ws, seeds, states)]
    infos = gibbs_sweep_group(models, 1, first_counter=9)
    for w, m, sd, s, inf in zip(ws, models, seeds, states, infos):
        check_chain(w, sd, s, m.get_state(), 9)
        assert inf.pcg_iterations_W > 0
        m.close()


@pytest.mark.parametrize("probe_in_group", [True, False])
def test_chains_and_probes_in_one_launch(probe_in_group):
    from paper_1606_00980_gb300.bfmri import gibbs_sweep_group_probes
    ws = subjects()
    chains_w = ws[:2]
    seeds = [601, 602]
    states = [state_for(w, np.random.default_rng(80 + i)) for i, w in enumerate(chains_w)]
    models = [make(w, sd, st) for w, sd, st in zip(chains_w, seeds, states)]
    if probe_in_group:
        pw, ps, pm, psd = chains_w[0], states[0], models[0], seeds[0]
    else:
        pw, psd = ws[2], 777
        ps = state_for(pw, np.random.default_rng(90))
        pm = make(pw, psd, ps)
    n_probes = 16
    infos, logdet, se, per = gibbs_sweep_group_probes(models, 9, pm, n_probes, 2000, probe_counter=6)
    for w, m, sd, s in zip(chains_w, models, seeds, states):
        check_chain(w, sd, s, m.get_state(), 9)
    # the probes saw the W system of the probe handle's state before the sweep
    lat = Lattice(pw.mask, pw.neighbourhood)
    Bd, _ = model.w_blocks_direct(pw.Y, pw.X, ps["A"], ps["lam"], pw.eps)
    V = probes.probe_vectors(lat, pw.K, n_probes, psd, 6)
    ldm, quad, _, ldb = probes.exact_probe_terms(lat, Bd, ps["alpha"], V)
    assert np.max(np.abs(per - quad) / np.abs(quad)) <= 1e-6
    assert abs(logdet - (ldm + quad.mean())) <= 1e-6 * abs(ldm + quad.mean())
    assert abs(logdet - ldb) <= 5 * max(se, 1e-9) + 1e-6 * abs(ldb)
    for m in models:
        m.close()
    if not probe_in_group:
        pm.close()
