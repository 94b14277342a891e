"""The multigrid V-cycle preconditioner on the GPU against the FP64 oracle (needs a GB300).

The GPU builds at most three levels of 2x2x2 aggregates (2x2 in-slice for the 4-neighbour
prior), adding a coarser level only while it keeps at least 64 voxels, and takes two
symmetric red-black Gauss-Seidel steps on the coarsest level; the oracle's hierarchy with the
same rule (max_levels = 3, min_coarse = 64, coarse_steps = 2) is the reference. One
application of the cycle matches the oracle's, on the oracle's own blocks, within the bound
that the blocks' assembly error allows (block_bounds); W and A draws with the multigrid
PCG reach the oracle's exact solve of the same perturbed system to 1e-8 (delta = 1e-12).
"""
import numpy as np
import pytest

from block_bounds import apply_tolerance
from oracle import gibbs, model, multigrid
from oracle.lattice import Lattice
from paper_1606_00980_gb300 import synth

pytestmark = pytest.mark.gpu

SEED = 8642


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def state_for(w, rng):
    N, K, P = w.N, w.K, w.P
    return dict(W=w.W_true + 0.2 * rng.standard_normal((K, N)),
                A=w.A_true + 0.02 * rng.standard_normal((P, N)),
                lam=rng.uniform(0.5, 2.0, N), alpha=rng.uniform(0.2, 3.0, K),
                beta=rng.uniform(2.0, 20.0, P))


def make(w, state, **opts):
    from paper_1606_00980_gb300 import bfmri
    from paper_1606_00980_gb300.bfmri import Model
    opts.setdefault("delta", 1e-12)
    m = Model.from_workload(w, seed=SEED, precond=bfmri.PRECOND_MULTIGRID, **opts)
    m.precompute_stats()
    m.set_state(W=state["W"], A=state["A"], lam=state["lam"], alpha=state["alpha"],
                beta=state["beta"])
    return m


CASES = {
    # three levels (about 5,900 -> 800 -> 110 voxels), K = 6, P = 3
    "three_levels_K6_P3": lambda: synth.request_workload(seed=51, N_target=6000, K=6, T=40, P=3),
    # two levels, holes and a ragged tail
    "two_levels_K4_P2": lambda: synth.small3d(seed=52, dims=(13, 12, 9), K=4, P=2, T=40),
    # slice-wise 2D prior (4 neighbours): 2x2 in-slice aggregates
    "slice2d_K3_P1": lambda: synth.make_workload("slice", (40, 36, 2), np.ones((2, 36, 40), np.uint8),
                                                 T=40, K=3, P=1, neighbourhood=4, seed=53,
                                                 ar_uniform=(0.1, 0.4)),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    w = CASES[request.param]()
    lat = Lattice(w.mask, w.neighbourhood)
    return w, lat, state_for(w, np.random.default_rng(61))


@pytest.mark.parametrize("which", [0, 1])
def test_vcycle_apply_matches_oracle(case, which):
    w, lat, s = case
    m = make(w, s)
    D = w.K if which == 0 else w.P
    x = np.random.default_rng(3).standard_normal((D, w.N))
    y = m.apply_preconditioner(which, x)
    m.close()
    if which == 0:
        Bd, _ = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"], w.eps)
        scale = s["alpha"]
        entry_err = 1e-12 * np.abs(Bd).max()
    else:
        Bd, _ = model.a_blocks_direct(w.Y, w.X, s["W"], s["lam"], w.P)
        scale = s["beta"]
        st = model.sufficient_stats(w.Y, w.X, w.P)
        entry_err = 1e-12 * (s["lam"] * st["Syy"][:, 0, 0]).max()
    levels = multigrid.hierarchy(lat, Bd, scale, n_min=0, max_levels=3, min_coarse=64)
    ref = multigrid.vcycle(levels, model.kmajor(x.T), coarse_steps=2).reshape(D, w.N)
    assert rel(y, ref) <= apply_tolerance(Bd, entry_err)


def test_draws_with_multigrid_reach_the_exact_solve(case):
    w, lat, s = case
    m = make(w, s)
    W, info = m.sample_W(counter=3)
    W_ref = gibbs.sample_W(lat, w.Y, w.X, s, SEED, 3, w.eps)
    assert info.rel_residual <= 1e-12
    assert rel(W, W_ref) <= 1e-8
    A, ia = m.sample_A(counter=4)
    A_ref = gibbs.sample_A(lat, w.Y, w.X, dict(s, W=W), SEED, 4, spatial=True)
    assert ia.rel_residual <= 1e-12
    assert rel(A, A_ref) <= 1e-8
    m.close()


def test_multigrid_sweep_matches_oracle_and_needs_fewer_iterations():
    """One Gibbs sweep with the multigrid solver on the three-level case, replayed by the
    oracle; and on a stiff prior the multigrid PCG needs fewer iterations than the reduced
    red-black solver (symmetric Gauss-Seidel's iterates) for the same draw."""
    from paper_1606_00980_gb300 import bfmri
    w = CASES["three_levels_K6_P3"]()
    lat = Lattice(w.mask, w.neighbourhood)
    s = state_for(w, np.random.default_rng(62))
    s["alpha"] = np.full(w.K, 200.0)           # strong spatial coupling
    m = make(w, s)
    m.gibbs_sweep(1, first_counter=5)
    g = m.get_state()
    m.close()
    assert rel(g["W"], gibbs.sample_W(lat, w.Y, w.X, s, SEED, 5, w.eps)) <= 1e-8
    its = {}
    for name, pc in (("mg", bfmri.PRECOND_MULTIGRID), ("reduced", bfmri.PRECOND_RB_REDUCED)):
        from paper_1606_00980_gb300.bfmri import Model
        mm = Model.from_workload(w, seed=SEED, precond=pc, delta=1e-10)
        mm.precompute_stats()
        mm.set_state(W=np.zeros_like(s["W"]), A=s["A"], lam=s["lam"], alpha=s["alpha"],
                     beta=s["beta"])
        _, info = mm.sample_W(counter=6)
        its[name] = info.iterations
        mm.close()
    assert its["mg"] < its["reduced"], its
