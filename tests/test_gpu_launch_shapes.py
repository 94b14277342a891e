"""The solvers' full-size launch shapes at sizes the oracle still solves exactly (needs a
GB300).

The whole-brain workload (49,928 voxels over 152 SMs) runs the resident reduced red-black
solvers with CTAs of 352 threads (11 warps, 329 voxels each); the small parity workloads
only reach CTAs of 64 threads. Capping the solvers at a few SMs (options.sm_budget) gives
an oracle-sized subject the headline's CTA shape: about 2,700 voxels over 8 SMs are CTAs of
352 threads, which takes the multi-warp colour phases and the partial-sum collection by the
last four (idle) warps of each CTA. Over 2 SMs the same subject no longer fits one CTA per
SM and runs the streaming solvers, whose grid spans several CTAs per SM. The multi-RHS
solver with 64 probes at K = 8 fills its whole cooperative grid (as the 96x96x60 workload
does). Every result is checked element by element against the FP64 oracle: W and A draws
1e-8 relative L2 (FP64, and mixed precision run to 1e-12), 1e-5 (mixed precision at
delta = 1e-8); per-probe Lanczos quadrature 1e-6 (FP64) and 1e-4 (FP32 storage).
"""
import numpy as np
import pytest

from oracle import gibbs, model, philox, probes
from oracle.lattice import Lattice
from paper_1606_00980_gb300 import synth

pytestmark = pytest.mark.gpu

SEED = 2468


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def state_for(w, rng):
    N, K, P = w.N, w.K, w.P
    return dict(W=w.W_true + 0.2 * rng.standard_normal((K, N)),
                A=w.A_true + 0.02 * rng.standard_normal((P, N)),
                lam=rng.uniform(0.5, 2.0, N), alpha=rng.uniform(0.2, 3.0, K),
                beta=rng.uniform(2.0, 20.0, P))


def make(w, state, seed=SEED, **opts):
    from paper_1606_00980_gb300.bfmri import Model
    opts.setdefault("delta", 1e-12)
    m = Model.from_workload(w, seed=seed, **opts)
    m.precompute_stats()
    m.set_state(W=state["W"], A=state["A"], lam=state["lam"], alpha=state["alpha"],
                beta=state["beta"])
    return m


# K = 6, P = 3 (the headline's K and P): 2,672 voxels -> 334 per CTA over 8 SMs -> 352 threads
W6 = synth.request_workload(seed=41, N_target=2700, K=6, T=60, P=3)
# K = 8, P = 3 (the batched workload's K and P)
W8 = synth.request_workload(seed=42, N_target=1300, K=8, T=60, P=3)


def test_shape_of_the_headline_cta():
    per = -(-W6.N // 8)
    assert 320 < per <= 352 and (per + 31) // 32 * 32 == 352


@pytest.fixture(scope="module")
def case6():
    lat = Lattice(W6.mask, W6.neighbourhood)
    s = state_for(W6, np.random.default_rng(51))
    W_ref = gibbs.sample_W(lat, W6.Y, W6.X, s, SEED, 3, W6.eps)
    return lat, s, W_ref


# (sm_budget, precision, delta, tolerance): 8 SMs = resident solvers with 352-thread CTAs,
# 2 SMs = streaming solvers over several CTAs per SM
CASES = [(8, "fp64", 1e-12, 1e-8), (8, "mixed", 1e-12, 1e-8), (8, "mixed", 1e-8, 1e-5),
         (2, "fp64", 1e-12, 1e-8), (2, "mixed", 1e-12, 1e-8), (2, "mixed", 1e-8, 1e-5)]


@pytest.mark.parametrize("sm,precision,delta,tol", CASES)
def test_reduced_solver_draws_at_full_cta_shape(case6, sm, precision, delta, tol):
    """The default solver (reduced red-black system) for W (D = 6: k_pcg_rbp /
    k_pcg_mixed_rbp resident, k_pcg_mixed_stream_rb or the SSOR streaming form over 2 SMs)
    and then A (D = 3) from the GPU's own W."""
    from paper_1606_00980_gb300 import bfmri
    lat, s, W_ref = case6
    m = make(W6, s, precond=bfmri.PRECOND_RB_REDUCED, sm_budget=sm, delta=delta,
             precision=bfmri.PREC_FP64 if precision == "fp64" else bfmri.PREC_MIXED)
    W, info = m.sample_W(counter=3)
    assert info.rel_residual <= delta
    assert rel(W, W_ref) <= tol
    A, ia = m.sample_A(counter=4)
    A_ref = gibbs.sample_A(lat, W6.Y, W6.X, dict(s, W=W), SEED, 4, spatial=True)
    assert ia.rel_residual <= delta
    assert rel(A, A_ref) <= tol
    m.close()


@pytest.mark.parametrize("lanes", [1, 2])
def test_one_lane_and_lane_pairs_at_full_cta_shape(case6, lanes):
    """The resident FP64 reduced solver with one lane per voxel (k_pcg_rbp) and with lane
    pairs (k_pcg_rbp2: one red and one black voxel per pair of lanes, each lane half of each
    voxel's components) at the headline CTA shape: W (D = 6) and A (D = 3, an odd D, where the
    second lane of a pair holds one component) against the oracle, and the same iteration
    count both ways."""
    from paper_1606_00980_gb300 import bfmri
    lat, s, W_ref = case6
    m = make(W6, s, precond=bfmri.PRECOND_RB_REDUCED, sm_budget=8, pcg_lanes=lanes)
    W, info = m.sample_W(counter=3)
    assert info.rel_residual <= 1e-12
    assert rel(W, W_ref) <= 1e-8
    A, ia = m.sample_A(counter=4)
    A_ref = gibbs.sample_A(lat, W6.Y, W6.X, dict(s, W=W), SEED, 4, spatial=True)
    assert ia.rel_residual <= 1e-12
    assert rel(A, A_ref) <= 1e-8
    m.close()
    other = make(W6, s, precond=bfmri.PRECOND_RB_REDUCED, sm_budget=8, pcg_lanes=3 - lanes)
    _, info2 = other.sample_W(counter=3)
    other.close()
    assert abs(info2.iterations - info.iterations) <= 1


@pytest.mark.parametrize("precond", ["bj", "ssor"])
def test_block_jacobi_and_ssor_at_full_cta_shape(case6, precond):
    """The resident block-Jacobi and SSOR solver (k_pcg_res) with 352-thread CTAs."""
    from paper_1606_00980_gb300 import bfmri
    lat, s, W_ref = case6
    pc = dict(precond=bfmri.PRECOND_BLOCK_JACOBI) if precond == "bj" else \
        dict(precond=bfmri.PRECOND_SSOR, ssor_omega=1.0)
    m = make(W6, s, sm_budget=8, **pc)
    W, info = m.sample_W(counter=3)
    assert info.rel_residual <= 1e-12
    assert rel(W, W_ref) <= 1e-8
    m.close()


def test_gibbs_sweep_at_full_cta_shape(case6):
    """One whole sweep with the headline's options (reduced solver, delta 1e-12 here) at the
    headline CTA shape, replayed step by step by the oracle from the GPU's own outputs."""
    from paper_1606_00980_gb300 import bfmri
    lat, s, W_ref = case6
    m = make(W6, s, precond=bfmri.PRECOND_RB_REDUCED, sm_budget=8)
    m.gibbs_sweep(1, first_counter=3)
    g = m.get_state()
    assert rel(g["W"], W_ref) <= 1e-8
    s1 = dict(s, W=g["W"])
    Ar = gibbs.sample_A(lat, W6.Y, W6.X, s1, SEED, 3, spatial=True)
    assert rel(g["A"], Ar) <= 1e-8
    s1["A"] = g["A"]
    lr = gibbs.sample_lambda(lat, W6.Y, W6.X, s1, SEED, 3)
    assert np.max(np.abs(g["lam"] / lr - 1)) <= 1e-10
    m.close()


@pytest.mark.parametrize("precision,tile", [("fp64", 1), ("fp32", 1), ("fp32", 2), ("fp32", 4)])
def test_64_probes_at_k8_fill_the_grid(precision, tile):
    """64 Rademacher probes of the K = 8 W system in one multi-RHS launch (the batched
    workload's probe count and K; 1,328 voxels give every one of the 64 right-hand sides 38
    voxel chunks over the full grid, as 250k voxels do). Eight sampled probes are checked
    against the oracle's converged Lanczos quadrature and exact trace terms; the estimates
    against the exact log det within 5 standard errors."""
    from paper_1606_00980_gb300 import bfmri
    w = W8
    lat = Lattice(w.mask, w.neighbourhood)
    rng = np.random.default_rng(4)
    s = dict(W=w.W_true + 0.1 * rng.standard_normal(w.W_true.shape), A=w.A_true,
             lam=rng.uniform(0.5, 2.0, w.N), alpha=rng.uniform(0.3, 3.0, w.K),
             beta=rng.uniform(2.0, 9.0, w.P))
    extra = dict(precision=bfmri.PREC_MIXED, delta=1e-5, mrhs_tile=tile) if precision == "fp32" else {}
    m = make(w, s, precond=bfmri.PRECOND_BLOCK_JACOBI, **extra)
    n_probes = 64
    res = m.logdet_probe(0, n_probes, 3000, counter=6)
    m.close()
    Bd, _ = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"], w.eps)
    V = probes.probe_vectors(lat, w.K, n_probes, SEED, 6)
    pick = list(range(0, n_probes, 9))
    ldm, quad, tr, ldb = probes.probe_terms_lanczos(lat, Bd, s["alpha"], [V[i] for i in pick])
    got = res["per_probe"][pick]
    tq = 1e-4 if precision == "fp32" else 1e-6
    assert np.max(np.abs(got - quad) / np.abs(quad)) <= tq
    assert np.all(res["iterations"] > 0)
    assert abs(res["logdet"] - ldb) <= 5 * max(res["stderr"], 1e-9) + 1e-6 * abs(ldb)


@pytest.mark.parametrize("sm", [0, 2])
def test_eight_grouped_chains_at_k8(sm):
    """Eight chains of the K = 8 subject advanced together (one multi-RHS launch with a matrix
    per chain); with 2 SMs every warp walks several chunks of its chain, as the 250k-voxel
    chains do. Each chain's W is checked against the oracle's exact draw."""
    from paper_1606_00980_gb300 import bfmri
    from paper_1606_00980_gb300.bfmri import gibbs_sweep_group
    w = W8
    lat = Lattice(w.mask, w.neighbourhood)
    seeds = [900 + c for c in range(8)]
    states = [state_for(w, np.random.default_rng(60 + c)) for c in range(8)]
    models = [make(w, st, seed=sd, precond=bfmri.PRECOND_RB_REDUCED, sm_budget=sm)
              for sd, st in zip(seeds, states)]
    gibbs_sweep_group(models, 1, first_counter=11)
    for m, sd, st in zip(models, seeds, states):
        W = m.get_state()["W"]
        W_ref = gibbs.sample_W(lat, w.Y, w.X, st, sd, 11, w.eps)
        assert rel(W, W_ref) <= 1e-8
        m.close()
