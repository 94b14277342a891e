"""Red-black symmetric SOR preconditioning on the GPU (needs a GB300).

The preconditioner apply is checked element by element against the oracle's factored form
(oracle.precond.ssor_apply, itself pinned to voxel-by-voxel SOR sweeps) on the oracle's own
blocks, within the bound that the GPU blocks' assembly error allows (block_bounds);
block-Jacobi the same way. Solves preconditioned with
SSOR, in both solver variants, reach the oracle's exact draw (1e-8 relative L2 at relative
residual 1e-12), as the block-Jacobi ones do, and take fewer iterations on the same system.
"""
import numpy as np
import pytest

from block_bounds import apply_tolerance
from oracle import gibbs, model, philox, precond, probes
from oracle.lattice import Lattice
from paper_1606_00980_gb300 import synth

pytestmark = pytest.mark.gpu

SEED = 777


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def state_for(w, rng):
    N, K, P = w.N, w.K, w.P
    return dict(W=w.W_true + 0.2 * rng.standard_normal((K, N)),
                A=w.A_true + 0.02 * rng.standard_normal((P, N)),
                lam=rng.uniform(0.5, 2.0, N), alpha=rng.uniform(0.2, 3.0, K),
                beta=rng.uniform(2.0, 20.0, P))


def make(w, state, **opts):
    from paper_1606_00980_gb300.bfmri import Model
    opts.setdefault("delta", 1e-12)
    m = Model.from_workload(w, seed=SEED, **opts)
    m.precompute_stats()
    m.set_state(W=state["W"], A=state["A"], lam=state["lam"], alpha=state["alpha"],
                beta=state["beta"] if w.P > 0 else None)
    return m


WL = {
    "small3d_K3_P2": synth.small3d(seed=31, dims=(9, 8, 6), K=3, P=2, T=40),
    "slab_K6_P3": synth.small3d(seed=32, dims=(13, 11, 7), K=6, P=3, T=60),
    "slice2d_K3_P1": synth.make_workload("slice", (17, 15, 1), synth.circle_mask(17, 15, 7.3),
                                         T=50, K=3, P=1, neighbourhood=4, seed=33,
                                         ar_uniform=(0.1, 0.4), eps=1e-6),
}


@pytest.fixture(scope="module", params=sorted(WL))
def case(request):
    w = WL[request.param]
    return w, Lattice(w.mask, w.neighbourhood), state_for(w, np.random.default_rng(8))


@pytest.mark.parametrize("omega", [1.0, 1.4])
@pytest.mark.parametrize("which", [0, 1])
def test_ssor_apply_matches_oracle(case, which, omega):
    from paper_1606_00980_gb300 import bfmri
    w, lat, s = case
    if which == 1 and w.P == 0:
        pytest.skip("no AR part")
    m = make(w, s, precond=bfmri.PRECOND_SSOR, ssor_omega=omega)
    D = w.K if which == 0 else w.P
    x = np.random.default_rng(4).standard_normal((D, w.N))
    got = m.apply_preconditioner(which, x)
    m.close()
    if which == 0:
        Bd, _ = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"], w.eps)
        scale, entry_err = s["alpha"], 1e-12 * np.abs(Bd).max()
    else:
        Bd, _ = model.a_blocks_direct(w.Y, w.X, s["W"], s["lam"], w.P)
        st = model.sufficient_stats(w.Y, w.X, w.P)
        scale, entry_err = s["beta"], 1e-12 * (s["lam"] * st["Syy"][:, 0, 0]).max()
    ref = precond.ssor_apply(lat, Bd, scale, x.T, omega).T
    assert rel(got, ref) <= apply_tolerance(Bd, entry_err)


def test_block_jacobi_apply_matches_oracle(case):
    w, lat, s = case
    m = make(w, s)
    x = np.random.default_rng(5).standard_normal((w.K, w.N))
    got = m.apply_preconditioner(0, x)
    m.close()
    Bd, _ = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"], w.eps)
    Mb = probes.precond_blocks(lat, Bd, s["alpha"])
    ref = np.stack([np.linalg.solve(Mb[n], x[:, n]) for n in range(w.N)], axis=1)
    assert rel(got, ref) <= apply_tolerance(Bd, 1e-12 * np.abs(Bd).max())


@pytest.mark.parametrize("variant", ["auto", "streaming"])
@pytest.mark.parametrize("omega", [1.0, 1.3])
def test_ssor_solves_reach_the_exact_draw(case, omega, variant):
    from paper_1606_00980_gb300 import bfmri
    w, lat, s = case
    m = make(w, s, precond=bfmri.PRECOND_SSOR, ssor_omega=omega,
             pcg_variant=bfmri.PCG_AUTO if variant == "auto" else bfmri.PCG_STREAMING)
    W, info = m.sample_W(counter=3)
    Bd, bw = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"], w.eps)
    ref, mu = gibbs.draw_gmrf(lat, Bd, bw, s["alpha"], SEED, 3, philox.TAG_W)
    assert info.rel_residual <= 1e-12
    assert rel(W, ref) <= 1e-8
    if w.P > 0:
        A, ia = m.sample_A(counter=4)
        s1 = dict(s, W=W)
        Ar = gibbs.sample_A(lat, w.Y, w.X, s1, SEED, 4, spatial=True)
        assert ia.rel_residual <= 1e-12
        assert rel(A, Ar) <= 1e-8
    m.close()


@pytest.mark.parametrize("variant", ["auto", "streaming"])
def test_ssor_takes_fewer_iterations_than_block_jacobi(variant):
    from paper_1606_00980_gb300 import bfmri
    w = WL["slab_K6_P3"]
    s = state_for(w, np.random.default_rng(9))
    pv = bfmri.PCG_AUTO if variant == "auto" else bfmri.PCG_STREAMING
    its = {}
    for name, pc in (("bj", bfmri.PRECOND_BLOCK_JACOBI), ("ssor", bfmri.PRECOND_SSOR)):
        m = make(w, s, precond=pc, delta=1e-10, pcg_variant=pv)
        _, info = m.sample_W(counter=1)
        its[name] = info.iterations
        m.close()
    assert its["ssor"] < its["bj"]


@pytest.mark.parametrize("variant", ["auto", "streaming"])
def test_mixed_ssor_reaches_the_exact_draw(case, variant):
    """The mixed solver preconditions its FP32 inner iterations with SSOR (FP32 factor and
    phases); the FP64 refinement still reaches the exact draw."""
    from paper_1606_00980_gb300 import bfmri
    w, lat, s = case
    m = make(w, s, precond=bfmri.PRECOND_SSOR, precision=bfmri.PREC_MIXED,
             pcg_variant=bfmri.PCG_AUTO if variant == "auto" else bfmri.PCG_STREAMING)
    W, info = m.sample_W(counter=3)
    Bd, bw = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"], w.eps)
    ref, _ = gibbs.draw_gmrf(lat, Bd, bw, s["alpha"], SEED, 3, philox.TAG_W)
    assert info.rel_residual <= 1e-12
    assert rel(W, ref) <= 1e-8
    assert info.refinements >= 1
    m.close()


def test_mixed_ssor_takes_fewer_inner_iterations():
    from paper_1606_00980_gb300 import bfmri
    w = WL["slab_K6_P3"]
    s = state_for(w, np.random.default_rng(10))
    its = {}
    for name, pc in (("bj", bfmri.PRECOND_BLOCK_JACOBI), ("ssor", bfmri.PRECOND_SSOR)):
        m = make(w, s, precond=pc, precision=bfmri.PREC_MIXED, delta=1e-8)
        _, info = m.sample_W(counter=1)
        its[name] = info.iterations
        m.close()
    assert its["ssor"] < its["bj"]


@pytest.mark.parametrize("variant", ["auto", "streaming"])
def test_reduced_system_solves_reach_the_exact_draw(case, variant):
    """PRECOND_RB_REDUCED: the resident FP64 solver runs CG on the black voxels' Schur
    complement and recovers the red voxels; the streaming solver runs SSOR with omega = 1.
    Both reach the oracle's exact draw and confirm on the full system's true residual."""
    from paper_1606_00980_gb300 import bfmri
    w, lat, s = case
    m = make(w, s, precond=bfmri.PRECOND_RB_REDUCED,
             pcg_variant=bfmri.PCG_AUTO if variant == "auto" else bfmri.PCG_STREAMING)
    W, info = m.sample_W(counter=3)
    Bd, bw = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"], w.eps)
    ref, _ = gibbs.draw_gmrf(lat, Bd, bw, s["alpha"], SEED, 3, philox.TAG_W)
    assert info.rel_residual <= 1e-12
    assert rel(W, ref) <= 1e-8
    s2 = s
    if w.P > 0:
        A, ia = m.sample_A(counter=4)
        Ar = gibbs.sample_A(lat, w.Y, w.X, dict(s, W=W), SEED, 4, spatial=True)
        assert ia.rel_residual <= 1e-12
        assert rel(A, Ar) <= 1e-8
        s2 = dict(s, A=A)
    # a second draw, warm-started from the first (the W system now sees the new A)
    W2, _ = m.sample_W(counter=5)
    Bd2, bw2 = model.w_blocks_direct(w.Y, w.X, s2["A"], s2["lam"], w.eps)
    ref2, _ = gibbs.draw_gmrf(lat, Bd2, bw2, s2["alpha"], SEED, 5, philox.TAG_W)
    assert rel(W2, ref2) <= 1e-8
    m.close()


@pytest.mark.parametrize("delta", [1e-8, 1e-12])
def test_reduced_system_iterates_like_ssor_omega1(delta):
    """Same Krylov spaces: the reduced solve needs as many iterations as SSOR with omega = 1
    (up to one for the red component of the start residual), about half of block-Jacobi's."""
    from paper_1606_00980_gb300 import bfmri
    w = WL["slab_K6_P3"]
    s = state_for(w, np.random.default_rng(9))
    its = {}
    for name, pc in (("bj", bfmri.PRECOND_BLOCK_JACOBI), ("ssor", bfmri.PRECOND_SSOR),
                     ("reduced", bfmri.PRECOND_RB_REDUCED)):
        m = make(w, s, precond=pc, delta=delta)
        _, info = m.sample_W(counter=1)
        its[name] = info.iterations
        m.close()
    assert abs(its["reduced"] - its["ssor"]) <= 2, its
    assert its["reduced"] < its["bj"], its


def test_reduced_system_sweeps_and_grouped_chains():
    """Whole sweeps with the reduced solver (W and A), against the same sweeps with SSOR at
    omega = 1 (different solvers, same stop rule): agreement to the solver tolerance; grouped
    chains with the option run their multi-RHS solves as SSOR with omega = 1."""
    from paper_1606_00980_gb300 import bfmri
    w = WL["slab_K6_P3"]
    s = state_for(w, np.random.default_rng(11))
    a = make(w, s, precond=bfmri.PRECOND_RB_REDUCED, delta=1e-11)
    b = make(w, s, precond=bfmri.PRECOND_SSOR, delta=1e-11)
    a.gibbs_sweep(3, 10)
    b.gibbs_sweep(3, 10)
    sa, sb = a.get_state(), b.get_state()
    assert rel(sa["W"], sb["W"]) <= 1e-8
    assert rel(sa["A"], sb["A"]) <= 1e-8
    assert np.max(np.abs(sa["lam"] / sb["lam"] - 1)) <= 1e-7
    c = make(w, s, precond=bfmri.PRECOND_RB_REDUCED, delta=1e-11)
    d = make(w, s, precond=bfmri.PRECOND_RB_REDUCED, delta=1e-11)
    bfmri.gibbs_sweep_group([c, d], 2, 10)
    c.close()
    d.close()
    a.close()
    b.close()


@pytest.mark.parametrize("variant", ["auto", "streaming"])
def test_mixed_reduced_system_reaches_the_exact_draw(case, variant):
    """Mixed precision with PRECOND_RB_REDUCED: FP32 CG on the reduced system for each
    correction (resident), SSOR with omega = 1 in the streaming variant; the FP64 refinement
    reaches the exact draw."""
    from paper_1606_00980_gb300 import bfmri
    w, lat, s = case
    m = make(w, s, precond=bfmri.PRECOND_RB_REDUCED, precision=bfmri.PREC_MIXED,
             pcg_variant=bfmri.PCG_AUTO if variant == "auto" else bfmri.PCG_STREAMING)
    W, info = m.sample_W(counter=3)
    Bd, bw = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"], w.eps)
    ref, _ = gibbs.draw_gmrf(lat, Bd, bw, s["alpha"], SEED, 3, philox.TAG_W)
    assert info.rel_residual <= 1e-12
    assert rel(W, ref) <= 1e-8
    assert info.refinements >= 1
    if w.P > 0:
        A, ia = m.sample_A(counter=4)
        Ar = gibbs.sample_A(lat, w.Y, w.X, dict(s, W=W), SEED, 4, spatial=True)
        assert ia.rel_residual <= 1e-12
        assert rel(A, Ar) <= 1e-8
    m.close()


def test_mixed_reduced_inner_iterations_match_mixed_ssor():
    from paper_1606_00980_gb300 import bfmri
    w = WL["slab_K6_P3"]
    s = state_for(w, np.random.default_rng(10))
    its = {}
    for name, pc in (("bj", bfmri.PRECOND_BLOCK_JACOBI), ("ssor", bfmri.PRECOND_SSOR),
                     ("reduced", bfmri.PRECOND_RB_REDUCED)):
        m = make(w, s, precond=pc, precision=bfmri.PREC_MIXED, delta=1e-8)
        _, info = m.sample_W(counter=1)
        its[name] = info.iterations
        m.close()
    assert its["reduced"] < its["bj"], its
    assert abs(its["reduced"] - its["ssor"]) <= max(3, its["ssor"] // 5), its


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_reduced_system_with_large_blocks(precision):
    """K = 8 runs the unpipelined reduced solver (the pipelined one keeps four extra vectors in
    shared memory and stops at D = 6); mixed precision runs the pipelined FP32 inner solver."""
    from paper_1606_00980_gb300 import bfmri
    w = synth.small3d(seed=34, dims=(9, 8, 6), K=8, P=1, T=60)
    lat = Lattice(w.mask, w.neighbourhood)
    s = state_for(w, np.random.default_rng(12))
    m = make(w, s, precond=bfmri.PRECOND_RB_REDUCED,
             precision=bfmri.PREC_FP64 if precision == "fp64" else bfmri.PREC_MIXED)
    W, info = m.sample_W(counter=3)
    Bd, bw = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"], w.eps)
    ref, _ = gibbs.draw_gmrf(lat, Bd, bw, s["alpha"], SEED, 3, philox.TAG_W)
    assert info.rel_residual <= 1e-12
    assert rel(W, ref) <= 1e-8
    m.close()
