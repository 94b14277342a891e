"""The anisotropic prior on the GPU (options.w_prior = PRIOR_ANISO; needs a GB300).

The Discussion's second variant gives W_k the prior precision G_w' C_k G_w with
C_k = diag(alpha_x,k I, alpha_y,k I, alpha_z,k I), the alphas random. W is drawn by the FP64
solvers (resident block-Jacobi and red-black reduced kernels, streaming block-Jacobi) with one
prior scale per direction and component; the alphas by the
exchange algorithm (Murray, Ghahramani & MacKay 2006): a log-normal proposal, an auxiliary
field drawn from the prior at the proposal by Algorithm 2's perturbation without a data term
and PCG from zero, and acceptance from the direction edge sums of W and of the field, after
an exact Gamma draw of the alphas' common scale along the ray alpha -> lam alpha.
Everything is checked against the oracle's anisotropic prior and alpha step (pinned in
tests/test_oracle_aniso.py): B~ x 1e-13, perturbed systems 1e-12, the block-Jacobi apply
within the blocks' assembly bound, W draws 1e-8 against the exact solve; for the alpha step
lam 1e-10 (the Gamma tests' bar), the edge sums of W 1e-12 and of the auxiliary field 1e-8
(a PCG solve to 1e-12 against the oracle's exact range solve, whose condition number on these
lattices is below 1e3), the field itself 1e-8 after removing each connected part's mean,
log a to 1e-6, the accept decisions the oracle's wherever |log u - log a| exceeds that bound
and the new alphas within lam's 1e-10; a sweep step by step; the captured sweep bitwise the
direct one. With equal alphas in every direction the precision and the W draw are the
graph-Laplacian prior's.
"""
import numpy as np
import pytest

from block_bounds import apply_tolerance
from oracle import gibbs, model, philox
from oracle.lattice import Lattice
from paper_1606_00980_gb300 import synth

pytestmark = pytest.mark.gpu

SEED = 7171
STEP = 0.05


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def state_for(w, rng):
    return dict(W=w.W_true + 0.2 * rng.standard_normal((w.K, w.N)),
                A=w.A_true + 0.02 * rng.standard_normal((w.P, w.N)),
                lam=rng.uniform(0.5, 2.0, w.N), alpha=rng.uniform(0.2, 3.0, (w.K, 3)),
                beta=rng.uniform(2.0, 20.0, w.P))


CASES = {
    "small3d_K3_P2": (synth.small3d(seed=71, dims=(9, 8, 6), K=3, P=2, T=40), (1.0, 1.0, 1.0)),
    "weighted3d_K4_P1": (synth.small3d(seed=72, dims=(8, 7, 6), K=4, P=1, T=40), (2.0, 0.5, 3.25)),
    "slice2d_K3_P1": (synth.make_workload("slice", (15, 13, 1), synth.circle_mask(15, 13, 6.1),
                                          T=40, K=3, P=1, neighbourhood=4, seed=73,
                                          ar_uniform=(0.1, 0.4), eps=1e-6), (1.0, 1.0, 1.0)),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    w, cw = CASES[request.param]
    lat = Lattice(w.mask, w.neighbourhood, weights=cw)
    rng = np.random.default_rng(74)
    s = dict(W=w.W_true + 0.2 * rng.standard_normal((w.K, w.N)),
             alpha=rng.uniform(0.2, 3.0, (w.K, 3)))
    s.update(A=w.A_true + 0.02 * rng.standard_normal((w.P, w.N)), lam=rng.uniform(0.5, 2.0, w.N),
             beta=rng.uniform(2.0, 20.0, w.P))
    return w, cw, lat, s


def make(w, cw, state, **opts):
    from paper_1606_00980_gb300 import bfmri
    from paper_1606_00980_gb300.bfmri import Model
    opts.setdefault("delta", 1e-12)
    opts.setdefault("precond", 1)
    opts.setdefault("aniso_step", STEP)
    m = Model.from_workload(w, seed=SEED, edge_weight=cw, w_prior=bfmri.PRIOR_ANISO, **opts)
    m.precompute_stats()
    m.set_state(W=state["W"], A=state["A"], lam=state["lam"], beta=state["beta"])
    m.set_alpha_dirs(state["alpha"])
    return m


def test_precision_and_perturbed_system(case):
    w, cw, lat, s = case
    m = make(w, cw, s)
    x = np.random.default_rng(1).standard_normal((w.K, w.N))
    y = m.apply_precision(0, x)
    _, _, bpert = m.build_system(0, counter=21)
    m.close()
    Bd, bw = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"], w.eps)
    B = model.precision(lat, Bd, s["alpha"], "aniso")
    assert rel(y, (B @ x.reshape(-1)).reshape(w.K, w.N)) <= 1e-13
    pert, _, _ = model.perturbation(lat, Bd, s["alpha"], SEED, 21, philox.TAG_W, 0, "aniso")
    assert rel(bpert, (model.kmajor(bw) + pert).reshape(bpert.shape)) <= 1e-12


def test_block_jacobi_apply(case):
    w, cw, lat, s = case
    m = make(w, cw, s)
    x = np.random.default_rng(2).standard_normal((w.K, w.N))
    got = m.apply_preconditioner(0, x)
    m.close()
    Bd, _ = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"], w.eps)
    degs = np.stack([L.diagonal() for L in model.direction_laplacians(lat)])     # (3, N)
    dk = s["alpha"] @ degs                                                        # (K, N)
    Mb = Bd + np.eye(w.K)[None] * dk.T[:, :, None]
    ref = np.stack([np.linalg.solve(Mb[n], x[:, n]) for n in range(w.N)], axis=1)
    assert rel(got, ref) <= apply_tolerance(Bd, 1e-12 * np.abs(Bd).max())


@pytest.mark.parametrize("variant", ["auto", "streaming"])
@pytest.mark.parametrize("precond", ["none", "bj", "reduced"])
def test_w_draw(case, precond, variant):
    """The register-resident kernels (auto at these sizes: block-Jacobi, or CG on the red-black
    reduced system) and the streaming kernel (block-Jacobi on the same blocks for both), with
    and without a preconditioner."""
    from paper_1606_00980_gb300 import bfmri
    w, cw, lat, s = case
    pc = dict(none=bfmri.PRECOND_NONE, bj=bfmri.PRECOND_BLOCK_JACOBI, reduced=bfmri.PRECOND_RB_REDUCED)
    m = make(w, cw, s, precond=pc[precond],
             pcg_variant=bfmri.PCG_AUTO if variant == "auto" else bfmri.PCG_STREAMING)
    W, info = m.sample_W(counter=3)
    m.close()
    assert info.rel_residual <= 1e-12
    assert rel(W, gibbs.sample_W(lat, w.Y, w.X, s, SEED, 3, w.eps, prior="aniso")) <= 1e-8


def parts_mean_removed(lat, v):
    """v with the mean of every connected part of the voxel graph subtracted (rows of v)."""
    J = gibbs.null_projector(lat)
    return v - (J @ v.T).T


def check_exchange(lat, m, state, counter, got_alpha, steps_seen):
    """The GPU alpha step from `state` against the oracle's; returns the oracle's new alphas."""
    new, acc, d = gibbs.aniso_alpha_step(lat, state, SEED, counter, STEP)
    ls = m.aniso_last_step()
    assert np.max(np.abs(ls["lam"] / d["lam"] - 1)) <= 1e-10
    assert rel(ls["Q"], d["Q"]) <= 1e-12
    assert rel(ls["Q_aux"], d["Qp"]) <= 1e-8
    assert rel(parts_mean_removed(lat, ls["w_aux"]), d["aux"]) <= 1e-8
    assert np.max(np.abs(ls["log_a"] - d["log_a"])) <= 1e-6
    margin = np.abs(np.log(d["u"]) - d["log_a"])
    for k in range(len(acc)):
        if margin[k] > 1e-6:
            assert np.allclose(got_alpha[k], new[k], rtol=1e-10, atol=0), (k, got_alpha[k], new[k])
            steps_seen.add(bool(acc[k]))
    return new, acc


@pytest.mark.parametrize("variant", ["auto", "streaming", "reduced"])
def test_exchange_steps(case, variant):
    from paper_1606_00980_gb300 import bfmri
    w, cw, lat, s = case
    m = make(w, cw, s, pcg_variant=bfmri.PCG_STREAMING if variant == "streaming" else bfmri.PCG_AUTO,
             precond=bfmri.PRECOND_RB_REDUCED if variant == "reduced" else bfmri.PRECOND_BLOCK_JACOBI)
    seen = set()
    cur = dict(s)
    acc_total = np.zeros(w.K, dtype=np.int64)
    for counter in (1, 2, 3, 4):
        m.sample_alpha(counter=counter)
        got, acc = m.get_alpha_dirs()
        new, acc_k = check_exchange(lat, m, cur, counter, got, seen)
        acc_total += acc_k
        cur = dict(cur, alpha=got)
    m.close()
    assert np.array_equal(acc, acc_total)
    assert seen == {True, False}


def test_sweep_step_by_step_and_captured(case):
    w, cw, lat, s = case
    m = make(w, cw, s)
    m.gibbs_sweep(1, first_counter=9)
    g = m.get_state()
    a3, _ = m.get_alpha_dirs()
    seen = set()
    assert rel(g["W"], gibbs.sample_W(lat, w.Y, w.X, s, SEED, 9, w.eps, prior="aniso")) <= 1e-8
    s1 = dict(s, W=g["W"])
    assert rel(g["A"], gibbs.sample_A(lat, w.Y, w.X, s1, SEED, 9, spatial=True)) <= 1e-8
    s1["A"] = g["A"]
    assert np.max(np.abs(g["lam"] / gibbs.sample_lambda(lat, w.Y, w.X, s1, SEED, 9) - 1)) <= 1e-10
    s1["lam"] = g["lam"]
    check_exchange(lat, m, s1, 9, a3, seen)
    m.close()
    s1["alpha"] = a3
    assert np.max(np.abs(g["beta"] / gibbs.sample_beta(lat, s1, SEED, 9) - 1)) <= 1e-10
    nd = w.neighbourhood // 2
    assert np.allclose(g["alpha"], a3[:, :nd].mean(axis=1), rtol=1e-15)
    runs = []
    for graph in (0, 1):
        mm = make(w, cw, s, use_graph=graph, delta=1e-10)
        mm.gibbs_sweep(3, first_counter=12)
        runs.append(dict(mm.get_state(), a3=mm.get_alpha_dirs()[0], acc=mm.get_alpha_dirs()[1]))
        mm.close()
    for k in runs[0]:
        assert np.array_equal(runs[0][k], runs[1][k]), k


def test_equal_alphas_are_the_graph_laplacian_prior():
    from paper_1606_00980_gb300.bfmri import Model
    w, cw = CASES["weighted3d_K4_P1"]
    rng = np.random.default_rng(75)
    s = state_for(w, rng)
    a = rng.uniform(0.3, 3.0, w.K)
    s["alpha"] = np.repeat(a[:, None], 3, axis=1)
    m = make(w, cw, s)
    u = Model.from_workload(w, seed=SEED, edge_weight=cw, precond=1, delta=1e-12)
    u.precompute_stats()
    u.set_state(W=s["W"], A=s["A"], lam=s["lam"], alpha=a, beta=s["beta"])
    x = rng.standard_normal((w.K, w.N))
    assert rel(m.apply_precision(0, x), u.apply_precision(0, x)) <= 1e-13
    Wa, _ = m.sample_W(counter=5)
    Wu, _ = u.sample_W(counter=5)
    m.close()
    u.close()
    assert rel(Wa, Wu) <= 1e-10


def test_options_and_calls_that_do_not_take_the_anisotropic_prior():
    from paper_1606_00980_gb300 import bfmri
    from paper_1606_00980_gb300.bfmri import Model, gibbs_sweep_group
    w, cw = CASES["small3d_K3_P2"]
    for bad in (dict(precond=bfmri.PRECOND_SSOR), dict(precond=bfmri.PRECOND_MULTIGRID),
                dict(precision=bfmri.PREC_MIXED), dict(precond=1, aniso_step=np.inf)):
        with pytest.raises(bfmri.BfmriError) as ei:
            Model.from_workload(w, w_prior=bfmri.PRIOR_ANISO, **bad)
        assert ei.value.status == -1
    u = Model.from_workload(w, precond=1)
    with pytest.raises(bfmri.BfmriError):
        u.set_alpha_dirs(np.ones((w.K, 3)))
    u.close()
    s = state_for(w, np.random.default_rng(76))
    ms = [make(w, cw, s), make(w, cw, s)]
    for v in (0.0, -1.0, np.nan):
        bad = np.ones((w.K, 3))
        bad[1, 2] = v
        with pytest.raises(bfmri.BfmriError):
            ms[0].set_alpha_dirs(bad)
    with pytest.raises(bfmri.BfmriError):
        ms[0].set_edge_factors(np.ones((3,) + np.asarray(w.mask).shape))
    with pytest.raises(bfmri.BfmriError):
        gibbs_sweep_group(ms, 1, 0)
    with pytest.raises(bfmri.BfmriError):
        ms[0].logdet_probe(0, 4, 100, counter=1)
    with pytest.raises(bfmri.BfmriError):
        ms[0].spvb_step(4, 1)
    for m in ms:
        m.close()
    mr = make(w, cw, s, precond=bfmri.PRECOND_RB_REDUCED)
    with pytest.raises(bfmri.BfmriError):
        mr.apply_preconditioner(0, np.ones((w.K, w.N)))
    mr.close()
