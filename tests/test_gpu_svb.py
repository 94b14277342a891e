"""Spatial-VB step through the C ABI vs the FP64 oracle (needs a GB300).

Single-step parity as for the Gibbs sweep: the oracle replays each stage of an SVB iteration
from the GPU's outputs of the previous stages (W samples -> A samples -> E[lambda] ->
E[alpha], E[beta]); draws within 1e-8 relative L2 of the oracle's exact solves of the same
averaged systems with the same random numbers, means within 1e-10. A second iteration checks
that the random numbers are reused and the previous samples serve as warm starts. The
Appendix C extrapolation is checked for self-consistency with the oracle's rule.
"""
import numpy as np
import pytest

from oracle import gibbs, philox
from oracle.lattice import Lattice
from paper_1606_00980_gb300 import synth

pytestmark = pytest.mark.gpu

SEED = 99


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


def setup(spatial=True, K=3, P=2, **opts):
    from paper_1606_00980_gb300 import bfmri
    from paper_1606_00980_gb300.bfmri import Model
    w = synth.small3d(seed=41, dims=(8, 7, 6), K=K, P=P, T=45)
    lat = Lattice(w.mask, w.neighbourhood)
    rng = np.random.default_rng(8)
    s = dict(W=w.W_true + 0.1 * rng.standard_normal(w.W_true.shape), A=w.A_true.copy(),
             lam=rng.uniform(0.5, 2.0, w.N), alpha=rng.uniform(0.3, 3.0, K),
             beta=rng.uniform(2.0, 9.0, P))
    m = Model.from_workload(w, delta=1e-12, seed=SEED,
                            ar_prior=bfmri.AR_SPATIAL if spatial else bfmri.AR_INDEPENDENT, **opts)
    m.precompute_stats()
    m.set_state(W=s["W"], A=s["A"], lam=s["lam"], alpha=s["alpha"], beta=s["beta"])
    return w, lat, s, m


@pytest.mark.parametrize("precond", [0, 2, 3])
@pytest.mark.parametrize("spatial", [True, False])
def test_svb_step_single_step_parity(spatial, precond):
    """precond 0: block-Jacobi multi-RHS solves; 2: red-black SSOR; 3: the reduced
    red-black system."""
    w, lat, s, m = setup(spatial, precond=precond)
    Ns, c = 4, 11
    avb, bvb, info = m.spvb_step(Ns, c, extrapolate=False)
    Wg, Ag = zip(*[m.svb_sample(j) for j in range(Ns)])
    Bd, bw = gibbs.svb_w_system(w.Y, w.X, [s["A"]] * Ns, s["lam"], w.eps)
    Wo = gibbs.svb_draw(lat, Bd, bw, s["alpha"], SEED, c, philox.TAG_W, Ns)
    for j in range(Ns):
        assert rel(Wg[j], Wo[j]) <= 1e-8
    assert rel(Wg[0], Wg[1]) > 1e-3          # different random numbers per sample
    Ja, ba = gibbs.svb_a_system(w.Y, w.X, list(Wg), s["lam"], w.P)
    Ao = gibbs.svb_draw(lat, Ja, ba, s["beta"] if spatial else np.zeros(w.P), SEED, c,
                        philox.TAG_A, Ns)
    for j in range(Ns):
        assert rel(Ag[j], Ao[j]) <= 1e-8
    st = m.get_state()
    lam_o = gibbs.svb_lambda_mean(w.Y, w.X, list(Wg), list(Ag))
    assert np.max(np.abs(st["lam"] / lam_o - 1)) <= 1e-10
    a_o, _ = gibbs.svb_hyper_mean(lat, list(Wg), 10.0, 0.1)
    assert np.max(np.abs(avb / a_o - 1)) <= 1e-10
    assert np.allclose(st["alpha"], avb, rtol=0, atol=0)      # no extrapolation requested
    if spatial:
        b_o, _ = gibbs.svb_hyper_mean(lat, list(Ag), 10000.0, 0.1)
        assert np.max(np.abs(bvb / b_o - 1)) <= 1e-10
    # second iteration: the same random numbers, the first iteration's samples as start values
    st1 = m.get_state()
    avb2, _, info2 = m.spvb_step(Ns, c, extrapolate=False)
    Wg2 = [m.svb_sample(j)[0] for j in range(Ns)]
    Bd2, bw2 = gibbs.svb_w_system(w.Y, w.X, list(Ag), st1["lam"], w.eps)
    Wo2 = gibbs.svb_draw(lat, Bd2, bw2, st1["alpha"], SEED, c, philox.TAG_W, Ns)
    for j in range(Ns):
        assert rel(Wg2[j], Wo2[j]) <= 1e-8
    # the same second iteration from cold (zero) samples needs more PCG iterations
    for j in range(Ns):
        m.svb_set_sample(j, W=np.zeros((w.K, w.N)), A=Ag[j])
    m.set_state(lam=st1["lam"], alpha=st1["alpha"], beta=st1["beta"] if w.P else None)
    _, _, info_cold = m.spvb_step(Ns, c, extrapolate=False)
    Wc = [m.svb_sample(j)[0] for j in range(Ns)]
    for j in range(Ns):
        assert rel(Wc[j], Wo2[j]) <= 1e-8
    assert info2.pcg_iterations_W < info_cold.pcg_iterations_W
    m.close()


def test_svb_extrapolation_follows_appendix_c_rule():
    w, lat, s, m = setup(True)
    used, vbs = [], []
    for it in range(3):
        avb, bvb, info = m.spvb_step(3, 5, extrapolate=True)
        vbs.append(avb.copy())
        used.append(m.get_state()["alpha"].copy())
        assert info.extrapolated == (1 if it == 2 else 0)
    ref = gibbs.svb_extrapolate((used[0], used[1]), vbs[2])
    assert np.allclose(used[2], ref, rtol=1e-12)
    assert np.allclose(used[0], vbs[0]) and np.allclose(used[1], vbs[1])
    m.close()
