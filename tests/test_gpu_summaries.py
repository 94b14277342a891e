"""Posterior summaries through the C ABI against the FP64 oracle (needs a GB300).

* Chain summaries (Eq. MCMCPPM, Eq. MCMCjointPPM): the device accumulators over a chain's
  sweeps against the oracle's summary of the same W draws (read back after every sweep):
  exceedance counts and joint counts bit-exact (the contrast values round identically on
  both sides), mean and covariance within 1e-12 / 1e-9 relative. Captured-graph sweeps,
  asynchronous sweeps and grouped chains accumulate exactly what direct sweeps do.
* SVB summaries (Section 3.3) against the oracle over the handle's N_s samples.
* The unnormalised log joint posterior (Eq. UnnormalisedJointPosterior) of the current state,
  term by term, within 1e-10 relative of the oracle's direct time-series evaluation.
"""
import numpy as np
import pytest

from oracle import summaries
from oracle.lattice import Lattice
from paper_1606_00980_gb300 import synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def make(w, seed=123, **opts):
    from paper_1606_00980_gb300.bfmri import Model
    opts.setdefault("delta", 1e-10)
    m = Model.from_workload(w, seed=seed, **opts)
    m.precompute_stats()
    return m


def contrasts(w, W):
    """Three contrasts with thresholds inside the spread of their values, so that the
    counts are neither all zero nor all n."""
    K = w.K
    C = np.zeros((3, K))
    C[0, 0] = 1.0
    C[1, 0], C[1, 1 % K] = 1.0, -1.0
    C[2] = np.linspace(0.5, -0.5, K)
    vals = summaries.contrast_values(C, W)
    gamma = np.median(vals, axis=1)
    return C, gamma


def compare_chain(got, ref, exact_moments=False):
    assert got["n"] == ref["n"]
    assert np.array_equal(got["ppm"], ref["count"] / ref["n"])
    assert np.array_equal(got["joint_count"], ref["joint_count"])
    assert rel(got["mean"], ref["mean"]) <= 1e-12
    assert rel(got["cov"], ref["cov"]) <= 1e-9


W6 = synth.small3d(seed=51, dims=(11, 9, 7), K=6, P=3, T=60)
W3 = synth.small3d(seed=52, dims=(9, 8, 6), K=3, P=1, T=40)


@pytest.mark.parametrize("w", [W6, W3], ids=["K6_P3", "K3_P1"])
def test_chain_summary_matches_oracle(w):
    m = make(w)
    m.gibbs_sweep(3, 0)                                   # burn-in
    C, gamma = contrasts(w, m.get_state()["W"])
    E = np.array([0, 5, 17, w.N // 2, w.N - 1])
    m.summary_begin(C, gamma, joint_set=E)
    samples = []
    for s in range(12):
        m.gibbs_sweep(1, 3 + s)
        samples.append(m.get_state()["W"])
    got = m.summary_get()
    ref = summaries.chain_summary(samples, C, gamma, E)
    compare_chain(got, ref)
    assert 0 < ref["count"].sum() < ref["count"].size * 12
    # one-voxel joint set = that voxel's marginal count; no set = every sample
    m.summary_begin(C, gamma, joint_set=[E[2]])
    m.gibbs_sweep(4, 20)
    one = m.summary_get()
    assert np.array_equal(one["joint_count"], np.rint(one["ppm"][:, E[2]] * one["n"]).astype(np.int64))
    m.summary_begin(C, gamma)
    m.gibbs_sweep(2, 30)
    assert np.all(m.summary_get()["joint_count"] == 2)
    m.close()


def test_summary_add_and_state_errors():
    from paper_1606_00980_gb300 import bfmri
    w = W3
    m = make(w)
    with pytest.raises(bfmri.BfmriError) as ei:
        m.summary_add()
    assert ei.value.status == -8
    C, gamma = contrasts(w, w.W_true)
    m.summary_begin(C, gamma)
    with pytest.raises(bfmri.BfmriError):
        m.summary_get()                                   # no sample yet
    samples = []
    for s in range(3):
        m.sample_W(40 + s)
        m.summary_add()
        samples.append(m.get_state()["W"])
    compare_chain(m.summary_get(), summaries.chain_summary(samples, C, gamma))
    with pytest.raises(bfmri.BfmriError) as ei:
        m.summary_begin(np.ones((17, w.K)), np.zeros(17))
    assert ei.value.status == -1
    with pytest.raises(bfmri.BfmriError):
        m.summary_begin(C, gamma, joint_set=[w.N])
    m.summary_end()
    with pytest.raises(bfmri.BfmriError):
        m.summary_get()
    m.close()


@pytest.mark.parametrize("opts", [dict(), dict(precond=2)], ids=["bj", "ssor"])
def test_captured_and_asynchronous_sweeps_accumulate_like_direct_ones(opts):
    w = W6
    direct = make(w, **opts)
    graph = make(w, use_graph=1, **opts)
    for m in (direct, graph):
        m.gibbs_sweep(2, 0)                               # the graph is captured here
    C, gamma = contrasts(w, direct.get_state()["W"])
    E = np.arange(0, w.N, 7)
    for m in (direct, graph):
        m.summary_begin(C, gamma, joint_set=E)            # drops the captured graph
    for s in range(5):
        direct.gibbs_sweep(1, 2 + s)
    graph.gibbs_sweep(3, 2, info=False)
    info = graph.gibbs_sweep(2, 5)
    assert info.captured == 1
    a, b = direct.summary_get(), graph.summary_get()
    assert a["n"] == b["n"] == 5
    for key in ("mean", "cov_packed", "ppm", "joint_count"):
        assert np.array_equal(a[key], b[key]), key
    # closing the summary re-captures a sweep without the accumulation
    graph.summary_end()
    direct.summary_end()
    assert graph.gibbs_sweep(1, 7).captured == 1
    direct.gibbs_sweep(1, 7)
    assert np.array_equal(direct.get_state()["W"], graph.get_state()["W"])
    direct.close()
    graph.close()


def test_grouped_chains_accumulate_per_chain():
    from paper_1606_00980_gb300.bfmri import gibbs_sweep_group
    w = W6
    models = [make(w, seed=900 + c) for c in range(3)]
    gibbs_sweep_group(models, 2, 0)
    C, gamma = contrasts(w, models[0].get_state()["W"])
    E = [1, 2, 3, 40]
    for m in models[:2]:                                  # the third chain keeps no summary
        m.summary_begin(C, gamma, joint_set=E)
    samples = [[], []]
    for s in range(6):
        gibbs_sweep_group(models, 1, 2 + s)
        for c in range(2):
            samples[c].append(models[c].get_state()["W"])
    for c in range(2):
        compare_chain(models[c].summary_get(), summaries.chain_summary(samples[c], C, gamma, E))
    for m in models:
        m.close()


@pytest.mark.parametrize("precond", [0, 2])
def test_svb_summary_matches_oracle(precond):
    w = W3
    m = make(w, delta=1e-10, precond=precond)
    m.gibbs_sweep(2, 0)
    m.spvb_step(6, 3, extrapolate=False)
    C, gamma = contrasts(w, m.get_state()["W"])
    got = m.svb_summary(C, gamma)
    samples = [m.svb_sample(j)[0] for j in range(6)]
    ref = summaries.svb_summary(samples, C, gamma)
    assert rel(got["mean"], ref["mean"]) <= 1e-12
    assert rel(got["cov"], ref["cov"]) <= 1e-9
    assert np.max(np.abs(got["ppm"] - ref["ppm"])) <= 1e-9
    m.close()


@pytest.mark.parametrize("ar", ["spatial", "independent"])
@pytest.mark.parametrize("w", [W6, W3, synth.make_workload("p0", (6, 5, 4), np.ones((4, 5, 6), np.uint8), T=30, K=2,
                                                           P=0, neighbourhood=6, seed=23)],
                         ids=["K6_P3", "K3_P1", "K2_P0"])
def test_log_joint_matches_oracle(w, ar):
    from paper_1606_00980_gb300 import bfmri
    spatial = ar == "spatial"
    m = make(w, ar_prior=bfmri.AR_SPATIAL if spatial else bfmri.AR_INDEPENDENT)
    lat = Lattice(w.mask, w.neighbourhood)
    for s in range(3):
        if s:
            m.gibbs_sweep(1, s)
        got = m.log_joint()
        st = m.get_state()
        ref = summaries.log_joint(lat, w.Y, w.X, st, w.T, spatial_ar=spatial)
        scale = sum(abs(ref[k]) for k in ("loglik", "W_prior", "A_prior", "lambda_prior",
                                           "alpha_prior", "beta_prior"))
        for key in ref:
            assert abs(got[key] - ref[key]) <= 1e-10 * scale, (key, got[key], ref[key])
    m.close()
