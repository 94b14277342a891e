"""Failure detection through status codes, with no GPU fault (needs a GB300).

* A grid barrier whose wait runs out: a test hook keeps one CTA from arriving; every other
  CTA gives up after the (shortened) limit, the call returns BFMRI_ERR_TIMEOUT, and the
  context stays usable: the next call succeeds and matches a fresh handle.
* A singular data block (an all-zero design column, no ridge: a zero pivot): BFMRI_ERR_NOT_SPD.
* An iteration cap below what the tolerance needs: BFMRI_ERR_NOT_CONVERGED.
* Asynchronous sweeps (no host wait): their errors and counts are read later.
* Checkpoint/resume: a chain stopped after s sweeps and resumed from its saved state in a new
  handle continues bit-identically (counter-based random numbers).
"""
import numpy as np
import pytest

from paper_1606_00980_gb300 import synth

pytestmark = pytest.mark.gpu


def model(w, **opts):
    from paper_1606_00980_gb300.bfmri import Model
    opts.setdefault("seed", 31)
    m = Model.from_workload(w, **opts)
    m.precompute_stats()
    return m


@pytest.mark.parametrize("variant", ["auto", "streaming"])
def test_barrier_timeout_is_reported_and_recoverable(variant):
    from paper_1606_00980_gb300 import bfmri
    w = synth.small3d(seed=3, dims=(12, 11, 9), K=3, P=1, T=40)
    pv = bfmri.PCG_AUTO if variant == "auto" else bfmri.PCG_STREAMING
    ref = model(w, pcg_variant=pv)
    # the hook fires on the first solve: CTA 0 never reaches its first barrier
    m = model(w, barrier_timeout_s=0.2, pcg_variant=pv, debug_skip_block=0)
    with pytest.raises(bfmri.BfmriError) as ei:
        m.sample_W(1)
    assert ei.value.status == -5
    # the hook fires once; the handle and the context remain usable
    W, info = m.sample_W(2)
    W_ref, _ = ref.sample_W(2)
    assert np.array_equal(W, W_ref)
    m.close()
    ref.close()


def test_singular_block_reports_not_spd():
    from paper_1606_00980_gb300 import bfmri
    w = synth.small3d(seed=4, dims=(6, 6, 5), K=3, P=0, T=30)
    w.X[:, 1] = 0.0                       # a zero column: X'X has an exactly zero pivot
    m = model(w, eps=0.0)
    with pytest.raises(bfmri.BfmriError) as ei:
        m.sample_W(1)
    assert ei.value.status == -3 and "voxel" in str(ei.value)
    m.close()


def test_iteration_cap_reports_not_converged():
    from paper_1606_00980_gb300 import bfmri
    w = synth.small3d(seed=5, dims=(9, 9, 7), K=3, P=1, T=40)
    m = model(w, max_iter=2, delta=1e-12)
    with pytest.raises(bfmri.BfmriError) as ei:
        m.sample_W(1)
    assert ei.value.status == -4
    m.close()


def test_checkpoint_resume_is_bitwise():
    w = synth.small3d(seed=6, dims=(9, 8, 6), K=3, P=2, T=40)
    full = model(w, delta=1e-10)
    full.gibbs_sweep(5, 100)
    end = full.get_state()
    full.close()
    first = model(w, delta=1e-10)
    first.gibbs_sweep(2, 100)
    ckpt = first.get_state()
    first.close()
    resumed = model(w, delta=1e-10)
    resumed.set_state(W=ckpt["W"], A=ckpt["A"], lam=ckpt["lam"], alpha=ckpt["alpha"], beta=ckpt["beta"])
    resumed.gibbs_sweep(3, 102)
    got = resumed.get_state()
    resumed.close()
    for k in end:
        assert np.array_equal(got[k], end[k]), k


def test_asynchronous_sweeps_match_and_report_at_synchronize():
    """Sweeps enqueued without info (no host wait) give the same states as synchronous
    sweeps; synchronize() reports the PCG counts of the whole asynchronous span."""
    w = synth.small3d(seed=7, dims=(10, 9, 7), K=3, P=2, T=40)
    sync = model(w, delta=1e-10)
    asyn = model(w, delta=1e-10)
    total_w = total_a = 0
    for s in range(4):
        inf = sync.gibbs_sweep(1, 50 + s)
        total_w += inf.pcg_iterations_W
        total_a += inf.pcg_iterations_A
        asyn.gibbs_sweep(1, 50 + s, info=False)
    got = asyn.synchronize()
    assert (got.pcg_iterations_W, got.pcg_iterations_A) == (total_w, total_a)
    a, b = sync.get_state(), asyn.get_state()
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    # nothing unread now: a second synchronize reports no work
    again = asyn.synchronize()
    assert (again.pcg_iterations_W, again.pcg_iterations_A) == (0, 0)
    sync.close()
    asyn.close()


def test_asynchronous_sweep_error_is_reported_later():
    """An iteration cap hit inside an asynchronous sweep: the enqueueing call succeeds, the
    next synchronising call raises NOT_CONVERGED, and the one after it starts clean."""
    from paper_1606_00980_gb300 import bfmri
    w = synth.small3d(seed=5, dims=(9, 9, 7), K=3, P=1, T=40)
    m = model(w, max_iter=2, delta=1e-12)
    m.gibbs_sweep(1, 0, info=False)
    with pytest.raises(bfmri.BfmriError) as ei:
        m.synchronize()
    assert ei.value.status == -4
    assert m.synchronize().pcg_iterations_W == 0
    m.close()
