"""Gibbs sweeps replayed from a captured CUDA graph (options.use_graph) against the same
sweeps launched directly: the same kernels with the same arguments and the same draw
counters, so the states agree bitwise, sweep after sweep and across calls (needs a GB300)."""
import numpy as np
import pytest

from paper_1606_00980_gb300 import synth

pytestmark = pytest.mark.gpu


def make(w, **opts):
    from paper_1606_00980_gb300.bfmri import Model
    m = Model.from_workload(w, seed=4321, delta=1e-10, **opts)
    m.precompute_stats()
    return m


CASES = {
    "resident_fp64_bj": dict(),
    "resident_fp64_ssor": dict(precond=2),
    "streaming_fp64_ssor": dict(precond=2, pcg_variant=1),
    "resident_mixed_ssor": dict(precond=2, precision=1),
    "resident_fp64_reduced": dict(precond=3),
    "resident_mixed_reduced": dict(precond=3, precision=1),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_captured_sweeps_equal_direct_launches(name):
    w = synth.small3d(seed=41, dims=(13, 11, 7), K=6, P=3, T=60)
    direct = make(w, **CASES[name])
    graph = make(w, use_graph=1, **CASES[name])
    for first, n in ((3, 4), (7, 3), (20, 1)):
        a = direct.gibbs_sweep(n, first)
        b = graph.gibbs_sweep(n, first)
        assert a.captured == 0
        assert b.captured == 1, graph.lib.bfmri_last_error(graph.handle)
        assert (a.pcg_iterations_W, a.pcg_iterations_A) == (b.pcg_iterations_W, b.pcg_iterations_A)
        sa, sb = direct.get_state(), graph.get_state()
        for key in ("W", "A", "lam", "alpha", "beta"):
            assert np.array_equal(sa[key], sb[key]), key
    direct.close()
    graph.close()


def test_graph_mode_is_skipped_while_profiling():
    w = synth.small3d(seed=42, dims=(8, 8, 6), K=3, P=2, T=40)
    m = make(w, use_graph=1, profile=1)
    info = m.gibbs_sweep(2, 0)
    assert info.captured == 0
    m.close()
