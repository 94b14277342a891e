"""Serving (continuous admission of subjects into slots under a memory budget), needs a GB300.

Each request's result must not depend on what else runs: the same request alone and in the
mix gives bit-identical W and alpha (fixed grids under the slot's SM budget, fixed-order
reductions, counter-based random numbers), and equals the single-handle API with the same
options. The device-memory estimate of the requests in flight never exceeds the budget.
"""
import numpy as np
import pytest

from paper_1606_00980_gb300 import synth

pytestmark = pytest.mark.gpu


def requests():
    out = []
    for i, (dims, K, P, T) in enumerate([((9, 8, 6), 3, 1, 40), ((12, 10, 8), 4, 2, 50),
                                          ((7, 7, 5), 2, 3, 36), ((14, 12, 9), 5, 2, 60),
                                          ((10, 9, 7), 6, 3, 48), ((8, 8, 8), 4, 1, 44)]):
        out.append(synth.small3d(seed=100 + i, dims=dims, K=K, P=P, T=T))
    return out


def run(server, ws, n_sweeps=3):
    from paper_1606_00980_gb300 import bfmri
    tickets = [server.submit(w, n_sweeps, first_counter=7 * i, precision=bfmri.PREC_MIXED,
                             delta=1e-8, seed=555 + i) for i, w in enumerate(ws)]
    return [server.poll(t) for t in tickets]


def test_result_is_the_same_alone_and_in_the_mix():
    from paper_1606_00980_gb300 import bfmri
    ws = requests()
    s = bfmri.Server(budget_bytes=8 << 30, slots=3, sm_budget=48)
    mixed = run(s, ws)
    st = s.stats()
    s.close()
    assert st["peak_running"] >= 2          # requests overlapped
    for i, w in enumerate(ws):
        s1 = bfmri.Server(budget_bytes=8 << 30, slots=3, sm_budget=48)
        tick = s1.submit(w, 3, first_counter=7 * i, precision=bfmri.PREC_MIXED, delta=1e-8,
                         seed=555 + i)
        alone = s1.poll(tick)
        s1.close()
        assert np.array_equal(alone["W"], mixed[i]["W"])
        assert np.array_equal(alone["alpha"], mixed[i]["alpha"])
        # and the same as the single-handle API with the same options
        m = bfmri.Model.from_workload(w, precision=bfmri.PREC_MIXED, delta=1e-8, seed=555 + i,
                                      sm_budget=48)
        m.precompute_stats()
        m.gibbs_sweep(3, 7 * i)
        assert np.array_equal(m.get_state()["W"], mixed[i]["W"])
        m.close()


def test_admission_respects_the_memory_budget():
    from paper_1606_00980_gb300 import bfmri
    ws = requests()
    lib = bfmri.load_library()
    sizes = [lib.bfmri_request_device_bytes(w.N, w.T, w.K, w.P, bfmri.BFMRI_F64, bfmri.PREC_MIXED)
             for w in ws]
    budget = int(max(sizes) * 1.6)          # at most one large request at a time
    s = bfmri.Server(budget_bytes=budget, slots=4, sm_budget=38)
    res = run(s, ws)
    st = s.stats()
    s.close()
    assert st["peak_bytes"] <= budget
    assert all(r["end_s"] >= r["start_s"] >= r["submit_s"] for r in res)
    with pytest.raises(bfmri.BfmriError):
        s2 = bfmri.Server(budget_bytes=min(sizes) // 2, slots=1)
        try:
            s2.submit(ws[0], 1)
        finally:
            s2.close()


def bench_like_pool():
    """Subjects shaped like the serving benchmark's pool at sizes the oracle solves in
    seconds: every K appears with two different (T, P), Y is FP32, and with four SMs per slot
    the larger subjects exceed one CTA per SM, so their W and A systems run the streaming
    mixed-precision solver on the reduced red-black system while the smaller ones run the
    resident one."""
    import numpy as np
    specs = [(1300, 4, 40, 1), (2600, 4, 80, 2), (1800, 6, 60, 3), (2400, 6, 120, 2),
             (900, 8, 50, 1), (2200, 8, 90, 3)]
    out = []
    for i, (n, K, T, P) in enumerate(specs):
        w = synth.request_workload(seed=700 + i, N_target=n, K=K, T=T, P=P)
        w.Y = w.Y.astype(np.float32)
        out.append(w)
    return out


def test_bench_shaped_mix_matches_alone_and_the_oracle():
    """Four slots of four SMs, reduced red-black preconditioner, mixed precision at
    delta = 1e-8 (the serving benchmark's options): every request's W is bit-identical alone
    and in the mix, and a one-sweep request's W equals the oracle's exact draw of the same
    perturbed system (Algorithm 2, from the prior-mean start state) to 1e-5 relative L2."""
    from oracle import gibbs, model, philox
    from oracle.lattice import Lattice
    from paper_1606_00980_gb300 import bfmri
    pool = bench_like_pool()
    opts = dict(precision=bfmri.PREC_MIXED, delta=1e-8, inner_tol=1e-6,
                precond=bfmri.PRECOND_RB_REDUCED)
    reqs = []                      # (pool index, sweeps, first counter, seed)
    for rep in range(2):
        for i in range(len(pool)):
            reqs.append((i, 1 if rep == 0 else 3, 11 * i + rep, 900 + 10 * i + rep))
    s = bfmri.Server(budget_bytes=8 << 30, slots=4, sm_budget=4)
    try:
        tickets = [s.submit(pool[i], n, first_counter=c, seed=sd, **opts) for i, n, c, sd in reqs]
        mixed = [s.poll(t) for t in tickets]
        st = s.stats()
    finally:
        s.close()
    assert st["peak_running"] >= 3
    for (i, n, c, sd), got in zip(reqs, mixed):
        s1 = bfmri.Server(budget_bytes=8 << 30, slots=1, sm_budget=4)
        try:
            alone = s1.poll(s1.submit(pool[i], n, first_counter=c, seed=sd, **opts))
        finally:
            s1.close()
        assert np.array_equal(alone["W"], got["W"]), (i, n)
        assert np.array_equal(alone["alpha"], got["alpha"]), (i, n)
        if n != 1:
            continue
        w = pool[i]
        lat = Lattice(w.mask, w.neighbourhood)
        state = gibbs.default_state(w.K, w.P, w.N)
        Y = w.Y.astype(np.float64)
        Bd, bw = model.w_blocks_direct(Y, w.X, state["A"], state["lam"], w.eps)
        W_ref, _ = gibbs.draw_gmrf(lat, Bd, bw, state["alpha"], seed=sd, counter=c,
                                   tag=philox.TAG_W)
        err = np.linalg.norm(got["W"] - W_ref) / np.linalg.norm(W_ref)
        assert err <= 1e-5, (i, err)


def test_admission_estimate_covers_every_allocation():
    """bfmri_request_device_bytes counts every allocation a request makes: for each subject of
    the bench-shaped pool (FP32 Y, mixed precision) and for FP64 requests, the estimate is at
    least the handle's own peak and the pool's high-water mark for that request run alone,
    and not far above them (the margin is 1/32 + 2 MiB)."""
    from paper_1606_00980_gb300 import bfmri
    lib = bfmri.load_library()
    pool = bench_like_pool()
    for w in pool:
        for prec in (bfmri.PREC_MIXED, bfmri.PREC_FP64):
            ydt = bfmri.BFMRI_F32 if w.Y.dtype == np.float32 else bfmri.BFMRI_F64
            est = lib.bfmri_request_device_bytes(w.N, w.T, w.K, w.P, ydt, prec)
            m = bfmri.Model.from_workload(w, precision=prec, delta=1e-8,
                                          precond=bfmri.PRECOND_RB_REDUCED, sm_budget=4)
            m.precompute_stats()
            m.gibbs_sweep(2, 0)
            now, peak = m.device_bytes()
            m.close()
            assert peak <= est <= peak * 33 // 32 + (2 << 20) + 4096, (w.N, prec, peak, est)
            with bfmri.Server(budget_bytes=8 << 30, slots=1, sm_budget=4) as s:
                s.pool_usage(reset=True)
                s.poll(s.submit(w, 2, first_counter=0, seed=3, precision=prec, delta=1e-8,
                                precond=bfmri.PRECOND_RB_REDUCED))
                high = s.pool_usage()
            assert high <= est, (w.N, prec, high, est)


def test_multigrid_request_estimate_covers_the_hierarchy():
    """A multigrid request builds its hierarchy on the first solve; the server's estimate for
    it (bfmri_result.device_bytes) adds those bytes, so it stays at least the handle's own
    peak and the pool's high-water mark for that request run alone. It counts Y and the
    hierarchy together although the statistics step releases Y before the first solve, so it
    may exceed the peak by Y's bytes beyond the usual margin."""
    from paper_1606_00980_gb300 import bfmri
    for w in bench_like_pool()[:3]:
        m = bfmri.Model.from_workload(w, precision=bfmri.PREC_FP64, delta=1e-8,
                                      precond=bfmri.PRECOND_MULTIGRID, sm_budget=4)
        m.precompute_stats()
        m.gibbs_sweep(2, 0)
        _, peak = m.device_bytes()
        m.close()
        with bfmri.Server(budget_bytes=8 << 30, slots=1, sm_budget=4) as s:
            s.pool_usage(reset=True)
            res = s.poll(s.submit(w, 2, first_counter=0, seed=3, precision=bfmri.PREC_FP64,
                                  delta=1e-8, precond=bfmri.PRECOND_MULTIGRID))
            high = s.pool_usage()
        est = res["device_bytes"]
        y_bytes = w.Y.size * w.Y.itemsize
        assert peak <= est <= peak * 33 // 32 + (2 << 20) + y_bytes + 8192, (w.N, peak, est)
        assert high <= est, (w.N, high, est)


def test_prior_request_estimates_cover_their_buffers():
    """Requests with the L'L prior (its [K][ld] plane for L v) and with the anisotropic prior
    (the exchange step's auxiliary field, its small per-k arrays and the direction partials):
    the server's estimate (bfmri_result.device_bytes) stays at least the handle's own peak and
    the pool's high-water mark for the request run alone, and within the usual margin of the
    peak (1/32 + 2 MiB, plus the 1024-row bound the server takes for the partials)."""
    from paper_1606_00980_gb300 import bfmri
    cases = [dict(w_prior=bfmri.PRIOR_LTL, precond=bfmri.PRECOND_BLOCK_JACOBI),
             dict(w_prior=bfmri.PRIOR_ANISO, precond=bfmri.PRECOND_RB_REDUCED)]
    for w in bench_like_pool()[:3]:
        for opts in cases:
            m = bfmri.Model.from_workload(w, precision=bfmri.PREC_FP64, delta=1e-8, sm_budget=4, **opts)
            m.precompute_stats()
            m.gibbs_sweep(2, 0)
            _, peak = m.device_bytes()
            m.close()
            with bfmri.Server(budget_bytes=8 << 30, slots=1, sm_budget=4) as s:
                s.pool_usage(reset=True)
                res = s.poll(s.submit(w, 2, first_counter=0, seed=3, precision=bfmri.PREC_FP64,
                                      delta=1e-8, **opts))
                high = s.pool_usage()
            est = res["device_bytes"]
            slack = 3 * 1024 * max(w.K, w.P) * 8 + 8192
            assert peak <= est <= peak * 33 // 32 + (2 << 20) + slack, (w.N, opts, peak, est)
            assert high <= est, (w.N, opts, high, est)
