"""Log-determinant and trace probes through the C ABI vs the FP64 oracle (needs a GB300).

Per probe, the GPU's Lanczos quadrature from the multi-right-hand-side PCG coefficients is
compared with the oracle's exact v' log(C) v (dense eigendecomposition); with the probe
solves run to relative residual 1e-12 the quadrature is converged to ~1e-8 relative. The
trace terms are compared with the oracle's exact per-probe values, and the estimates with
the exact log det and traces within 5 standard errors.
"""
import numpy as np
import pytest

from oracle import model, probes
from oracle.lattice import Lattice
from paper_1606_00980_gb300 import synth

pytestmark = pytest.mark.gpu

SEED = 777


def make(w, state, **opts):
    from paper_1606_00980_gb300.bfmri import Model
    opts.setdefault("delta", 1e-12)
    m = Model.from_workload(w, seed=SEED, **opts)
    m.precompute_stats()
    m.set_state(W=state["W"], A=state["A"], lam=state["lam"], alpha=state["alpha"],
                beta=state["beta"] if w.P > 0 else None)
    return m


CASES = {
    "small3d_K3_P2": lambda: synth.small3d(seed=31, dims=(8, 7, 5), K=3, P=2, T=40),
    "slice2d_K2_P1": lambda: synth.make_workload("slice", (11, 9, 1), synth.circle_mask(11, 9, 4.6),
                                                 T=40, K=2, P=1, neighbourhood=4, seed=32,
                                                 ar_uniform=(0.1, 0.4), eps=1e-6),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("which", [0, 1])
@pytest.mark.parametrize("variant", ["pcg", "nopre", "fp32"])
def test_logdet_probe_matches_oracle(name, which, variant):
    """fp32: the mixed-precision handle runs the probe solves in FP32 to delta 1e-5; the
    per-probe quadrature then agrees with the exact value to 1e-4 and the traces to 1e-3."""
    from paper_1606_00980_gb300 import bfmri
    w = CASES[name]()
    lat = Lattice(w.mask, w.neighbourhood)
    rng = np.random.default_rng(4)
    s = dict(W=w.W_true + 0.1 * rng.standard_normal(w.W_true.shape), A=w.A_true,
             lam=rng.uniform(0.5, 2.0, w.N), alpha=rng.uniform(0.3, 3.0, w.K),
             beta=rng.uniform(2.0, 9.0, w.P))
    extra = dict(precision=bfmri.PREC_MIXED, delta=1e-5) if variant == "fp32" else {}
    m = make(w, s, precond=bfmri.PRECOND_NONE if variant == "nopre" else bfmri.PRECOND_BLOCK_JACOBI,
             **extra)
    n_probes = 12
    res = m.logdet_probe(which, n_probes, 2000, counter=6)
    D = w.K if which == 0 else w.P
    if which == 0:
        Bd, _ = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"], w.eps)
        scale = s["alpha"]
    else:
        Bd, _ = model.a_blocks_direct(w.Y, w.X, s["W"], s["lam"], w.P)
        scale = s["beta"]
    V = probes.probe_vectors(lat, D, n_probes, SEED, 6)
    if variant == "nopre":
        # no preconditioner: M = I, C = B~
        eye = np.broadcast_to(np.eye(D), Bd.shape)
        B = model.precision(lat, Bd, scale).toarray()
        lam, Q = np.linalg.eigh(B)
        quad = np.array([np.sum((Q.T @ model.kmajor(v)) ** 2 * np.log(lam)) for v in V])
        ldm = 0.0
        ldb = float(np.sum(np.log(lam)))
        Dw = lat.D().toarray()
        tr = np.array([[float(model.kmajor(v).reshape(D, -1)[k] @ (Dw @ np.linalg.solve(
            B, model.kmajor(v)).reshape(D, -1)[k])) for k in range(D)] for v in V])
    else:
        ldm, quad, tr, ldb = probes.exact_probe_terms(lat, Bd, scale, V)
    got = res["per_probe"]
    tq, tt = (1e-4, 1e-3) if variant == "fp32" else (1e-6, 1e-8)
    assert np.max(np.abs(got - quad) / np.abs(quad)) <= tq
    assert abs(res["logdet"] - (ldm + quad.mean())) <= tq * abs(ldm + quad.mean()) + 1e-6
    assert np.allclose(res["traces"], tr.mean(axis=0), rtol=tt, atol=tt * np.abs(tr).mean())
    assert np.all(res["iterations"] > 0)
    assert abs(res["logdet"] - ldb) <= 5 * max(res["stderr"], 1e-9) + 1e-6 * abs(ldb)
    m.close()


@pytest.mark.parametrize("tile", [2, 4])
@pytest.mark.parametrize("which", [0, 1])
def test_tiled_fp32_probes_match_oracle(tile, which):
    """FP32 probe solves with 2 or 4 right-hand sides interleaved per thread (the tile the
    autotuner chooses among): per-probe quadrature within 1e-4 of the exact value, traces
    within 1e-3, and the tile reported back."""
    from paper_1606_00980_gb300 import bfmri
    w = CASES["small3d_K3_P2"]()
    lat = Lattice(w.mask, w.neighbourhood)
    rng = np.random.default_rng(4)
    s = dict(W=w.W_true + 0.1 * rng.standard_normal(w.W_true.shape), A=w.A_true,
             lam=rng.uniform(0.5, 2.0, w.N), alpha=rng.uniform(0.3, 3.0, w.K),
             beta=rng.uniform(2.0, 9.0, w.P))
    m = make(w, s, precond=bfmri.PRECOND_BLOCK_JACOBI, precision=bfmri.PREC_MIXED, delta=1e-5,
             mrhs_tile=tile)
    n_probes = 12
    res = m.logdet_probe(which, n_probes, 2000, counter=6)
    assert m.probe_tuning()[0] == tile
    m.close()
    D = w.K if which == 0 else w.P
    if which == 0:
        Bd, _ = model.w_blocks_direct(w.Y, w.X, s["A"], s["lam"], w.eps)
        scale = s["alpha"]
    else:
        Bd, _ = model.a_blocks_direct(w.Y, w.X, s["W"], s["lam"], w.P)
        scale = s["beta"]
    V = probes.probe_vectors(lat, D, n_probes, SEED, 6)
    ldm, quad, tr, ldb = probes.exact_probe_terms(lat, Bd, scale, V)
    assert np.max(np.abs(res["per_probe"] - quad) / np.abs(quad)) <= 1e-4
    assert np.allclose(res["traces"], tr.mean(axis=0), rtol=1e-3, atol=1e-3 * np.abs(tr).mean())


def test_autotuner_times_every_tile_and_keeps_the_fastest():
    from paper_1606_00980_gb300 import bfmri
    w = synth.small3d(seed=33, dims=(9, 8, 7), K=4, P=1, T=40)
    rng = np.random.default_rng(5)
    s = dict(W=w.W_true, A=w.A_true, lam=rng.uniform(0.5, 2.0, w.N),
             alpha=rng.uniform(0.3, 3.0, w.K), beta=rng.uniform(2.0, 9.0, w.P))
    m = make(w, s, precond=bfmri.PRECOND_BLOCK_JACOBI, precision=bfmri.PREC_MIXED, delta=1e-5)
    r1 = m.logdet_probe(0, 8, 2000, counter=3)
    tile, ms = m.probe_tuning()
    assert all(t > 0 for t in ms) and tile in (1, 2, 4)
    assert ms[(1, 2, 4).index(tile)] == min(ms)
    r2 = m.logdet_probe(0, 8, 2000, counter=3)          # cached: same tile, no new timing
    assert m.probe_tuning()[0] == tile
    assert np.array_equal(r1["per_probe"], r2["per_probe"])
    m.close()
