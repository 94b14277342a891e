"""The C ABI library builds, loads without a GPU and exports every function include/bfmri.h
declares; the Python binding declares exactly that set (CPU only)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(bfmri_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1606_00980_gb300 import build
    build.build()
    from paper_1606_00980_gb300 import bfmri
    return bfmri.load_library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["bfmri_create", "bfmri_precompute_stats", "bfmri_sample_W",
                     "bfmri_gibbs_sweep", "bfmri_destroy", "bfmri_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in sorted(declared_functions()):
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_binding_matches_header(lib):
    from paper_1606_00980_gb300 import bfmri
    bound = {n for n, _, _ in bfmri.SIGNATURES}
    assert bound == declared_functions()


def test_default_options_without_gpu(lib):
    from paper_1606_00980_gb300 import bfmri
    o = bfmri.bfmri_default_options()
    assert (o.q1, o.q2, o.u1, o.u2, o.r1, o.r2) == (10.0, 0.1, 10.0, 0.1, 10000.0, 0.1)
    assert o.delta == 1e-8 and o.precond == bfmri.PRECOND_BLOCK_JACOBI
    assert o.debug_skip_block == -1 and o.inner_tol == 1e-6 and o.ssor_omega == 1.0
    assert list(o.edge_weight) == [1.0, 1.0, 1.0]
    # the trailing fields, read back through the same layout (a mismatch shows here first)
    assert o.w_prior == bfmri.PRIOR_UGL and o.pcg_lanes == 0 and o.aniso_step == 0.0
    assert o.mrhs_tile == 0 and o.stats_kernel == 0


def test_create_rejects_bad_arguments_without_touching_the_gpu(lib):
    """Host-side validation runs before any device call: these fail with INVALID_ARG."""
    import numpy as np
    from paper_1606_00980_gb300 import bfmri
    mask = np.ones((2, 3, 4), np.uint8)
    X = np.ones((20, 2))
    Y = np.ones((20, 24))
    cases = [((4, 3, 2, 5), mask, X, Y, 2, 1),      # bad neighbourhood
             ((4, 3, 2, 6), mask, X, Y, 13, 1),     # K too large
             ((4, 3, 2, 6), mask, X, Y, 2, 5),      # P too large
             ((4, 3, 2, 6), np.zeros_like(mask), X, Y, 2, 1)]   # empty mask
    for lat, m, x, y, K, P in cases:
        with pytest.raises(bfmri.BfmriError) as ei:
            bfmri.bfmri_create(lat, m, x[:, :K] if K <= 2 else np.ones((20, K)), y, K, P,
                               torch_memory=False)
        assert ei.value.status == -1
    for fields in (dict(precond=2, ssor_omega=2.0), dict(precond=2, ssor_omega=0.0),
                   dict(precond=5), dict(edge_weight=(1.0, 0.0, 1.0)),
                   dict(edge_weight=(1.0, 1.0, float("inf")))):
        o = bfmri.bfmri_default_options()
        for k, v in fields.items():
            setattr(o, k, v)
        with pytest.raises(bfmri.BfmriError) as ei:
            bfmri.bfmri_create((4, 3, 2, 6), mask, X, Y, 2, 1, opts=o, torch_memory=False)
        assert ei.value.status == -1
    Yn = Y.copy()
    Yn[3, 5] = np.nan
    with pytest.raises(bfmri.BfmriError) as ei:
        bfmri.bfmri_create((4, 3, 2, 6), mask, X, Yn, 2, 1, torch_memory=False)
    assert ei.value.status == -1 and "non-finite" in str(ei.value)
    # FP32 series, infinities, and a series long enough for the multi-threaded scan (the
    # offending value in its last block and in the middle)
    T = 200000
    XL = np.ones((T, 2))
    for dt in (np.float64, np.float32):
        for pos, val in (((3, 5), np.inf), ((T - 1, 23), -np.inf), ((T // 2, 11), np.nan)):
            YL = np.ones((T if pos[0] >= 20 else 20, 24), dt)
            YL[pos] = val
            with pytest.raises(bfmri.BfmriError) as ei:
                bfmri.bfmri_create((4, 3, 2, 6), mask, XL[:YL.shape[0]], YL, 2, 1, torch_memory=False)
            assert ei.value.status == -1 and "non-finite" in str(ei.value), (dt, pos)


def test_summary_bindings_marshal_without_a_gpu(lib):
    """The summary and synchronisation bindings build their ctypes arguments and reach the
    library, which rejects the NULL handle with INVALID_ARG before any device call."""
    import numpy as np
    from paper_1606_00980_gb300 import bfmri
    m = object.__new__(bfmri.Model)
    m.handle, m.lib, m.K, m.N, m.P, m._n_contrasts = None, lib, 3, 10, 1, 2
    calls = [lambda: m.summary_begin(np.ones((2, 3)), [0.1, 0.2], joint_set=[1, 2]),
             lambda: m.summary_begin(np.ones(3), 0.5),
             m.summary_add, m.summary_get, m.summary_end, m.log_joint, m.synchronize,
             lambda: m.svb_summary(np.ones((2, 3)), [0.1, 0.2])]
    for call in calls:
        with pytest.raises(bfmri.BfmriError) as ei:
            call()
        assert ei.value.status == -1


def test_prior_options_rejected_without_touching_the_gpu(lib):
    """The W-prior options are validated on the host at create: an unknown prior, the L'L and
    anisotropic priors with a solver they do not run on, and a non-finite proposal step."""
    import numpy as np
    from paper_1606_00980_gb300 import bfmri
    mask = np.ones((2, 3, 4), np.uint8)
    X = np.ones((20, 2))
    Y = np.ones((20, 24))
    bad = [dict(w_prior=3), dict(w_prior=-1),
           dict(w_prior=bfmri.PRIOR_LTL, precond=bfmri.PRECOND_SSOR),
           dict(w_prior=bfmri.PRIOR_LTL, precond=bfmri.PRECOND_RB_REDUCED),
           dict(w_prior=bfmri.PRIOR_LTL, precision=bfmri.PREC_MIXED),
           dict(w_prior=bfmri.PRIOR_ANISO, precond=bfmri.PRECOND_SSOR),
           dict(w_prior=bfmri.PRIOR_ANISO, precond=bfmri.PRECOND_MULTIGRID),
           dict(w_prior=bfmri.PRIOR_ANISO, precision=bfmri.PREC_MIXED),
           dict(w_prior=bfmri.PRIOR_ANISO, aniso_step=float("nan")),
           dict(w_prior=bfmri.PRIOR_ANISO, aniso_step=float("inf"))]
    for fields in bad:
        o = bfmri.bfmri_default_options()
        for k, v in fields.items():
            setattr(o, k, v)
        with pytest.raises(bfmri.BfmriError) as ei:
            bfmri.bfmri_create((4, 3, 2, 6), mask, X, Y, 2, 1, opts=o, torch_memory=False)
        assert ei.value.status == -1, fields


def test_prior_bindings_marshal_without_a_gpu(lib):
    """The per-edge factor and anisotropic-prior bindings build their ctypes arguments and
    reach the library, which rejects the NULL handle with INVALID_ARG before any device call."""
    import numpy as np
    from paper_1606_00980_gb300 import bfmri
    m = object.__new__(bfmri.Model)
    m.handle, m.lib, m.K, m.N, m.P, m.sites = None, lib, 3, 10, 1, 24
    calls = [lambda: m.set_edge_factors(np.ones((3, 24))), lambda: m.set_edge_factors(None),
             lambda: m.set_alpha_dirs(np.ones((3, 3))), m.get_alpha_dirs, m.aniso_last_step]
    for call in calls:
        with pytest.raises(bfmri.BfmriError) as ei:
            call()
        assert ei.value.status == -1
    with pytest.raises(ValueError):
        m.set_edge_factors(np.ones((3, 23)))
