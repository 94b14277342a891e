"""Python binding of the bfmri C ABI (include/bfmri.h): argument marshalling only.

Every step of the sampler runs in the CUDA library ``_lib/libbfmri.so``; this module only
converts numpy arrays to pointers, routes the library's device allocations to PyTorch's
caching allocator, and passes PyTorch's current CUDA stream. There is no CPU fallback:
if the library is missing, ``load_library`` raises.

The function names are those of the C ABI; ``Model`` is a small convenience wrapper that
owns a handle.
"""
from __future__ import annotations

import atexit
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libbfmri.so")

BFMRI_OK = 0
STATUS_NAMES = {0: "OK", -1: "INVALID_ARG", -2: "OOM", -3: "NOT_SPD", -4: "NOT_CONVERGED",
                -5: "TIMEOUT", -6: "CUDA", -7: "INTERNAL", -8: "STATE"}
BFMRI_F32, BFMRI_F64 = 0, 1
PRECOND_NONE, PRECOND_BLOCK_JACOBI, PRECOND_SSOR, PRECOND_RB_REDUCED, PRECOND_MULTIGRID = 0, 1, 2, 3, 4
PRIOR_UGL, PRIOR_LTL, PRIOR_ANISO = 0, 1, 2
PREC_FP64, PREC_MIXED = 0, 1
AR_SPATIAL, AR_INDEPENDENT = 0, 1
Y_MASKED, Y_LATTICE = 0, 1
PCG_AUTO, PCG_STREAMING = 0, 1
STATS_AUTO, STATS_FP64, STATS_TENSOR = 0, 1, 2

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class bfmri_lattice(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("neighbourhood", C.c_int)]


class bfmri_options(C.Structure):
    _fields_ = [("q1", C.c_double), ("q2", C.c_double), ("u1", C.c_double), ("u2", C.c_double),
                ("r1", C.c_double), ("r2", C.c_double), ("eps", C.c_double),
                ("delta", C.c_double), ("max_iter", C.c_int), ("precond", C.c_int),
                ("precision", C.c_int), ("ar_prior", C.c_int), ("y_layout", C.c_int),
                ("inner_tol", C.c_double), ("seed", C.c_uint64), ("stream_id", C.c_uint32),
                ("cuda_stream", C.c_void_p), ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN),
                ("alloc_ctx", C.c_void_p), ("barrier_timeout_s", C.c_double),
                ("debug_skip_block", C.c_int), ("profile", C.c_int), ("pcg_variant", C.c_int),
                ("sm_budget", C.c_int), ("ssor_omega", C.c_double),
                ("use_graph", C.c_int), ("edge_weight", C.c_double * 3),
                ("stats_kernel", C.c_int), ("mrhs_tile", C.c_int),
                ("w_prior", C.c_int), ("pcg_lanes", C.c_int), ("aniso_step", C.c_double)]


class bfmri_solve_info(C.Structure):
    _fields_ = [("iterations", C.c_int), ("refinements", C.c_int),
                ("rel_residual", C.c_double), ("rel_residual0", C.c_double)]


class bfmri_svb_info(C.Structure):
    _fields_ = [("iteration", C.c_int), ("samples", C.c_int), ("pcg_iterations_W", C.c_longlong),
                ("pcg_iterations_A", C.c_longlong), ("max_rel_residual_W", C.c_double),
                ("extrapolated", C.c_int)]


class bfmri_sweep_info(C.Structure):
    _fields_ = [("sweeps", C.c_int), ("pcg_iterations_W", C.c_longlong),
                ("pcg_iterations_A", C.c_longlong), ("last_rel_residual_W", C.c_double),
                ("gamma_exhausted", C.c_longlong), ("captured", C.c_int)]


T_CLASSES = ["stats", "assemble_W", "pcg_W", "assemble_A", "pcg_A", "lambda", "hyper", "other",
             "summary"]
MAX_CONTRASTS = 16
LOG_JOINT_TERMS = ["loglik", "W_prior", "A_prior", "lambda_prior", "alpha_prior", "beta_prior",
                   "total"]


class bfmri_timing(C.Structure):
    _fields_ = [("ms", C.c_double * 9), ("launches", C.c_longlong * 9),
                ("pcg_iterations", C.c_longlong * 9)]


class bfmri_request(C.Structure):
    _fields_ = [("lat", bfmri_lattice), ("mask", C.c_void_p), ("X", C.c_void_p), ("Y", C.c_void_p),
                ("y_dtype", C.c_int), ("T", C.c_int), ("K", C.c_int), ("P", C.c_int),
                ("opt", bfmri_options), ("n_sweeps", C.c_int), ("first_counter", C.c_uint64),
                ("W_out", C.c_void_p), ("alpha_out", C.c_void_p)]


class bfmri_result(C.Structure):
    _fields_ = [("status", C.c_int), ("N", C.c_int), ("submit_s", C.c_double),
                ("start_s", C.c_double), ("end_s", C.c_double), ("pcg_iterations", C.c_longlong),
                ("device_bytes", C.c_size_t)]


BFMRI_PENDING = 1
_P = C.POINTER
_dp = _P(C.c_double)
_vp = C.c_void_p
_h = C.c_void_p

# (name, restype, argtypes): the ABI as declared in include/bfmri.h
SIGNATURES = [
    ("bfmri_default_options", None, [_P(bfmri_options)]),
    ("bfmri_create", C.c_int, [_P(bfmri_lattice), _P(C.c_uint8), _dp, _vp, C.c_int, C.c_int,
                               C.c_int, C.c_int, _P(bfmri_options), _P(_h)]),
    ("bfmri_destroy", C.c_int, [_h]),
    ("bfmri_last_error", C.c_char_p, [_h]),
    ("bfmri_num_voxels", C.c_int, [_h]),
    ("bfmri_sizes", C.c_int, [_h, _P(C.c_int), _P(C.c_int), _P(C.c_int), _P(C.c_int)]),
    ("bfmri_precompute_stats", C.c_int, [_h]),
    ("bfmri_get_stats", C.c_int, [_h, _dp]),
    ("bfmri_set_edge_factors", C.c_int, [_h, _P(C.c_float)]),
    ("bfmri_set_alpha_dirs", C.c_int, [_h, _dp]),
    ("bfmri_get_alpha_dirs", C.c_int, [_h, _dp, _P(C.c_longlong)]),
    ("bfmri_aniso_last_step", C.c_int, [_h, _dp, _dp, _dp, _dp, _dp]),
    ("bfmri_set_state", C.c_int, [_h, _dp, _dp, _dp, _dp, _dp]),
    ("bfmri_get_state", C.c_int, [_h, _dp, _dp, _dp, _dp, _dp]),
    ("bfmri_sample_W", C.c_int, [_h, C.c_uint64, _dp, _P(bfmri_solve_info)]),
    ("bfmri_sample_A", C.c_int, [_h, C.c_uint64, _dp, _P(bfmri_solve_info)]),
    ("bfmri_sample_lambda", C.c_int, [_h, C.c_uint64, _dp]),
    ("bfmri_sample_alpha", C.c_int, [_h, C.c_uint64, _dp]),
    ("bfmri_sample_beta", C.c_int, [_h, C.c_uint64, _dp]),
    ("bfmri_gibbs_sweep", C.c_int, [_h, C.c_int, C.c_uint64, _P(bfmri_sweep_info)]),
    ("bfmri_gibbs_sweep_group", C.c_int, [_P(_h), C.c_int, C.c_int, C.c_uint64, _P(bfmri_sweep_info)]),
    ("bfmri_gibbs_sweep_group_probes", C.c_int, [_P(_h), C.c_int, C.c_uint64, _h, C.c_int, C.c_int,
                                                 C.c_uint64, _dp, _dp, _dp, _P(bfmri_sweep_info)]),
    ("bfmri_synchronize", C.c_int, [_h, _P(bfmri_sweep_info)]),
    ("bfmri_summary_begin", C.c_int, [_h, C.c_int, _P(C.c_double), _P(C.c_double), _P(C.c_int), C.c_int]),
    ("bfmri_summary_add", C.c_int, [_h]),
    ("bfmri_summary_get", C.c_int, [_h, _P(C.c_longlong), _P(C.c_double), _P(C.c_double),
                                    _P(C.c_double), _P(C.c_longlong)]),
    ("bfmri_summary_end", C.c_int, [_h]),
    ("bfmri_svb_summary", C.c_int, [_h, C.c_int, _P(C.c_double), _P(C.c_double), _P(C.c_double),
                                    _P(C.c_double), _P(C.c_double)]),
    ("bfmri_log_joint", C.c_int, [_h, _P(C.c_double)]),
    ("bfmri_logdet_probe", C.c_int, [_h, C.c_int, C.c_int, C.c_int, C.c_uint64, _dp, _dp, _dp, _dp,
                                     _P(C.c_int)]),
    ("bfmri_lanczos_log_quadrature", C.c_int, [C.c_int, _dp, _dp, _dp]),
    ("bfmri_spvb_step", C.c_int, [_h, C.c_int, C.c_uint64, C.c_int, _dp, _dp, _P(bfmri_svb_info)]),
    ("bfmri_svb_get_sample", C.c_int, [_h, C.c_int, _dp, _dp]),
    ("bfmri_svb_set_sample", C.c_int, [_h, C.c_int, _dp, _dp]),
    ("bfmri_get_timing", C.c_int, [_h, _P(bfmri_timing)]),
    ("bfmri_reset_timing", C.c_int, [_h]),
    ("bfmri_apply_precision", C.c_int, [_h, C.c_int, _dp, _dp]),
    ("bfmri_apply_preconditioner", C.c_int, [_h, C.c_int, _dp, _dp]),
    ("bfmri_build_system", C.c_int, [_h, C.c_int, C.c_uint64, _dp, _dp, _dp]),
    ("bfmri_request_device_bytes", C.c_size_t, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]),
    ("bfmri_server_create", C.c_int, [C.c_size_t, C.c_int, C.c_int, _P(C.c_void_p)]),
    ("bfmri_server_submit", C.c_int, [C.c_void_p, _P(bfmri_request), _P(C.c_longlong)]),
    ("bfmri_server_poll", C.c_int, [C.c_void_p, C.c_longlong, C.c_int, _P(bfmri_result)]),
    ("bfmri_server_stats", C.c_int, [C.c_void_p, _P(C.c_size_t), _P(C.c_int), _P(C.c_size_t)]),
    ("bfmri_server_pool_usage", C.c_int, [C.c_void_p, _P(C.c_size_t), C.c_int]),
    ("bfmri_device_bytes", C.c_int, [_h, _P(C.c_size_t), _P(C.c_size_t)]),
    ("bfmri_probe_tuning", C.c_int, [_h, _P(C.c_int), _dp]),
    ("bfmri_server_destroy", C.c_int, [C.c_void_p]),
    ("bfmri_pcg_static_capacity", C.c_size_t, []),
    ("bfmri_pcg_static_bytes", C.c_size_t, [C.c_size_t, C.c_int]),
    ("bfmri_pcg_solve_static", C.c_int, [C.c_int, C.c_int, C.c_int, _vp, C.c_size_t, _vp, _vp,
                                         _vp, _vp, C.c_double, C.c_int, _vp,
                                         _P(bfmri_solve_info)]),
]

_lib = None


def load_library(path: str = LIB_PATH):
    """Loads libbfmri.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"bfmri CUDA library not found at {path}; build it first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class BfmriError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def _check(status, handle=None):
    if status != BFMRI_OK:
        msg = load_library().bfmri_last_error(handle)
        raise BfmriError(status, msg.decode() if msg else "")


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_dp)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != tuple(shape):
        a = a.reshape(shape)
    return a


class TorchDeviceMemory:
    """Device allocator callbacks backed by PyTorch's caching allocator."""

    def __init__(self):
        import torch
        self._torch = torch
        self._live = {}
        self.alloc = ALLOC_FN(self._alloc)
        self.free = FREE_FN(self._free)

    def _alloc(self, nbytes, ctx):
        try:
            t = self._torch.empty(int(nbytes), dtype=self._torch.uint8, device="cuda")
        except Exception:   # OOM -> NULL, the library reports BFMRI_ERR_OOM
            return None
        p = t.data_ptr()
        self._live[p] = t
        return p

    def _free(self, ptr, ctx):
        self._live.pop(ptr, None)

    @property
    def bytes_held(self):
        return sum(t.numel() for t in self._live.values())


def bfmri_default_options():
    o = bfmri_options()
    load_library().bfmri_default_options(C.byref(o))
    return o


def bfmri_create(lattice, mask, X, Y, K, P, opts=None, torch_memory=True):
    """Returns (handle, keepalive). lattice = (nx, ny, nz, neighbourhood); mask is an
    (nz, ny, nx) uint8 array; X is T x K; Y is T x N (float32 or float64)."""
    lib = load_library()
    nx, ny, nz, nb = lattice
    lat = bfmri_lattice(nx, ny, nz, nb)
    mask = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
    X = np.asfortranarray(np.asarray(X, dtype=np.float64))
    T = X.shape[0]
    Y = np.ascontiguousarray(Y)
    if Y.dtype == np.float64:
        ydt = BFMRI_F64
    elif Y.dtype == np.float32:
        ydt = BFMRI_F32
    else:
        Y = Y.astype(np.float64)
        ydt = BFMRI_F64
    if opts is None:
        opts = bfmri_default_options()
    mem = None
    if torch_memory:
        import torch
        mem = TorchDeviceMemory()
        opts.dev_alloc = mem.alloc
        opts.dev_free = mem.free
        if opts.cuda_stream is None:
            opts.cuda_stream = torch.cuda.current_stream().cuda_stream
    h = _h()
    st = lib.bfmri_create(C.byref(lat), mask.ctypes.data_as(_P(C.c_uint8)),
                          X.ctypes.data_as(_dp), Y.ctypes.data_as(_vp), ydt, T, K, P,
                          C.byref(opts), C.byref(h))
    _check(st, None)
    return h, (mem, opts)


def bfmri_destroy(h):
    _check(load_library().bfmri_destroy(h))


class Server:
    """A bfmri_server: requests (synthetic workloads) are submitted with their host arrays,
    which this object keeps alive until the request has finished."""

    def __init__(self, budget_bytes, slots, sm_budget=0):
        self.lib = load_library()
        h = C.c_void_p()
        _check(self.lib.bfmri_server_create(int(budget_bytes), slots, sm_budget, C.byref(h)))
        self.h = h
        self._keep = {}
        # the slots' threads read the host arrays in _keep and write W and alpha into them:
        # a server left open at interpreter exit is drained first (destroy waits for every
        # admitted and queued request), before those arrays or the CUDA context go away
        atexit.register(self.close)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def submit(self, w, n_sweeps, first_counter=0, **opt_fields):
        o = bfmri_default_options()
        o.eps = w.eps
        o.delta = w.delta
        for k, v in opt_fields.items():
            setattr(o, k, v)
        mask = np.ascontiguousarray(w.mask, dtype=np.uint8).reshape(-1)
        X = np.asfortranarray(w.X, dtype=np.float64)
        Y = np.ascontiguousarray(w.Y)
        W = np.empty((w.K, w.N))
        alpha = np.empty(w.K)
        nx, ny, nz = w.dims
        r = bfmri_request(lat=bfmri_lattice(nx, ny, nz, w.neighbourhood),
                          mask=mask.ctypes.data, X=X.ctypes.data, Y=Y.ctypes.data,
                          y_dtype=BFMRI_F64 if Y.dtype == np.float64 else BFMRI_F32,
                          T=w.T, K=w.K, P=w.P, opt=o, n_sweeps=n_sweeps,
                          first_counter=first_counter, W_out=W.ctypes.data,
                          alpha_out=alpha.ctypes.data)
        t = C.c_longlong()
        _check(self.lib.bfmri_server_submit(self.h, C.byref(r), C.byref(t)))
        self._keep[t.value] = (mask, X, Y, W, alpha, r)
        return t.value

    def poll(self, ticket, wait=True):
        res = bfmri_result()
        st = self.lib.bfmri_server_poll(self.h, ticket, 1 if wait else 0, C.byref(res))
        if st == BFMRI_PENDING:
            return None
        _check(st)
        if res.status != BFMRI_OK:
            raise BfmriError(res.status, "request failed")
        mask, X, Y, W, alpha, r = self._keep.pop(ticket)
        return dict(W=W, alpha=alpha, N=res.N, submit_s=res.submit_s, start_s=res.start_s,
                    end_s=res.end_s, pcg_iterations=res.pcg_iterations,
                    device_bytes=res.device_bytes)

    def stats(self):
        pb, pr, iu = C.c_size_t(), C.c_int(), C.c_size_t()
        _check(self.lib.bfmri_server_stats(self.h, C.byref(pb), C.byref(pr), C.byref(iu)))
        return dict(peak_bytes=pb.value, peak_running=pr.value, in_use=iu.value)

    def pool_usage(self, reset=False):
        """High-water mark of the bytes in use from the server's memory pool."""
        v = C.c_size_t()
        _check(self.lib.bfmri_server_pool_usage(self.h, C.byref(v), 1 if reset else 0))
        return v.value

    def close(self):
        if self.h:
            h, self.h = self.h, None
            _check(self.lib.bfmri_server_destroy(h))
            self._keep.clear()
            atexit.unregister(self.close)


def bfmri_pcg_solve_static(N, D, neighbourhood, nbr_ptr, ld, blocks_ptr, scale_ptr, b_ptr,
                           x_ptr, delta, max_iter, stream=None):
    """The allocation-free solve on caller-owned device arrays (pointers as integers)."""
    info = bfmri_solve_info()
    st = load_library().bfmri_pcg_solve_static(N, D, neighbourhood, nbr_ptr, ld, blocks_ptr,
                                               scale_ptr, b_ptr, x_ptr, delta, max_iter, stream,
                                               C.byref(info))
    _check(st, None)
    return info


def unpack_cov(packed, K):
    """(K(K+1)/2, N) packed lower triangles (row i(i+1)/2 + j, j <= i) -> (N, K, K)."""
    N = packed.shape[1]
    out = np.empty((N, K, K))
    for i in range(K):
        for j in range(i + 1):
            out[:, i, j] = out[:, j, i] = packed[i * (i + 1) // 2 + j]
    return out


def gibbs_sweep_group(models, n_sweeps, first_counter=0):
    """Advances the chains of `models` (Model objects, on one lattice or on several) together
    by n_sweeps Gibbs sweeps, their W and A systems solved as one multi-RHS launch per step
    (bfmri_gibbs_sweep_group); returns one bfmri_sweep_info per chain."""
    lib = load_library()
    n = len(models)
    hs = (_h * n)(*[m.handle for m in models])
    infos = (bfmri_sweep_info * n)()
    st = lib.bfmri_gibbs_sweep_group(hs, n, n_sweeps, first_counter, infos)
    if st != BFMRI_OK:
        _check(st, models[0].handle)
    return list(infos)


def gibbs_sweep_group_probes(models, counter, probe_model, n_probes, lanczos_steps,
                             probe_counter=0):
    """One sweep of the chains of `models` (which may be subjects on different lattices)
    whose W systems share one multi-RHS launch with n_probes log-det probes of probe_model's
    W system (bfmri_gibbs_sweep_group_probes); returns (infos, logdet, std_err, per_probe)."""
    import numpy as np
    lib = load_library()
    n = len(models)
    hs = (_h * n)(*[m.handle for m in models])
    infos = (bfmri_sweep_info * n)()
    ld, se = C.c_double(), C.c_double()
    per = np.empty(n_probes)
    st = lib.bfmri_gibbs_sweep_group_probes(hs, n, counter, probe_model.handle, n_probes,
                                            lanczos_steps, probe_counter, C.byref(ld),
                                            C.byref(se), _ptr(per), infos)
    if st != BFMRI_OK:
        _check(st, models[0].handle)
    return list(infos), ld.value, se.value, per


def lanczos_log_quadrature(cg_alpha, cg_beta):
    a = _f64(cg_alpha)
    b = _f64(cg_beta) if len(cg_beta) else np.zeros(1)
    v = C.c_double()
    _check(load_library().bfmri_lanczos_log_quadrature(len(a), _ptr(a), _ptr(b), C.byref(v)))
    return v.value


class Model:
    """Owns one handle: a subject's data, its statistics and its chain state on the GPU."""

    def __init__(self, lattice, mask, X, Y, K, P, opts=None, **opt_fields):
        o = opts if opts is not None else bfmri_default_options()
        for k, v in opt_fields.items():
            setattr(o, k, v)
        self.handle, self._keep = bfmri_create(lattice, mask, X, Y, K, P, o)
        self.lib = load_library()
        N, T, Kc, Pc = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        _check(self.lib.bfmri_sizes(self.handle, C.byref(N), C.byref(T), C.byref(Kc), C.byref(Pc)), self.handle)
        self.N, self.T, self.K, self.P = N.value, T.value, Kc.value, Pc.value
        self.sites = int(np.prod(lattice[:3]))

    @classmethod
    def from_workload(cls, w, **opt_fields):
        nx, ny, nz = w.dims
        opt_fields.setdefault("eps", w.eps)
        opt_fields.setdefault("delta", w.delta)
        return cls((nx, ny, nz, w.neighbourhood), w.mask, w.X, w.Y, w.K, w.P, **opt_fields)

    def close(self):
        if self.handle:
            bfmri_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _c(self, st):
        _check(st, self.handle)

    def probe_tuning(self):
        """(tile of the last probe solve, autotuner times in ms for tiles 1, 2, 4 or -1)."""
        t = C.c_int()
        ms = np.empty(3)
        self._c(self.lib.bfmri_probe_tuning(self.handle, C.byref(t), _ptr(ms)))
        return t.value, ms.tolist()

    def device_bytes(self):
        """(bytes held now, peak so far) of the handle's own device allocations."""
        a, b = C.c_size_t(), C.c_size_t()
        self._c(self.lib.bfmri_device_bytes(self.handle, C.byref(a), C.byref(b)))
        return a.value, b.value

    def precompute_stats(self):
        self._c(self.lib.bfmri_precompute_stats(self.handle))

    def get_stats(self):
        from_s = (self.P + 1) * (self.P + 2) // 2 + self.K * (self.P + 1) ** 2
        out = np.empty((self.N, from_s))
        self._c(self.lib.bfmri_get_stats(self.handle, _ptr(out)))
        return out

    def set_edge_factors(self, factors):
        """Per-edge factors of C, shape (3, nz, ny, nx) (or (3, nx*ny*nz)), entry [d, site]
        for the +d edge from that site; None removes them. Stored as BF16."""
        if factors is None:
            self._c(self.lib.bfmri_set_edge_factors(self.handle, None))
            return
        f = np.ascontiguousarray(np.asarray(factors, dtype=np.float32).reshape(3, -1))
        if f.shape[1] != self.sites:
            raise ValueError("edge factors: shape (3, nz, ny, nx)")
        self._c(self.lib.bfmri_set_edge_factors(self.handle, f.ctypes.data_as(_P(C.c_float))))

    def set_alpha_dirs(self, alpha):
        """Anisotropic prior: alpha_{d,k} as a K x 3 array (x, y, z per k)."""
        a = _f64(alpha, (self.K, 3))
        self._c(self.lib.bfmri_set_alpha_dirs(self.handle, _ptr(a)))

    def get_alpha_dirs(self):
        """Anisotropic prior: (alpha K x 3, accepted exchange steps per k)."""
        a = np.empty((self.K, 3))
        acc = np.zeros(self.K, dtype=np.int64)
        self._c(self.lib.bfmri_get_alpha_dirs(self.handle, _ptr(a), acc.ctypes.data_as(_P(C.c_longlong))))
        return a, acc

    def aniso_last_step(self):
        """Anisotropic prior: dict of the last alpha step's Q, Q_aux (K x 3), log_a, lam (K)
        and the auxiliary field w_aux (K x N)."""
        Q = np.empty((self.K, 3))
        Qa = np.empty((self.K, 3))
        la = np.empty(self.K)
        lam = np.empty(self.K)
        wa = np.empty((self.K, self.N))
        self._c(self.lib.bfmri_aniso_last_step(self.handle, _ptr(Q), _ptr(Qa), _ptr(la), _ptr(lam), _ptr(wa)))
        return dict(Q=Q, Q_aux=Qa, log_a=la, lam=lam, w_aux=wa)

    def set_state(self, W=None, A=None, lam=None, alpha=None, beta=None):
        arrs = [None if v is None else _f64(v) for v in (W, A, lam, alpha, beta)]
        self._c(self.lib.bfmri_set_state(self.handle, *[_ptr(a) for a in arrs]))

    def get_state(self):
        W = np.empty((self.K, self.N))
        A = np.empty((self.P, self.N))
        lam = np.empty(self.N)
        alpha = np.empty(self.K)
        beta = np.empty(max(self.P, 1))
        self._c(self.lib.bfmri_get_state(self.handle, _ptr(W), _ptr(A), _ptr(lam), _ptr(alpha), _ptr(beta)))
        return dict(W=W, A=A, lam=lam, alpha=alpha, beta=beta[:self.P])

    def get_W(self, out=None):
        """The current W (K x N) into `out` (a C-contiguous float64 array, e.g. in pinned host
        memory for a fast copy) or a new array."""
        W = np.empty((self.K, self.N)) if out is None else out
        if W.shape != (self.K, self.N) or W.dtype != np.float64 or not W.flags["C_CONTIGUOUS"]:
            raise ValueError("out must be a C-contiguous float64 array of shape (K, N)")
        self._c(self.lib.bfmri_get_state(self.handle, _ptr(W), None, None, None, None))
        return W

    def sample_W(self, counter, out=True):
        W = np.empty((self.K, self.N)) if out else None
        info = bfmri_solve_info()
        self._c(self.lib.bfmri_sample_W(self.handle, counter, _ptr(W), C.byref(info)))
        return W, info

    def sample_A(self, counter, out=True):
        A = np.empty((self.P, self.N)) if out else None
        info = bfmri_solve_info()
        self._c(self.lib.bfmri_sample_A(self.handle, counter, _ptr(A), C.byref(info)))
        return A, info

    def sample_lambda(self, counter):
        lam = np.empty(self.N)
        self._c(self.lib.bfmri_sample_lambda(self.handle, counter, _ptr(lam)))
        return lam

    def sample_alpha(self, counter):
        a = np.empty(self.K)
        self._c(self.lib.bfmri_sample_alpha(self.handle, counter, _ptr(a)))
        return a

    def sample_beta(self, counter):
        b = np.empty(max(self.P, 1))
        self._c(self.lib.bfmri_sample_beta(self.handle, counter, _ptr(b)))
        return b[:self.P]

    def gibbs_sweep(self, n_sweeps, first_counter=0, info=True):
        """info=False only enqueues the sweeps (no host wait); their errors and PCG counts are
        read by the next synchronising call, e.g. synchronize()."""
        inf = bfmri_sweep_info()
        self._c(self.lib.bfmri_gibbs_sweep(self.handle, n_sweeps, first_counter,
                                           C.byref(inf) if info else None))
        return inf

    def _contrasts(self, contrast, gamma):
        cm = np.ascontiguousarray(np.atleast_2d(np.asarray(contrast, dtype=np.float64)))
        gamma = np.ascontiguousarray(np.atleast_1d(np.asarray(gamma, dtype=np.float64)))
        return cm, gamma

    def summary_begin(self, contrast, gamma, joint_set=None):
        """Opens a chain summary (marginal / joint contrast PPMs and moments of W); every later
        sweep adds its draw. joint_set: compact voxel indices of the joint-PPM set."""
        cm, gamma = self._contrasts(contrast, gamma)
        js = np.ascontiguousarray(np.asarray([] if joint_set is None else joint_set, dtype=np.int32))
        self._c(self.lib.bfmri_summary_begin(self.handle, len(gamma), _ptr(cm), _ptr(gamma),
                                             js.ctypes.data_as(_P(C.c_int)) if len(js) else None,
                                             len(js)))
        self._n_contrasts = len(gamma)

    def summary_add(self):
        self._c(self.lib.bfmri_summary_add(self.handle))

    def summary_get(self):
        K, N, nc = self.K, self.N, self._n_contrasts
        n = C.c_longlong()
        mean = np.empty((K, N))
        covp = np.empty((K * (K + 1) // 2, N))
        ppm = np.empty((nc, N))
        jc = (C.c_longlong * max(nc, 1))()
        self._c(self.lib.bfmri_summary_get(self.handle, C.byref(n), _ptr(mean), _ptr(covp),
                                           _ptr(ppm), jc))
        return dict(n=n.value, mean=mean, cov_packed=covp, cov=unpack_cov(covp, K), ppm=ppm,
                    joint_count=np.array(jc[:nc], dtype=np.int64))

    def summary_end(self):
        self._c(self.lib.bfmri_summary_end(self.handle))

    def svb_summary(self, contrast, gamma):
        """Moments of the SVB samples and the Gaussian contrast PPMs (Section 3.3)."""
        cm, gamma = self._contrasts(contrast, gamma)
        K, N = self.K, self.N
        mean = np.empty((K, N))
        covp = np.empty((K * (K + 1) // 2, N))
        ppm = np.empty((len(gamma), N))
        self._c(self.lib.bfmri_svb_summary(self.handle, len(gamma), _ptr(cm), _ptr(gamma),
                                           _ptr(mean), _ptr(covp), _ptr(ppm)))
        return dict(mean=mean, cov_packed=covp, cov=unpack_cov(covp, K), ppm=ppm)

    def log_joint(self):
        """Unnormalised log joint posterior of the current state, by term."""
        t = np.empty(7)
        self._c(self.lib.bfmri_log_joint(self.handle, _ptr(t)))
        return dict(zip(LOG_JOINT_TERMS, (float(v) for v in t)))

    def synchronize(self):
        """Waits for the enqueued work; raises the first error of the asynchronous sweeps
        since the last synchronising call and returns their PCG counts."""
        inf = bfmri_sweep_info()
        self._c(self.lib.bfmri_synchronize(self.handle, C.byref(inf)))
        return inf

    def logdet_probe(self, which, n_probes, lanczos_steps, counter, traces=True):
        D = self.K if which == 0 else self.P
        ld = C.c_double()
        se = C.c_double()
        tr = np.empty(D) if traces else None
        pp = np.empty(n_probes)
        its = np.empty(n_probes, dtype=np.int32)
        self._c(self.lib.bfmri_logdet_probe(self.handle, which, n_probes, lanczos_steps, counter,
                                            C.byref(ld), C.byref(se), _ptr(tr), _ptr(pp),
                                            its.ctypes.data_as(_P(C.c_int))))
        return dict(logdet=ld.value, stderr=se.value, traces=tr, per_probe=pp, iterations=its)

    def spvb_step(self, n_samples, counter, extrapolate=True):
        avb = np.empty(self.K)
        bvb = np.empty(max(self.P, 1))
        info = bfmri_svb_info()
        self._c(self.lib.bfmri_spvb_step(self.handle, n_samples, counter, 1 if extrapolate else 0,
                                         _ptr(avb), _ptr(bvb), C.byref(info)))
        return avb, bvb[:self.P], info

    def svb_set_sample(self, j, W=None, A=None):
        W = None if W is None else _f64(W)
        A = None if A is None else _f64(A)
        self._c(self.lib.bfmri_svb_set_sample(self.handle, j, _ptr(W), _ptr(A)))

    def svb_sample(self, j):
        W = np.empty((self.K, self.N))
        A = np.empty((self.P, self.N))
        self._c(self.lib.bfmri_svb_get_sample(self.handle, j, _ptr(W), _ptr(A)))
        return W, A

    def timing(self):
        t = bfmri_timing()
        self._c(self.lib.bfmri_get_timing(self.handle, C.byref(t)))
        return {name: dict(ms=t.ms[i], launches=t.launches[i], pcg_iterations=t.pcg_iterations[i])
                for i, name in enumerate(T_CLASSES)}

    def reset_timing(self):
        self._c(self.lib.bfmri_reset_timing(self.handle))

    def apply_precision(self, which, x):
        D = self.K if which == 0 else self.P
        x = _f64(x, (D, self.N))
        y = np.empty((D, self.N))
        self._c(self.lib.bfmri_apply_precision(self.handle, which, _ptr(x), _ptr(y)))
        return y

    def apply_preconditioner(self, which, x):
        D = self.K if which == 0 else self.P
        x = _f64(x, (D, self.N))
        y = np.empty((D, self.N))
        self._c(self.lib.bfmri_apply_preconditioner(self.handle, which, _ptr(x), _ptr(y)))
        return y

    def build_system(self, which, counter):
        D = self.K if which == 0 else self.P
        blocks = np.empty((self.N, D, D))
        bmean = np.empty((D, self.N))
        bpert = np.empty((D, self.N))
        self._c(self.lib.bfmri_build_system(self.handle, which, counter, _ptr(blocks),
                                            _ptr(bmean), _ptr(bpert)))
        return blocks, bmean, bpert
