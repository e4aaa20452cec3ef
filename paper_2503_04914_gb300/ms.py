"""Thin ctypes binding of libms.so (include/ms.h) with the same entry-point names.

Argument marshalling only: every step of the fit runs in the library's CUDA
kernels.  Host arrays are numpy float64; device arrays are torch CUDA tensors
(float64, contiguous), whose data pointers and current stream are passed to the
``*_dev`` entry points.  If the library is missing this module raises on import
of the library (there is no fallback).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

MS_MAX_LEVELS = 32
MS_OK, MS_ERR_ARG, MS_ERR_CUDA, MS_ERR_OOM, MS_ERR_NOT_SPD, MS_ERR_NOT_CONVERGED, MS_ERR_TIMEOUT, \
    MS_ERR_NUMERIC, MS_ERR_STATE = range(9)
MS_OP_CSR, MS_OP_MATRIX_FREE, MS_OP_AUTO = range(3)
MS_PREC_FP64, MS_PREC_MIXED = range(2)
MS_PRECOND_NONE, MS_PRECOND_LEARNED, MS_PRECOND_EXACT = range(3)
MS_INSPECT_PATTERN, MS_INSPECT_TARGETS, MS_INSPECT_PREDICT, MS_INSPECT_GRAD, MS_INSPECT_PATCHES, \
    MS_INSPECT_CANDIDATES = range(6)
PC_K, PC_OUT, PC_HIDDEN = 16, 17, 64
MS_APPLY_A64, MS_APPLY_A32, MS_APPLY_AMF32, MS_APPLY_B64, MS_APPLY_B32, MS_APPLY_BMF32, MS_APPLY_BMFDF = range(7)

STATUS_NAMES = {0: "MS_OK", 1: "MS_ERR_ARG", 2: "MS_ERR_CUDA", 3: "MS_ERR_OOM", 4: "MS_ERR_NOT_SPD",
                5: "MS_ERR_NOT_CONVERGED", 6: "MS_ERR_TIMEOUT", 7: "MS_ERR_NUMERIC", 8: "MS_ERR_STATE"}

# the symbols include/ms.h declares (checked by the tests)
EXPORTED = ["ms_default_opts", "ms_build_hierarchy", "ms_build_hierarchy_dev", "ms_fit", "ms_fit_dev",
            "ms_fit_static_dev", "ms_fit_batch", "ms_fit_batch_dev", "ms_batch_plan_create", "ms_batch_plan_launch",
            "ms_batch_plan_stats", "ms_batch_plan_destroy", "ms_default_train_opts", "ms_train_precond", "ms_precond_params",
            "ms_precond_inspect", "ms_evaluate", "ms_evaluate_dev", "ms_apply_dev", "ms_get_permutation", "ms_hierarchy_info",
            "ms_peak_probe", "ms_wait_selftest", "ms_launch_count", "ms_last_error", "ms_destroy",
            "ms_trim_memory"]


class ms_opts(C.Structure):
    _fields_ = [("wendland_d", C.c_int), ("wendland_k", C.c_int), ("nu", C.c_double), ("op", C.c_int),
                ("precision", C.c_int), ("precond", C.c_int), ("max_iters", C.c_int),
                ("jacobi_sweeps", C.c_int), ("inter_tol", C.c_double), ("inner_tol", C.c_double),
                ("cell_split", C.c_int), ("threads_per_row", C.c_int), ("lower_fp32", C.c_int),
                ("solve_ctas_per_sm", C.c_int), ("autotune", C.c_int), ("lower_op", C.c_int),
                ("reserved", C.c_int * 4)]


class ms_fit_stats(C.Structure):
    _fields_ = [("L", C.c_int32), ("sweeps", C.c_int32), ("cg_iterations", C.c_int64 * MS_MAX_LEVELS),
                ("refinements", C.c_int32 * MS_MAX_LEVELS), ("rel_residual", C.c_double * MS_MAX_LEVELS),
                ("precond_fallbacks", C.c_int32), ("fp64_fallbacks", C.c_int32), ("device_status", C.c_int32),
                ("fit_ms", C.c_double),
                ("matvec_bytes", C.c_double), ("kernel_launches", C.c_int64), ("phase_ms", C.c_double * 8),
                ("solve_launches", C.c_int32), ("rhs_per_launch", C.c_int32)]

    PHASES = ("resid64", "matvec", "update", "barrier", "lower", "other", "scalar")

    def as_dict(self):
        L = self.L
        return {"L": L, "sweeps": self.sweeps, "cg_iterations": list(self.cg_iterations[:L]),
                "refinements": list(self.refinements[:L]), "rel_residual": list(self.rel_residual[:L]),
                "precond_fallbacks": self.precond_fallbacks, "fp64_fallbacks": self.fp64_fallbacks,
                "device_status": self.device_status,
                "fit_ms": self.fit_ms, "matvec_bytes": self.matvec_bytes,
                "kernel_launches": self.kernel_launches, "solve_launches": self.solve_launches,
                "rhs_per_launch": self.rhs_per_launch,
                "phase_ms": {n: self.phase_ms[i] for i, n in enumerate(self.PHASES)}}


class ms_info(C.Structure):
    _fields_ = [("d", C.c_int32), ("L", C.c_int32), ("N", C.c_int64),
                ("n_per_level", C.c_int64 * MS_MAX_LEVELS), ("delta", C.c_double * MS_MAX_LEVELS),
                ("nnz_A", C.c_int64), ("nnz_B", C.c_int64), ("device_bytes", C.c_int64),
                ("build_ms", C.c_double), ("tpr_A", C.c_int32 * MS_MAX_LEVELS), ("pc_basis", C.c_int32),
                ("cell_split", C.c_int32), ("solve_ctas_per_sm", C.c_int32)]


class ms_train_opts(C.Structure):
    _fields_ = [("epochs", C.c_int), ("batch", C.c_int), ("lr", C.c_double), ("lr_final", C.c_double),
                ("seed", C.c_uint64), ("fp32_weights", C.c_int), ("input_noise", C.c_float),
                ("augment", C.c_int), ("n_basis", C.c_int), ("reserved", C.c_int * 4)]


class ms_train_stats(C.Structure):
    _fields_ = [("samples", C.c_int64), ("steps", C.c_int64), ("loss_first", C.c_double),
                ("loss_last", C.c_double), ("train_ms", C.c_double), ("n_params", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None
_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I64 = C.POINTER(C.c_int64)


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libms.so (built by build.build()); raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libms.so not found at {path}: run paper_2503_04914_gb300.build.build() first")
    lib = C.CDLL(path)
    lib.ms_default_opts.argtypes = [C.POINTER(ms_opts)]
    lib.ms_default_opts.restype = None
    lib.ms_build_hierarchy.argtypes = [C.c_int, C.c_int, _I64, _D, _D, C.POINTER(ms_opts), C.POINTER(_P)]
    lib.ms_build_hierarchy_dev.argtypes = [C.c_int, C.c_int, _I64, _P, _D, C.POINTER(ms_opts), _P, C.POINTER(_P)]
    lib.ms_fit.argtypes = [_P, _D, C.c_int, C.c_double, _D, C.POINTER(ms_fit_stats)]
    lib.ms_fit_dev.argtypes = [_P, _P, C.c_int, C.c_double, _P, C.POINTER(ms_fit_stats), _P]
    lib.ms_fit_static_dev.argtypes = [_P, _P, C.c_double, _P, C.POINTER(ms_fit_stats), _P]
    lib.ms_fit_batch.argtypes = [C.POINTER(_P), C.c_int, C.POINTER(_D), C.c_double, C.POINTER(_D),
                                 C.POINTER(ms_fit_stats)]
    lib.ms_fit_batch_dev.argtypes = [C.POINTER(_P), C.c_int, C.POINTER(C.c_void_p), C.c_double,
                                     C.POINTER(C.c_void_p), C.POINTER(ms_fit_stats), _P]
    lib.ms_batch_plan_create.argtypes = [C.POINTER(_P), C.c_int, C.POINTER(C.c_void_p), C.c_double,
                                         C.POINTER(C.c_void_p), _P, C.POINTER(_P)]
    lib.ms_batch_plan_launch.argtypes = [_P, _P, C.c_int]
    lib.ms_batch_plan_stats.argtypes = [_P, _P, C.POINTER(ms_fit_stats)]
    lib.ms_batch_plan_destroy.argtypes = [_P]
    lib.ms_batch_plan_destroy.restype = None
    lib.ms_default_train_opts.argtypes = [C.POINTER(ms_train_opts)]
    lib.ms_default_train_opts.restype = None
    lib.ms_train_precond.argtypes = [_P, C.POINTER(C.c_int), C.c_int, C.POINTER(ms_train_opts),
                                     C.POINTER(ms_train_stats)]
    lib.ms_precond_params.argtypes = [_P, C.POINTER(C.c_float), C.c_int64, C.c_int]
    lib.ms_precond_inspect.argtypes = [_P, C.c_int, C.POINTER(C.c_int), C.c_int, C.c_void_p, C.c_int64]
    lib.ms_evaluate.argtypes = [_P, _D, C.c_int, _D, C.c_int64, _D]
    lib.ms_evaluate_dev.argtypes = [_P, _P, C.c_int, _P, C.c_int64, _P, _P]
    lib.ms_apply_dev.argtypes = [_P, C.c_int, _P, _P, C.c_int, _P]
    lib.ms_get_permutation.argtypes = [_P, _I64]
    lib.ms_hierarchy_info.argtypes = [_P, C.POINTER(ms_info)]
    lib.ms_peak_probe.argtypes = [C.c_int, C.POINTER(C.c_double)]
    lib.ms_wait_selftest.argtypes = [C.c_double, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double)]
    lib.ms_last_error.argtypes = []
    lib.ms_last_error.restype = C.c_char_p
    lib.ms_destroy.argtypes = [_P]
    lib.ms_destroy.restype = None
    for name in EXPORTED:
        if name not in ("ms_default_opts", "ms_last_error", "ms_destroy", "ms_launch_count",
                        "ms_default_train_opts", "ms_batch_plan_destroy"):
            getattr(lib, name).restype = C.c_int  # ms_status
    lib.ms_trim_memory.argtypes = []
    lib.ms_launch_count.argtypes = []
    lib.ms_launch_count.restype = C.c_uint64
    _lib = lib
    return lib


def _check(status):
    if status != MS_OK:
        raise MsError(status, load().ms_last_error().decode(errors="replace"))


def _host(a, dtype=np.float64):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(C.POINTER(C.c_double if dtype == np.float64 else C.c_int64))


def _is_dev(t):
    return hasattr(t, "is_cuda") and t.is_cuda


def _dev_ptr(t):
    import torch
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError("device arrays must be contiguous torch.float64 CUDA tensors")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is not None:
        return C.c_void_p(int(stream))
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


# ------------------------------------------------------------------ entry points


def ms_default_opts(**overrides) -> ms_opts:
    o = ms_opts()
    load().ms_default_opts(C.byref(o))
    names = {n for n, _ in ms_opts._fields_}
    for k, v in overrides.items():
        if k not in names:
            raise TypeError(f"ms_opts has no field {k!r}")
        setattr(o, k, v)
    return o


def ms_build_hierarchy(d, n_per_level, points, h_per_level, opts: ms_opts | None = None, stream=None):
    """Returns an opaque handle (int).  points: numpy [N, d] (host) or torch CUDA [N, d] (device)."""
    lib = load()
    n, n_p = _host(n_per_level, np.int64)
    hh, h_p = _host(h_per_level)
    out = C.c_void_p()
    L = len(n)
    optp = C.byref(opts) if opts is not None else None
    if _is_dev(points):
        _check(lib.ms_build_hierarchy_dev(d, L, n_p, _dev_ptr(points), h_p, optp, _stream(stream), C.byref(out)))
    else:
        pts, p_p = _host(points)
        _check(lib.ms_build_hierarchy(d, L, n_p, p_p, h_p, optp, C.byref(out)))
    return out.value


def ms_fit(handle, f, rel_tol=1e-10, alpha_out=None, stream=None):
    """Solve for the coefficients; returns (alpha, stats dict).  f: [N] or [N, nrhs]."""
    lib = load()
    st = ms_fit_stats()
    nrhs = 1 if f.ndim == 1 else f.shape[1]
    if _is_dev(f):
        import torch
        if alpha_out is None:
            alpha_out = torch.empty_like(f)
        _check(lib.ms_fit_dev(C.c_void_p(handle), _dev_ptr(f), nrhs, rel_tol, _dev_ptr(alpha_out), C.byref(st),
                              _stream(stream)))
        return alpha_out, st.as_dict()
    fa, f_p = _host(f)
    out = np.empty_like(fa) if alpha_out is None else alpha_out
    _check(lib.ms_fit(C.c_void_p(handle), f_p, nrhs, rel_tol, out.ctypes.data_as(_D), C.byref(st)))
    return out, st.as_dict()


def ms_fit_static_dev(handle, f, rel_tol=1e-10, alpha_out=None, stream=None):
    """Allocation-free fit of one right-hand side (device tensors only); see include/ms.h.
    The call itself allocates nothing; pass alpha_out to keep this wrapper allocation-free too."""
    import torch
    st = ms_fit_stats()
    if alpha_out is None:
        alpha_out = torch.empty_like(f)
    _check(load().ms_fit_static_dev(C.c_void_p(handle), _dev_ptr(f), rel_tol, _dev_ptr(alpha_out), C.byref(st),
                                    _stream(stream)))
    return alpha_out, st.as_dict()


def ms_fit_batch(handles, fs, rel_tol=1e-10, alpha_out=None, stream=None):
    """Fit nh hierarchies (one right-hand side each) in one launch; returns (alphas, stats dicts).
    fs: list of [N_i] numpy arrays (host API) or contiguous float64 CUDA tensors (device API)."""
    lib = load()
    nh = len(handles)
    hs = (_P * nh)(*[C.c_void_p(h) for h in handles])
    st = (ms_fit_stats * nh)()
    if nh and _is_dev(fs[0]):
        import torch
        outs = alpha_out if alpha_out is not None else [torch.empty_like(f) for f in fs]
        fp = (C.c_void_p * nh)(*[_dev_ptr(f) for f in fs])
        ap = (C.c_void_p * nh)(*[_dev_ptr(a) for a in outs])
        _check(lib.ms_fit_batch_dev(hs, nh, fp, rel_tol, ap, st, _stream(stream)))
        return outs, [s.as_dict() for s in st]
    fa = [np.ascontiguousarray(f, dtype=np.float64) for f in fs]
    outs = alpha_out if alpha_out is not None else [np.empty_like(f) for f in fa]
    fp = (_D * nh)(*[f.ctypes.data_as(_D) for f in fa])
    ap = (_D * nh)(*[a.ctypes.data_as(_D) for a in outs])
    _check(lib.ms_fit_batch(hs, nh, fp, rel_tol, ap, st))
    return outs, [s.as_dict() for s in st]


class BatchPlan:
    """A prepared batched fit (ms_batch_plan_*): binds the device tensors fs[i] (right-hand
    sides, input order) and alphas[i] (coefficients, written by each launch)."""

    def __init__(self, handles, fs, rel_tol=1e-10, alphas=None, stream=None):
        import torch
        lib = load()
        self.nh = len(handles)
        self.fs = fs
        self.alphas = alphas if alphas is not None else [torch.empty_like(f) for f in fs]
        hs = (_P * self.nh)(*[C.c_void_p(h) for h in handles])
        fp = (C.c_void_p * self.nh)(*[_dev_ptr(f) for f in fs])
        ap = (C.c_void_p * self.nh)(*[_dev_ptr(a) for a in self.alphas])
        out = _P()
        _check(lib.ms_batch_plan_create(hs, self.nh, fp, rel_tol, ap, _stream(stream), C.byref(out)))
        self.plan = out.value

    def launch(self, stream=None, use_graph=False):
        _check(load().ms_batch_plan_launch(C.c_void_p(self.plan), _stream(stream), int(bool(use_graph))))

    def stats(self, stream=None):
        st = (ms_fit_stats * self.nh)()
        _check(load().ms_batch_plan_stats(C.c_void_p(self.plan), _stream(stream), st))
        return [s.as_dict() for s in st]

    def close(self):
        if self.plan:
            load().ms_batch_plan_destroy(C.c_void_p(self.plan))
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ms_evaluate(handle, alpha, query, out=None, stream=None):
    lib = load()
    d = ms_hierarchy_info(handle)["d"]
    if query.ndim != 2 or query.shape[1] != d:
        raise MsError(MS_ERR_ARG, f"query must be [nq][{d}] for this hierarchy (got shape {tuple(query.shape)})")
    nrhs = 1 if alpha.ndim == 1 else alpha.shape[1]
    nq = query.shape[0]
    if _is_dev(alpha):
        import torch
        if out is None:
            out = torch.empty((nq,) if nrhs == 1 else (nq, nrhs), dtype=torch.float64, device=alpha.device)
        _check(lib.ms_evaluate_dev(C.c_void_p(handle), _dev_ptr(alpha), nrhs, _dev_ptr(query), nq, _dev_ptr(out),
                                   _stream(stream)))
        return out
    a, a_p = _host(alpha)
    q, q_p = _host(query)
    o = np.empty((nq,) if nrhs == 1 else (nq, nrhs)) if out is None else out
    _check(lib.ms_evaluate(C.c_void_p(handle), a_p, nrhs, q_p, nq, o.ctypes.data_as(_D)))
    return o


def ms_apply_dev(handle, op, x, y=None, sorted_order=False, stream=None):
    import torch
    if y is None:
        y = torch.empty_like(x)
    _check(load().ms_apply_dev(C.c_void_p(handle), op, _dev_ptr(x), _dev_ptr(y), int(bool(sorted_order)),
                               _stream(stream)))
    return y


def ms_get_permutation(handle, N):
    out = np.empty(N, dtype=np.int64)
    _check(load().ms_get_permutation(C.c_void_p(handle), out.ctypes.data_as(_I64)))
    return out


def ms_hierarchy_info(handle) -> dict:
    info = ms_info()
    _check(load().ms_hierarchy_info(C.c_void_p(handle), C.byref(info)))
    L = info.L
    return {"d": info.d, "L": L, "N": info.N, "n_per_level": list(info.n_per_level[:L]),
            "delta": list(info.delta[:L]), "nnz_A": info.nnz_A, "nnz_B": info.nnz_B,
            "device_bytes": info.device_bytes, "build_ms": info.build_ms,
            "tpr_A": list(info.tpr_A[:L]), "pc_basis": info.pc_basis, "cell_split": info.cell_split,
            "solve_ctas_per_sm": info.solve_ctas_per_sm}


def ms_default_train_opts(**overrides) -> ms_train_opts:
    o = ms_train_opts()
    load().ms_default_train_opts(C.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def _levels(levels):
    arr = (C.c_int * len(levels))(*[int(x) for x in levels])
    return arr, len(levels)


def ms_train_precond(handle, levels, opts: ms_train_opts | None = None, **overrides) -> dict:
    if opts is None:
        opts = ms_default_train_opts(**overrides)
    lv, n = _levels(levels)
    st = ms_train_stats()
    _check(load().ms_train_precond(C.c_void_p(handle), lv, n, C.byref(opts), C.byref(st)))
    return st.as_dict()


def precond_n_values(d: int, m: int) -> int:
    """Values of an exported network with m candidate rows: weights, then 17 means and 17 deviations."""
    n_in = PC_K * d
    return (PC_HIDDEN * n_in + PC_HIDDEN + PC_HIDDEN * PC_HIDDEN + PC_HIDDEN + m * PC_OUT * PC_HIDDEN + m * PC_OUT
            + 2 * PC_OUT)


def ms_precond_params(handle, d, params=None):
    """Get (params None) or set the network weights + output standardisation (float32 array).
    Setting takes the candidate count from the array's length."""
    n = precond_n_values(d, ms_hierarchy_info(handle)["pc_basis"])
    if params is None:
        out = np.empty(n, dtype=np.float32)
        _check(load().ms_precond_params(C.c_void_p(handle), out.ctypes.data_as(C.POINTER(C.c_float)), n, 0))
        return out
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(load().ms_precond_params(C.c_void_p(handle), p.ctypes.data_as(C.POINTER(C.c_float)), len(p), 1))
    return p


def ms_precond_inspect(handle, what, N, d, levels=(0,), augment=4):
    """augment: the extra patches per point of the last training (MS_INSPECT_PATCHES only)."""
    lv, n = _levels(levels)
    if what == MS_INSPECT_PATCHES:
        npl = ms_hierarchy_info(handle)["n_per_level"]
        out = np.empty(((1 + augment) * sum(npl[l] for l in levels), 18), dtype=np.int32)
    elif what == MS_INSPECT_PATTERN:
        out = np.empty((N, PC_K), dtype=np.int32)
    elif what == MS_INSPECT_TARGETS:
        out = np.empty((N, PC_OUT), dtype=np.float64)
    elif what == MS_INSPECT_PREDICT:
        out = np.empty((N, PC_OUT), dtype=np.float32)
    elif what == MS_INSPECT_CANDIDATES:
        out = np.empty((N, PC_OUT * ms_hierarchy_info(handle)["pc_basis"]), dtype=np.float32)
    else:
        out = np.empty(precond_n_values(d, ms_hierarchy_info(handle)["pc_basis"]) - 2 * PC_OUT + 1, dtype=np.float32)
    _check(load().ms_precond_inspect(C.c_void_p(handle), what, lv, n, out.ctypes.data_as(C.c_void_p), out.size))
    return out


MS_PROBE_FP32, MS_PROBE_FP64, MS_PROBE_XU = range(3)


def ms_peak_probe(kind) -> float:
    """Warp-lane instructions per second of the FP32-FMA, FP64-FMA or XU (rsqrt) probe."""
    v = C.c_double()
    _check(load().ms_peak_probe(int(kind), C.byref(v)))
    return v.value


def ms_wait_selftest(timeout_s, peer_timed_out=False):
    """Runs the solve kernel's grid barrier with a partner CTA that never arrives; returns
    (device status word, seconds the kernel ran)."""
    st = C.c_int(-1)
    w = C.c_double()
    _check(load().ms_wait_selftest(float(timeout_s), int(bool(peer_timed_out)), C.byref(st), C.byref(w)))
    return st.value, w.value


def ms_launch_count() -> int:
    return int(load().ms_launch_count())


def ms_last_error() -> str:
    return load().ms_last_error().decode(errors="replace")


def ms_trim_memory() -> None:
    """Return the library pool's unused device memory (build scratch, freed handles)."""
    _check(load().ms_trim_memory())


def ms_destroy(handle) -> None:
    if handle:
        load().ms_destroy(C.c_void_p(handle))


class Hierarchy:
    """Owns one ms_hierarchy handle (freed on close / garbage collection)."""

    def __init__(self, d, n_per_level, points, h_per_level, opts=None, stream=None, **overrides):
        if opts is None:
            opts = ms_default_opts(**overrides)
        self.opts = opts
        self.d = int(d)
        self.N = int(np.sum(n_per_level))
        self.handle = ms_build_hierarchy(d, n_per_level, points, h_per_level, opts, stream)

    @classmethod
    def from_workload(cls, w, device=False, **overrides):
        opts = ms_default_opts(wendland_d=w.wendland_d, wendland_k=w.wendland_k, nu=w.nu, **overrides)
        pts = w.points
        if device:
            import torch
            pts = torch.from_numpy(pts).cuda()
        return cls(w.d, w.n_per_level, pts, w.h, opts=opts)

    def fit(self, f, rel_tol=1e-10, alpha_out=None, stream=None):
        return ms_fit(self.handle, f, rel_tol, alpha_out, stream)

    def evaluate(self, alpha, query, out=None, stream=None):
        return ms_evaluate(self.handle, alpha, query, out, stream)

    def apply(self, op, x, y=None, sorted_order=False, stream=None):
        return ms_apply_dev(self.handle, op, x, y, sorted_order, stream)

    def permutation(self):
        return ms_get_permutation(self.handle, self.N)

    def info(self):
        return ms_hierarchy_info(self.handle)

    def train_precond(self, levels, **overrides):
        return ms_train_precond(self.handle, levels, **overrides)

    def precond_params(self, params=None):
        return ms_precond_params(self.handle, self.d, params)

    def inspect(self, what, levels=(0,), augment=4):
        return ms_precond_inspect(self.handle, what, self.N, self.d, levels, augment)

    def close(self):
        if getattr(self, "handle", None):
            ms_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
