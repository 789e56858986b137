"""Thin ctypes binding of ``libtls.so`` (include/tls.h, include/tls_debug.h).

Argument marshalling only: every step of the solve runs in the library's CUDA kernels. The
functions keep the C names. Host arrays are numpy float64; device inputs may be torch CUDA
tensors (their data pointers are passed with ``on_device=1``). There is no CPU fallback: if
the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

TLS_FP16, TLS_BF16, TLS_FP32, TLS_FP64 = 0, 1, 2, 3
TLS_AUTO = 4
PREC = {"fp16": TLS_FP16, "bf16": TLS_BF16, "fp32": TLS_FP32, "fp64": TLS_FP64, "auto": TLS_AUTO}
MLP_PARAMS = 5508
N_FEATURES = 16
STOP_TOL, STOP_PSI_UP, STOP_MAX_RQI, STOP_STALL = 1, 2, 3, 4
TRIGGER_NONE, TRIGGER_MAX_RQI, TRIGGER_STALL, TRIGGER_NOT_SPD, TRIGGER_CONSTRAINT = 0, 1, 2, 3, 4

STATUS = ["TLS_OK", "TLS_ERR_ARG", "TLS_ERR_CUDA", "TLS_ERR_OOM", "TLS_ERR_STATE",
          "TLS_ERR_FACTOR_BREAKDOWN", "TLS_ERR_NOT_SPD", "TLS_ERR_NOT_UNIQUE",
          "TLS_ERR_NO_CONVERGENCE", "TLS_ERR_TIMEOUT"]

# every symbol the headers declare (checked by the CPU test suite)
EXPORTS = ["tls_default_options", "tls_create_dense", "tls_create_csr", "tls_factor", "tls_solve",
           "tls_solve_device", "tls_solve_batched", "tls_destroy", "tls_status_str",
           "tls_last_error", "tls_shape", "tls_set_allocator", "tls_export_factor",
           "tls_residual", "tls_pcgtls", "tls_precond", "tls_profile_enable", "tls_profile_get",
           "tls_kernel_launches", "tls_residual_noalloc", "tls_export_working_copy",
           "tls_condition", "tls_factor_batched", "tls_batch_create_dense", "tls_batch_factor",
           "tls_batch_solve", "tls_batch_destroy", "tls_batch_last_error",
           "tls_batch_export_factor", "tls_batch_profile_enable", "tls_batch_profile_get",
           "tls_batch_profile_elems", "tls_mlp_forward", "tls_mlp_grad", "tls_mlp_adam",
           "tls_batch_set_selector", "tls_batch_features", "tls_set_pass_variant",
           "tls_set_selector", "tls_features", "tls_pool_enable", "tls_pool_trim",
           "tls_pool_stats", "tls_pool_poison", "tls_set_small_path", "tls_profile_units",
           "tls_set_pcg_fused", "tls_trace_enable", "tls_trace_get", "tls_set_pcg_l2_keep",
           "tls_set_factor_chain", "tls_set_factor_tc", "tls_precond_trsv", "tls_options_check"]

PROF_CLASSES = ["scale", "gram", "chol", "trtri", "resid_pass", "resid_reduce", "pcg_pass2",
                "pcg_pass1", "pcg_reduce", "pcg_gemv", "vec", "pcg_solve2", "pcg_solve1"]


class tls_options(C.Structure):
    _fields_ = [("u", C.c_int), ("mode_A", C.c_int), ("cg_fixed", C.c_int),
                ("cg_tol", C.c_double), ("cg_max", C.c_int), ("psi_rule_ge", C.c_int),
                ("ls_iters", C.c_int), ("max_shifts", C.c_int), ("gram_simt", C.c_int),
                ("psi_accept", C.c_double), ("shift_first", C.c_int), ("fallback", C.c_int),
                ("constr_guard", C.c_double), ("stall_fallback", C.c_int),
                ("stall_ratio", C.c_double), ("constraint_iters", C.c_int),
                ("hybrid_ratio", C.c_double), ("reproducible", C.c_int), ("factor", C.c_int)]


class tls_info(C.Structure):
    _fields_ = [("stop_reason", C.c_int), ("rqi_steps", C.c_int), ("best_k", C.c_int),
                ("cg_iters", C.c_int), ("shifts", C.c_int), ("not_spd", C.c_int),
                ("u_f_used", C.c_int), ("psi_final", C.c_double), ("sigma2", C.c_double),
                ("shift", C.c_double), ("t_factor_ms", C.c_double), ("t_solve_ms", C.c_double),
                ("fail_pivot", C.c_int), ("pass_variant", C.c_int * 2), ("n_psi", C.c_int),
                ("psi_hist", C.c_double * 24), ("fallbacks", C.c_int),
                ("fallback_trigger", C.c_int), ("escalations", C.c_int), ("constr1", C.c_double),
                ("constr2", C.c_double), ("constr2_scaled", C.c_double),
                ("mode_switch_k", C.c_int)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("psi_hist", "pass_variant")}
        d["pass_variant"] = [self.pass_variant[0], self.pass_variant[1]]
        d["psi_hist"] = [self.psi_hist[i] for i in range(min(self.n_psi, 24))]
        return d


class TLSError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        name = STATUS[status] if 0 <= status < len(STATUS) else str(status)
        super().__init__(f"{name}: {message}")


_LIB = None
_ALLOC_REFS: list = []
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


def load(path: str | None = None, build_if_missing: bool = True) -> C.CDLL:
    """Load libtls.so (building it in-tree first if it is missing or stale)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    lib_path = path or _build.LIB
    if build_if_missing and path is None:
        _build.build()
    if not os.path.exists(lib_path):
        raise RuntimeError(f"libtls.so not found at {lib_path}; run __graft_entry__.build()")
    lib = C.CDLL(lib_path)
    v, vp, i64 = C.c_void_p, C.POINTER(C.c_void_p), C.c_int64
    sig = {
        "tls_default_options": (None, [C.POINTER(tls_options)]),
        "tls_options_check": (C.c_char_p, [C.POINTER(tls_options)]),
        "tls_create_dense": (C.c_int, [vp, i64, i64, v, i64, v, C.c_int, v]),
        "tls_create_csr": (C.c_int, [vp, i64, i64, i64, v, v, v, v, C.c_int, v]),
        "tls_factor": (C.c_int, [v, C.c_int, C.POINTER(tls_options)]),
        "tls_solve": (C.c_int, [v, C.c_double, C.c_int, _dp, _dp, C.POINTER(tls_info)]),
        "tls_solve_device": (C.c_int, [v, C.c_double, C.c_int, v, _dp, C.POINTER(tls_info)]),
        "tls_solve_batched": (C.c_int, [C.c_int, vp, C.c_double, C.c_int, C.POINTER(_dp), _dp,
                                        C.POINTER(tls_info), _ip]),
        "tls_destroy": (None, [v]),
        "tls_status_str": (C.c_char_p, [C.c_int]),
        "tls_last_error": (C.c_char_p, [v]),
        "tls_shape": (None, [v, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]),
        "tls_set_allocator": (None, [v, v, v]),
        "tls_pool_enable": (None, [C.c_int]),
        "tls_pool_trim": (C.c_uint64, []),
        "tls_pool_stats": (None, [C.POINTER(C.c_uint64)] * 3),
        "tls_pool_poison": (None, [C.c_int]),
        "tls_export_factor": (C.c_int, [v, _dp, _dp, _dp]),
        "tls_residual": (C.c_int, [v, _dp, _dp, _dp]),
        "tls_pcgtls": (C.c_int, [v, C.c_int, C.c_double, _dp, _dp, C.c_int, C.c_double, _dp, _dp,
                                 _ip, _ip]),
        "tls_precond": (C.c_int, [v, _dp, _dp, _dp]),
        "tls_precond_trsv": (C.c_int, [v, _dp, _dp, _dp]),
        "tls_profile_enable": (C.c_int, [v, C.c_int]),
        "tls_profile_get": (C.c_int, [v, C.c_int, C.POINTER(i64), _dp]),
        "tls_kernel_launches": (C.c_uint64, []),
        "tls_residual_noalloc": (C.c_int, [i64, i64, v, i64, v, v, v, v, v]),
        "tls_export_working_copy": (C.c_int, [v, C.POINTER(C.c_float)]),
        "tls_condition": (C.c_int, [v, C.c_int, _dp]),
        "tls_set_selector": (C.c_int, [v, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                       C.POINTER(C.c_float)]),
        "tls_features": (C.c_int, [v, C.POINTER(C.c_float)]),
        "tls_factor_batched": (C.c_int, [C.c_int, vp, C.c_int, C.POINTER(tls_options), _ip]),
        "tls_batch_create_dense": (C.c_int, [vp, C.c_int, C.POINTER(i64), C.POINTER(i64), vp,
                                             C.POINTER(i64), vp, C.c_int, v]),
        "tls_batch_factor": (C.c_int, [v, C.c_int, C.POINTER(tls_options)]),
        "tls_batch_solve": (C.c_int, [v, C.c_double, C.c_int, C.POINTER(_dp), _dp,
                                      C.POINTER(tls_info), _ip]),
        "tls_batch_destroy": (None, [v]),
        "tls_batch_last_error": (C.c_char_p, [v]),
        "tls_batch_export_factor": (C.c_int, [v, C.c_int, _dp, _dp, _dp]),
        "tls_batch_profile_enable": (C.c_int, [v, C.c_int]),
        "tls_batch_profile_get": (C.c_int, [v, C.c_int, C.POINTER(i64), _dp]),
        "tls_batch_profile_elems": (C.c_int, [v, C.c_int, C.POINTER(i64)]),
        "tls_mlp_forward": (C.c_int, [v, C.c_int, v, v, v]),
        "tls_mlp_grad": (C.c_int, [v, C.c_int, v, v, v, v, v, C.c_float, v, v, v, v]),
        "tls_mlp_adam": (C.c_int, [v, v, v, v, C.c_int, C.c_float, C.c_float, C.c_float,
                                   C.c_float, v]),
        "tls_batch_set_selector": (C.c_int, [v, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                             C.POINTER(C.c_float)]),
        "tls_batch_features": (C.c_int, [v, C.POINTER(C.c_float)]),
        "tls_set_pass_variant": (C.c_int, [v, C.c_int, C.c_int]),
        "tls_set_small_path": (C.c_int, [v, C.c_int]),
        "tls_profile_units": (C.c_int, [v, C.c_int, C.POINTER(i64)]),
        "tls_set_pcg_fused": (C.c_int, [v, C.c_int]),
        "tls_trace_enable": (C.c_int, [v, C.c_int]),
        "tls_set_pcg_l2_keep": (C.c_int, [v, i64]),
        "tls_set_factor_chain": (C.c_int, [v, C.c_int]),
        "tls_set_factor_tc": (C.c_int, [v, C.c_int]),
        "tls_trace_get": (C.c_int, [v, C.POINTER(C.c_uint64), C.c_int, C.POINTER(C.c_int)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _check(status: int, ctx=None):
    if status != 0:
        msg = ""
        if ctx:
            msg = (load().tls_last_error(ctx) or b"").decode()
        raise TLSError(status, msg)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _arg_error(fn: str, msg: str):
    raise TLSError(1, f"{fn}: {msg}")


def _host_vec(fn: str, name: str, a, need: int) -> np.ndarray:
    """A contiguous float64 copy (or view) of a host vector with exactly `need` entries: the
    library reads that many, so a shorter array would be read past its end."""
    v = _f64(a)
    if v.size != need:
        _arg_error(fn, f"{name} has {v.size} entries, {need} required")
    return v


def _host_dense(fn: str, A, b) -> tuple[np.ndarray, np.ndarray]:
    A = _f64(A)
    if A.ndim != 2:
        _arg_error(fn, f"A must be 2-D (got {A.ndim}-D)")
    return A, _host_vec(fn, "b", b, A.shape[0])


def _check_device_tensors(fn: str, named: dict, dtype=None) -> None:
    """Every tensor a torch tensor of `dtype` (default float64) on the current CUDA device (the
    library reads device pointers as arrays of the stated type and sizes and cannot check them
    itself)."""
    import torch

    dtype = torch.float64 if dtype is None else dtype
    for nm, t in named.items():
        if not isinstance(t, torch.Tensor):
            _arg_error(fn, f"{nm} is not a torch tensor")
        if t.dtype != dtype:
            _arg_error(fn, f"{nm} has dtype {t.dtype}, {str(dtype).replace('torch.', '')} required")
        if t.device.type != "cuda":
            _arg_error(fn, f"{nm} is not on a CUDA device")
    cur = torch.cuda.current_device()
    for nm, t in named.items():
        if t.device.index != cur:
            _arg_error(fn, f"{nm} is on cuda:{t.device.index}, the current device is cuda:{cur}")


def _device_dense(fn: str, A, b) -> tuple[int, int, int]:
    """(m, n, row stride) of a device problem: A (m, n) row-major with unit column stride and
    row stride >= n, b contiguous with m entries."""
    _check_device_tensors(fn, {"A": A, "b": b})
    if A.dim() != 2:
        _arg_error(fn, f"A must be 2-D (got {A.dim()}-D)")
    m, n = A.shape
    if m < 1 or n < 1:
        _arg_error(fn, f"A is {m} x {n}")
    if (n > 1 and A.stride(1) != 1) or A.stride(0) < n:
        _arg_error(fn, f"A must be row-major with unit column stride and row stride >= n "
                       f"(strides {A.stride()})")
    if not b.is_contiguous() or b.numel() != m:
        _arg_error(fn, f"b must be contiguous with {m} entries (got {b.numel()})")
    return m, n, A.stride(0)


def tls_default_options(**overrides) -> tls_options:
    o = tls_options()
    load().tls_default_options(C.byref(o))
    for k, val in overrides.items():
        if k == "u" and isinstance(val, str):
            val = PREC[val]
        setattr(o, k, val)
    return o


def tls_create_dense(A, b, stream=None) -> C.c_void_p:
    """A: (m, n) float64 numpy array (host) or torch CUDA tensor (device); b likewise."""
    lib = load()
    ctx = C.c_void_p()
    st = C.c_void_p(stream) if stream else None
    if hasattr(A, "is_cuda") and A.is_cuda:
        m, n, lda = _device_dense("tls_create_dense", A, b)
        _check(lib.tls_create_dense(C.byref(ctx), m, n, C.c_void_p(A.data_ptr()), lda,
                                    C.c_void_p(b.data_ptr()), 1, st))
    else:
        A, b = _host_dense("tls_create_dense", A, b)
        m, n = A.shape
        _check(lib.tls_create_dense(C.byref(ctx), m, n, A.ctypes.data_as(C.c_void_p), n,
                                    b.ctypes.data_as(C.c_void_p), 0, st))
    return ctx


def tls_create_csr(m: int, n: int, row_ptr, col_idx, val, b, stream=None) -> C.c_void_p:
    lib = load()
    ctx = C.c_void_p()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    fn = "tls_create_csr"
    if rp.ndim != 1 or rp.size != m + 1:
        _arg_error(fn, f"row_ptr has {rp.size} entries, m + 1 = {m + 1} required")
    nnz = int(rp[-1])
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    if ci.size < nnz:
        _arg_error(fn, f"col_idx has {ci.size} entries, row_ptr[m] = {nnz} required")
    va = _f64(val)
    if va.size < nnz:
        _arg_error(fn, f"val has {va.size} entries, row_ptr[m] = {nnz} required")
    bb = _host_vec(fn, "b", b, m)
    st = C.c_void_p(stream) if stream else None
    _check(lib.tls_create_csr(C.byref(ctx), m, n, nnz, rp.ctypes.data_as(C.c_void_p),
                              ci.ctypes.data_as(C.c_void_p), va.ctypes.data_as(C.c_void_p),
                              bb.ctypes.data_as(C.c_void_p), 0, st))
    return ctx


def tls_options_check(opt: tls_options) -> str | None:
    """None when every field of opt is in range, else what is not (host only, no GPU)."""
    why = load().tls_options_check(C.byref(opt))
    return why.decode() if why else None


def tls_factor(ctx, u_f="fp16", opt: tls_options | None = None):
    uf = PREC[u_f] if isinstance(u_f, str) else int(u_f)
    _check(load().tls_factor(ctx, uf, C.byref(opt) if opt is not None else None), ctx)


def tls_shape(ctx) -> tuple[int, int, int]:
    m, n, nnz = C.c_int64(), C.c_int64(), C.c_int64()
    load().tls_shape(ctx, C.byref(m), C.byref(n), C.byref(nnz))
    return m.value, n.value, nnz.value


def tls_solve(ctx, tol: float = 0.0, max_rqi: int = 10):
    """Returns (x, sigma, info dict)."""
    _, n, _ = tls_shape(ctx)
    x = np.zeros(n)
    sigma = C.c_double()
    info = tls_info()
    _check(load().tls_solve(ctx, tol, max_rqi, _ptr(x), C.byref(sigma), C.byref(info)), ctx)
    return x, sigma.value, info.as_dict()


def tls_solve_device(ctx, x_dev, tol: float = 0.0, max_rqi: int = 10):
    """tls_solve with x written to device memory. x_dev: a float64 torch CUDA tensor on the
    current device, contiguous with n entries (checked), or a raw device address (an int) of
    n float64 values, which the caller vouches for. The copy is ordered on the context's
    stream and finished when this returns. Returns (sigma, info dict)."""
    if isinstance(x_dev, int):
        ptr = x_dev
    else:
        _, n, _ = tls_shape(ctx)
        _check_device_tensors("tls_solve_device", {"x": x_dev})
        if not x_dev.is_contiguous() or x_dev.numel() != n:
            _arg_error("tls_solve_device",
                       f"x must be contiguous with {n} entries (got {x_dev.numel()})")
        ptr = x_dev.data_ptr()
    sigma = C.c_double()
    info = tls_info()
    _check(load().tls_solve_device(ctx, tol, max_rqi, C.c_void_p(ptr), C.byref(sigma),
                                   C.byref(info)), ctx)
    return sigma.value, info.as_dict()


def tls_solve_batched(ctxs, tol: float = 0.0, max_rqi: int = 10):
    k = len(ctxs)
    arr = (C.c_void_p * k)(*[c.value for c in ctxs])
    xs = [np.zeros(tls_shape(c)[1]) for c in ctxs]
    xp = (_dp * k)(*[_ptr(x) for x in xs])
    sig = np.zeros(k)
    infos = (tls_info * k)()
    per = (C.c_int * k)()
    st = load().tls_solve_batched(k, arr, tol, max_rqi, xp, _ptr(sig), infos, per)
    return xs, sig, [i.as_dict() for i in infos], list(per), st


def tls_factor_batched(ctxs, u_f="fp16", opt: tls_options | None = None):
    """Factor several contexts concurrently; returns the per-problem status list."""
    k = len(ctxs)
    arr = (C.c_void_p * k)(*[c.value for c in ctxs])
    per = (C.c_int * k)()
    uf = PREC[u_f] if isinstance(u_f, str) else int(u_f)
    load().tls_factor_batched(k, arr, uf, C.byref(opt) if opt is not None else None, per)
    return list(per)


def tls_destroy(ctx):
    if ctx:
        load().tls_destroy(ctx)


def tls_status_str(status: int) -> str:
    return load().tls_status_str(status).decode()


def tls_last_error(ctx) -> str:
    return (load().tls_last_error(ctx) or b"").decode()


def tls_export_factor(ctx):
    """Returns (R_H, d, H) as float64 numpy arrays."""
    _, n, _ = tls_shape(ctx)
    R = np.zeros((n, n))
    d = np.zeros(n)
    H = np.zeros((n, n))
    _check(load().tls_export_factor(ctx, _ptr(R), _ptr(d), _ptr(H)), ctx)
    return R, d, H


COND_KEYS = ["sigma1", "sigma_n", "kappa", "norm_F", "pinv_norm_F", "kappa_F", "sigma_n1",
             "constr1", "constr2"]


def tls_condition(ctx, iters: int = 30) -> dict:
    """Estimates of Sec. 3.1: see include/tls.h."""
    out = np.zeros(9)
    _check(load().tls_condition(ctx, iters, _ptr(out)), ctx)
    return dict(zip(COND_KEYS, out.tolist()))


def tls_set_selector(ctx, params, mean, scale):
    """Install the selector network (FP32 params, feature mean and scale) for tls_factor(..., "auto")."""
    fp = C.POINTER(C.c_float)
    P = np.ascontiguousarray(params, dtype=np.float32)
    mu = np.ascontiguousarray(mean, dtype=np.float32)
    sd = np.ascontiguousarray(scale, dtype=np.float32)
    if P.size != MLP_PARAMS or mu.size != N_FEATURES or sd.size != N_FEATURES:
        raise ValueError("selector: wrong parameter or feature sizes")
    _check(load().tls_set_selector(ctx, P.ctypes.data_as(fp), mu.ctypes.data_as(fp),
                                   sd.ctypes.data_as(fp)), ctx)


def tls_features(ctx) -> np.ndarray:
    """The 16 raw selector features of the current factor."""
    F = np.zeros(N_FEATURES, dtype=np.float32)
    _check(load().tls_features(ctx, F.ctypes.data_as(C.POINTER(C.c_float))), ctx)
    return F


def tls_export_working_copy(ctx):
    """The FP32 working copy of A (m x n float32)."""
    m, n, _ = tls_shape(ctx)
    out = np.zeros((m, n), dtype=np.float32)
    _check(load().tls_export_working_copy(ctx, out.ctypes.data_as(C.POINTER(C.c_float))), ctx)
    return out


def tls_residual(ctx, x):
    _, n, _ = tls_shape(ctx)
    x = _host_vec("tls_residual", "x", x, n)
    f = np.zeros(n)
    sc = np.zeros(5)
    _check(load().tls_residual(ctx, _ptr(x), _ptr(f), _ptr(sc)), ctx)
    return f, {"sigma2": sc[0], "g": sc[1], "psi": sc[2], "rr": sc[3], "br": sc[4]}


def tls_pcgtls(ctx, sigma2: float, f0, f1=None, steps: int = 1, cg_tol: float = 0.0):
    _, n, _ = tls_shape(ctx)
    nr = 1 if f1 is None else 2
    f0 = _host_vec("tls_pcgtls", "f0", f0, n)
    f1a = _host_vec("tls_pcgtls", "f1", f1, n) if f1 is not None else np.zeros(n)
    w0 = np.zeros(n)
    w1 = np.zeros(n)
    it = (C.c_int * 2)()
    bad = (C.c_int * 2)()
    _check(load().tls_pcgtls(ctx, nr, sigma2, _ptr(f0), _ptr(f1a), steps, cg_tol, _ptr(w0),
                             _ptr(w1), it, bad), ctx)
    return w0, (w1 if nr == 2 else None), list(it), list(bad)


def tls_precond(ctx, y):
    _, n, _ = tls_shape(ctx)
    y = _host_vec("tls_precond", "y", y, n)
    s0 = np.zeros(n)
    u = np.zeros(n)
    _check(load().tls_precond(ctx, _ptr(y), _ptr(s0), _ptr(u)), ctx)
    return s0, u


def tls_precond_trsv(ctx, y):
    """s0 = R^{-T} y and u = R^{-1} s0 by triangular solves with the factor (not its inverse)."""
    _, n, _ = tls_shape(ctx)
    y = _host_vec("tls_precond_trsv", "y", y, n)
    s0 = np.zeros(n)
    u = np.zeros(n)
    _check(load().tls_precond_trsv(ctx, _ptr(y), _ptr(s0), _ptr(u)), ctx)
    return s0, u


def tls_profile_enable(ctx, on: bool = True):
    _check(load().tls_profile_enable(ctx, 1 if on else 0), ctx)


def tls_profile_get(ctx) -> dict:
    """{class name: (launches, device ms)} summed since tls_profile_enable."""
    out = {}
    for i, name in enumerate(PROF_CLASSES):
        cnt = C.c_int64()
        ms = C.c_double()
        _check(load().tls_profile_get(ctx, i, C.byref(cnt), C.byref(ms)), ctx)
        out[name] = (cnt.value, ms.value)
    return out


def tls_profile_units(ctx) -> dict:
    """{class name: units of work behind its timed launches} (PCGTLS steps for pcg_solve*)."""
    out = {}
    for i, name in enumerate(PROF_CLASSES):
        u = C.c_int64()
        _check(load().tls_profile_units(ctx, i, C.byref(u)), ctx)
        out[name] = u.value
    return out


def tls_set_pcg_fused(ctx, mode: int) -> None:
    """0 automatic, 1 one persistent launch per PCGTLS solve, 2 the multi-launch path."""
    _check(load().tls_set_pcg_fused(ctx, int(mode)), ctx)


def tls_set_factor_chain(ctx, per_sm: int) -> None:
    """Block steps of the FP32 factor in one persistent launch of up to per_sm CTAs per SM
    (default 2), or one launch each (0)."""
    _check(load().tls_set_factor_chain(ctx, int(per_sm)), ctx)


def tls_set_factor_tc(ctx, on: int) -> None:
    """Trailing updates of the wide block steps of an FP16/BF16 factor on the tensor cores (1,
    default) or on the CUDA cores in FP32 (0)."""
    _check(load().tls_set_factor_tc(ctx, int(on)), ctx)


def tls_set_pcg_l2_keep(ctx, nbytes: int) -> None:
    """Bytes of A the one-launch PCGTLS solve keeps resident in L2 across its steps."""
    _check(load().tls_set_pcg_l2_keep(ctx, int(nbytes)), ctx)


def tls_trace_enable(ctx, on: bool = True) -> None:
    _check(load().tls_trace_enable(ctx, 1 if on else 0), ctx)


def tls_trace_get(ctx) -> np.ndarray:
    """Phase timestamps (ns) of the last one-launch PCGTLS solve (see tls_debug.h)."""
    cnt = C.c_int()
    buf = (C.c_uint64 * 16384)()
    _check(load().tls_trace_get(ctx, buf, 16384, C.byref(cnt)), ctx)
    return np.array(buf[:cnt.value], dtype=np.uint64)


def tls_kernel_launches() -> int:
    return int(load().tls_kernel_launches())


def tls_residual_noalloc(A, b, x, f, scal, stream=None):
    """The residual block with caller-provided device buffers and no device allocation.
    A (m, n), b (m,), x (n,), f (n,), scal (5,): torch CUDA float64 tensors on the current
    device (A row-major with unit column stride, any row stride >= n; the vectors contiguous).
    Every tensor is checked before the call (dtype, device, shape, strides), so the kernels
    never index past the end of a buffer; a mismatch raises TLSError (TLS_ERR_ARG). Returns the
    status code (0 on success); raises on error."""

    def bad(msg):
        _arg_error("tls_residual_noalloc", msg)

    _check_device_tensors("tls_residual_noalloc", {"A": A, "b": b, "x": x, "f": f, "scal": scal})
    if A.dim() != 2:
        bad("A must be 2-D")
    m, n = A.shape
    if m < 1 or n < 1:
        bad(f"A is {m} x {n}")
    if A.stride(1) != 1 or A.stride(0) < n:
        bad(f"A must be row-major with unit column stride and row stride >= n "
            f"(strides {A.stride()})")
    for nm, t, need in (("b", b, m), ("x", x, n), ("f", f, n)):
        if not t.is_contiguous() or t.numel() != need:
            bad(f"{nm} must be contiguous with {need} elements (got {t.numel()})")
    if not scal.is_contiguous() or scal.numel() < 5:
        bad("scal must be contiguous with at least 5 elements")
    st = C.c_void_p(stream) if stream else None
    status = load().tls_residual_noalloc(m, n, C.c_void_p(A.data_ptr()), A.stride(0),
                                         C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()),
                                         C.c_void_p(f.data_ptr()), C.c_void_p(scal.data_ptr()),
                                         st)
    _check(status)
    return status


def tls_pool_enable(on: bool = True) -> None:
    """Cache freed device / pinned host blocks for later contexts (default on)."""
    load().tls_pool_enable(1 if on else 0)


def tls_pool_trim() -> int:
    """Release every cached block; returns the bytes released."""
    return int(load().tls_pool_trim())


def tls_pool_stats() -> dict:
    cd, ch, ld = C.c_uint64(), C.c_uint64(), C.c_uint64()
    load().tls_pool_stats(C.byref(cd), C.byref(ch), C.byref(ld))
    return {"cached_device": cd.value, "cached_host": ch.value, "live_device": ld.value}


def tls_pool_poison(value: int | None) -> None:
    """Fill every newly allocated block with the byte `value` (None: off)."""
    load().tls_pool_poison(-1 if value is None else int(value))


def use_torch_allocator(enable: bool = True):
    """Route the library's device allocations through torch's caching allocator."""
    lib = load()
    if not enable:
        lib.tls_set_allocator(None, None, None)
        return
    import torch

    ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p)
    FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p)

    def _alloc(nbytes, stream, user):
        try:
            dev = torch.cuda.current_device()
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream or 0)
        except Exception:     # out of memory: the library reports TLS_ERR_OOM
            return None

    def _free(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(ptr)

    a, f = ALLOC(_alloc), FREE(_free)
    # kept for the life of the process: blocks made through them return to them when freed,
    # whatever allocator is set by then
    _ALLOC_REFS.append((a, f))
    lib.tls_set_allocator(C.cast(a, C.c_void_p), C.cast(f, C.c_void_p), None)


class Batch:
    """A packed batch of dense problems (n <= 512) solved together (tls_batch_* entry points).

    problems: sequence of (A, b) host arrays, or pass device=True with torch CUDA tensors."""

    def __init__(self, problems, stream=None):
        lib = load()
        k = len(problems)
        self.k = k
        self.shapes = []
        self._keep = []
        ms = (C.c_int64 * k)()
        ns = (C.c_int64 * k)()
        ld = (C.c_int64 * k)()
        ap = (C.c_void_p * k)()
        bp = (C.c_void_p * k)()
        # one flag covers every problem's pointers: all on the device or all on the host
        on_dev = 1 if k and hasattr(problems[0][0], "is_cuda") and problems[0][0].is_cuda else 0
        for i, (A, b) in enumerate(problems):
            fn = f"tls_batch_create_dense (problem {i})"
            if bool(hasattr(A, "is_cuda") and A.is_cuda) != bool(on_dev):
                _arg_error(fn, "problems must be all on the device or all on the host")
            if on_dev:
                m, n, lda = _device_dense(fn, A, b)
                ms[i], ns[i], ld[i] = m, n, lda
                ap[i], bp[i] = A.data_ptr(), b.data_ptr()
            else:
                A, b = _host_dense(fn, A, b)
                m, n = A.shape
                ms[i], ns[i], ld[i] = m, n, n
                ap[i], bp[i] = A.ctypes.data, b.ctypes.data
            self._keep.append((A, b))
            self.shapes.append((m, n))
        h = C.c_void_p()
        st = lib.tls_batch_create_dense(C.byref(h), k, ms, ns, ap, ld, bp, on_dev,
                                        C.c_void_p(stream) if stream else None)
        self._keep = None
        if st != 0:
            raise TLSError(st, "tls_batch_create_dense")
        self.h = h

    def _err(self, st):
        if st != 0:
            raise TLSError(st, (load().tls_batch_last_error(self.h) or b"").decode())

    def factor(self, u_f="fp16", **opt):
        o = tls_default_options(**opt)
        uf = PREC[u_f] if isinstance(u_f, str) else int(u_f)
        self._err(load().tls_batch_factor(self.h, uf, C.byref(o)))

    def solve(self, tol: float = 0.0, max_rqi: int = 10, check: bool = True):
        """Returns (list of x, sigma array, list of info dicts, per-problem statuses)."""
        k = self.k
        xs = [np.zeros(n) for _, n in self.shapes]
        xp = (_dp * k)(*[_ptr(x) for x in xs])
        sig = np.zeros(k)
        infos = (tls_info * k)()
        per = (C.c_int * k)()
        st = load().tls_batch_solve(self.h, tol, max_rqi, xp, _ptr(sig), infos, per)
        if check:
            self._err(st)
        return xs, sig, [i.as_dict() for i in infos], list(per)

    def set_selector(self, params, mean, scale):
        """Install the selector network (FP32 params, feature mean and scale) for factor("auto")."""
        fp = C.POINTER(C.c_float)
        P = np.ascontiguousarray(params, dtype=np.float32)
        mu = np.ascontiguousarray(mean, dtype=np.float32)
        sd = np.ascontiguousarray(scale, dtype=np.float32)
        if P.size != MLP_PARAMS or mu.size != N_FEATURES or sd.size != N_FEATURES:
            raise ValueError("selector: wrong parameter or feature sizes")
        self._err(load().tls_batch_set_selector(self.h, P.ctypes.data_as(fp), mu.ctypes.data_as(fp),
                                                sd.ctypes.data_as(fp)))

    def features(self) -> np.ndarray:
        """Raw selector features (count x 16) from the current factor."""
        F = np.zeros((self.k, N_FEATURES), dtype=np.float32)
        self._err(load().tls_batch_features(self.h, F.ctypes.data_as(C.POINTER(C.c_float))))
        return F

    def profile(self, on: bool = True):
        load().tls_batch_profile_enable(self.h, int(on))

    def profile_get(self) -> dict:
        """{class name: (launches, device ms, entries of A read)} for classes with launches."""
        out = {}
        for k, name in enumerate(PROF_CLASSES):
            c = C.c_int64()
            ms = C.c_double()
            el = C.c_int64()
            load().tls_batch_profile_get(self.h, k, C.byref(c), C.byref(ms))
            load().tls_batch_profile_elems(self.h, k, C.byref(el))
            if c.value:
                out[name] = (c.value, ms.value, el.value)
        return out

    def export_factor(self, i: int):
        """(R_H, d, H) of problem i, as tls_export_factor."""
        n = self.shapes[i][1]
        R = np.zeros((n, n))
        H = np.zeros((n, n))
        d = np.zeros(n)
        self._err(load().tls_batch_export_factor(self.h, i, _ptr(R), _ptr(d), _ptr(H)))
        return R, d, H

    def close(self):
        if getattr(self, "h", None):
            load().tls_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """Convenience owner of one context: create -> factor -> solve."""

    def __init__(self, A, b, u_f="fp16", u="fp32", stream=None, **opts):
        self.ctx = tls_create_dense(A, b, stream=stream)
        self.opt = tls_default_options(u=u, **opts)
        self.u_f = u_f

    def factor(self):
        tls_factor(self.ctx, self.u_f, self.opt)
        return self

    def solve(self, tol=0.0, max_rqi=10):
        return tls_solve(self.ctx, tol, max_rqi)

    def close(self):
        tls_destroy(self.ctx)
        self.ctx = None

    def __del__(self):
        try:
            if self.ctx:
                self.close()
        except Exception:
            pass
