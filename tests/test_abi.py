"""Host-side checks of the C ABI that need no GPU: the library builds and loads, it exports
every function the headers declare, and argument validation rejects bad input before any
device work."""
from __future__ import annotations

import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

from paper_2305_19028_gb300 import tls
from tests.conftest import ROOT


def _declared_functions() -> set[str]:
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(tls_[a-z_0-9]+)\s*\(", src):
            names.add(m.group(1))
    # typedef'd callback types are not functions
    return {n for n in names if not n.endswith("_fn")}


def test_library_exports_every_declared_symbol():
    lib = tls.load()
    declared = _declared_functions()
    assert declared, "no declarations found"
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"
    assert set(tls.EXPORTS) == declared


def test_status_strings():
    assert tls.tls_status_str(0) == "TLS_OK"
    assert tls.tls_status_str(5) == "TLS_ERR_FACTOR_BREAKDOWN"
    assert tls.tls_status_str(9) == "TLS_ERR_TIMEOUT"


def test_default_options():
    o = tls.tls_default_options()
    assert o.u == tls.TLS_FP32 and o.mode_A == 1 and o.cg_fixed == 1 and o.ls_iters > 0


def _create(m, n, A, b):
    lib = tls.load()
    ctx = C.c_void_p()
    st = lib.tls_create_dense(C.byref(ctx), m, n, A.ctypes.data_as(C.c_void_p), n,
                              b.ctypes.data_as(C.c_void_p), 0, None)
    return st, ctx


def test_create_rejects_bad_shapes_without_device():
    A = np.ones((3, 5))
    b = np.ones(3)
    st, ctx = _create(3, 5, A, b)          # m < n
    assert st == 1 and not ctx.value
    st, ctx = _create(0, 0, A, b)
    assert st == 1


@pytest.mark.gpu
def test_create_rejects_nan_inf():
    """NaN / Inf in A or b: TLS_ERR_ARG from the device-side check of the copy, for host and
    device pointers, the single context and the packed batch; the pool keeps working after."""
    import torch
    A = np.ones((70, 5))
    A[::3, 1] = 2.0
    b = np.arange(70.0)
    for where in ("A", "b"):
        for bad in (np.nan, np.inf, -np.inf):
            A2, b2 = A.copy(), b.copy()
            if where == "A":
                A2[69, 4] = bad
            else:
                b2[0] = bad
            st, ctx = _create(70, 5, A2, b2)
            assert st == 1 and not ctx.value
            with pytest.raises(tls.TLSError) as ei:
                tls.tls_create_dense(torch.from_numpy(A2).cuda(), torch.from_numpy(b2).cuda())
            assert ei.value.status == 1
            with pytest.raises(tls.TLSError) as ei:
                tls.Batch([(A, b), (A2, b2)])
            assert ei.value.status == 1
    ctx = tls.tls_create_dense(A, b)        # a clean problem still creates
    tls.tls_destroy(ctx)


def _create_csr(m, n, rp, ci, va, b):
    lib = tls.load()
    ctx = C.c_void_p()
    rp = np.ascontiguousarray(rp, dtype=np.int64)
    ci = np.ascontiguousarray(ci, dtype=np.int32)
    va = np.ascontiguousarray(va, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    st = lib.tls_create_csr(C.byref(ctx), m, n, int(rp[-1]), rp.ctypes.data_as(C.c_void_p),
                            ci.ctypes.data_as(C.c_void_p), va.ctypes.data_as(C.c_void_p),
                            b.ctypes.data_as(C.c_void_p), 0, None)
    if st == 0:
        lib.tls_destroy(ctx)
    return st, ctx


def test_csr_validation_on_host():
    """The checks made before any device work: sizes and the two end offsets."""
    va = np.ones(3)
    st, ctx = _create_csr(2, 2, [1, 2, 3], [0, 1, 0], va, np.ones(2))      # row_ptr[0] != 0
    assert st == 1 and not ctx.value
    st, _ = _create_csr(1, 2, [0, 3], [0, 1, 0], va, np.ones(1))           # m < n
    assert st == 1
    n = 60000                                                             # n above the limit
    st, _ = _create_csr(n, n, np.zeros(n + 1), np.zeros(0), np.zeros(0), np.ones(n))
    assert st == 1


@pytest.mark.gpu
def test_csr_validation_on_device():
    """Malformed structure or non-finite data: TLS_ERR_ARG from the device check, before the
    column index is built; a well-formed matrix still creates afterwards."""
    m, n = 5, 3
    rp = [0, 2, 3, 5, 6, 7]
    ci = [0, 2, 1, 0, 2, 1, 0]
    va = np.arange(1.0, 8.0)
    b = np.ones(m)
    st, _ = _create_csr(m, n, rp, ci, va, b)
    assert st == 0
    bad_cases = {
        "not increasing": (rp, [2, 0, 1, 0, 2, 1, 0], va, b),
        "duplicate": (rp, [0, 0, 1, 0, 2, 1, 0], va, b),
        "column >= n": (rp, [0, 3, 1, 0, 2, 1, 0], va, b),
        "negative column": (rp, [-1, 2, 1, 0, 2, 1, 0], va, b),
        "row_ptr decreasing": ([0, 2, 1, 5, 6, 7], ci, va, b),
        "row_ptr beyond nnz": ([0, 2, 9, 5, 6, 7], ci, va, b),
        "NaN value": (rp, ci, np.where(np.arange(7) == 4, np.nan, va), b),
        "Inf in b": (rp, ci, va, np.where(np.arange(m) == 4, np.inf, b)),
    }
    for name, (rp2, ci2, va2, b2) in bad_cases.items():
        st, ctx = _create_csr(m, n, rp2, ci2, va2, b2)
        assert st == 1 and not ctx.value, name
    st, _ = _create_csr(m, n, rp, ci, va, b)
    assert st == 0


def test_noalloc_binding_refuses_host_and_mistyped_tensors():
    # the binding checks dtype and device before it loads or calls the library
    torch = pytest.importorskip("torch")
    A = torch.zeros((8, 4), dtype=torch.float64)
    v8 = torch.zeros(8, dtype=torch.float64)
    v4 = torch.zeros(4, dtype=torch.float64)
    s5 = torch.zeros(5, dtype=torch.float64)
    with pytest.raises(tls.TLSError, match="float64 required"):
        tls.tls_residual_noalloc(A.float(), v8, v4, v4, s5)
    with pytest.raises(tls.TLSError, match="not on a CUDA device"):
        tls.tls_residual_noalloc(A, v8, v4, v4, s5)
    with pytest.raises(tls.TLSError, match="not a torch tensor"):
        tls.tls_residual_noalloc(A.numpy(), v8, v4, v4, s5)


def test_binding_checks_host_lengths_before_the_library_reads():
    """The library reads m, n or nnz entries from host pointers; the binding refuses arrays
    that are shorter (or longer) before the call, so nothing is read past an array's end."""
    A = np.ones((10, 3))
    with pytest.raises(tls.TLSError, match="b has 9 entries, 10 required"):
        tls.tls_create_dense(A, np.ones(9))
    with pytest.raises(tls.TLSError, match="A must be 2-D"):
        tls.tls_create_dense(np.ones(10), np.ones(10))
    rp, ci, va = [0, 1, 2, 3], [0, 1, 0], np.ones(3)
    with pytest.raises(tls.TLSError, match="row_ptr has 4 entries"):
        tls.tls_create_csr(4, 2, rp, ci, va, np.ones(4))
    with pytest.raises(tls.TLSError, match="col_idx has 2 entries"):
        tls.tls_create_csr(3, 2, rp, ci[:2], va, np.ones(3))
    with pytest.raises(tls.TLSError, match="val has 1 entries"):
        tls.tls_create_csr(3, 2, rp, ci, va[:1], np.ones(3))
    with pytest.raises(tls.TLSError, match="b has 2 entries"):
        tls.tls_create_csr(3, 2, rp, ci, va, np.ones(2))
    with pytest.raises(tls.TLSError, match="problem 1"):
        tls.Batch([(A, np.ones(10)), (A, np.ones(3))])
    with pytest.raises(tls.TLSError, match="y has 4 entries, 3 required"):
        tls._host_vec("tls_precond", "y", np.ones(4), 3)


def test_binding_checks_device_tensors_before_the_library_reads():
    """Device pointers are read as float64 arrays of the stated shape: dtype, placement,
    layout and lengths are checked in the binding (here on CPU tensors and stand-ins, so the
    checks run without a GPU)."""
    torch = pytest.importorskip("torch")
    A = torch.zeros((8, 4), dtype=torch.float64)
    b = torch.zeros(8, dtype=torch.float64)
    with pytest.raises(tls.TLSError, match="float64 required"):
        tls._device_dense("f", A.float(), b)
    with pytest.raises(tls.TLSError, match="not on a CUDA device"):
        tls._device_dense("f", A, b)
    with pytest.raises(tls.TLSError, match="not a torch tensor"):
        tls._device_dense("f", A.numpy(), b)

    class OnDevice:   # looks like a CUDA tensor to the placement test, is not a tensor
        is_cuda = True

    with pytest.raises(tls.TLSError, match="all on the device or all on the host"):
        tls.Batch([(np.ones((10, 3)), np.ones(10)), (OnDevice(), OnDevice())])
    with pytest.raises(tls.TLSError, match="not a torch tensor"):
        tls.Batch([(OnDevice(), OnDevice())])


def test_option_ranges_are_checked_on_the_host():
    """tls_options_check (the check tls_factor and tls_batch_factor apply before any device
    work): the defaults pass; a switch outside {0, 1}, an unbounded count or a non-finite or
    negative real is named."""
    assert tls.tls_options_check(tls.tls_default_options()) is None
    assert tls.tls_options_check(tls.tls_default_options(u="fp64", mode_A=2, factor=1,
                                                         cg_fixed=0, cg_max=100000,
                                                         max_shifts=30, psi_accept=float("inf"),
                                                         constraint_iters=60)) is None
    bad = {"u": 0, "mode_A": 3, "factor": 2, "cg_fixed": 2, "reproducible": -1, "cg_max": 0,
           "ls_iters": -1, "max_shifts": 31, "constraint_iters": 100001,
           "cg_tol": float("nan"), "psi_accept": -1.0, "constr_guard": float("inf"),
           "stall_ratio": -0.5, "hybrid_ratio": float("nan")}
    for field, value in bad.items():
        why = tls.tls_options_check(tls.tls_default_options(**{field: value}))
        assert why is not None and field in why, (field, value, why)


def test_selector_trainer_checks_its_tensors_before_the_kernels():
    """The training kernels read X, labels and indices by device pointer: the trainer refuses
    a wrong dtype, shape or placement before any call (checked here without a GPU)."""
    torch = pytest.importorskip("torch")
    from paper_2305_19028_gb300 import selector
    tr = selector.Trainer.__new__(selector.Trainer)   # no device parameters needed for the checks
    tr.torch = torch
    X = torch.zeros((5, 16), dtype=torch.float32)
    with pytest.raises(tls.TLSError, match="not on a CUDA device"):
        tr._check_X("f", X)
    with pytest.raises(tls.TLSError, match="float32 required"):
        tr._check_X("f", X.double())
    with pytest.raises(tls.TLSError, match="not a torch tensor"):
        tr.grad(X.numpy(), None, None, None)
    with pytest.raises(tls.TLSError, match="not on a CUDA device"):
        tr.forward(X)


def test_no_device_means_an_error_not_a_fallback():
    """Without a GPU the library reports the CUDA failure (a non-zero status, TLSError in the
    binding) instead of computing on the host; without libtls.so the binding raises at load."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    p_A = np.random.default_rng(0).standard_normal((50, 5))
    with pytest.raises(tls.TLSError) as ei:
        tls.tls_create_dense(p_A, np.ones(50))
    assert ei.value.status != 0
    import subprocess
    import sys
    code = ("from paper_2305_19028_gb300 import tls\n"
            "try:\n"
            "    tls.load(path='/nonexistent/libtls.so', build_if_missing=False)\n"
            "except RuntimeError as e:\n"
            "    print('raised:', e)\n")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT,
                       timeout=120)
    assert "raised: libtls.so not found" in r.stdout, r.stdout + r.stderr
