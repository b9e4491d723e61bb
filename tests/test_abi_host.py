"""Host-side argument checks of the C ABI, called through the library without a GPU: every check
here returns before any CUDA call (a NULL context, the allocation-free column entry's argument
checks, an empty column batch), so these run on a machine with no device."""
import ctypes as ct
import os
import shutil

import numpy as np
import pytest

from paper_2104_03968_gb300 import fld, inputs

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="needs nvcc to build the library")

OK, INVALID, UNSUPPORTED = 0, 1, 7


@pytest.fixture(scope="module")
def lib():
    lib = fld.load()
    lib.fld_ctx_create.argtypes = [ct.POINTER(ct.c_void_p), ct.c_int]
    lib.fld_trace_enable.argtypes = [ct.c_void_p, ct.c_int]
    lib.fld_trace_enable.restype = ct.c_int
    lib.fld_trace_report.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_int, ct.c_void_p]
    lib.fld_trace_report.restype = ct.c_int
    lib.fld_columns_step_static.argtypes = [ct.c_int, ct.c_int, ct.c_void_p, ct.c_int, ct.c_int, ct.c_int] + \
        [ct.c_void_p] * 9
    lib.fld_columns_step_static.restype = ct.c_int
    return lib


def test_null_context_is_rejected_by_every_entry_point(lib):
    for name, args in fld._SIGS.items():
        if name in ("fld_ctx_create", "fld_ctx_destroy"):
            continue
        zeros = [0.0 if a is ct.c_double else 0 for a in args]
        zeros = [None if a is ct.c_void_p else z for a, z in zip(args, zeros)]
        assert getattr(lib, name)(*zeros) == INVALID, name
    assert lib.fld_ctx_create(None, 0) == INVALID
    assert lib.fld_ctx_destroy(None) == OK
    assert lib.fld_trace_enable(None, 1) == INVALID
    n = ct.c_int(-1)
    assert lib.fld_trace_report(None, None, 0, ct.byref(n)) == INVALID
    assert lib.fld_last_error(None) == b"null context"


def _params(**kw):
    return fld.params_struct(dict(inputs.cgs_units(0.6), opacity="const", kappa0=0.4, **kw), [], None)


def _static(lib, ncol, ncell, p, geometry=1, bc=(2, 2), arrays=True, info=None):
    buf = np.ones(max(1, ncol * ncell) + ncell + 1)  # host memory: never read on these paths
    ptr = buf.ctypes.data if arrays else None
    return lib.fld_columns_step_static(ncol, ncell, buf.ctypes.data, geometry, bc[0], bc[1], ptr, ptr,
                                       ct.byref(p), ptr, ptr, ptr, ptr,
                                       None if info is None else ct.byref(info), None)


def test_static_column_entry_checks_its_arguments_on_the_host(lib):
    p = _params()
    assert _static(lib, 4, fld.STATIC_MAX_CELLS + 1, p) == UNSUPPORTED
    assert _static(lib, -1, 64, p) == INVALID
    assert _static(lib, 4, 1, p) == INVALID          # at least two cells per column
    assert _static(lib, 4, 64, p, geometry=5) == INVALID
    assert _static(lib, 4, 64, p, bc=(2, 4)) == INVALID  # the luminosity face is the inner one
    assert _static(lib, 4, 64, p, bc=(0, 2)) == INVALID  # columns take no periodic face
    assert _static(lib, 4, 64, p, arrays=False) == INVALID
    bad = _params()
    bad.c = 0.0
    assert _static(lib, 0, 64, bad) == INVALID       # parameters are checked even for no columns


def test_empty_column_batch_returns_ok_without_the_device(lib):
    info = fld.Info()
    info.status, info.exch_max_iters, info.cycles = 9, 9, 9
    n0 = lib.fld_launch_count()
    assert _static(lib, 0, 64, _params(), arrays=False, info=info) == OK
    assert (info.status, info.exch_max_iters, info.cycles) == (0, 0, 0)
    assert lib.fld_launch_count() == n0
