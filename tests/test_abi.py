"""The C-ABI library builds for sm_103a and exports every entry point of include/fld.h;
the oracle builds.  No compute calls: these run without a GPU."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, "include", "fld.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"^FLD_API\s+[\w\s\*]+?\b(fld_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("fld_coeffs", "fld_diffuse", "fld_exchange", "fld_step", "fld_step_batched", "fld_columns_step",
                 "fld_ctx_create", "fld_ctx_destroy", "fld_last_error"):
        assert must in names


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="needs nvcc")
def test_library_exports_every_declared_symbol():
    from paper_2104_03968_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_oracle_builds_and_loads():
    import oracle
    path = oracle.build()
    assert os.path.exists(path)
    assert oracle.lam(0.0) == 1.0 / 3.0


def test_product_path_does_not_import_the_oracle():
    """The CUDA binding and the benchmark's GPU leg never reach the oracle package."""
    pkg = os.path.join(ROOT, "paper_2104_03968_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), f
                assert "fld_oracle" not in src, f
