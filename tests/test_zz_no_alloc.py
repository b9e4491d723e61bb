"""The allocation-free column entry point, fld_columns_step_static.

Callers that cannot allocate device memory while they step the radiation field (a host code
whose memory pool owns the GPU, a runtime that forbids allocation inside its time-step loop)
use this entry point: it takes the same arguments as fld_columns_step minus the context and
keeps its scratch in a static device array.  This file runs last so that a failure here does
not hide the other GPU tests; it also passes when run alone in a fresh process.
"""
import numpy as np
import pytest
import torch

import lp_dt
from paper_2104_03968_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def _relerr(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("order", ["diffuse_then_exchange", "exchange_then_diffuse", "imex_midpoint"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_static_entry_matches_context_entry_twice(order, precision):
    from paper_2104_03968_gb300 import fld
    ctx = fld.Context(0)
    case = lp_dt.columns_dt(inputs.wind_columns(ncol=37, ncell=2048, seed=6))
    p = dict(case["phys"], order=order, precision=precision)
    bc = tuple(case["bc"])
    # reference: the context entry point, two steps in a row
    eps_r, E_r = _dev(case["eps"]), _dev(case["E"])
    rho = _dev(case["rho"])
    for _ in range(2):
        fld.columns_step(ctx, case["r_faces"], "spherical", bc, case["bc_lo"], case["bc_hi"], p, case["dt"], rho,
                         eps_r, E_r)
    # the allocation-free entry point on caller-owned buffers, two calls in a row
    rf, vlo, vhi, dt = (_dev(case[k]) for k in ("r_faces", "bc_lo", "bc_hi", "dt"))
    eps_s, E_s = _dev(case["eps"]), _dev(case["E"])
    infos = []
    for _ in range(2):
        infos.append(fld.columns_step_static(rf, "spherical", bc, vlo, vhi, p, dt, rho, eps_s, E_s))
    torch.cuda.synchronize()
    for info in infos:
        assert info["status"] == 0 and info["bisection_fallbacks"] == 0
    assert _relerr(E_s, E_r) < TOL
    assert _relerr(eps_s, eps_r) < TOL
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_static_entry_matches_oracle(precision):
    """One step of the allocation-free entry point against the oracle's column step, column by
    column (the paper's order: exchange, then the implicit diffusion)."""
    import oracle
    from paper_2104_03968_gb300 import fld
    case = lp_dt.columns_dt(inputs.wind_columns(ncol=5, ncell=2048, seed=7))
    order = "exchange_then_diffuse"
    p = dict(case["phys"], order=order, precision=precision)
    bc = tuple(case["bc"])
    rf, vlo, vhi, dt = (_dev(case[k]) for k in ("r_faces", "bc_lo", "bc_hi", "dt"))
    eps, E = _dev(case["eps"]), _dev(case["E"])
    info = fld.columns_step_static(rf, "spherical", bc, vlo, vhi, p, dt, _dev(case["rho"]), eps, E)
    torch.cuda.synchronize()
    assert info["status"] == 0
    col = {"r_faces": case["r_faces"], "geometry": "spherical", "bc": case["bc"]}
    for j in range(5):
        e_o, E_o, _ = oracle.column_step(col, p, case["dt"][j], case["rho"][j], case["eps"][j], case["E"][j],
                                         case["bc_lo"][j], case["bc_hi"][j], order=order)
        got_E, got_e = E[j].cpu().numpy(), eps[j].cpu().numpy()
        assert float(np.abs(got_E - E_o).max() / np.abs(E_o).max()) < TOL
        assert float(np.abs(got_e - e_o).max() / np.abs(e_o).max()) < TOL


def test_static_entry_rejects_oversized_columns():
    from paper_2104_03968_gb300 import fld
    n = fld.STATIC_MAX_CELLS + 1
    rf = _dev(np.linspace(1.0, 2.0, n + 1))
    one = _dev(np.ones((1, n)))
    v = _dev(np.ones(1))
    with pytest.raises(fld.FldError) as e:
        fld.columns_step_static(rf, "cartesian", ("dirichlet", "dirichlet"), v, v, inputs.code_units(), v, one,
                                one.clone(), one.clone())
    assert e.value.status == 7
