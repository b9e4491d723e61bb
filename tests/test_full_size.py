"""Full-size certification: the benchmark's workloads, solved on the GPU in the benchmark's launch
configuration, checked against the oracle's operator.

At these sizes the oracle cannot solve the systems itself (its CG would take hours), but it can
apply its operator: with the exchange first (Sect. 3.1's order), the step's final E is the result
of the implicit diffusion solve (Sect. 3.4), so the oracle's exchanged state and its D give the
true relative residual ||b - A E|| / ||b|| of the GPU result, which must meet the tolerance the
solve was asked for.  The exchanged gas energy is compared cell by cell.
"""
import numpy as np
import pytest
import torch

import lp_dt
import oracle
from paper_2104_03968_gb300 import inputs

pytestmark = pytest.mark.gpu

RTOL = 1e-8  # the benchmark's tolerance


def _host(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def ctx():
    from paper_2104_03968_gb300 import fld
    c = fld.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def lognormal512():
    """The 512^3 benchmark inputs (built on the GPU like the benchmark's) and the oracle's
    exchanged state and D on the host."""
    case = inputs.lognormal_3d(n=512, seed=2, device="cuda", dt_exp=lp_dt.stored("lognormal_3d_512_seed2"))
    g, p, dt = case["grid"], case["phys"], case["dt"]
    rho, eps, E = _host(case["rho"]), _host(case["eps"]), _host(case["E"])
    e1, E1, _ = oracle.exchange(p, dt, rho, oracle.opacity(p, rho, eps), eps, E)
    D1 = oracle.coeffs(g, p, E1, rho, oracle.opacity(p, rho, e1))
    yield {"case": case, "e1": e1, "E1": E1, "D1": D1}


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_lognormal512_step_meets_rtol_under_the_oracle_operator(ctx, lognormal512, precision):
    from paper_2104_03968_gb300 import fld
    case = lognormal512["case"]
    g, p, dt = case["grid"], case["phys"], case["dt"]
    eps, E = case["eps"].clone(), case["E"].clone()
    info = fld.step(ctx, g, dict(p, precision=precision, rtol=RTOL, order="exchange_then_diffuse"), dt, case["rho"],
                    eps, E)
    assert info["status"] == 0, info
    true = oracle.relres(g, dt, lognormal512["D1"], lognormal512["E1"], _host(E))
    # the oracle's exchanged state differs from the GPU's at the 1e-12 level, which moves the
    # residual by as much
    assert true <= RTOL * 1.01, (true, info)
    e_gpu = _host(eps)
    e1 = lognormal512["e1"]
    assert float(np.abs(e_gpu - e1).max() / np.abs(e1).max()) < 1e-12
    assert float((np.abs(e_gpu - e1) / np.abs(e1)).max()) < 1e-11


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_batched512_each_grid_meets_rtol_under_the_oracle_operator(ctx, precision):
    """All 512 uneven 2-D grids of the batched benchmark, in one call, grid by grid."""
    from paper_2104_03968_gb300 import fld
    cases = inputs.batched_2d(ngrids=512, seed=3, dt_exp=lp_dt.stored("batched_2d_512_seed3"))
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    params = [dict(c["phys"], precision=precision, rtol=RTOL, order="exchange_then_diffuse") for c in cases]
    E = [dev(c["E"]) for c in cases]
    eps = [dev(c["eps"]) for c in cases]
    infos = fld.step_batched(ctx, [c["grid"] for c in cases], params, [c["dt"] for c in cases],
                             [dev(c["rho"]) for c in cases], eps, E)
    worst = 0.0
    for c, i, tE in zip(cases, infos, E):
        assert i["status"] == 0, i
        p = c["phys"]
        e1, E1, _ = oracle.exchange(p, c["dt"], c["rho"], oracle.opacity(p, c["rho"], c["eps"]), c["eps"], c["E"])
        D = oracle.coeffs(c["grid"], p, E1, c["rho"], oracle.opacity(p, c["rho"], e1))
        true = oracle.relres(c["grid"], c["dt"], D, E1, _host(tE).reshape(E1.shape))
        worst = max(worst, true / RTOL)
    assert worst <= 1.01, worst
