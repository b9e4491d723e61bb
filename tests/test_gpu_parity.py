"""CUDA path (through the C ABI) against the FP64 CPU oracle on the same seeded inputs.

Tolerances: FP64 results within 1e-10 relative (max-norm over the field, so cells at the
1e-6 floor do not dominate); the mixed form's residual, measured with the oracle's own FP64
operator, within its rtol.  Integer diagnostics are compared exactly where they are unique.
"""
import numpy as np
import pytest
import torch

import oracle
import lp_dt
from paper_2104_03968_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def ctx():
    from paper_2104_03968_gb300 import fld
    c = fld.Context(0)
    yield c
    c.close()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def relerr(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def solver(phys, **kw):
    p = dict(phys)
    p.update(kw)
    return p


BCS = {
    "periodic": (["periodic"] * 6, [0.0] * 6),
    "neumann": (["neumann"] * 6, [0.05, -0.02, 0.0, 0.1, 0.03, 0.0]),
    "dirichlet": (["dirichlet"] * 6, [0.8, 1.2, 0.5, 0.9, 1.1, 0.3]),
    "mixed": (["dirichlet", "neumann", "periodic", "periodic", "neumann", "dirichlet"], [1.5, 0.2, 0, 0, -0.1, 0.7]),
    "continuous": (["continuous"] * 4 + ["periodic"] * 2, [0.0] * 6),
}


# ----------------------------------------------------------------------------- coefficients

@pytest.mark.parametrize("shape", [(70, 45), (24, 20, 18), (300,)])
@pytest.mark.parametrize("bcname", ["periodic", "neumann", "dirichlet", "mixed", "continuous"])
@pytest.mark.parametrize("limiter", ["lp", "third", "minerbo"])
def test_coeffs_parity(ctx, shape, bcname, limiter):
    from paper_2104_03968_gb300 import fld
    case = inputs.random_small(shape, seed=len(shape) * 7 + len(bcname), bc=BCS[bcname], limiter=limiter)
    g, p = case["grid"], case["phys"]
    kap_o = oracle.opacity(p, case["rho"], case["eps"])
    D_o = oracle.coeffs(g, p, case["E"], case["rho"], kap_o)
    kap, D = fld.coeffs(ctx, g, p, dev(case["E"]), dev(case["rho"]), dev(case["eps"]))
    torch.cuda.synchronize()
    assert relerr(host(kap).reshape(kap_o.shape), kap_o) < 1e-13
    assert np.abs(host(D).reshape(D_o.shape) / D_o - 1).max() < 1e-12


@pytest.mark.parametrize("scaling", ["cgs", "per_cell"])
@pytest.mark.parametrize("limiter", ["lp", "third", "minerbo"])
def test_coeffs_unit_scales(ctx, scaling, limiter):
    """Coefficients in cgs units (values from 1e-21 to 1e25: the double-float path throughout) and
    with per-cell factors over tens of decades (cells whose values leave the double-float window
    take the FP64 path): every cell matches the oracle."""
    from paper_2104_03968_gb300 import fld
    rng = np.random.default_rng(23)
    shape = (40, 36, 12)
    arr = tuple(reversed(shape))
    phys = inputs.cgs_units(0.6, limiter=limiter)
    phys.update(opacity="kramers", kappa0=4e25, kr_a=1.0, kr_b=-3.5)
    rho = 1e-9 * np.exp(0.8 * inputs.smooth_field(rng, arr))
    T = 1e6 * (1 + 0.3 * inputs.smooth_field(rng, arr))
    E = inputs.rad_energy(phys, T * (1 + 0.1 * inputs.smooth_field(rng, arr)))
    eps = inputs.equilibrium_eps(phys, rho, T)
    if scaling == "per_cell":
        E = E * 10 ** rng.uniform(-12, 12, arr)
        rho = rho * 10 ** rng.uniform(-4, 4, arr)
        eps = eps * 10 ** rng.uniform(-4, 4, arr)
    g = inputs.periodic_grid(shape, dx=1e10)
    kap_o = oracle.opacity(phys, rho, eps)
    D_o = oracle.coeffs(g, phys, E, rho, kap_o)
    assert np.isfinite(D_o).all() and (D_o > 0).all()  # the case stays inside FP64's range
    kap, D = fld.coeffs(ctx, g, phys, dev(E), dev(rho), dev(eps))
    torch.cuda.synchronize()
    assert np.abs(host(kap).reshape(kap_o.shape) / kap_o - 1).max() < 1e-13
    assert np.abs(host(D).reshape(D_o.shape) / D_o - 1).max() < 1e-12


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_opacity_table_over_its_range(ctx, precision):
    """The tabulated opacity (bilinear in log10 rho, log10 T on log10 kappa, clamped at the edges)
    over and beyond the table's range: the mixed precision's double-float logarithms and power
    of ten, and the FP64 ones, against the oracle."""
    from paper_2104_03968_gb300 import fld
    case = inputs.wind_columns(ncol=2, ncell=64)
    p = dict(case["phys"], precision=precision)
    rng = np.random.default_rng(11)
    n = 200000
    lrho = rng.uniform(-17.0, -5.0, n)   # the table covers -16 .. -6
    lT = rng.uniform(3.5, 6.8, n)        # and 3.7 .. 6.5
    # grid nodes and cell midpoints of the table exactly, where the interpolation weights are 0 or 1/2
    lrho[:128] = np.linspace(-16.0, -6.0, 128)
    lT[128:256] = np.linspace(3.7, 6.5, 128)
    rho = 10.0 ** lrho
    T = 10.0 ** lT
    eps = rho * p["gas_R"] * T / (p["gamma"] - 1.0)  # T = (gamma - 1) eps / (rho gas_R)
    kap_o = oracle.opacity(case["phys"], rho, eps)
    kap = host(fld.opacity(ctx, p, dev(rho), dev(eps)))
    assert np.abs(kap / kap_o - 1).max() < 1e-13


def test_coeffs_table_opacity(ctx):
    from paper_2104_03968_gb300 import fld
    case = inputs.wind_columns(ncol=4, ncell=64)
    p = case["phys"]
    n = case["rho"].size
    g = {"ndim": 1, "n": [n, 1, 1], "dx": [1.0, 1, 1], "bc": ["continuous"] * 2 + ["periodic"] * 4,
         "bc_val": [0.0] * 6}
    rho, eps, E = case["rho"].ravel(), case["eps"].ravel(), case["E"].ravel()
    kap_o = oracle.opacity(p, rho, eps)
    kap, D = fld.coeffs(ctx, g, p, dev(E), dev(rho), dev(eps))
    torch.cuda.synchronize()
    assert np.abs(host(kap) / kap_o - 1).max() < 1e-12


# ----------------------------------------------------------------------------- exchange

@pytest.mark.parametrize("units", ["code", "cgs"])
def test_exchange_parity(ctx, units):
    from paper_2104_03968_gb300 import fld
    rng = np.random.default_rng(17)
    n = 100_003  # several blocks and a ragged tail
    if units == "code":
        phys = inputs.code_units()
        rho, kap = 10 ** rng.uniform(-3, 3, n), 10 ** rng.uniform(-3, 3, n)
        eps, E = 10 ** rng.uniform(-4, 4, n), 10 ** rng.uniform(-4, 4, n)
        dts = (1e-4, 1.0, 1e4)
    else:
        phys = inputs.cgs_units(0.6)
        rho, kap = 10 ** rng.uniform(-12, -4, n), 10 ** rng.uniform(-1, 2, n)
        T = 10 ** rng.uniform(3.5, 7, n)
        eps = inputs.equilibrium_eps(phys, rho, T * 10 ** rng.uniform(-2, 2, n))
        E = inputs.rad_energy(phys, T)
        dts = (1e-14, 1e-10, 1e-6)
    for dt in dts:
        e_o, E_o, _ = oracle.exchange(phys, dt, rho, kap, eps, E)
        te, tE = dev(eps), dev(E)
        info = fld.exchange(ctx, phys, dt, dev(rho), te, tE, kappa=dev(kap))
        assert np.abs(host(te) / e_o - 1).max() < 1e-12
        assert np.abs(host(tE) / E_o - 1).max() < 1e-12
        assert info["bisection_fallbacks"] == 0
        assert info["status"] == 0


def test_exchange_extreme_coefficients_take_fp64_path(ctx):
    """Coefficients outside the FP32-safe range (very hot gas with a huge dt) still give the
    root of the quartic."""
    from paper_2104_03968_gb300 import fld
    phys = inputs.code_units()
    rho = np.array([1e-8, 1.0, 1e6, 1.0])
    kap = np.array([1e8, 1e-9, 1e3, 1.0])
    eps = np.array([1e10, 1e-20, 1e-12, 0.0])
    E = np.array([1e-10, 1e20, 1e12, 2.0])
    for dt in (1e-8, 1e8):
        e_o, E_o, _ = oracle.exchange(phys, dt, rho, kap, eps, E)
        te, tE = dev(eps), dev(E)
        fld.exchange(ctx, phys, dt, dev(rho), te, tE, kappa=dev(kap))
        assert np.allclose(host(te), e_o, rtol=1e-12, atol=0)
        assert np.allclose(host(tE), E_o, rtol=1e-12, atol=0)


def test_exchange_heating_cooling_setup(ctx):
    """The paper's heating/cooling relaxation (Sect. 4.1) stepped on the GPU matches the oracle
    step by step."""
    from paper_2104_03968_gb300 import fld
    for ratio in (1e-6, 1e2):
        for dt in (1e-12, 1e-11):
            case = inputs.heating_cooling(ratio, dt)
            p = case["phys"]
            kap = np.full_like(case["rho"], 0.4)
            eo, Eo = case["eps"].copy(), case["E"].copy()
            te, tE = dev(eo), dev(Eo)
            for _ in range(50):
                eo, Eo, _ = oracle.exchange(p, dt, case["rho"], kap, eo, Eo)
                fld.exchange(ctx, p, dt, dev(case["rho"]), te, tE, kappa=dev(kap))
            assert np.abs(host(te) / eo - 1).max() < 1e-11
            assert np.abs(host(tE) / Eo - 1).max() < 1e-11


# ----------------------------------------------------------------------------- diffusion

@pytest.mark.parametrize("shape", [(64, 48), (32, 24, 16), (256,)])
@pytest.mark.parametrize("bcname", ["periodic", "neumann", "dirichlet", "mixed"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_diffuse_parity(ctx, shape, bcname, precision):
    from paper_2104_03968_gb300 import fld
    case = inputs.random_small(shape, seed=3 + len(shape), bc=BCS[bcname], dt_factor=100.0)
    g, p = case["grid"], case["phys"]
    kap = oracle.opacity(p, case["rho"], case["eps"])
    D = oracle.coeffs(g, p, case["E"], case["rho"], kap)
    ref = oracle.diffuse(g, case["dt"], D, case["E"], rtol=1e-14)
    rtol = 1e-13 if precision == "fp64" else 1e-12
    out, info = fld.diffuse(ctx, g, solver(p, precision=precision, rtol=rtol), case["dt"], dev(D), dev(case["E"]))
    x = host(out).reshape(ref.shape)
    assert info["status"] == 0, info
    assert info["rel_residual"] <= rtol
    assert oracle.relres(g, case["dt"], D, case["E"], x) < 3 * rtol
    assert relerr(x, ref) < TOL


@pytest.mark.parametrize("shape,bcname", [((256, 40, 8), "periodic"), ((128, 36, 20), "mixed"),
                                           ((96, 24, 16), "dirichlet")])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_wavefront_sweep_equals_two_pass(shape, bcname, precision, monkeypatch):
    """The wavefront sweep (large 3-D levels) against the two-launch red-black sweep, forced on
    and off by the level-size threshold: the same per-cell arithmetic in the same colour order,
    so the iterates agree bit for bit; and both against the oracle.  The shapes give ragged row
    chunks (x rows of 128 and 64 colour cells) and a periodic and two bounded z axes."""
    from paper_2104_03968_gb300 import fld
    case = inputs.random_small(shape, seed=40 + len(bcname), bc=BCS[bcname], dt_factor=100.0)
    g, p = case["grid"], case["phys"]
    kap = oracle.opacity(p, case["rho"], case["eps"])
    D = oracle.coeffs(g, p, case["E"], case["rho"], kap)
    ref = oracle.diffuse(g, case["dt"], D, case["E"], rtol=1e-14)
    rtol = 1e-13 if precision == "fp64" else 1e-12
    res = []
    for threshold in ("1000000000000", "1"):
        monkeypatch.setenv("FLD_WAVE_MIN_CELLS", threshold)
        c = fld.Context(0)
        # fixed sweep counts: the autotuner could pick different ones for the two contexts
        out, info = fld.diffuse(c, g, solver(p, precision=precision, rtol=rtol, nu1=2, nu2=2), case["dt"], dev(D),
                                dev(case["E"]))
        torch.cuda.synchronize()
        res.append((host(out).reshape(ref.shape), info))
        c.close()
    (x0, i0), (x1, i1) = res
    assert i0["status"] == 0 and i1["status"] == 0
    assert i0["cycles"] == i1["cycles"]
    assert np.array_equal(x0, x1)
    assert relerr(x1, ref) < TOL


@pytest.mark.parametrize("shape,bcname", [((64, 64, 64), "periodic"), ((96, 64), "mixed"), ((128,), "dirichlet")])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fmg_start(ctx, shape, bcname, precision):
    """Full-multigrid first cycle (Sect. 3.4) and plain V-cycle start reach the same discrete
    solution; the FMG start needs no more cycles."""
    from paper_2104_03968_gb300 import fld
    case = inputs.random_small(shape, seed=60 + len(shape), bc=BCS[bcname], dt_factor=100.0)
    g, p = case["grid"], case["phys"]
    kap = oracle.opacity(p, case["rho"], case["eps"])
    D = oracle.coeffs(g, p, case["E"], case["rho"], kap)
    ref = oracle.diffuse(g, case["dt"], D, case["E"], rtol=1e-14)
    rtol = 1e-13 if precision == "fp64" else 1e-12
    cyc = {}
    for start in ("vcycle", "fmg"):
        out, info = fld.diffuse(ctx, g, solver(p, precision=precision, rtol=rtol, start=start, nu1=2, nu2=2),
                                case["dt"], dev(D), dev(case["E"]))
        assert info["status"] == 0, (start, info)
        assert relerr(host(out).reshape(ref.shape), ref) < TOL
        cyc[start] = info["cycles"]
    assert cyc["fmg"] <= cyc["vcycle"]


@pytest.mark.parametrize("shape,bcname", [((32, 24, 16), "periodic"), ((64, 48), "mixed"), ((48, 32, 24), "dirichlet")])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_diffuse_diagonal_tensor(ctx, shape, bcname, precision):
    """fld_diffuse_aniso: one heterogeneous D per axis, against the oracle's per-axis operator."""
    from paper_2104_03968_gb300 import fld
    case = inputs.random_small(shape, seed=90 + len(shape), bc=BCS[bcname], dt_factor=50.0)
    g, p = case["grid"], case["phys"]
    kap = oracle.opacity(p, case["rho"], case["eps"])
    D = oracle.coeffs(g, p, case["E"], case["rho"], kap)
    rng = np.random.default_rng(91)
    Dax = [D * np.exp(0.5 * rng.standard_normal(D.shape)) * f for f in (1.0, 0.3, 2.0)[:len(shape)]]
    ref = oracle.diffuse(g, case["dt"], Dax, case["E"], rtol=1e-14)
    rtol = 1e-13 if precision == "fp64" else 1e-12
    out, info = fld.diffuse_aniso(ctx, g, solver(p, precision=precision, rtol=rtol), case["dt"], [dev(d) for d in Dax],
                                  dev(case["E"]))
    assert info["status"] == 0, info
    x = host(out).reshape(ref.shape)
    assert oracle.relres(g, case["dt"], Dax, case["E"], x) < 3 * rtol
    assert relerr(x, ref) < TOL


def test_launch_count(ctx):
    """fld_launch_count counts the kernels of a step, those replayed in CUDA graphs included: two
    identical steps (same state, same cycles) count the same, and a 3-D multigrid step with
    several levels launches more kernels than it has levels x sweeps."""
    from paper_2104_03968_gb300 import fld
    case = inputs.random_small((64, 48, 40), seed=3, dt_factor=30.0)
    p = solver(case["phys"], rtol=1e-8, nu1=2, nu2=2)
    counts, cycles = [], []
    for _ in range(3):
        eps, E = dev(case["eps"]), dev(case["E"])
        n0 = fld.launch_count()
        info = fld.step(ctx, case["grid"], p, case["dt"], dev(case["rho"]), eps, E)
        torch.cuda.synchronize()
        counts.append(fld.launch_count() - n0)
        cycles.append(info["cycles"])
    assert cycles[1] == cycles[2] and counts[1] == counts[2], (counts, cycles)
    assert counts[2] > 4 * 2 * 2 * cycles[2]
    cases = lp_dt.batched_dt(inputs.batched_2d(ngrids=6, seed=9, nmin=64, nmax=128))
    args = ([c["grid"] for c in cases], [solver(c["phys"], rtol=1e-8) for c in cases], [c["dt"] for c in cases],
            [dev(c["rho"]) for c in cases])
    fld.step_batched(ctx, *args, [dev(c["eps"]) for c in cases], [dev(c["E"]) for c in cases])  # builds the graph
    n0 = fld.launch_count()
    fld.step_batched(ctx, *args, [dev(c["eps"]) for c in cases], [dev(c["E"]) for c in cases])
    assert fld.launch_count() - n0 > 10


@pytest.mark.parametrize("order", ["diffuse_then_exchange", "exchange_then_diffuse"])
@pytest.mark.parametrize("kind", ["numpy", "pinned"])
def test_step_on_host_arrays_equals_device_step(ctx, order, kind):
    """fld_step_host (host arrays, copies pipelined with the coefficient and exchange kernels over
    8 cell ranges) gives bit for bit the result of fld_step on device arrays."""
    from paper_2104_03968_gb300 import fld
    case = inputs.random_small((48, 40, 32), seed=5, bc=BCS["mixed"], dt_factor=30.0)
    g = case["grid"]
    p = solver(case["phys"], rtol=1e-10, nu1=2, nu2=2, order=order)
    eps_d, E_d = dev(case["eps"]), dev(case["E"])
    info_d = fld.step(ctx, g, p, case["dt"], dev(case["rho"]), eps_d, E_d)
    if kind == "numpy":
        rho_h, eps_h, E_h = case["rho"].copy(), case["eps"].copy(), case["E"].copy()
    else:
        rho_h, eps_h, E_h = (torch.as_tensor(np.ascontiguousarray(a)).pin_memory()
                             for a in (case["rho"], case["eps"], case["E"]))
    info_h = fld.step(ctx, g, p, case["dt"], rho_h, eps_h, E_h)
    assert info_h["status"] == info_d["status"] == 0
    assert info_h["cycles"] == info_d["cycles"]
    assert np.array_equal(np.asarray(eps_h).ravel(), host(eps_d).ravel())
    assert np.array_equal(np.asarray(E_h).ravel(), host(E_d).ravel())
    assert np.array_equal(np.asarray(rho_h).ravel(), np.asarray(case["rho"]).ravel())  # rho is read only


@pytest.mark.parametrize("shape,bcname", [((64, 48, 40), "periodic"), ((48, 40, 32), "neumann"), ((96, 64), "mixed")])
@pytest.mark.parametrize("start", ["fmg", "vcycle"])
def test_mixed_reported_residual_is_the_true_one(ctx, shape, bcname, start):
    """The relative residual the mixed solver reports after its double-float residual updates is
    the oracle's ||b - A x|| / ||b|| of the returned x (E of order 1, so that a wrong scaling by
    rms(b) would show), for several stopping points."""
    from paper_2104_03968_gb300 import fld
    case = inputs.random_small(shape, seed=100 + len(shape) + len(bcname), bc=BCS[bcname], dt_factor=100.0)
    g, p = case["grid"], case["phys"]
    kap = oracle.opacity(p, case["rho"], case["eps"])
    D = oracle.coeffs(g, p, case["E"], case["rho"], kap)
    for rtol in (1e-3, 1e-6, 1e-8):
        out, info = fld.diffuse(ctx, g, solver(p, precision="mixed", rtol=rtol, nu1=2, nu2=2, start=start), case["dt"],
                                dev(D), dev(case["E"]))
        assert info["status"] == 0 and info["cycles"] >= 1, info
        x = host(out).reshape(case["E"].shape)
        true = oracle.relres(g, case["dt"], D, case["E"], x)
        assert abs(true / info["rel_residual"] - 1) < 1e-3, (rtol, true, info)
        assert true <= rtol


@pytest.mark.parametrize("shape,bcname", [((64, 48, 40), "periodic"), ((96, 64), "mixed"), ((48, 40, 32), "neumann"),
                                          ((40, 32, 24), "dirichlet"), ((80, 48), "continuous"), ((512,), "mixed")])
@pytest.mark.parametrize("rtol", [1e-8, 1e-10])
def test_mixed_double_float_setup(ctx, shape, bcname, rtol):
    """At rtol >= 1e-10 the mixed solver builds its finest level (weights, diagonal, rhs, first
    residual) in double-float arithmetic; the oracle's FP64 operator applied to the result must
    meet rtol, whatever the boundary conditions."""
    from paper_2104_03968_gb300 import fld
    case = inputs.random_small(shape, seed=100 + len(shape) + len(bcname), bc=BCS[bcname], dt_factor=100.0)
    g, p = case["grid"], case["phys"]
    kap = oracle.opacity(p, case["rho"], case["eps"])
    D = oracle.coeffs(g, p, case["E"], case["rho"], kap)
    out, info = fld.diffuse(ctx, g, solver(p, precision="mixed", rtol=rtol), case["dt"], dev(D), dev(case["E"]))
    assert info["status"] == 0, info
    x = host(out).reshape(case["E"].shape)
    assert oracle.relres(g, case["dt"], D, case["E"], x) <= 1.01 * rtol
    if bcname != "continuous":  # the oracle's CG needs a symmetric operator
        ref = oracle.diffuse(g, case["dt"], D, case["E"], rtol=1e-14)
        assert relerr(x, ref) < 1e3 * rtol


@pytest.mark.parametrize("scale", [1e-25, 1e30])
def test_mixed_double_float_setup_out_of_window(ctx, scale):
    """E outside the double-float window [2^-77, 2^90) (|E| ~ 1e-25 or 1e30): the setup falls back to
    FP64 and the solve still meets rtol (the problem is linear, so the solution scales with E)."""
    from paper_2104_03968_gb300 import fld
    case = inputs.random_small((48, 40, 32), seed=7, bc=BCS["periodic"], dt_factor=100.0)
    g, p = case["grid"], case["phys"]
    kap = oracle.opacity(p, case["rho"], case["eps"])
    D = oracle.coeffs(g, p, case["E"], case["rho"], kap)
    E = case["E"] * scale
    out, info = fld.diffuse(ctx, g, solver(p, precision="mixed", rtol=1e-8), case["dt"], dev(D), dev(E))
    assert info["status"] == 0, info
    x = host(out).reshape(E.shape)
    assert oracle.relres(g, case["dt"], D, E, x) <= 1.01e-8


def test_diffuse_continuous_boundary(ctx):
    from paper_2104_03968_gb300 import fld
    case = inputs.random_small((32, 16), seed=5, bc=BCS["continuous"], dt_factor=2.0)
    g, p = case["grid"], case["phys"]
    kap = oracle.opacity(p, case["rho"], case["eps"])
    D = oracle.coeffs(g, p, case["E"], case["rho"], kap)
    ref = oracle.diffuse(g, case["dt"], D, case["E"], method="dense")
    out, info = fld.diffuse(ctx, g, solver(p, rtol=1e-13), case["dt"], dev(D), dev(case["E"]))
    assert info["status"] == 0, info
    assert relerr(host(out).reshape(ref.shape), ref) < TOL


def test_diffuse_fourier_closed_form(ctx):
    """Uniform D, periodic: the GPU solve hits the Fourier closed form of backward Euler."""
    from paper_2104_03968_gb300 import fld
    rng = np.random.default_rng(1)
    n = (40, 24, 32)
    g = {"ndim": 3, "n": list(n), "dx": [1.0, 0.5, 2.0], "bc": ["periodic"] * 6, "bc_val": [0.0] * 6}
    E = 1 + rng.random(tuple(reversed(n)))
    Dval, dt = 0.37, 3.3
    out, info = fld.diffuse(ctx, g, solver(inputs.code_units(), rtol=1e-14, max_cycles=200), dt,
                            dev(np.full(E.shape, Dval)), dev(E))
    shape = E.shape
    sym = np.zeros(shape)
    for ax, dxa in zip(range(3), (2.0, 0.5, 1.0)):
        k = 2 * np.pi * np.fft.fftfreq(shape[ax])
        s = (4.0 / dxa ** 2) * np.sin(k / 2) ** 2
        sl = [None] * 3
        sl[ax] = slice(None)
        sym = sym + s[tuple(sl)]
    ref = np.real(np.fft.ifftn(np.fft.fftn(E) / (1 + dt * Dval * sym)))
    assert relerr(host(out), ref) < 1e-12


def test_diffuse_in_place_alias(ctx):
    from paper_2104_03968_gb300 import fld
    case = inputs.random_small((32, 32), seed=9)
    g, p = case["grid"], case["phys"]
    kap = oracle.opacity(p, case["rho"], case["eps"])
    D = oracle.coeffs(g, p, case["E"], case["rho"], kap)
    ref = oracle.diffuse(g, case["dt"], D, case["E"], rtol=1e-14)
    E = dev(case["E"])
    fld.diffuse(ctx, g, solver(p, rtol=1e-13), case["dt"], dev(D), E, out=E)
    assert relerr(host(E), ref) < TOL


# ----------------------------------------------------------------------------- full step

@pytest.mark.parametrize("order", ["diffuse_then_exchange", "exchange_then_diffuse", "imex_midpoint"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_step_parity_lognormal(ctx, order, precision):
    from paper_2104_03968_gb300 import fld
    case = lp_dt.grid_dt(inputs.lognormal_3d(n=32, seed=11))
    g, p = case["grid"], case["phys"]
    e_o, E_o, _ = oracle.step(g, p, case["dt"], case["rho"], case["eps"], case["E"], order=order, rtol=1e-14)
    eps, E = dev(case["eps"]), dev(case["E"])
    rtol = 1e-13 if precision == "fp64" else 1e-12
    info = fld.step(ctx, g, solver(p, precision=precision, rtol=rtol, order=order), case["dt"], dev(case["rho"]), eps, E)
    assert info["status"] == 0
    assert relerr(host(E), E_o) < TOL
    assert relerr(host(eps), e_o) < TOL


def test_gaussian_pulse_twenty_steps(ctx):
    """64x64 Gaussian pulse: 20 steps at 10x the explicit limit to 1e-12, then 10 exchange steps
    from T_gas = 2 T_rad; every step against the oracle."""
    from paper_2104_03968_gb300 import fld
    case = inputs.gaussian_pulse_2d()
    g, p = case["grid"], case["phys"]
    sp = solver(p, rtol=1e-12)
    Eo, eo = case["E"].copy(), case["eps"].copy()
    E, eps, rho = dev(Eo), dev(eo), dev(case["rho"])
    for _ in range(20):
        kap = oracle.opacity(p, case["rho"], eo)
        D = oracle.coeffs(g, p, Eo, case["rho"], kap)
        Eo = oracle.diffuse(g, case["dt"], D, Eo, rtol=1e-14)
        _, D_g = fld.coeffs(ctx, g, p, E, rho, eps)
        E, info = fld.diffuse(ctx, g, sp, case["dt"], D_g, E)
        assert info["rel_residual"] <= 1e-12
    assert relerr(host(E), Eo) < TOL
    # exchange phase: T_gas = 2 T_rad
    T = inputs.rad_temperature(p, Eo)
    eo = inputs.equilibrium_eps(p, case["rho"], 2 * T)
    eps = dev(eo)
    E = dev(Eo)
    kap = np.full_like(Eo, p["kappa0"])
    for _ in range(10):
        eo, Eo, _ = oracle.exchange(p, case["dt"], case["rho"], kap, eo, Eo)
        fld.exchange(ctx, p, case["dt"], rho, eps, E, kappa=dev(kap))
    assert relerr(host(E), Eo) < TOL and relerr(host(eps), eo) < TOL


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_step_full_size_128(ctx, precision):
    """The 128^3 lognormal workload at its full size and rtol: the oracle's FP64 operator applied
    to the GPU result meets rtol, and sampled cells of the exchange match the oracle."""
    from paper_2104_03968_gb300 import fld
    case = inputs.lognormal_3d(n=128, seed=1, dt_exp=lp_dt.stored("lognormal_3d_128_seed1"))
    g, p = case["grid"], case["phys"]
    rtol = 1e-10 if precision == "fp64" else 1e-8
    kap = oracle.opacity(p, case["rho"], case["eps"])
    D = oracle.coeffs(g, p, case["E"], case["rho"], kap)
    out, info = fld.diffuse(ctx, g, solver(p, precision=precision, rtol=rtol), case["dt"], dev(D), dev(case["E"]))
    x = host(out).reshape(case["E"].shape)
    assert info["status"] == 0
    assert oracle.relres(g, case["dt"], D, case["E"], x) <= 1.01 * rtol
    # full step: coefficients on the GPU, exchange on sampled cells against the oracle
    eps, E = dev(case["eps"]), dev(case["E"])
    info = fld.step(ctx, g, solver(p, precision=precision, rtol=rtol), case["dt"], dev(case["rho"]), eps, E)
    assert info["status"] == 0
    rng = np.random.default_rng(0)
    idx = rng.choice(x.size, 4096, replace=False)
    e_s, E_s, _ = oracle.exchange(p, case["dt"], case["rho"].ravel()[idx], kap.ravel()[idx],
                                  case["eps"].ravel()[idx], x.ravel()[idx])
    # the GPU's diffusion result differs from x by at most the solve tolerance amplification
    tol = 1e-7 if precision == "fp64" else 1e-5
    assert np.abs(host(E).ravel()[idx] / E_s - 1).max() < tol
    assert np.abs(host(eps).ravel()[idx] / e_s - 1).max() < tol


# ----------------------------------------------------------------------------- explicit terms

@pytest.mark.parametrize("shape,bcname", [((24, 20, 18), "periodic"), ((70, 45), "mixed"), ((40, 24, 16), "dirichlet"),
                                          ((300,), "neumann")])
@pytest.mark.parametrize("limiter", ["lp", "minerbo"])
def test_radiation_terms_parity(ctx, shape, bcname, limiter):
    """Flux, force, work, Eddington factor and tensor, photon tiring (Sect. 2.1-2.2, 3.2)."""
    from paper_2104_03968_gb300 import fld
    case = inputs.random_small(shape, seed=80 + len(shape), bc=BCS[bcname], limiter=limiter)
    g, p = case["grid"], case["phys"]
    rng = np.random.default_rng(81)
    v = [rng.standard_normal(case["E"].shape) for _ in range(len(shape))]
    kap = oracle.opacity(p, case["rho"], case["eps"])
    ref = oracle.radiation_sources(g, p, case["E"], case["rho"], kap, v=v)
    out = fld.radiation_terms(ctx, g, p, dev(case["E"]), dev(case["rho"]), dev(case["eps"]), v=[dev(c) for c in v])
    torch.cuda.synchronize()
    for key in ("F", "fr", "P"):
        for a, (o, r) in enumerate(zip(out[key], ref[key])):
            if key == "P" and len(shape) < 3 and a in (4, 5):
                continue  # components with a z index are 0 in 2-D / 1-D on both sides
            assert relerr(host(o).reshape(r.shape), r) < 1e-12, (key, a)
    for key in ("work", "fedd", "tiring"):
        assert relerr(host(out[key]).reshape(ref[key].shape), ref[key]) < 1e-12, key
    # the explicit step E <- E - dt P : grad v
    dt = 1e-3
    E = dev(case["E"])
    fld.photon_tiring_step(ctx, g, p, dt, dev(case["rho"]), dev(case["eps"]), [dev(c) for c in v], E)
    assert relerr(host(E).reshape(case["E"].shape), case["E"] - dt * ref["tiring"]) < 1e-13


@pytest.mark.parametrize("shape,bcname", [((24, 20, 18), "periodic"), ((70, 45), "mixed"), ((300,), "neumann"),
                                          ((1000,), "dirichlet")])
@pytest.mark.parametrize("x0", [0.0, 7.5])
def test_pseudo_planar_parity(ctx, shape, bcname, x0):
    """The pseudo-planar source of E (Appendix A), with and without a velocity field, and the
    explicit step E <- E + dt S; x0 < 0 is rejected before any launch."""
    from paper_2104_03968_gb300 import fld
    case = inputs.random_small(shape, seed=90 + len(shape), bc=BCS[bcname])
    g, p = case["grid"], case["phys"]
    rng = np.random.default_rng(91)
    v = [rng.standard_normal(case["E"].shape) for _ in range(len(shape))]
    kap = oracle.opacity(p, case["rho"], case["eps"])
    args = (dev(case["E"]), dev(case["rho"]), dev(case["eps"]))
    for vel in (None, v):
        ref = oracle.pseudo_planar_source(g, p, x0, case["E"], case["rho"], kap, v=vel)
        S = fld.pseudo_planar_source(ctx, g, p, x0, *args, v=None if vel is None else [dev(c) for c in vel])
        torch.cuda.synchronize()
        assert relerr(host(S).reshape(ref.shape), ref) < 1e-12
    dt = 1e-4 * float(np.min(case["E"] / np.maximum(np.abs(ref), 1e-300)))
    E = dev(case["E"])
    fld.pseudo_planar_step(ctx, g, p, dt, x0, dev(case["rho"]), dev(case["eps"]), [dev(c) for c in v], E)
    assert relerr(host(E).reshape(case["E"].shape), case["E"] + dt * ref) < 1e-13
    with pytest.raises(fld.FldError):
        fld.pseudo_planar_source(ctx, g, p, -1.0, *args)


# ----------------------------------------------------------------------------- columns

def _column_case(ncol, ncell, seed=0):
    case = lp_dt.columns_dt(inputs.wind_columns(ncol=ncol, ncell=ncell, seed=seed))
    return case


def test_step_parity_minerbo(ctx):
    """The Minerbo limiter through a full 3-D step (both branches of the limiter are met)."""
    from paper_2104_03968_gb300 import fld
    case = lp_dt.grid_dt(inputs.lognormal_3d(n=32, seed=12))
    g, p = case["grid"], dict(case["phys"], limiter="minerbo")
    e_o, E_o, _ = oracle.step(g, p, case["dt"], case["rho"], case["eps"], case["E"], rtol=1e-14)
    eps, E = dev(case["eps"]), dev(case["E"])
    info = fld.step(ctx, g, solver(p, precision="mixed", rtol=1e-13), case["dt"], dev(case["rho"]), eps, E)
    assert info["status"] == 0
    assert relerr(host(E), E_o) < TOL
    assert relerr(host(eps), e_o) < TOL


@pytest.mark.parametrize("ncell", [64, 100, 2048])
@pytest.mark.parametrize("order", ["diffuse_then_exchange", "exchange_then_diffuse", "imex_midpoint"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_columns_step_parity(ctx, ncell, order, precision):
    """The mixed form (FP32 tridiagonal solves inside two FP64 refinement passes) is held to the
    same FP64 tolerance: the refinement reaches FP64 round-off on these columns."""
    from paper_2104_03968_gb300 import fld
    ncol = 6
    case = _column_case(ncol, ncell)
    # the Minerbo limiter rides along on one configuration
    lim = "minerbo" if (ncell, order, precision) == (100, "exchange_then_diffuse", "mixed") else "lp"
    p = solver(case["phys"], order=order, precision=precision, limiter=lim)
    col = {"r_faces": case["r_faces"], "geometry": "spherical", "bc": case["bc"]}
    eps, E = dev(case["eps"]), dev(case["E"])
    info = fld.columns_step(ctx, case["r_faces"], "spherical", tuple(case["bc"]), case["bc_lo"], case["bc_hi"], p,
                            case["dt"], dev(case["rho"]), eps, E)
    assert info["status"] == 0
    for j in range(ncol):
        e_o, E_o, _ = oracle.column_step(col, p, case["dt"][j], case["rho"][j], case["eps"][j], case["E"][j],
                                         case["bc_lo"][j], case["bc_hi"][j], order=order)
        assert relerr(host(E)[j], E_o) < TOL
        assert relerr(host(eps)[j], e_o) < TOL


@pytest.mark.parametrize("order", ["diffuse_then_exchange", "exchange_then_diffuse", "imex_midpoint"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_columns_wind_cak_and_luminosity(ctx, order, precision):
    """Sect. 5.1-5.2: CAK line opacity from the wind velocity added to the table opacity, and the
    fixed-luminosity inner boundary, through the fused column kernel."""
    from paper_2104_03968_gb300 import fld
    ncol, ncell = 4, 512
    case = _column_case(ncol, ncell, seed=2)
    cak = inputs.wind_cak(case)
    p = solver(case["phys"], order=order, precision=precision, cak=cak)
    L = np.full(ncol, case["L"])
    eps, E = dev(case["eps"]), dev(case["E"])
    info = fld.columns_step(ctx, case["r_faces"], "spherical", ("luminosity", "dirichlet"), L, case["bc_hi"], p,
                            case["dt"], dev(case["rho"]), eps, E)
    assert info["status"] == 0
    col = {"r_faces": case["r_faces"], "geometry": "spherical", "bc": ("luminosity", "dirichlet")}
    for j in range(ncol):
        cj = dict(cak, v=case["v"][j])
        e_o, E_o, _ = oracle.column_step(col, case["phys"], case["dt"][j], case["rho"][j], case["eps"][j],
                                         case["E"][j], L[j], case["bc_hi"][j], order=order, cak=cj)
        assert relerr(host(E)[j], E_o) < TOL
        assert relerr(host(eps)[j], e_o) < TOL


@pytest.mark.parametrize("geometry", ["spherical", "cartesian"])
@pytest.mark.parametrize("bc", [("dirichlet", "dirichlet"), ("neumann", "dirichlet"), ("continuous", "neumann")])
def test_columns_diffuse_parity(ctx, geometry, bc):
    from paper_2104_03968_gb300 import fld
    rng = np.random.default_rng(2)
    ncol, n = 5, 333
    rf = 1.0 * 3.0 ** (np.arange(n + 1) / n)
    D = 10 ** rng.uniform(-1, 1, (ncol, n))
    E_old = 1 + rng.random((ncol, n))
    vlo, vhi = rng.random(ncol) + 0.5, rng.random(ncol)
    dts = 10 ** rng.uniform(-3, 0, ncol)
    p = inputs.code_units()
    out = fld.columns_diffuse(ctx, rf, geometry, bc, vlo, vhi, p, dts, dev(D), dev(E_old))
    col = {"r_faces": rf, "geometry": geometry, "bc": list(bc)}
    for j in range(ncol):
        ref = oracle.column_diffuse(col, dts[j], D[j], E_old[j], vlo[j], vhi[j], method="dense")
        assert relerr(host(out)[j], ref) < 1e-12


def test_columns_thin_front(ctx):
    """The optically thin front (Sect. 4.4) on a uniform Cartesian column, GPU vs oracle."""
    from paper_2104_03968_gb300 import fld
    case = inputs.thin_front()
    p = case["phys"]
    n = case["E"].size
    rf = np.linspace(-0.5, 1.5, n + 1)
    col = {"r_faces": rf, "geometry": "cartesian", "bc": ["dirichlet", "dirichlet"]}
    vlo, vhi = case["E0"] + case["E1"], case["E0"]
    Eo, eo = case["E"].copy(), case["eps"].copy()
    E = dev(Eo[None, :])
    for _ in range(20):
        kap = oracle.opacity(p, case["rho"], eo)
        D = oracle.column_coeffs(col, p, Eo, case["rho"], kap, vlo, vhi)
        Eo = oracle.column_diffuse(col, case["dt"], D, Eo, vlo, vhi)
        E = fld.columns_diffuse(ctx, rf, "cartesian", ("dirichlet", "dirichlet"), [vlo], [vhi], p, [case["dt"]],
                                dev(D[None, :]), E)
    assert relerr(host(E)[0], Eo) < 1e-12


# ----------------------------------------------------------------------------- batched

@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_step_batched_parity(ctx, precision):
    """Five uneven grids in one graph launch (the first call also autotunes), each against the
    oracle; a second call on the same shape reuses the graph."""
    from paper_2104_03968_gb300 import fld
    cases = lp_dt.batched_dt(inputs.batched_2d(ngrids=5, nmin=32, nmax=96, seed=21))
    params = [solver(c["phys"], rtol=1e-13 if precision == "fp64" else 1e-12, precision=precision) for c in cases]
    eps = [dev(c["eps"]) for c in cases]
    E = [dev(c["E"]) for c in cases]
    infos = fld.step_batched(ctx, [c["grid"] for c in cases], params, [c["dt"] for c in cases],
                             [dev(c["rho"]) for c in cases], eps, E)
    for c, i, te, tE in zip(cases, infos, eps, E):
        assert i["status"] == 0
        e_o, E_o, _ = oracle.step(c["grid"], c["phys"], c["dt"], c["rho"], c["eps"], c["E"], rtol=1e-14)
        assert relerr(host(tE), E_o) < TOL
        assert relerr(host(te), e_o) < TOL
    # second step through the cached graph, against a second oracle step
    infos2 = fld.step_batched(ctx, [c["grid"] for c in cases], params, [c["dt"] for c in cases],
                              [dev(c["rho"]) for c in cases], eps, E)
    for c, i, te, tE in zip(cases, infos2, eps, E):
        assert i["status"] == 0
        e1, E1, _ = oracle.step(c["grid"], c["phys"], c["dt"], c["rho"], c["eps"], c["E"], rtol=1e-14)
        e2, E2, _ = oracle.step(c["grid"], c["phys"], c["dt"], c["rho"], e1, E1, rtol=1e-14)
        assert relerr(host(tE), E2) < TOL
        assert relerr(host(te), e2) < TOL


def _scaled(case, s):
    """The same problem in units where every energy density and the density are s times larger:
    rho, eps, E and a_rad times s, kappa0 over s^2.  T, kappa rho, D, the limiter's R and the
    exchange's a2 are unchanged, so the solution is s times the unscaled one."""
    c = dict(case)
    c["phys"] = dict(case["phys"], a_rad=case["phys"]["a_rad"] * s, kappa0=case["phys"]["kappa0"] / (s * s))
    for k in ("rho", "eps", "E"):
        c[k] = case[k] * s
    return c


@pytest.mark.parametrize("scale", [1.0, 1e-20])
def test_step_batched_mixed_certified_residual(ctx, scale):
    """Mixed batched residuals are double-float, with a bound on their error: a grid stops when the
    residual plus the bound meets rtol, so the true relative residual of its diffusion solve is
    below rtol.  With the exchange first the final E is the solve's result, and the oracle gives
    the true residual from the exchanged state.  At scale 1e-20 the squares of the residuals and
    of their bounds are far below the FP32 range unless the solver scales them."""
    from paper_2104_03968_gb300 import fld
    rtol = 1e-9
    cases = lp_dt.batched_dt(inputs.batched_2d(ngrids=6, nmin=64, nmax=160, seed=23))
    cases = [_scaled(c, scale) for c in cases]
    params = [solver(c["phys"], rtol=rtol, precision="mixed", order="exchange_then_diffuse") for c in cases]
    E = [dev(c["E"]) for c in cases]
    infos = fld.step_batched(ctx, [c["grid"] for c in cases], params, [c["dt"] for c in cases],
                             [dev(c["rho"]) for c in cases], [dev(c["eps"]) for c in cases], E)
    for c, i, tE in zip(cases, infos, E):
        assert i["status"] == 0 and i["cycles"] >= 1
        p = c["phys"]
        e1, E1, _ = oracle.exchange(p, c["dt"], c["rho"], oracle.opacity(p, c["rho"], c["eps"]), c["eps"], c["E"])
        D = oracle.coeffs(c["grid"], p, E1, c["rho"], oracle.opacity(p, c["rho"], e1))
        true = oracle.relres(c["grid"], c["dt"], D, E1, host(tE).reshape(E1.shape))
        # the oracle's exchanged state differs from the GPU's at the 1e-12 level, which moves the
        # residual by as much
        assert true <= rtol * 1.01, (true, i)
        # the reported residual is the double-float estimate of the true one
        assert abs(i["rel_residual"] - true) <= 1e-3 * true + 1e-11, (true, i)


def test_step_batched_mixed_dims_and_boundaries(ctx):
    """A batch mixing 2-D and 3-D grids, different boundary conditions and both step orders."""
    from paper_2104_03968_gb300 import fld
    shapes = [((48, 32), "periodic", "diffuse_then_exchange"), ((16, 16, 8), "dirichlet", "exchange_then_diffuse"),
              ((40, 24), "mixed", "diffuse_then_exchange"), ((24, 16, 16), "neumann", "diffuse_then_exchange")]
    cases, params = [], []
    for k, (shape, bcname, order) in enumerate(shapes):
        c = inputs.random_small(shape, seed=40 + k, bc=BCS[bcname], dt_factor=50.0)
        cases.append(c)
        params.append(solver(c["phys"], rtol=1e-13, order=order))
    eps = [dev(c["eps"]) for c in cases]
    E = [dev(c["E"]) for c in cases]
    infos = fld.step_batched(ctx, [c["grid"] for c in cases], params, [c["dt"] for c in cases],
                             [dev(c["rho"]) for c in cases], eps, E)
    for c, p, i, te, tE in zip(cases, params, infos, eps, E):
        assert i["status"] == 0, i
        e_o, E_o, _ = oracle.step(c["grid"], c["phys"], c["dt"], c["rho"], c["eps"], c["E"], order=p["order"],
                                  rtol=1e-14)
        assert relerr(host(tE).reshape(E_o.shape), E_o) < TOL
        assert relerr(host(te).reshape(e_o.shape), e_o) < TOL


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_step_batched_conjugate_gradient_and_plain_grids(ctx, precision):
    """Grids with symmetric operators (periodic, Dirichlet, Neumann faces) run the conjugate-
    gradient outer loop, grids with a linear-extrapolation face the plain one, in the same batch:
    both meet the oracle, on stiff time steps."""
    from paper_2104_03968_gb300 import fld
    shapes = [((64, 48), "periodic"), ((40, 24), "continuous"), ((16, 16, 8), "neumann"), ((32, 32), "dirichlet"),
              ((12, 8, 8), "continuous")]
    cases, params = [], []
    for k, (shape, bcname) in enumerate(shapes):
        c = inputs.random_small(shape, seed=70 + k, bc=BCS[bcname], dt_factor=300.0)
        cases.append(c)
        params.append(solver(c["phys"], precision=precision, rtol=1e-13))
    eps = [dev(c["eps"]) for c in cases]
    E = [dev(c["E"]) for c in cases]
    infos = fld.step_batched(ctx, [c["grid"] for c in cases], params, [c["dt"] for c in cases],
                             [dev(c["rho"]) for c in cases], eps, E)
    for (shape, bcname), c, i, te, tE in zip(shapes, cases, infos, eps, E):
        assert i["status"] == 0, i
        # the oracle's CG needs a symmetric operator: the extrapolated grids take its dense solve
        e_o, E_o, _ = oracle.step(c["grid"], c["phys"], c["dt"], c["rho"], c["eps"], c["E"], rtol=1e-14,
                                  method="dense" if bcname == "continuous" else "cg")
        assert relerr(host(tE).reshape(E_o.shape), E_o) < TOL
        assert relerr(host(te).reshape(e_o.shape), e_o) < TOL


# ----------------------------------------------------------------------------- errors

def test_invalid_arguments_are_rejected(ctx):
    from paper_2104_03968_gb300 import fld
    g = inputs.periodic_grid((16, 16))
    p = solver(inputs.code_units(), rtol=1e-10)
    t = dev(np.ones((16, 16)))
    with pytest.raises(fld.FldError) as e:
        fld.step(ctx, dict(g, ndim=4), p, 1.0, t, t.clone(), t.clone())
    assert e.value.status == 1
    with pytest.raises(fld.FldError):
        fld.step(ctx, g, dict(p, rtol=0.0), 1.0, t, t.clone(), t.clone())
    with pytest.raises(fld.FldError):
        fld.step(ctx, g, p, -1.0, t, t.clone(), t.clone())
    # a state with E <= 0 is reported, not solved
    bad = dev(np.full((16, 16), -1.0))
    with pytest.raises(fld.FldError) as e:
        fld.step(ctx, g, p, 1.0, t, t.clone(), bad)
    assert e.value.status == 2


def test_empty_batches_launch_nothing(ctx):
    """Zero cells, zero columns and zero grids are valid calls: FLD_OK, no kernel launched, the
    data arrays may be NULL (an empty tensor's data pointer), the info zeroed."""
    from paper_2104_03968_gb300 import fld
    case = _column_case(2, 64)
    p = solver(case["phys"])
    empty = torch.empty(0, dtype=torch.float64, device="cuda")
    n0 = fld.launch_count()
    info = fld.exchange(ctx, p, 1.0, empty, empty.clone(), empty.clone())
    assert info["status"] == 0 and info["exch_max_iters"] == 0
    assert fld.opacity(ctx, dict(p, precision="mixed"), empty, empty.clone()).numel() == 0
    assert fld.step_batched(ctx, [], [], [], [], [], []) == []
    no_col = torch.empty((0, 64), dtype=torch.float64, device="cuda")
    for precision in ("fp64", "mixed"):
        info = fld.columns_step(ctx, case["r_faces"], "spherical", tuple(case["bc"]), case["bc_lo"][:0],
                                case["bc_hi"][:0], dict(p, precision=precision), case["dt"][:0], no_col,
                                no_col.clone(), no_col.clone())
        assert info["status"] == 0
    out = fld.columns_diffuse(ctx, case["r_faces"], "spherical", tuple(case["bc"]), case["bc_lo"][:0],
                              case["bc_hi"][:0], p, case["dt"][:0], no_col, no_col.clone())
    assert out.shape == (0, 64)
    info = fld.columns_step_static(dev(case["r_faces"]), "spherical", tuple(case["bc"]), empty, empty.clone(), p,
                                   empty.clone(), no_col, no_col.clone(), no_col.clone())
    assert info["status"] == 0
    assert fld.launch_count() == n0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_steps_enqueued_back_to_back(ctx, precision):
    """fld_step is asynchronous: two steps enqueued one after the other with no host wait between
    them (the outcome of each arrives in its fld_info in stream order) give the oracle's two steps."""
    from paper_2104_03968_gb300 import fld
    case = lp_dt.grid_dt(inputs.lognormal_3d(n=32, seed=13))
    g, p = case["grid"], solver(case["phys"], precision=precision, rtol=1e-13 if precision == "fp64" else 1e-12)
    rho = dev(case["rho"])
    # the first call of a configuration autotunes its sweep counts (that part synchronises)
    fld.step(ctx, g, p, case["dt"], rho, dev(case["eps"]), dev(case["E"]))
    eps, E = dev(case["eps"]), dev(case["E"])
    infos = [fld.step(ctx, g, p, case["dt"], rho, eps, E, sync=False) for _ in range(2)]
    torch.cuda.synchronize()
    outs = [fld.outcome(ctx, i, allow_unconverged=False) for i in infos]
    assert all(o["cycles"] >= 1 for o in outs), outs
    e_o, E_o = case["eps"], case["E"]
    for _ in range(2):
        e_o, E_o, _ = oracle.step(g, case["phys"], case["dt"], case["rho"], e_o, E_o, rtol=1e-14)
    assert relerr(host(E), E_o) < TOL and relerr(host(eps), e_o) < TOL


def test_diffuse_same_arrays_new_contents(ctx):
    """Solves that reuse one set of device arrays with new contents each time (the solver keeps its
    CUDA graph while the arrays and parameters stay the same), crossing the double-float window
    both ways: every result must meet rtol under the oracle's operator for its own inputs."""
    from paper_2104_03968_gb300 import fld
    case = inputs.random_small((48, 40, 32), seed=11, bc=BCS["periodic"], dt_factor=100.0)
    g, p = case["grid"], case["phys"]
    other = inputs.random_small((48, 40, 32), seed=12, bc=BCS["periodic"], dt_factor=100.0)
    Ds = [oracle.coeffs(g, p, c["E"], c["rho"], oracle.opacity(p, c["rho"], c["eps"])) for c in (case, other)]
    D_t, E_t = dev(Ds[0]), dev(case["E"])
    out = torch.empty_like(E_t)
    seq = [(0, case["E"]), (0, case["E"] * 1e30), (0, case["E"] * 2.0), (1, other["E"]), (0, case["E"] * 1e-25),
           (1, other["E"] * 3.0)]
    for which, E in seq:
        D_t.copy_(torch.as_tensor(Ds[which]))
        E_t.copy_(torch.as_tensor(E))
        out.fill_(0.0)
        _, info = fld.diffuse(ctx, g, solver(p, precision="mixed", rtol=1e-8), case["dt"], D_t, E_t, out=out)
        assert info["status"] == 0, info
        true = oracle.relres(g, case["dt"], Ds[which], E, host(out).reshape(E.shape))
        assert true <= 1.01e-8, (which, float(np.abs(E).max()), true, info)


def test_not_converged_is_reported(ctx):
    from paper_2104_03968_gb300 import fld
    case = inputs.random_small((64, 64), seed=2, dt_factor=300.0)
    g, p = case["grid"], case["phys"]
    kap = oracle.opacity(p, case["rho"], case["eps"])
    D = oracle.coeffs(g, p, case["E"], case["rho"], kap)
    out, info = fld.diffuse(ctx, g, solver(p, rtol=1e-14, max_cycles=1), case["dt"], dev(D), dev(case["E"]))
    assert info["status"] == 4 and info["cycles"] == 1

# ----------------------------------------------------------------------------- tiled 3-D smoother

def _gs_sweep(D, r, x, dt, dx, bc, first):
    """One red-black Gauss-Seidel sweep of x + dt (-div D grad x) = r written from Sect. 3.4's
    operator (harmonic-mean faces, homogeneous boundary faces), vectorised in FP64: each colour is
    updated from the current values of the other.  Also returns, per cell, the magnitude M that
    bounds an FP32 evaluation's error as a multiple of its unit roundoff: (|r| + sum |w x_nb| +
    |x| (1 + sum |w|)) / |diag|, plus sum |w| M_nb / |diag| for the second colour, whose neighbours
    carry the first colour's errors."""
    codes = {"periodic": 0, "neumann": 1, "dirichlet": 2, "continuous": 3}
    nz, ny, nx = D.shape
    x = x.astype(np.float64).copy()
    D = D.astype(np.float64)
    M = np.zeros_like(x)
    par = (np.arange(nx)[None, None, :] + np.arange(ny)[None, :, None] + np.arange(nz)[:, None, None]) & 1
    for col in (first, 1 - first):
        a = r.astype(np.float64).copy()
        d = np.ones_like(a)
        ma = np.abs(a)
        wsum = np.ones_like(a)
        mprop = np.zeros_like(a)
        for ax_phys in range(3):
            arr_ax = 2 - ax_phys
            s = dt / dx[ax_phys] ** 2
            n = D.shape[arr_ax]
            idx = np.arange(n).reshape([-1 if q == arr_ax else 1 for q in range(3)])
            for side in (0, 1):
                shift = 1 if side == 0 else -1  # roll by +1 brings x[i-1] to position i
                nb, Dn, mir = np.roll(x, shift, arr_ax), np.roll(D, shift, arr_ax), np.roll(x, -shift, arr_ax)
                Mn, Mm = np.roll(M, shift, arr_ax), np.roll(M, -shift, arr_ax)
                at_bnd = np.broadcast_to(idx == (0 if side == 0 else n - 1), D.shape)
                kind = codes[bc[2 * ax_phys + side]]
                w = s * 2 * D * Dn / (D + Dn)
                pair = ~at_bnd if kind != 0 else np.ones_like(at_bnd)
                a += np.where(pair, w * nb, 0.0)
                d += np.where(pair, w, 0.0)
                ma += np.where(pair, np.abs(w * nb), 0.0)
                wsum += np.where(pair, w, 0.0)
                mprop += np.where(pair, w * Mn, 0.0)
                if kind == 2:
                    d += np.where(at_bnd, s * D, 0.0)
                    wsum += np.where(at_bnd, s * D, 0.0)
                elif kind == 3:
                    a -= np.where(at_bnd, s * D * mir, 0.0)
                    d -= np.where(at_bnd, s * D, 0.0)
                    ma += np.where(at_bnd, np.abs(s * D * mir), 0.0)
                    wsum += np.where(at_bnd, s * D, 0.0)
                    mprop += np.where(at_bnd, s * D * Mm, 0.0)
        xn = a / d
        Mc = (ma + np.abs(xn) * wsum + mprop) / np.abs(d)
        x = np.where(par == col, xn, x)
        M = np.where(par == col, Mc, M)
    return x, M


# (192, 48, 8) periodic has a tile whose halo does not wrap (staged by TMA boxes); the others wrap
# or cross non-periodic faces
TILED_CASES = [((64, 16, 6), "periodic"), ((192, 48, 8), "periodic"), ((128, 32, 8), "mixed"),
               ((64, 48, 4), "dirichlet"),
               ((192, 16, 10), "continuous"), ((64, 32, 8), "neumann")]


@pytest.mark.parametrize("shape,bcname", TILED_CASES)
@pytest.mark.parametrize("zero", [False, True])
def test_tiled_sweep_matches_gauss_seidel(ctx, shape, bcname, zero):
    """The finest-level smoother of the mixed solver on 3-D grids (one launch per sweep, tiles
    staged in shared memory, face means formed on chip) is one red-black Gauss-Seidel sweep, for
    both colour orders, with and without a starting iterate, on every boundary type."""
    from paper_2104_03968_gb300 import fld
    rng = np.random.default_rng(7 + len(bcname) + shape[2])
    nx, ny, nz = shape
    grid = {"ndim": 3, "n": list(shape), "dx": [1.0, 0.8, 1.3], "bc": BCS[bcname][0], "bc_val": [0.0] * 6}
    D = 10 ** rng.uniform(-1, 1, (nz, ny, nx))
    r = rng.standard_normal((nz, ny, nx)).astype(np.float32)
    x0 = rng.standard_normal((nz, ny, nx)).astype(np.float32)
    dt = 0.7
    for first in (0, 1):
        out = torch.empty((nz, ny, nx), dtype=torch.float32, device="cuda")
        fld.smooth_sweep(ctx, grid, dt, dev(D), torch.as_tensor(r, device="cuda"),
                         None if zero else torch.as_tensor(x0, device="cuda"), out, first)
        ref, M = _gs_sweep(D, r, np.zeros_like(x0) if zero else x0, dt, grid["dx"], grid["bc"], first)
        got = out.cpu().numpy().astype(np.float64)
        # FP32 inputs rounded once (dc), ~a dozen roundings per cell: 64 unit roundoffs of M
        excess = np.abs(got - ref) / (64 * 2.0 ** -24 * M)
        assert excess.max() <= 1.0, (first, excess.max(), relerr(got, ref))


def test_tiled_sweep_rejects_unsupported_shapes(ctx):
    from paper_2104_03968_gb300 import fld
    grid = {"ndim": 3, "n": [48, 16, 8], "dx": [1.0] * 3, "bc": ["periodic"] * 6, "bc_val": [0.0] * 6}
    z = torch.zeros((8, 16, 48), dtype=torch.float32, device="cuda")
    with pytest.raises(fld.FldError) as e:
        fld.smooth_sweep(ctx, grid, 1.0, torch.ones((8, 16, 48), dtype=torch.float64, device="cuda"), z, None,
                         torch.empty_like(z))
    assert e.value.status == 7


@pytest.mark.parametrize("shape,bcname", TILED_CASES)
def test_tiled_solve_parity(monkeypatch, shape, bcname):
    """Diffusion solves whose finest level uses the tiled sweep (forced onto these small grids)
    meet the oracle's operator: its relative residual of the GPU result is at the solver's
    tolerance, and where the operator is symmetric (no extrapolated boundary) the result equals
    the oracle's CG solution."""
    from paper_2104_03968_gb300 import fld
    monkeypatch.setenv("FLD_SWEEP3D_MIN_CELLS", "0")
    c = fld.Context(0)
    try:
        case = inputs.random_small(shape, seed=200 + shape[2], bc=BCS[bcname], dt_factor=100.0)
        g, p = case["grid"], case["phys"]
        kap = oracle.opacity(p, case["rho"], case["eps"])
        D = oracle.coeffs(g, p, case["E"], case["rho"], kap)
        out, info = fld.diffuse(c, g, solver(p, precision="mixed", rtol=1e-13), case["dt"], dev(D), dev(case["E"]))
        assert info["status"] == 0
        x = host(out).reshape(case["E"].shape)
        assert oracle.relres(g, case["dt"], D, case["E"], x) < 2e-13
        if bcname != "continuous":
            ref = oracle.diffuse(g, case["dt"], D, case["E"], rtol=1e-14)
            assert relerr(x, ref) < TOL
    finally:
        c.close()
