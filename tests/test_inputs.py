"""The seeded input recipes hold the statistics and structure they are documented to have (no GPU):
the lognormal density's exact log-moments, the k^-4 band-limited Gaussian field, the batched
grids' size, opacity and time-step ranges, the wind columns' geometric grid, mass flux and
velocity law, and the torch path of the large grids against the numpy path."""
import math

import numpy as np
import pytest
import torch

from paper_2104_03968_gb300 import inputs


def _shell_power(f):
    """Mean |F(k)|^2 over the shells |k| in [m, m + 1) of a periodic field."""
    F = np.fft.fftn(f)
    k = np.sqrt(sum(q * q for q in np.meshgrid(*[np.fft.fftfreq(s) * s for s in f.shape], indexing="ij")))
    m = np.floor(k).astype(int)
    p = np.bincount(m.ravel(), weights=(np.abs(F) ** 2).ravel())
    c = np.bincount(m.ravel())
    return k, np.abs(F) ** 2, p / np.maximum(c, 1)


def test_gaussian_field_is_unit_variance_and_band_limited_k4():
    n = 48
    rng = np.random.default_rng(7)
    G = inputs.gaussian_random_field(rng, (n, n, n))
    assert abs(G.mean()) < 1e-14 and G.std() == pytest.approx(1.0, abs=1e-13)
    k, P, shells = _shell_power(G)
    assert P[(k > n / 4) | (k < 1)].max() < 1e-20 * P.max()  # outside 1 <= |k| <= N/4: nothing
    # shell power of white noise filtered by k^-2 in amplitude: a slope of -4 in log-log
    m = np.arange(2, n // 4)
    slope = np.polyfit(np.log(m + 0.5), np.log(shells[m]), 1)[0]
    assert slope == pytest.approx(-4.0, abs=0.3)


def test_torch_path_of_the_fields_equals_the_numpy_path():
    """The large grids filter the same numpy noise with torch FFTs; on the CPU device both paths
    give the same fields."""
    a = inputs.lognormal_3d(n=24, seed=5)
    b = inputs.lognormal_3d(n=24, seed=5, device="cpu")
    for key in ("rho", "eps", "E"):
        t = b[key].numpy()
        assert np.abs(t - a[key]).max() <= 1e-13 * np.abs(a[key]).max()
    assert b["dt_exp_thick"] == pytest.approx(a["dt_exp_thick"], rel=1e-12)


def test_lognormal_density_log_moments_and_temperatures():
    case = inputs.lognormal_3d(n=32, seed=2)
    rho, eps, E, phys = case["rho"], case["eps"], case["E"], case["phys"]
    assert rho.shape == (32, 32, 32) and rho.flags.c_contiguous and rho.dtype == np.float64
    # rho = exp(G - 1/2) with G of mean 0 and variance 1 exactly (normalised on the grid)
    assert np.log(rho).mean() == pytest.approx(-0.5, abs=1e-13)
    assert np.log(rho).std() == pytest.approx(1.0, abs=1e-13)
    Tg = eps * (phys["gamma"] - 1.0) / (rho * phys["gas_R"])
    Tr = (E / phys["a_rad"]) ** 0.25
    for T in (Tg, Tr):  # 1 + 0.3 S with max |S| = 1: one extreme is reached
        assert T.min() >= 0.7 - 1e-12 and T.max() <= 1.3 + 1e-12
        assert min(abs(T.min() - 0.7), abs(T.max() - 1.3)) < 1e-12
    kr_min = (phys["kappa0"] * rho * Tg ** -3.5 * rho).min()
    assert case["dt_exp_thick"] == pytest.approx(1.0 / (2 * 3 * phys["c"] / (3 * kr_min)), rel=1e-12)
    assert case["dt"] is None and case["dt_factor"] == 100.0
    inputs.with_explicit_dt(case, 0.25)
    assert case["dt"] == 25.0 and case["dt_exp"] == 0.25


def test_recipes_are_seeded():
    a, b, c = (inputs.lognormal_3d(n=16, seed=s) for s in (1, 1, 2))
    assert np.array_equal(a["rho"], b["rho"]) and np.array_equal(a["E"], b["E"])
    assert not np.array_equal(a["rho"], c["rho"])
    w1, w2 = inputs.wind_columns(ncol=3, ncell=64), inputs.wind_columns(ncol=3, ncell=64)
    assert np.array_equal(w1["rho"], w2["rho"]) and np.array_equal(w1["eps"], w2["eps"])


def test_batched_grid_sizes_opacities_and_time_steps():
    grids = inputs.batched_2d(ngrids=48, seed=3, nmin=64, nmax=512)
    ns = [g["grid"]["n"][0] for g in grids]
    for g, n in zip(grids, ns):
        assert g["grid"]["ndim"] == 2 and g["grid"]["n"] == [n, n, 1] and g["grid"]["bc"] == ["periodic"] * 6
        assert n % 16 == 0 and 64 <= n <= 512
        assert g["rho"].shape == (n, n)
        assert 1e-2 <= g["phys"]["kappa0"] <= 1e4 and g["phys"]["opacity"] == "kramers"
        assert 10.0 <= g["dt_factor"] <= 1000.0 and g["dt"] is None
    assert len(set(ns)) >= 8  # uneven sizes
    # log-uniform: as many grids below the geometric midpoint sqrt(64 * 512) as above, roughly
    below = sum(n < math.sqrt(64 * 512) for n in ns)
    assert 12 <= below <= 36
    dts = np.linspace(1.0, 2.0, 4)
    with_dt = inputs.batched_2d(ngrids=4, seed=3, dt_exp=dts)
    for g, d, h in zip(with_dt, dts, grids):
        assert g["dt"] == pytest.approx(h["dt_factor"] * d)


def test_wind_columns_grid_mass_flux_and_velocity_law():
    ncol, ncell = 6, 256
    w = inputs.wind_columns(ncol=ncol, ncell=ncell, seed=4)
    rf, Rs = w["r_faces"], w["r_star"]
    assert rf.shape == (ncell + 1,) and rf[0] == Rs and rf[-1] == pytest.approx(100 * Rs, rel=1e-14)
    ratio = rf[1:] / rf[:-1]
    assert np.allclose(ratio, 100.0 ** (1.0 / ncell), rtol=1e-13, atol=0)  # geometric faces
    rc = 0.5 * (rf[1:] + rf[:-1])
    v, rho, E = w["v"], w["rho"], w["E"]
    wind = rc > 1.3 * Rs  # beyond every column's sonic radius (at most 1.3 R*)
    yr_msun = inputs.M_SUN / inputs.YEAR
    for j in range(ncol):
        mdot = 4 * np.pi * rc[wind] ** 2 * rho[j, wind] * v[j, wind]
        assert np.ptp(mdot) <= 1e-12 * mdot.max()  # rho = Mdot / (4 pi r^2 v)
        assert 0.8 * 1.87e-5 <= mdot[0] / yr_msun <= 1.2 * 1.87e-5
        # beta = 1/2 velocity law v = v_inf sqrt(1 - R*/r), floored at 1e-3 v_inf
        vinf2 = v[j, wind] ** 2 / (1 - Rs / rc[wind])
        assert np.ptp(vinf2) <= 1e-12 * vinf2.max()
        vinf = math.sqrt(vinf2[0])
        assert 0.8e8 <= vinf <= 1.2e8 and v[j].min() >= 1e-3 * vinf * (1 - 1e-15)
        assert np.all(np.diff(E[j]) < 0)  # the inward diffusion integral: E falls outward
    assert np.all(E[:, -1] > inputs.A_RAD * 5.0e4 ** 4)
    Tr = (E / inputs.A_RAD) ** 0.25
    Tg = w["eps"] * (w["phys"]["gamma"] - 1.0) / (rho * w["phys"]["gas_R"])
    assert np.abs(Tg / Tr - 1).max() <= 0.05 + 1e-12
    assert np.array_equal(w["bc_lo"], E[:, 0]) and np.array_equal(w["bc_hi"], E[:, -1])
    tab, tlo, thi = w["phys"]["table"], w["phys"]["tlo"], w["phys"]["thi"]
    assert tab.shape == (128, 128) and tlo == [-16.0, 3.7] and thi == [-6.0, 6.5]
    assert tab.min() >= math.log10(0.2) - 1e-12  # electron scattering is the floor of the table


def test_heating_cooling_and_thin_front_setups():
    hc = inputs.heating_cooling(2.0, dt=1e-12)
    T_r = (1e12 / hc["phys"]["a_rad"]) ** 0.25
    assert hc["e_equil"] == pytest.approx(1e-7 * hc["phys"]["gas_R"] * T_r / (2.0 / 3.0), rel=1e-14)
    assert np.allclose(hc["eps"], 2.0 * hc["e_equil"], rtol=1e-15)
    tf = inputs.thin_front()
    assert tf["grid"]["n"][0] == 256 and tf["grid"]["dx"][0] == pytest.approx(2.0 / 256)
    assert tf["x"][0] == pytest.approx(-0.5 + 1.0 / 256) and tf["x"][-1] == pytest.approx(1.5 - 1.0 / 256)
    assert tf["E"][0] == pytest.approx(tf["E0"] + tf["E1"], rel=1e-12)
    assert tf["E"][-1] == pytest.approx(tf["E0"], rel=1e-12)
    assert np.all(np.diff(tf["E"]) <= 0)


def test_gaussian_pulse_setup():
    c = inputs.gaussian_pulse_2d()
    assert c["E"].shape == (64, 64)
    i = np.unravel_index(np.argmax(c["E"]), c["E"].shape)
    assert c["E"].max() == pytest.approx(1e-6 + math.exp(-0.5 / 32), rel=1e-14)  # centre at (32, 32), 2 sigma^2 = 32
    assert i in {(31, 31), (31, 32), (32, 31), (32, 32)}
    assert c["dt_exp"] == pytest.approx(750.0) and c["dt"] == pytest.approx(7500.0)


def test_wind_table_reproduces_its_opacity_law_at_the_nodes():
    """The wind recipe's table, read through the oracle's lookup with the recipe's parameters,
    gives back electron scattering + Kramers + the bump at log T = 5.3 at every node: the ranges
    reach the lookup in the parameters' order (rows log10 rho over [-16, -6], columns log10 T over
    [3.7, 6.5])."""
    import oracle
    phys = inputs.wind_columns(ncol=1, ncell=16)["phys"]
    lr, lt = np.linspace(-16.0, -6.0, 128), np.linspace(3.7, 6.5, 128)
    rng = np.random.default_rng(3)
    i, j = rng.integers(0, 128, 64), rng.integers(0, 128, 64)
    rho, T = 10.0 ** lr[i], 10.0 ** lt[j]
    kap = oracle.opacity(phys, rho, inputs.equilibrium_eps(phys, rho, T))
    kK = 0.2 / (1e-10 * 1e5 ** -3.5)  # the Kramers term is 0.2 at rho = 1e-10, T = 1e5
    law = 0.2 + kK * rho * T ** -3.5 + np.exp(-(np.log10(T) - 5.3) ** 2 / (2 * 0.15 ** 2)) * (rho / 1e-10) ** 0.25
    assert np.abs(kap / law - 1).max() < 1e-9
