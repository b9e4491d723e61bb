"""Seeded synthetic inputs for the FLD radiation-energy update.

This module is the only code shared by the CUDA path's tests/benchmark and the
CPU oracle's tests.  It holds workload recipes (fields, grids, units, time steps)
and none of the method's arithmetic: no limiter, no diffusion coefficient, no
operator, no exchange.  Every array is float64 and C-contiguous, x fastest.

Recipes (numpy ``default_rng``; the seeds are the workloads' names):

* ``gaussian_pulse_2d``  64x64 periodic, rho=1, kappa=1e3, c=1: a Gaussian E pulse
  (sigma=4 cells, amplitude 1 on a 1e-6 floor), dt = 10x the explicit limit.
* ``lognormal_3d``       n^3 periodic, lognormal density (sigma_ln=1, P(k) ~ k^-4
  Gaussian field), smooth T_gas and T_rad fields, Kramers opacity
  kappa = kappa0 rho T^-3.5, dt = 100x the explicit limit.
* ``batched_2d``         many square periodic grids, n log-uniform in [64, 512]
  (multiples of 16), kappa0 = 10^U(-2,4), dt = 10^U(1,3) x the explicit limit.
* ``wind_columns``       spherically symmetric wind-like columns on a geometric
  radial grid r = R*..100 R*, rho ~ r^-2 beyond a seeded sonic point, E from the
  inward diffusion integral, a synthetic 128x128 (log rho, log T) opacity table.
* ``heating_cooling``    uniform static gas out of radiative equilibrium.
* ``thin_front``         1-D optically thin slab lit by an erf profile.

The "explicit limit" of the 3-D, batched 2-D and column workloads is the smallest explicit
diffusion step of the initial state, dt_exp = min over cells of dx^2 / (2 d D_cell), with
D_cell the flux-limited (Levermore-Pomraning) coefficient of that state.  This module holds no
limiter, so the recipes take dt_exp (or D_cell) from the caller: the tests compute D_cell with
the oracle, and the full-size workloads read dt_exp from a table written by a script that runs
the oracle on these same recipes.  A recipe called without dt_exp returns dt = None.  The
optically thick bound dx^2 / (2 d D_thick), D_thick = c / (3 min kappa rho), is kept as a
secondary time scale (``dt_exp_thick``); the Gaussian pulse (R ~ 0, so the two agree) and the
small brute-force grids of ``random_small`` use it.
"""
from __future__ import annotations

import math

import numpy as np

# CODATA-style cgs constants
C_LIGHT = 2.99792458e10       # cm/s
K_B = 1.380649e-16            # erg/K
M_P = 1.67262192e-24          # g
SIGMA_SB = 5.670374419e-5     # erg/cm^2/s/K^4
A_RAD = 4.0 * SIGMA_SB / C_LIGHT
R_SUN = 6.957e10              # cm
L_SUN = 3.828e33              # erg/s
M_SUN = 1.98847e33            # g
YEAR = 3.15576e7              # s

SEED_BASE = 2104039680


def code_units(limiter: str = "lp") -> dict:
    """Dimensionless units: c = 1, a_r = 1, k_b/(mu m_p) = 1, gamma = 5/3."""
    return {"c": 1.0, "a_rad": 1.0, "gamma": 5.0 / 3.0, "gas_R": 1.0, "limiter": limiter,
            "opacity": "const", "kappa0": 1.0, "kr_a": 1.0, "kr_b": -3.5}


def cgs_units(mu: float, gamma: float = 5.0 / 3.0, limiter: str = "lp") -> dict:
    return {"c": C_LIGHT, "a_rad": A_RAD, "gamma": gamma, "gas_R": K_B / (mu * M_P),
            "limiter": limiter, "opacity": "const", "kappa0": 1.0, "kr_a": 1.0, "kr_b": -3.5}


def periodic_grid(shape, dx: float = 1.0) -> dict:
    """shape is (nx,), (nx, ny) or (nx, ny, nz); arrays are stored x fastest."""
    nd = len(shape)
    n = list(shape) + [1] * (3 - nd)
    return {"ndim": nd, "n": n, "dx": [dx] * 3, "bc": ["periodic"] * 6, "bc_val": [0.0] * 6}


def _array_shape(grid: dict):
    nx, ny, nz = grid["n"]
    return {1: (nx,), 2: (ny, nx), 3: (nz, ny, nx)}[grid["ndim"]]


def equilibrium_eps(phys: dict, rho, T):
    """Gas internal energy density at temperature T (ideal gas)."""
    return rho * phys["gas_R"] * T / (phys["gamma"] - 1.0)


def rad_energy(phys: dict, T):
    return phys["a_rad"] * T ** 4


def rad_temperature(phys: dict, E):
    return (E / phys["a_rad"]) ** 0.25


def thick_explicit_dt(dx2_min, ndim: int, c: float, kr_min: float) -> float:
    """dx^2 / (2 d D_thick) with the largest optically thick D = c / (3 min(kappa rho))."""
    return float(dx2_min / (2.0 * ndim * c / (3.0 * kr_min)))


def explicit_dt(D_cell, dx2, ndim: int) -> float:
    """The explicit diffusion limit of a grid, min over cells of dx^2 / (2 d D_cell), from the
    caller's cell-centred D (uniform spacing, dx2 = dx^2)."""
    return float(dx2 / (2.0 * ndim * float(np.max(D_cell))))


def column_explicit_dt(D_cell, r_faces) -> np.ndarray:
    """Per column (rows of D_cell), min over cells of dr_i^2 / (2 D_i), dr_i the cell width."""
    dr = np.diff(np.asarray(r_faces, dtype=np.float64))
    return (dr[None, :] ** 2 / (2.0 * np.asarray(D_cell))).min(axis=1)


def with_explicit_dt(case: dict, dt_exp) -> dict:
    """Set a recipe's time step to its dt_factor times the given explicit limit(s)."""
    case["dt_exp"] = dt_exp
    case["dt"] = case["dt_factor"] * dt_exp
    return case


# ----------------------------------------------------------------------------- fields

def _kgrid(shape, device=None):
    if device is None:
        ks = np.meshgrid(*[np.fft.fftfreq(s) * s for s in shape], indexing="ij")
        return np.sqrt(sum(k * k for k in ks))
    import torch
    ks = torch.meshgrid(*[torch.fft.fftfreq(s, device=device, dtype=torch.float64) * s for s in shape],
                        indexing="ij")
    return torch.sqrt(sum(k * k for k in ks))


def gaussian_random_field(rng, shape, kmax_frac: float = 0.25, device=None):
    """Unit-variance Gaussian field: white noise filtered to P(k) ~ k^-4, 1 <= |k| <= N/4.
    With a torch ``device`` the same numpy noise is filtered there (large grids)."""
    k = _kgrid(shape, device)
    kmax = kmax_frac * min(shape)
    noise = rng.standard_normal(shape)
    if device is None:
        amp = np.zeros_like(k)
        sel = (k >= 1.0) & (k <= kmax)
        amp[sel] = k[sel] ** -2.0
        f = np.real(np.fft.ifftn(np.fft.fftn(noise) * amp))
    else:
        import torch
        sel = (k >= 1.0) & (k <= kmax)
        amp = torch.where(sel, k.clamp(min=1.0) ** -2.0, torch.zeros_like(k))
        del k, sel
        f = torch.fft.fftn(torch.from_numpy(noise).to(device))
        del noise
        f *= amp
        del amp
        f = torch.fft.ifftn(f).real.contiguous()
        f = f - f.mean()
        return f / f.std(correction=0)
    f = f - f.mean()
    return f / f.std()


def smooth_field(rng, shape, kmax: float = 4.0, device=None) -> np.ndarray:
    """Sum of the Fourier modes with |k| <= kmax, random phases, scaled to max |S| = 1."""
    k = _kgrid(shape)  # host: the selection is tiny
    sel = (k > 0) & (k <= kmax)
    ph = rng.uniform(0, 2 * np.pi, size=int(sel.sum()))
    if device is None:
        coef = np.zeros(shape, dtype=np.complex128)
        coef[sel] = np.exp(1j * ph)
        f = np.real(np.fft.ifftn(coef))
        return f / np.abs(f).max()
    import torch
    coef = torch.zeros(shape, dtype=torch.complex128, device=device)
    idx = torch.from_numpy(np.nonzero(sel.ravel())[0]).to(device)
    coef.view(-1)[idx] = torch.from_numpy(np.exp(1j * ph)).to(device)
    f = torch.fft.ifftn(coef).real.contiguous()
    return f / f.abs().max()


# ----------------------------------------------------------------------------- workloads

def gaussian_pulse_2d(n: int = 64, kappa: float = 1e3, sigma: float = 4.0, floor: float = 1e-6,
                      dt_factor: float = 10.0, limiter: str = "lp") -> dict:
    """Gaussian E_r pulse on a uniform static periodic medium (code units)."""
    grid = periodic_grid((n, n))
    phys = code_units(limiter)
    phys["opacity"] = "const"
    phys["kappa0"] = kappa
    x = np.arange(n) + 0.5
    X, Y = np.meshgrid(x, x, indexing="xy")  # arrays (ny, nx), x fastest
    r2 = (X - n / 2) ** 2 + (Y - n / 2) ** 2
    E = floor + np.exp(-r2 / (2 * sigma ** 2))
    rho = np.ones_like(E)
    eps = equilibrium_eps(phys, rho, rad_temperature(phys, E))
    dt_exp = thick_explicit_dt(1.0, 2, phys["c"], kappa * 1.0)
    return {"name": f"gaussian_pulse_2d_{n}", "grid": grid, "phys": phys, "rho": rho, "eps": eps,
            "E": E, "dt": dt_factor * dt_exp, "dt_exp": dt_exp, "sigma": sigma, "floor": floor,
            "D_thick": phys["c"] / (3 * kappa)}


def lognormal_fields(rng, shape, phys: dict, kappa0: float, sigma_ln: float = 1.0, device=None):
    G = gaussian_random_field(rng, shape, device=device)
    xp = np if device is None else __import__("torch")
    rho = xp.exp(sigma_ln * G - sigma_ln ** 2 / 2)
    del G
    Tg = 1.0 + 0.3 * smooth_field(rng, shape, device=device)
    Tr = 1.0 + 0.3 * smooth_field(rng, shape, device=device)
    E = rad_energy(phys, Tr)
    del Tr
    eps = equilibrium_eps(phys, rho, Tg)
    kr_min = float((kappa0 * rho * Tg ** -3.5 * rho).min())
    return rho, eps, E, kr_min


def lognormal_3d(n: int = 128, seed: int = 1, kappa0: float = 1.0, dt_factor: float = 100.0,
                 ndim: int = 3, limiter: str = "lp", device=None, dt_exp=None) -> dict:
    """Lognormal density with Kramers opacity; periodic n^ndim (code units); dt = dt_factor x the
    explicit limit dt_exp of the initial state (None: dt is None until ``with_explicit_dt``).
    With a torch ``device`` the fields are built there (same noise and recipe) as tensors."""
    rng = np.random.default_rng(SEED_BASE + seed)
    shape = (n,) * ndim
    grid = periodic_grid(shape)
    phys = code_units(limiter)
    phys.update(opacity="kramers", kappa0=kappa0, kr_a=1.0, kr_b=-3.5)
    rho, eps, E, kr_min = lognormal_fields(rng, shape, phys, kappa0, device=device)
    case = {"name": f"lognormal_{ndim}d_{n}", "seed": seed, "grid": grid, "phys": phys, "rho": rho,
            "eps": eps, "E": E, "dt_factor": dt_factor, "dt": None, "dt_exp": None,
            "dt_exp_thick": thick_explicit_dt(1.0, ndim, phys["c"], kr_min)}
    return case if dt_exp is None else with_explicit_dt(case, dt_exp)


def batched_2d(ngrids: int = 512, seed: int = 3, nmin: int = 64, nmax: int = 512,
               limiter: str = "lp", dt_exp=None) -> list:
    """Independent square periodic 2-D grids of uneven size, opacity and time step
    (dt = 10^U(1,3) x each grid's explicit limit; dt_exp: one per grid, or None)."""
    rng = np.random.default_rng(SEED_BASE + seed)
    out = []
    for g in range(ngrids):
        n = int(16 * round(math.exp(rng.uniform(math.log(nmin), math.log(nmax))) / 16))
        n = max(16, n)
        kappa0 = 10.0 ** rng.uniform(-2, 4)
        fac = 10.0 ** rng.uniform(1, 3)
        grid = periodic_grid((n, n))
        phys = code_units(limiter)
        phys.update(opacity="kramers", kappa0=kappa0, kr_a=1.0, kr_b=-3.5)
        rho, eps, E, kr_min = lognormal_fields(rng, (n, n), phys, kappa0)
        case = {"name": f"batched_2d_{g}", "grid": grid, "phys": phys, "rho": rho, "eps": eps, "E": E,
                "dt_factor": fac, "dt": None, "dt_exp": None,
                "dt_exp_thick": thick_explicit_dt(1.0, 2, phys["c"], kr_min)}
        out.append(case if dt_exp is None else with_explicit_dt(case, float(dt_exp[g])))
    return out


def opacity_table(nrho: int = 128, nT: int = 128, lrho=(-16.0, -6.0), lT=(3.7, 6.5)):
    """Synthetic log10 kappa table: electron scattering + Kramers + an iron-like bump at
    log T = 5.3.  Rows are log10 rho, columns log10 T.  Returns (table, tlo, thi) with the
    parameters' convention: tlo = [lowest log10 rho, lowest log10 T], thi = the highest."""
    lr = np.linspace(lrho[0], lrho[1], nrho)
    lt = np.linspace(lT[0], lT[1], nT)
    R, T = np.meshgrid(10.0 ** lr, 10.0 ** lt, indexing="ij")
    kK = 0.2 / (1e-10 * (1e5) ** -3.5)
    bump = 1.0 * np.exp(-(np.log10(T) - 5.3) ** 2 / (2 * 0.15 ** 2)) * (R / 1e-10) ** 0.25
    kap = 0.2 + kK * R * T ** -3.5 + bump
    return np.ascontiguousarray(np.log10(kap)), [lrho[0], lT[0]], [lrho[1], lT[1]]


def wind_columns(ncol: int = 4096, ncell: int = 2048, seed: int = 4, dt_factor: float = 100.0,
                 limiter: str = "lp", dt_exp=None) -> dict:
    """Spherically symmetric wind-like radial columns (cgs).  Arrays are (ncol, ncell).  dt per
    column = dt_factor x its explicit limit (dt_exp: ncol values, or None)."""
    rng = np.random.default_rng(SEED_BASE + seed)
    mu = 4.0 / 3.0  # fully ionised helium
    phys = cgs_units(mu, limiter=limiter)
    tab, tlo, thi = opacity_table()
    phys.update(opacity="table", table=tab, tlo=tlo, thi=thi)
    Rs = R_SUN
    rf = Rs * 100.0 ** (np.arange(ncell + 1) / ncell)
    rc = 0.5 * (rf[1:] + rf[:-1])
    dr = rf[1:] - rf[:-1]
    L = 10 ** 5.416 * L_SUN
    kappa_es = 0.2
    Mdot0 = 1.87e-5 * M_SUN / YEAR
    vinf0 = 1.0e8
    rho = np.empty((ncol, ncell))
    E = np.empty((ncol, ncell))
    Tg = np.empty((ncol, ncell))
    vel = np.empty((ncol, ncell))
    for j in range(ncol):
        Mdot = Mdot0 * rng.uniform(0.8, 1.2)
        vinf = vinf0 * rng.uniform(0.8, 1.2)
        rs = Rs * rng.uniform(1.02, 1.3)
        v = np.maximum(vinf * np.sqrt(np.maximum(1 - Rs / rc, 0.0)), 1e-3 * vinf)
        vel[j] = v
        r_wind = Mdot / (4 * np.pi * rc ** 2 * v)
        vs = max(vinf * math.sqrt(1 - Rs / rs), 1e-3 * vinf)
        rho_s = Mdot / (4 * np.pi * rs ** 2 * vs)
        inner = rho_s * np.exp(np.minimum((rs - rc) / (0.01 * Rs), 10.0))
        rho[j] = np.where(rc < rs, inner, r_wind)
        # E from the inward integral of the Eddington-approximation flux, T(r_max) = 5e4 K
        integrand = 3 * kappa_es * rho[j] * L / (4 * np.pi * rc ** 2 * C_LIGHT) * dr
        tail = np.cumsum(integrand[::-1])[::-1]
        E[j] = A_RAD * 5.0e4 ** 4 + tail
        Tr = (E[j] / A_RAD) ** 0.25
        noise = np.interp(np.arange(ncell), np.linspace(0, ncell - 1, 17), rng.uniform(-1, 1, 17))
        Tg[j] = Tr * (1 + 0.05 * noise)
    eps = rho * phys["gas_R"] * Tg / (phys["gamma"] - 1.0)
    # electron scattering is the smallest opacity the table holds: the optically thick bound
    dt_thick = (dr[None, :] ** 2 * 3 * kappa_es * rho / (2 * C_LIGHT)).min(axis=1)
    case = {"name": f"wind_columns_{ncol}x{ncell}", "seed": seed, "phys": phys, "r_faces": rf,
            "geometry": "spherical", "bc": ["dirichlet", "dirichlet"], "rho": rho, "eps": eps,
            "E": E, "bc_lo": E[:, 0].copy(), "bc_hi": E[:, -1].copy(), "dt_factor": dt_factor,
            "dt": None, "dt_exp": None, "dt_exp_thick": dt_thick, "v": vel, "L": L, "r_star": Rs}
    return case if dt_exp is None else with_explicit_dt(case, np.asarray(dt_exp, dtype=np.float64))


def wind_cak(case: dict, Qbar: float = 2000.0) -> dict:
    """CAK line-opacity parameters of the wind columns (Sect. 5.1): kappa_e Qbar with electron
    scattering kappa_e = 0.2 cm^2/g, alpha 0.66 -> 0.5 between 1 - R*/r = 0.4 and 0.65."""
    return {"v": case["v"], "kappa_e_Qbar": 0.2 * Qbar, "r_star": case["r_star"], "alpha_in": 0.66,
            "alpha_out": 0.5, "x_in": 0.4, "x_out": 0.65}


def heating_cooling(e_ratio: float, dt: float, ncell: int = 16) -> dict:
    """Uniform static gas: rho = 1e-7, kappa = 0.4, gamma = 5/3, mu = 0.6, E = 1e12 (cgs);
    gas energy e_ratio times the equilibrium value set by the radiation temperature."""
    phys = cgs_units(0.6)
    phys.update(opacity="const", kappa0=0.4)
    rho = np.full(ncell, 1e-7)
    E = np.full(ncell, 1e12)
    Tr = rad_temperature(phys, E)
    e_eq = equilibrium_eps(phys, rho, Tr)
    return {"name": f"heating_cooling_{e_ratio:g}", "phys": phys, "rho": rho, "E": E,
            "eps": e_ratio * e_eq, "e_equil": e_eq, "dt": dt}


def thin_front(ncell: int = 256) -> dict:
    """Optically thin slab: rho = 0.025, kappa = 0.4 on [-0.5, 1.5] cm, erf-lit from the left."""
    from math import erf
    phys = cgs_units(0.6)
    phys.update(opacity="const", kappa0=0.4)
    dx = 2.0 / ncell
    x = -0.5 + (np.arange(ncell) + 0.5) * dx
    E0, E1, d = 1.4e-11, 1.4e11, 0.05
    E = E0 + 0.5 * (1 - np.array([erf(v / d) for v in x])) * E1
    rho = np.full(ncell, 0.025)
    eps = equilibrium_eps(phys, rho, rad_temperature(phys, np.full(ncell, E0)))
    grid = {"ndim": 1, "n": [ncell, 1, 1], "dx": [dx, 1.0, 1.0],
            "bc": ["dirichlet", "dirichlet"] + ["periodic"] * 4, "bc_val": [E0 + E1, E0, 0, 0, 0, 0]}
    return {"name": "thin_front", "grid": grid, "phys": phys, "rho": rho, "eps": eps, "E": E,
            "x": x, "dt": 1e-13, "E0": E0, "E1": E1}


def random_small(shape, seed: int, bc=None, kappa0: float = 1.0, dt_factor: float = 30.0,
                 limiter: str = "lp") -> dict:
    """Small heterogeneous grid for brute-force checks (code units, Kramers opacity)."""
    rng = np.random.default_rng(SEED_BASE + 1000 + seed)
    nd = len(shape)
    grid = periodic_grid(shape)
    if bc is not None:
        grid["bc"] = list(bc[0])
        grid["bc_val"] = list(bc[1])
    phys = code_units(limiter)
    phys.update(opacity="kramers", kappa0=kappa0)
    arr_shape = tuple(reversed(shape))
    rho, eps, E, kr_min = lognormal_fields(rng, arr_shape, phys, kappa0)
    # the optically thick time scale (these brute-force cases fix their stiffness by dt_factor)
    dt_exp = thick_explicit_dt(1.0, nd, phys["c"], kr_min)
    return {"name": f"random_{'x'.join(map(str, shape))}_{seed}", "grid": grid, "phys": phys,
            "rho": rho, "eps": eps, "E": E, "dt": dt_factor * dt_exp, "dt_exp": dt_exp}
