"""Plain FP64 CPU oracle for the FLD radiation-energy update (arXiv 2104.03968).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library never
loads it and shares no source with it.

The arithmetic lives in ``fld_oracle.c`` (plain loops, double precision); this
module compiles it with gcc on first use and marshals numpy arrays through ctypes.
Parameter dictionaries use the plain-data schema of the seeded input generators:

    grid = {"ndim": 3, "n": [nx, ny, nz], "dx": [..], "bc": ["periodic"] * 6,
            "bc_val": [0.0] * 6}
    phys = {"c": .., "a_rad": .., "gamma": .., "gas_R": .., "limiter": "lp",
            "opacity": "kramers", "kappa0": .., "kr_a": 1.0, "kr_b": -3.5,
            "table": None | 2-D array of log10 kappa, "tlo": [..], "thi": [..]}

``step`` composes the oracle's functions in the order of a full radiation-energy
update: opacity, coefficients (Sect. 2.2), implicit diffusion (Sect. 3.4) and the
point-implicit exchange (Sect. 3.3).
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fld_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

BC = {"periodic": 0, "neumann": 1, "dirichlet": 2, "continuous": 3, "luminosity": 4}
LIMITER = {"lp": 0, "third": 1, "minerbo": 2}
OPACITY = {"const": 0, "kramers": 1, "table": 2}
GEOMETRY = {"cartesian": 0, "spherical": 1}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no CUDA).  Returns the library path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "fld_oracle.h")))
    if force or stale:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Grid(ct.Structure):
    _fields_ = [("ndim", ct.c_int), ("n", ct.c_int * 3), ("dx", ct.c_double * 3),
                ("bc", ct.c_int * 6), ("bc_val", ct.c_double * 6)]


class _Phys(ct.Structure):
    _fields_ = [("c", ct.c_double), ("a_rad", ct.c_double), ("gamma", ct.c_double),
                ("gas_R", ct.c_double), ("limiter", ct.c_int), ("opacity", ct.c_int),
                ("kappa0", ct.c_double), ("kr_a", ct.c_double), ("kr_b", ct.c_double),
                ("table", ct.POINTER(ct.c_double)), ("tn", ct.c_int * 2),
                ("tlo", ct.c_double * 2), ("thi", ct.c_double * 2)]


_D = ct.POINTER(ct.c_double)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ct.CDLL(build())
            P = ct.c_void_p
            sig = {
                "ora_lambda": (ct.c_double, [ct.c_double]),
                "ora_lambda_minerbo": (ct.c_double, [ct.c_double]),
                "ora_temperature": (ct.c_double, [P, ct.c_double, ct.c_double]),
                "ora_kappa": (ct.c_double, [P, ct.c_double, ct.c_double]),
                "ora_opacity": (None, [ct.c_size_t, P, _D, _D, _D]),
                "ora_coeffs": (ct.c_int, [P, P, _D, _D, _D, _D, _D]),
                "ora_radiation_sources": (ct.c_int, [P, P, _D, _D, _D, P, P, P, _D, _D, P, _D]),
                "ora_pseudo_planar_source": (ct.c_int, [P, P, ct.c_double, _D, _D, _D, P, _D]),
                "ora_apply": (None, [P, ct.c_double, _D, _D, _D]),
                "ora_rhs": (None, [P, ct.c_double, _D, _D, _D]),
                "ora_relres": (ct.c_double, [P, ct.c_double, _D, _D, _D]),
                "ora_diffuse_cg": (ct.c_int, [P, ct.c_double, _D, _D, _D, ct.c_double, ct.c_int,
                                              _D, ct.POINTER(ct.c_int)]),
                "ora_diffuse_dense": (ct.c_int, [P, ct.c_double, _D, _D, _D]),
                "ora_apply_aniso": (None, [P, ct.c_double, P, _D, _D]),
                "ora_relres_aniso": (ct.c_double, [P, ct.c_double, P, _D, _D]),
                "ora_diffuse_cg_aniso": (ct.c_int, [P, ct.c_double, P, _D, _D, ct.c_double, ct.c_int,
                                                    _D, ct.POINTER(ct.c_int)]),
                "ora_kappa_cak": (None, [ct.c_int, _D, _D, _D, ct.c_double, ct.c_double, ct.c_double,
                                         ct.c_double, ct.c_double, ct.c_double, ct.c_double, _D]),
                "ora_column_coeffs": (ct.c_int, [ct.c_int, _D, ct.c_int, ct.c_int, ct.c_double,
                                                 ct.c_double, P, _D, _D, _D, _D]),
                "ora_column_diffuse": (ct.c_int, [ct.c_int, _D, ct.c_int, ct.c_int, ct.c_int,
                                                  ct.c_double, ct.c_double, ct.c_double, _D, _D, _D]),
                "ora_column_diffuse_dense": (ct.c_int, [ct.c_int, _D, ct.c_int, ct.c_int, ct.c_int,
                                                        ct.c_double, ct.c_double, ct.c_double, _D, _D,
                                                        _D]),
                "ora_column_relres": (ct.c_double, [ct.c_int, _D, ct.c_int, ct.c_int, ct.c_int,
                                                    ct.c_double, ct.c_double, ct.c_double, _D, _D, _D]),
                "ora_exchange": (ct.c_int, [ct.c_size_t, P, ct.c_double, _D, _D, _D, _D, ct.c_int,
                                            ct.POINTER(ct.c_int), ct.POINTER(ct.c_int)]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _grid(g: dict) -> _Grid:
    s = _Grid()
    s.ndim = int(g["ndim"])
    n = list(g["n"]) + [1] * (3 - len(g["n"]))
    dx = list(g.get("dx", [1.0] * 3)) + [1.0] * (3 - len(g.get("dx", [1.0] * 3)))
    bc = list(g.get("bc", ["periodic"] * 6))
    bv = list(g.get("bc_val", [0.0] * 6))
    for a in range(3):
        s.n[a] = int(n[a])
        s.dx[a] = float(dx[a])
    for f in range(6):
        s.bc[f] = BC[bc[f]] if isinstance(bc[f], str) else int(bc[f])
        s.bc_val[f] = float(bv[f])
    return s


def _phys(p: dict, keep: list) -> _Phys:
    s = _Phys()
    s.c = p["c"]
    s.a_rad = p["a_rad"]
    s.gamma = p["gamma"]
    s.gas_R = p["gas_R"]
    s.limiter = LIMITER[p.get("limiter", "lp")]
    s.opacity = OPACITY[p.get("opacity", "const")]
    s.kappa0 = p.get("kappa0", 1.0)
    s.kr_a = p.get("kr_a", 1.0)
    s.kr_b = p.get("kr_b", -3.5)
    if s.opacity == OPACITY["table"]:
        t = _f64(p["table"])
        keep.append(t)
        s.table = _ptr(t)
        s.tn[0], s.tn[1] = t.shape
        s.tlo[0], s.tlo[1] = p["tlo"]
        s.thi[0], s.thi[1] = p["thi"]
    return s


def _ref(s):
    return ct.cast(ct.pointer(s), ct.c_void_p)


# ----------------------------------------------------------------------------- physics

def lam(R: float) -> float:
    """Levermore-Pomraning limiter, Sect. 2.2, Eq. (fld_lambda)."""
    return _load().ora_lambda(float(R))


def lam_minerbo(R: float) -> float:
    """Minerbo limiter, the alternative Sect. 2.2 names."""
    return _load().ora_lambda_minerbo(float(R))


def temperature(phys: dict, rho: float, eps: float) -> float:
    keep = []
    return _load().ora_temperature(_ref(_phys(phys, keep)), float(rho), float(eps))


def opacity(phys: dict, rho, eps) -> np.ndarray:
    """kappa per cell from rho and the gas internal energy density eps."""
    rho, eps = _f64(rho), _f64(eps)
    out = np.empty_like(rho)
    keep = []
    _load().ora_opacity(rho.size, _ref(_phys(phys, keep)), _ptr(rho), _ptr(eps), _ptr(out))
    return out


def coeffs(grid: dict, phys: dict, E, rho, kappa, with_grad: bool = False):
    """Cell-centred D = c lambda(R) / (kappa rho) (Sect. 2.2), R from the 5-point gradient."""
    E, rho, kappa = _f64(E), _f64(rho), _f64(kappa)
    D = np.empty_like(E)
    gm = np.empty_like(E)
    keep = []
    st = _load().ora_coeffs(_ref(_grid(grid)), _ref(_phys(phys, keep)), _ptr(E), _ptr(rho), _ptr(kappa),
                            _ptr(D), _ptr(gm))
    if st:
        raise ValueError(f"oracle coeffs: status {st}")
    return (D, gm) if with_grad else D


def _ptr_array(arrays):
    """A C array of double pointers (None -> NULL array)."""
    if arrays is None:
        return None
    arr = (_D * len(arrays))(*[_ptr(a) for a in arrays])
    return ct.cast(arr, ct.c_void_p), arr


def radiation_sources(grid: dict, phys: dict, E, rho, kappa, v=None) -> dict:
    """Sect. 2.1-2.2 and 3.2: per cell the flux F = -D grad E, the force density f_r = rho kappa
    F / c, its work v . f_r, the Eddington factor f = lambda + lambda^2 R^2, the pressure tensor
    P = E [(1-f)/2 I + (3f-1)/2 n n] (xx, yy, zz, xy, xz, yz) and the photon-tiring term
    P : grad v (5-point gradients; velocity ghosts by linear extrapolation)."""
    E, rho, kappa = _f64(E), _f64(rho), _f64(kappa)
    nd = int(grid["ndim"])
    out = {"F": [np.empty_like(E) for _ in range(nd)], "fr": [np.empty_like(E) for _ in range(nd)],
           "work": np.empty_like(E), "fedd": np.empty_like(E), "P": [np.empty_like(E) for _ in range(6)],
           "tiring": np.empty_like(E)}
    vs = None if v is None else [_f64(c) for c in v]
    keep = []
    pv = _ptr_array(vs)
    pF, pfr, pP = _ptr_array(out["F"]), _ptr_array(out["fr"]), _ptr_array(out["P"])
    st = _load().ora_radiation_sources(_ref(_grid(grid)), _ref(_phys(phys, keep)), _ptr(E), _ptr(rho), _ptr(kappa),
                                       pv[0] if pv else None, pF[0], pfr[0], _ptr(out["work"]), _ptr(out["fedd"]),
                                       pP[0], _ptr(out["tiring"]))
    if st:
        raise ValueError(f"oracle radiation_sources: status {st}")
    return out



def pseudo_planar_source(grid: dict, phys: dict, x0: float, E, rho, kappa, v=None) -> np.ndarray:
    """Appendix A: the geometric source of the radiation energy on a Cartesian grid whose x axis
    stands for the radius, S = -2 (E v_x + F_x) / x + 2 v_x P_xx / x, x = x0 + (i + 1/2) dx_x the
    cell centre's radius; F and P as in radiation_sources; v = None means v = 0."""
    E, rho, kappa = _f64(E), _f64(rho), _f64(kappa)
    S = np.empty_like(E)
    vs = None if v is None else [_f64(c) for c in v]
    pv = _ptr_array(vs)
    keep = []
    st = _load().ora_pseudo_planar_source(_ref(_grid(grid)), _ref(_phys(phys, keep)), float(x0), _ptr(E), _ptr(rho),
                                          _ptr(kappa), pv[0] if pv else None, _ptr(S))
    if st:
        raise ValueError(f"oracle pseudo_planar_source: status {st}")
    return S


# ----------------------------------------------------------------------------- diffusion

def apply(grid: dict, dt: float, D, x) -> np.ndarray:
    D, x = _f64(D), _f64(x)
    out = np.empty_like(x)
    _load().ora_apply(_ref(_grid(grid)), float(dt), _ptr(D), _ptr(x), _ptr(out))
    return out


def rhs(grid: dict, dt: float, D, E_old) -> np.ndarray:
    D, E_old = _f64(D), _f64(E_old)
    out = np.empty_like(E_old)
    _load().ora_rhs(_ref(_grid(grid)), float(dt), _ptr(D), _ptr(E_old), _ptr(out))
    return out


def _axes(grid: dict, D):
    """A list of per-axis D arrays (a diagonal tensor), or None for one scalar D field."""
    if isinstance(D, (list, tuple)):
        if len(D) != int(grid["ndim"]):
            raise ValueError("a diagonal-tensor D needs one array per axis")
        arrs = [_f64(d) for d in D]
        return arrs + [arrs[0]] * (3 - len(arrs))
    return None


def relres(grid: dict, dt: float, D, E_old, x) -> float:
    """||b - A x||_2 / ||b||_2 of the backward-Euler system of Sect. 3.4 (D: one array, or one
    per axis for a diagonal-tensor D)."""
    E_old, x = _f64(E_old), _f64(x)
    ax = _axes(grid, D)
    if ax is not None:
        pa = _ptr_array(ax)
        return _load().ora_relres_aniso(_ref(_grid(grid)), float(dt), pa[0], _ptr(E_old), _ptr(x))
    D = _f64(D)
    return _load().ora_relres(_ref(_grid(grid)), float(dt), _ptr(D), _ptr(E_old), _ptr(x))


def diffuse(grid: dict, dt: float, D, E_old, rtol: float = 1e-13, maxit: int = 100000,
            method: str = "cg") -> np.ndarray:
    """E^{n+1} solving Eq. (discdiff) (times dt) by Jacobi-CG or dense LU.  D: one array, or one
    per axis (a diagonal-tensor D, Jacobi-CG only)."""
    E_old = _f64(E_old)
    x = np.empty_like(E_old)
    lib = _load()
    g = _ref(_grid(grid))
    ax = _axes(grid, D)
    if ax is not None:
        pa = _ptr_array(ax)
        rr = ct.c_double()
        it = ct.c_int()
        st = lib.ora_diffuse_cg_aniso(g, float(dt), pa[0], _ptr(E_old), _ptr(x), float(rtol), int(maxit),
                                      ct.byref(rr), ct.byref(it))
        if st not in (0, 4):
            raise ValueError(f"oracle CG: status {st}")
        diffuse.last_relres = rr.value
        diffuse.last_iters = it.value
        return x
    D = _f64(D)
    if method == "dense":
        st = lib.ora_diffuse_dense(g, float(dt), _ptr(D), _ptr(E_old), _ptr(x))
        if st:
            raise ValueError(f"oracle dense solve: status {st}")
        return x
    rr = ct.c_double()
    it = ct.c_int()
    st = lib.ora_diffuse_cg(g, float(dt), _ptr(D), _ptr(E_old), _ptr(x), float(rtol), int(maxit),
                            ct.byref(rr), ct.byref(it))
    if st not in (0, 4):
        raise ValueError(f"oracle CG: status {st}")
    diffuse.last_relres = rr.value
    diffuse.last_iters = it.value
    return x


def _col_args(col: dict):
    rf = _f64(col["r_faces"])
    return (rf.size - 1, rf, GEOMETRY[col.get("geometry", "spherical")], BC[col["bc"][0]], BC[col["bc"][1]])


def column_coeffs(col: dict, phys: dict, E, rho, kappa, v_lo: float = 0.0, v_hi: float = 0.0) -> np.ndarray:
    n, rf, _, blo, bhi = _col_args(col)
    E, rho, kappa = _f64(E), _f64(rho), _f64(kappa)
    D = np.empty_like(E)
    keep = []
    st = _load().ora_column_coeffs(n, _ptr(rf), blo, bhi, float(v_lo), float(v_hi), _ref(_phys(phys, keep)),
                                   _ptr(E), _ptr(rho), _ptr(kappa), _ptr(D))
    if st:
        raise ValueError(f"oracle column coeffs: status {st}")
    return D


def column_diffuse(col: dict, dt: float, D, E_old, v_lo: float = 0.0, v_hi: float = 0.0,
                   method: str = "thomas") -> np.ndarray:
    n, rf, geom, blo, bhi = _col_args(col)
    D, E_old = _f64(D), _f64(E_old)
    x = np.empty_like(E_old)
    fn = _load().ora_column_diffuse_dense if method == "dense" else _load().ora_column_diffuse
    st = fn(n, _ptr(rf), geom, blo, bhi, float(v_lo), float(v_hi), float(dt), _ptr(D), _ptr(E_old), _ptr(x))
    if st:
        raise ValueError(f"oracle column solve: status {st}")
    return x


def column_relres(col: dict, dt: float, D, E_old, x, v_lo: float = 0.0, v_hi: float = 0.0) -> float:
    n, rf, geom, blo, bhi = _col_args(col)
    D, E_old, x = _f64(D), _f64(E_old), _f64(x)
    return _load().ora_column_relres(n, _ptr(rf), geom, blo, bhi, float(v_lo), float(v_hi), float(dt),
                                     _ptr(D), _ptr(E_old), _ptr(x))


# ----------------------------------------------------------------------------- exchange

def exchange(phys: dict, dt: float, rho, kappa, eps, E, maxit: int = 100):
    """Point-implicit heating/cooling of Sect. 3.3.  Returns (eps_new, E_new, info)."""
    rho, kappa = _f64(rho), _f64(kappa)
    eps = _f64(eps).copy()
    E = _f64(E).copy()
    mi = ct.c_int()
    nb = ct.c_int()
    keep = []
    st = _load().ora_exchange(rho.size, _ref(_phys(phys, keep)), float(dt), _ptr(rho), _ptr(kappa),
                              _ptr(eps), _ptr(E), int(maxit), ct.byref(mi), ct.byref(nb))
    if st:
        raise ValueError(f"oracle exchange: status {st}")
    return eps, E, {"max_iters": mi.value, "bisections": nb.value}


# ----------------------------------------------------------------------------- full update

def step(grid: dict, phys: dict, dt: float, rho, eps, E, order: str = "diffuse_then_exchange",
         rtol: float = 1e-13, method: str = "cg", exch_maxit: int = 100):
    """One radiation-energy update.  D is lagged (built from the state entering the
    diffusion stage); kappa^n for the exchange is built from the state entering it."""
    rho = _f64(rho)
    eps = _f64(eps)
    E = _f64(E)
    info = {}

    def diffusion(eps_, E_, h=dt):
        kap = opacity(phys, rho, eps_)
        D = coeffs(grid, phys, E_, rho, kap)
        En = diffuse(grid, h, D, E_, rtol=rtol, method=method)
        info["relres"] = relres(grid, h, D, E_, En)
        return En

    def exch(eps_, E_, h=dt):
        kap = opacity(phys, rho, eps_)
        e2, E2, inf = exchange(phys, h, rho, kap, eps_, E_, maxit=exch_maxit)
        info.update(inf)
        return e2, E2

    if order == "diffuse_then_exchange":
        E = diffusion(eps, E)
        eps, E = exch(eps, E)
    elif order == "exchange_then_diffuse":
        eps, E = exch(eps, E)
        E = diffusion(eps, E)
    elif order == "imex_midpoint":
        eps, E = imex_midpoint(eps, E, dt, exch, diffusion)
    else:
        raise ValueError(f"unknown order {order}")
    return eps, E, info


def imex_midpoint(eps, E, dt, exch, diffusion):
    """Sect. 3.1, the midpoint IMEX scheme for the radiation-energy subsystem of a static
    medium.  The explicit operator is the local implicit exchange (no advection, no explicit
    sources here), the implicit operator the diffusion:
      u+      = u^n advanced by the explicit operator over dt/2,
      u^{1/2} = u+ advanced by the implicit diffusion over dt/2,
      u^{n+1} = u^n + dt G_im(u^{1/2}) (the half-step diffusion increment, doubled), then the
                explicit operator over the full dt from that state."""
    eps_h, E_h = exch(eps, E, dt / 2)
    E_mid = diffusion(eps_h, E_h, dt / 2)
    E_star = E + 2.0 * (E_mid - E_h)
    return exch(eps, E_star, dt)


def kappa_cak(col: dict, phys: dict, rho, cak: dict) -> np.ndarray:
    """Sect. 5.1, Eq. (kap_cak): the CAK line opacity of one column.  cak: {"v": radial velocity
    at the cell centres, "kappa_e_Qbar", "r_star", "alpha_in", "alpha_out", "x_in", "x_out"}."""
    rf = _f64(col["r_faces"])
    rho, v = _f64(rho), _f64(cak["v"])
    out = np.empty_like(rho)
    _load().ora_kappa_cak(rf.size - 1, _ptr(rf), _ptr(rho), _ptr(v), float(phys["c"]), float(cak["kappa_e_Qbar"]),
                          float(cak["r_star"]), float(cak["alpha_in"]), float(cak["alpha_out"]), float(cak["x_in"]),
                          float(cak["x_out"]), _ptr(out))
    return out


def column_step(col: dict, phys: dict, dt: float, rho, eps, E, v_lo: float, v_hi: float,
                order: str = "diffuse_then_exchange", exch_maxit: int = 100, cak: dict = None):
    """One radiation-energy update of a single 1-D column (tridiagonal diffusion).  With cak, the
    CAK line opacity (Sect. 5.1) is added to the opacity model everywhere the opacity enters."""
    rho, eps, E = _f64(rho), _f64(eps), _f64(E)
    info = {}
    k_line = kappa_cak(col, phys, rho, cak) if cak is not None else 0.0

    def kappa_of(eps_):
        return opacity(phys, rho, eps_) + k_line

    def diffusion(eps_, E_, h=dt):
        kap = kappa_of(eps_)
        D = column_coeffs(col, phys, E_, rho, kap, v_lo, v_hi)
        En = column_diffuse(col, h, D, E_, v_lo, v_hi)
        info["relres"] = column_relres(col, h, D, E_, En, v_lo, v_hi)
        return En

    def exch(eps_, E_, h=dt):
        kap = kappa_of(eps_)
        e2, E2, inf = exchange(phys, h, rho, kap, eps_, E_, maxit=exch_maxit)
        info.update(inf)
        return e2, E2

    if order == "diffuse_then_exchange":
        E = diffusion(eps, E)
        eps, E = exch(eps, E)
    elif order == "exchange_then_diffuse":
        eps, E = exch(eps, E)
        E = diffusion(eps, E)
    elif order == "imex_midpoint":
        eps, E = imex_midpoint(eps, E, dt, exch, diffusion)
    else:
        raise ValueError(f"unknown order {order}")
    return eps, E, info
