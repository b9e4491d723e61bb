"""Thin ctypes binding over the C ABI of ``include/fld.h`` (libfld.so, sm_103a).

Argument marshalling only: every step of the update runs in the CUDA library.
Device arrays are float64, contiguous torch CUDA tensors (x fastest, i.e. a torch
tensor of shape (nz, ny, nx)); the stream is torch's current stream.  Host arrays
(numpy or CPU tensors) are accepted by ``step`` / ``columns_step`` / ``step_batched``,
which then copy them to the device and back around the call.

Parameter dictionaries follow the plain-data schema of ``inputs``: a grid dict
(ndim, n, dx, bc names, bc_val) and a physics dict (c, a_rad, gamma, gas_R, limiter,
opacity, kappa0, kr_a, kr_b, table, tlo, thi) extended by solver keys (precision
"fp64" | "mixed", rtol, max_cycles, nu1, nu2, exch_maxit, order, start "fmg" | "vcycle").
"""
from __future__ import annotations

import ctypes as ct
import os
import threading

import numpy as np
import torch

from . import build as _build

BC = {"periodic": 0, "neumann": 1, "dirichlet": 2, "continuous": 3, "luminosity": 4}
LIMITER = {"lp": 0, "third": 1, "minerbo": 2}
OPACITY = {"const": 0, "kramers": 1, "table": 2}
PRECISION = {"fp64": 0, "mixed": 1}
ORDER = {"diffuse_then_exchange": 0, "exchange_then_diffuse": 1, "imex_midpoint": 2}
GEOMETRY = {"cartesian": 0, "spherical": 1}
START = {"fmg": 0, "vcycle": 1}
STATUS = {0: "ok", 1: "invalid argument", 2: "non-positive input", 3: "non-finite residual",
          4: "not converged", 5: "CUDA error", 6: "device timeout", 7: "unsupported"}


class FldError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"fld status {status} ({STATUS.get(status, '?')}): {msg}")
        self.status = status


class Grid(ct.Structure):
    _fields_ = [("ndim", ct.c_int), ("n", ct.c_int * 3), ("dx", ct.c_double * 3), ("bc", ct.c_int * 6),
                ("bc_val", ct.c_double * 6)]


class Cak(ct.Structure):
    _fields_ = [("v", ct.c_void_p), ("kappa_e_Qbar", ct.c_double), ("r_star", ct.c_double),
                ("alpha_in", ct.c_double), ("alpha_out", ct.c_double), ("x_in", ct.c_double), ("x_out", ct.c_double)]


class Params(ct.Structure):
    _fields_ = [("c", ct.c_double), ("a_rad", ct.c_double), ("gamma", ct.c_double), ("gas_R", ct.c_double),
                ("limiter", ct.c_int), ("opacity", ct.c_int), ("kappa0", ct.c_double), ("kr_a", ct.c_double),
                ("kr_b", ct.c_double), ("table", ct.c_void_p), ("tn", ct.c_int * 2), ("tlo", ct.c_double * 2),
                ("thi", ct.c_double * 2), ("precision", ct.c_int), ("rtol", ct.c_double),
                ("max_cycles", ct.c_int), ("nu1", ct.c_int), ("nu2", ct.c_int), ("exch_maxit", ct.c_int),
                ("order", ct.c_int), ("start", ct.c_int), ("cak", ct.c_void_p)]


class Info(ct.Structure):
    _fields_ = [("cycles", ct.c_int), ("rel_residual", ct.c_double), ("exch_max_iters", ct.c_int),
                ("bisection_fallbacks", ct.c_int), ("status", ct.c_int), ("nu1", ct.c_int), ("nu2", ct.c_int),
                ("nu1_coarse", ct.c_int), ("nu2_coarse", ct.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_lock = threading.Lock()
P = ct.c_void_p
_SIGS = {
    "fld_ctx_create": [ct.POINTER(ct.c_void_p), ct.c_int],
    "fld_ctx_destroy": [P],
    "fld_coeffs": [P, P, P, P, P, P, P, P, P],
    "fld_diffuse": [P, P, P, ct.c_double, P, P, P, P, P],
    "fld_exchange": [P, ct.c_size_t, P, ct.c_double, P, P, P, P, P, P],
    "fld_opacity": [P, ct.c_size_t, P, P, P, P, P],
    "fld_step": [P, P, P, ct.c_double, P, P, P, P, P],
    "fld_step_host": [P, P, P, ct.c_double, P, P, P, P, P],
    "fld_step_batched": [P, ct.c_int, P, P, P, P, P, P, P, P],
    "fld_columns_step": [P, ct.c_int, ct.c_int, P, ct.c_int, ct.c_int, ct.c_int, P, P, P, P, P, P, P, P, P],
    "fld_columns_diffuse": [P, ct.c_int, ct.c_int, P, ct.c_int, ct.c_int, ct.c_int, P, P, P, P, P, P, P, P],
    "fld_radiation_terms": [P, P, P, P, P, P, P, P, P, P, P, P, P, ct.c_int, P],
    "fld_diffuse_aniso": [P, P, P, ct.c_double, P, P, P, P, P],
    "fld_photon_tiring_step": [P, P, P, ct.c_double, P, P, P, P, P],
    "fld_pseudo_planar_source": [P, P, P, ct.c_double, P, P, P, P, P, ct.c_int, P],
    "fld_pseudo_planar_step": [P, P, P, ct.c_double, ct.c_double, P, P, P, P, P],
    "fld_smooth_sweep": [P, P, ct.c_double, P, P, P, P, ct.c_int, P],
}


def library_path() -> str:
    return _build.LIB


def load():
    """Load libfld.so (building it with nvcc if it is missing or stale).  Raises if the CUDA
    library cannot be built or loaded: there is no CPU fallback."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library {path} is missing")
            lib = ct.CDLL(path)
            for name, args in _SIGS.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = ct.c_int
            lib.fld_last_error.argtypes = [P]
            lib.fld_last_error.restype = ct.c_char_p
            lib.fld_launch_count.argtypes = []
            lib.fld_launch_count.restype = ct.c_ulonglong
            _lib = lib
    return _lib


class Context:
    """An fld_ctx bound to one CUDA device."""

    def __init__(self, device: int = 0):
        self.lib = load()
        self.device = device
        h = ct.c_void_p()
        st = self.lib.fld_ctx_create(ct.byref(h), int(device))
        if st:
            raise FldError(st, f"fld_ctx_create(device={device}) failed")
        self.h = h
        self._keep = []

    def close(self):
        if getattr(self, "h", None):
            self.lib.fld_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, st: int):
        if st:
            raise FldError(st, self.lib.fld_last_error(self.h).decode())


# ----------------------------------------------------------------------------- marshalling

def launch_count() -> int:
    """Kernels the library has launched in this process so far (graph replays included)."""
    return int(load().fld_launch_count())


def _stream():
    return ct.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return ct.c_void_p(t.data_ptr())


def grid_struct(g: dict) -> Grid:
    s = Grid()
    s.ndim = int(g["ndim"])
    n = list(g["n"]) + [1] * (3 - len(g["n"]))
    dx = list(g.get("dx", [1.0] * 3))
    dx = dx + [1.0] * (3 - len(dx))
    for a in range(3):
        s.n[a] = int(n[a])
        s.dx[a] = float(dx[a])
    bc = list(g.get("bc", ["periodic"] * 6))
    bv = list(g.get("bc_val", [0.0] * 6))
    for f in range(6):
        s.bc[f] = BC[bc[f]] if isinstance(bc[f], str) else int(bc[f])
        s.bc_val[f] = float(bv[f])
    return s


def params_struct(p: dict, keep: list, device) -> Params:
    s = Params()
    s.c, s.a_rad, s.gamma, s.gas_R = (float(p[k]) for k in ("c", "a_rad", "gamma", "gas_R"))
    s.limiter = LIMITER[p.get("limiter", "lp")]
    s.opacity = OPACITY[p.get("opacity", "const")]
    s.kappa0 = float(p.get("kappa0", 1.0))
    s.kr_a = float(p.get("kr_a", 1.0))
    s.kr_b = float(p.get("kr_b", -3.5))
    if s.opacity == OPACITY["table"]:
        tab = p["table"]
        if not isinstance(tab, torch.Tensor) or not tab.is_cuda:
            tab = torch.as_tensor(np.ascontiguousarray(tab), dtype=torch.float64, device=device)
        tab = tab.contiguous()
        keep.append(tab)
        s.table = tab.data_ptr()
        s.tn[0], s.tn[1] = tab.shape
        s.tlo[0], s.tlo[1] = (float(v) for v in p["tlo"])
        s.thi[0], s.thi[1] = (float(v) for v in p["thi"])
    s.precision = PRECISION[p.get("precision", "fp64")]
    s.rtol = float(p.get("rtol", 1e-10))
    s.max_cycles = int(p.get("max_cycles", 0))
    s.nu1 = int(p.get("nu1", 0))
    s.nu2 = int(p.get("nu2", 0))
    s.exch_maxit = int(p.get("exch_maxit", 0))
    s.order = ORDER[p.get("order", "diffuse_then_exchange")]
    s.start = START[p.get("start", "fmg")]
    cak = p.get("cak")
    if cak is not None:
        v = cak["v"]
        if not isinstance(v, torch.Tensor) or not v.is_cuda:
            v = torch.as_tensor(np.ascontiguousarray(v, dtype=np.float64), device=device)
        v = v.contiguous()
        c = Cak(v.data_ptr(), float(cak["kappa_e_Qbar"]), float(cak["r_star"]), float(cak["alpha_in"]),
                float(cak["alpha_out"]), float(cak["x_in"]), float(cak["x_out"]))
        keep.extend([v, c])
        s.cak = ct.cast(ct.pointer(c), ct.c_void_p)
    return s


def _device_of(ctx: Context):
    return torch.device("cuda", ctx.device)


def to_device(a, ctx: Context) -> torch.Tensor:
    if isinstance(a, torch.Tensor):
        return a.to(device=_device_of(ctx), dtype=torch.float64).contiguous()
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=_device_of(ctx))


# ----------------------------------------------------------------------------- calls

def coeffs(ctx: Context, grid: dict, params: dict, E, rho, eps):
    """Per-cell (kappa, D) on the device (Sect. 2.2).  Inputs are CUDA tensors."""
    keep = []
    g, p = grid_struct(grid), params_struct(params, keep, _device_of(ctx))
    kappa = torch.empty_like(E)
    D = torch.empty_like(E)
    ctx.check(ctx.lib.fld_coeffs(ctx.h, ct.byref(g), ct.byref(p), _dptr(E), _dptr(rho), _dptr(eps), _dptr(kappa),
                                 _dptr(D), _stream()))
    return kappa, D


def outcome(ctx: Context, info: Info, allow_unconverged: bool = True) -> dict:
    """The outcome of an asynchronous call as a dict, once its stream has been synchronised; raises
    FldError for a failed solve or invalid input (a solve that missed rtol only if
    allow_unconverged is false)."""
    d = info.as_dict()
    st = d["status"]
    if st and not (allow_unconverged and st == 4):
        if st == 2:
            msg = "rho, kappa or E <= 0 (or eps < 0) in the input or an intermediate state"
        else:
            msg = f"diffusion solve stopped at relative residual {d['rel_residual']:.3e} after {d['cycles']} cycles"
        raise FldError(st, msg)
    return d


def diffuse(ctx: Context, grid: dict, params: dict, dt: float, D, E_old, out=None):
    """Backward-Euler diffusion solve (Sect. 3.4) by multigrid.  Returns (E_new, info); the call is
    asynchronous on torch's current stream, which this function synchronises to read info."""
    keep = []
    g, p = grid_struct(grid), params_struct(params, keep, _device_of(ctx))
    E_new = torch.empty_like(E_old) if out is None else out
    info = Info()
    ctx.check(ctx.lib.fld_diffuse(ctx.h, ct.byref(g), ct.byref(p), float(dt), _dptr(D), _dptr(E_old), _dptr(E_new),
                                  ct.byref(info), _stream()))
    torch.cuda.current_stream().synchronize()
    return E_new, outcome(ctx, info)


def _fptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError("expected a contiguous float32 CUDA tensor")
    return ct.c_void_p(t.data_ptr())


def smooth_sweep(ctx: Context, grid: dict, dt: float, D, r, x_in, x_out, first_colour: int = 0):
    """One red-black Gauss-Seidel sweep of the mixed solver's FP32 smoother (Sect. 3.4) on a 3-D
    grid: D float64, r / x_in / x_out float32 CUDA tensors (x_in None: start from zero).
    Synchronises the stream (FLD_ERR_DEVICE_TIMEOUT if the kernel's wait for staged planes ran out
    of its bound)."""
    g = grid_struct(grid)
    ctx.check(ctx.lib.fld_smooth_sweep(ctx.h, ct.byref(g), float(dt), _dptr(D), _fptr(r), _fptr(x_in), _fptr(x_out),
                                       int(first_colour), _stream()))
    return x_out


def diffuse_aniso(ctx: Context, grid: dict, params: dict, dt: float, D_axis, E_old, out=None):
    """Backward-Euler diffusion with a diagonal-tensor D (one CUDA tensor per axis)."""
    keep = []
    g, p = grid_struct(grid), params_struct(params, keep, _device_of(ctx))
    for d in D_axis:
        _dptr(d)
    arr = (ct.c_void_p * len(D_axis))(*[d.data_ptr() for d in D_axis])
    E_new = torch.empty_like(E_old) if out is None else out
    info = Info()
    ctx.check(ctx.lib.fld_diffuse_aniso(ctx.h, ct.byref(g), ct.byref(p), float(dt), ct.cast(arr, ct.c_void_p),
                                        _dptr(E_old), _dptr(E_new), ct.byref(info), _stream()))
    torch.cuda.current_stream().synchronize()
    return E_new, outcome(ctx, info)


def exchange(ctx: Context, params: dict, dt: float, rho, eps, E, kappa=None) -> dict:
    """Point-implicit exchange (Sect. 3.3), in place on eps and E (CUDA tensors)."""
    keep = []
    p = params_struct(params, keep, _device_of(ctx))
    info = Info()
    ctx.check(ctx.lib.fld_exchange(ctx.h, E.numel(), ct.byref(p), float(dt), _dptr(rho), _dptr(kappa), _dptr(eps),
                                   _dptr(E), ct.byref(info), _stream()))
    return info.as_dict()


def opacity(ctx: Context, params: dict, rho, eps, out=None):
    """kappa per cell from rho and eps (CUDA float64 tensors) with the opacity model of params
    (the table's logarithms in double-float with precision "mixed")."""
    keep = []
    p = params_struct(params, keep, _device_of(ctx))
    if out is None:
        out = rho.new_empty(rho.shape)
    ctx.check(ctx.lib.fld_opacity(ctx.h, rho.numel(), ct.byref(p), _dptr(rho), _dptr(eps), _dptr(out), _stream()))
    return out


def _host_buffer(a, writable: bool):
    """(pointer, temporary) for a host array: the array's own float64 C-contiguous memory, or a
    contiguous float64 copy (temporary, to be copied back when writable)."""
    if isinstance(a, torch.Tensor):
        if a.is_cuda:
            raise TypeError("mixed CUDA and host arrays")
        if a.dtype == torch.float64 and a.is_contiguous():
            return ct.c_void_p(a.data_ptr()), None
        t = a.to(torch.float64).contiguous()
        return ct.c_void_p(t.data_ptr()), t
    arr = np.asarray(a)
    if arr.dtype == np.float64 and arr.flags.c_contiguous and (arr.flags.writeable or not writable):
        return ct.c_void_p(arr.ctypes.data), None
    tmp = np.ascontiguousarray(arr, dtype=np.float64)
    return ct.c_void_p(tmp.ctypes.data), tmp


def _assign_back(host, tmp):
    if isinstance(host, torch.Tensor):
        host.copy_(tmp.reshape(host.shape))
    else:
        host[...] = np.asarray(tmp).reshape(np.shape(host))


def step(ctx: Context, grid: dict, params: dict, dt: float, rho, eps, E, allow_unconverged: bool = False,
         sync: bool = True):
    """One full update in place on eps and E.  CUDA tensors are updated in place on the device;
    host arrays (numpy, or CPU tensors -- pinned ones let the copies overlap the kernels) go through
    fld_step_host, which copies them in, steps and copies eps and E back into the same buffers.
    On the device the call is asynchronous: with sync (the default) this function synchronises
    torch's current stream and returns the outcome as a dict; without, it returns the Info that the
    library fills in stream order (keep it until the stream is synchronised, then pass it to
    ``outcome``)."""
    host = not (isinstance(E, torch.Tensor) and E.is_cuda)
    keep = []
    g, p = grid_struct(grid), params_struct(params, keep, _device_of(ctx))
    info = Info()
    if host:
        pr, _tr = _host_buffer(rho, False)
        pe, te = _host_buffer(eps, True)
        pE, tE = _host_buffer(E, True)
        st = ctx.lib.fld_step_host(ctx.h, ct.byref(g), ct.byref(p), float(dt), pr, pe, pE, ct.byref(info),
                                   _stream())
        if te is not None:
            _assign_back(eps, te)
        if tE is not None:
            _assign_back(E, tE)
        if st and not (allow_unconverged and st == 4):
            ctx.check(st)
        return info.as_dict()
    ctx.check(ctx.lib.fld_step(ctx.h, ct.byref(g), ct.byref(p), float(dt), _dptr(rho), _dptr(eps), _dptr(E),
                               ct.byref(info), _stream()))
    if not sync:
        return info
    torch.cuda.current_stream().synchronize()
    return outcome(ctx, info, allow_unconverged)


def _copy_back(host, dev: torch.Tensor):
    if isinstance(host, torch.Tensor):
        host.copy_(dev.reshape(host.shape))
    else:
        host[...] = dev.cpu().numpy().reshape(host.shape)


def step_batched(ctx: Context, grids: list, params: list, dts, rhos: list, epss: list, Es: list) -> list:
    """fld_step on many independent grids (CUDA tensors, updated in place)."""
    n = len(grids)
    keep = []
    G = (Grid * n)(*[grid_struct(g) for g in grids])
    Pp = (Params * n)(*[params_struct(p, keep, _device_of(ctx)) for p in params])
    DT = (ct.c_double * n)(*[float(d) for d in dts])
    R = (ct.c_void_p * n)(*[r.data_ptr() for r in rhos])
    EP = (ct.c_void_p * n)(*[e.data_ptr() for e in epss])
    EE = (ct.c_void_p * n)(*[e.data_ptr() for e in Es])
    for t in list(rhos) + list(epss) + list(Es):
        _dptr(t)
    infos = (Info * n)()
    ctx.check(ctx.lib.fld_step_batched(ctx.h, n, G, Pp, DT, R, EP, EE, infos, _stream()))
    return [i.as_dict() for i in infos]


def columns_step(ctx: Context, r_faces, geometry: str, bc: tuple, v_lo, v_hi, params: dict, dt, rho, eps, E) -> dict:
    """Full update of many 1-D radial columns: rho, eps, E of shape (ncol, ncell) updated in place
    (CUDA tensors) or copied through the device (host arrays)."""
    host = not (isinstance(E, torch.Tensor) and E.is_cuda)
    if host:
        he, hE = eps, E
        rho, eps, E = to_device(rho, ctx), to_device(eps, ctx), to_device(E, ctx)
    ncol, ncell = E.shape
    keep = []
    rf = to_device(r_faces, ctx)
    vl = None if v_lo is None else to_device(v_lo, ctx)
    vh = None if v_hi is None else to_device(v_hi, ctx)
    dtt = to_device(np.broadcast_to(np.asarray(dt, dtype=np.float64), (ncol,)).copy() if not isinstance(dt, torch.Tensor) else dt, ctx)
    keep += [rf, vl, vh, dtt]
    p = params_struct(params, keep, _device_of(ctx))
    info = Info()
    ctx.check(ctx.lib.fld_columns_step(ctx.h, ncol, ncell, _dptr(rf), GEOMETRY[geometry], BC[bc[0]], BC[bc[1]],
                                       _dptr(vl), _dptr(vh), ct.byref(p), _dptr(dtt), _dptr(rho), _dptr(eps),
                                       _dptr(E), ct.byref(info), _stream()))
    if host:
        _copy_back(he, eps)
        _copy_back(hE, E)
    return info.as_dict()


def columns_diffuse(ctx: Context, r_faces, geometry: str, bc: tuple, v_lo, v_hi, params: dict, dt, D, E_old):
    """Tridiagonal diffusion stage of many columns with a given cell D.  Returns E_new."""
    ncol, ncell = E_old.shape
    keep = []
    rf = to_device(r_faces, ctx)
    vl = None if v_lo is None else to_device(v_lo, ctx)
    vh = None if v_hi is None else to_device(v_hi, ctx)
    dtt = to_device(np.broadcast_to(np.asarray(dt, dtype=np.float64), (ncol,)).copy() if not isinstance(dt, torch.Tensor) else dt, ctx)
    keep += [rf, vl, vh, dtt]
    p = params_struct(params, keep, _device_of(ctx))
    E_new = torch.empty_like(E_old)
    ctx.check(ctx.lib.fld_columns_diffuse(ctx.h, ncol, ncell, _dptr(rf), GEOMETRY[geometry], BC[bc[0]], BC[bc[1]],
                                          _dptr(vl), _dptr(vh), ct.byref(p), _dptr(dtt), _dptr(D), _dptr(E_old),
                                          _dptr(E_new), _stream()))
    torch.cuda.current_stream().synchronize()
    return E_new


class TraceEntry(ct.Structure):
    _fields_ = [("name", ct.c_char * 32), ("launches", ct.c_int), ("total_ms", ct.c_double)]


def trace_enable(ctx: Context, on: bool = True, major_only: bool = False):
    """Start (clearing the record) or stop per-kernel launch timing with CUDA events; major_only
    skips the coarse-level and bookkeeping kernels."""
    ctx.lib.fld_trace_enable.argtypes = [P, ct.c_int]
    ctx.check(ctx.lib.fld_trace_enable(ctx.h, (2 if major_only else 1) if on else 0))


def trace_report(ctx: Context) -> dict:
    """{kernel name: (launches, total device ms)} since the last trace_enable(True)."""
    ctx.lib.fld_trace_report.argtypes = [P, P, ct.c_int, ct.POINTER(ct.c_int)]
    buf = (TraceEntry * 256)()
    n = ct.c_int()
    ctx.check(ctx.lib.fld_trace_report(ctx.h, buf, 256, ct.byref(n)))
    return {buf[i].name.decode(): (buf[i].launches, buf[i].total_ms) for i in range(n.value)}


STATIC_MAX_CELLS = 2048


def columns_step_static(r_faces, geometry: str, bc: tuple, v_lo, v_hi, params: dict, dt, rho, eps, E,
                        device: int = 0) -> dict:
    """fld_columns_step_static: the column update without a context and without any device
    allocation inside the library (its scratch is a static device array).  All array arguments
    must already be contiguous float64 CUDA tensors; eps and E ([ncol][ncell]) are updated in
    place.  The caller owns every buffer, including the per-column dt and boundary values."""
    lib = load()
    lib.fld_columns_step_static.argtypes = [ct.c_int, ct.c_int, P, ct.c_int, ct.c_int, ct.c_int, P, P, P, P, P, P,
                                            P, P, P]
    lib.fld_columns_step_static.restype = ct.c_int
    ncol, ncell = E.shape
    keep = []
    p = params_struct(params, keep, torch.device("cuda", device))
    info = Info()
    st = lib.fld_columns_step_static(ncol, ncell, _dptr(r_faces), GEOMETRY[geometry], BC[bc[0]], BC[bc[1]],
                                     _dptr(v_lo), _dptr(v_hi), ct.byref(p), _dptr(dt), _dptr(rho), _dptr(eps),
                                     _dptr(E), ct.byref(info), _stream())
    if st:
        raise FldError(st, "fld_columns_step_static failed" +
                       (f" (ncell {ncell} > {STATIC_MAX_CELLS})" if ncell > STATIC_MAX_CELLS else ""))
    return info.as_dict()


def _dev_ptr_array(tensors):
    """A host array of device pointers (None -> NULL)."""
    if tensors is None:
        return None, None
    arr = (ct.c_void_p * len(tensors))(*[t.data_ptr() for t in tensors])
    return ct.cast(arr, ct.c_void_p), arr


def radiation_terms(ctx: Context, grid: dict, params: dict, E, rho, eps, v=None) -> dict:
    """Explicit radiation terms (Sect. 2.1-2.2, 3.2) of the state: F, f_r (ndim components each),
    work, fedd (Eddington factor), P (xx, yy, zz, xy, xz, yz) and tiring (P : grad v).  v: list of
    ndim velocity tensors or None.  Returns CUDA tensors shaped like E."""
    keep = []
    g, p = grid_struct(grid), params_struct(params, keep, _device_of(ctx))
    nd = int(grid["ndim"])
    out = {"F": [torch.empty_like(E) for _ in range(nd)], "fr": [torch.empty_like(E) for _ in range(nd)],
           "work": torch.empty_like(E), "fedd": torch.empty_like(E), "P": [torch.empty_like(E) for _ in range(6)],
           "tiring": torch.empty_like(E)}
    if v is not None:
        for c in v:
            _dptr(c)
    pv, kv = _dev_ptr_array(v)
    pF, kF = _dev_ptr_array(out["F"])
    pr, kr = _dev_ptr_array(out["fr"])
    pP, kP = _dev_ptr_array(out["P"])
    ctx.check(ctx.lib.fld_radiation_terms(ctx.h, ct.byref(g), ct.byref(p), _dptr(E), _dptr(rho), _dptr(eps), pv, pF,
                                          pr, _dptr(out["work"]), _dptr(out["fedd"]), pP, _dptr(out["tiring"]), 1,
                                          _stream()))
    return out


def photon_tiring_step(ctx: Context, grid: dict, params: dict, dt: float, rho, eps, v, E) -> None:
    """E <- E - dt P : grad v in place (the explicit radiation-energy source, Sect. 3.1-3.2)."""
    keep = []
    g, p = grid_struct(grid), params_struct(params, keep, _device_of(ctx))
    for c in v:
        _dptr(c)
    pv, kv = _dev_ptr_array(v)
    ctx.check(ctx.lib.fld_photon_tiring_step(ctx.h, ct.byref(g), ct.byref(p), float(dt), _dptr(rho), _dptr(eps), pv,
                                             _dptr(E), _stream()))


def pseudo_planar_source(ctx: Context, grid: dict, params: dict, x0: float, E, rho, eps, v=None):
    """Pseudo-planar geometric source of E (Appendix A) on a grid whose x axis stands for the
    radius: -2 (E v_x + F_x) / x + 2 v_x P_xx / x, x = x0 + (i + 1/2) dx_x.  v: list of ndim
    velocity tensors or None.  Returns a CUDA tensor shaped like E."""
    keep = []
    g, p = grid_struct(grid), params_struct(params, keep, _device_of(ctx))
    if v is not None:
        for c in v:
            _dptr(c)
    pv, kv = _dev_ptr_array(v)
    S = torch.empty_like(E)
    ctx.check(ctx.lib.fld_pseudo_planar_source(ctx.h, ct.byref(g), ct.byref(p), float(x0), _dptr(E), _dptr(rho),
                                               _dptr(eps), pv, _dptr(S), 1, _stream()))
    return S


def pseudo_planar_step(ctx: Context, grid: dict, params: dict, dt: float, x0: float, rho, eps, v, E) -> None:
    """E <- E + dt S in place, S the pseudo-planar source of the state on entry (Appendix A)."""
    keep = []
    g, p = grid_struct(grid), params_struct(params, keep, _device_of(ctx))
    if v is not None:
        for c in v:
            _dptr(c)
    pv, kv = _dev_ptr_array(v)
    ctx.check(ctx.lib.fld_pseudo_planar_step(ctx.h, ct.byref(g), ct.byref(p), float(dt), float(x0), _dptr(rho),
                                             _dptr(eps), pv, _dptr(E), _stream()))
