"""FP64 CPU oracle for the adjoint-guided shallow-water path (ctypes binding).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the bench's
CPU-baseline leg are the only callers.  The product library never imports,
links or executes anything in this directory, and this directory shares no
source with the CUDA library.

Every function follows the paper's method step by step (see swe_oracle.c for
the passage each routine follows).  Parity status of each function and the
pins that fix it are listed in the test modules `tests/test_oracle_*.py`.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "swe_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

BC_EXTRAP, BC_WALL = 0, 1
FLAG_INTERP, FLAG_BRACKET = 0, 1
SCHEME_SPLIT, SCHEME_CTU = 0, 1   # 2D forward step: split, unsplit with transverse waves


def build(force: bool = False, out: str = _LIB, plant: int = 0) -> str:
    """Compile the oracle with gcc (FP64, no contraction, OpenMP).  plant > 0
    compiles one of the deliberately wrong variants listed at ORC_PLANT in
    swe_oracle.c (used only by tests showing that a pin catches it)."""
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(_SRC)):
        return out
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-shared", "-fPIC", f"-DORC_PLANT={int(plant)}",
           "-o", out + ".tmp", _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(out + ".tmp", out)
    return out


@contextlib.contextmanager
def planted(plant: int, workdir: str):
    """Run the block against the oracle compiled with mistake `plant`
    (ORC_PLANT in swe_oracle.c), built into workdir."""
    global _lib
    path = os.path.join(workdir, f"liboracle_plant{int(plant)}.so")
    build(force=True, out=path, plant=plant)
    saved = _load()
    _lib = _bind(ctypes.CDLL(path))
    try:
        yield
    finally:
        _lib = saved


class _Grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("x_lo", ctypes.c_double), ("y_lo", ctypes.c_double),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("order", ctypes.c_int), ("bc", ctypes.c_int * 4),
                ("g", ctypes.c_double), ("cfl", ctypes.c_double),
                ("dry_tol", ctypes.c_double), ("lin_nu", ctypes.c_double * 2),
                ("scheme", ctypes.c_int), ("tw_scale", ctypes.c_double),
                ("wetdry", ctypes.c_int)]


@dataclass
class Grid:
    ndim: int
    nx: int
    ny: int
    x_lo: float = 0.0
    y_lo: float = 0.0
    dx: float = 1.0
    dy: float = 1.0
    order: int = 2
    bc: tuple = (BC_EXTRAP,) * 4
    g: float = 9.81
    cfl: float = 0.75
    dry_tol: float = 1e-3
    scheme: int = SCHEME_SPLIT
    tw_scale: float = 1.0   # transverse terms; tests set 0 / -1 to plant a mistake
    wetdry: int = 0         # split step: shore solver at dry and transonic edges

    @property
    def n(self):
        return self.nx * self.ny

    def c(self):
        s = _Grid()
        s.ndim, s.nx, s.ny = self.ndim, self.nx, self.ny
        s.x_lo, s.y_lo, s.dx, s.dy = self.x_lo, self.y_lo, self.dx, self.dy
        s.order = self.order
        for k in range(4):
            s.bc[k] = int(self.bc[k])
        s.g, s.cfl, s.dry_tol = self.g, self.cfl, self.dry_tol
        s.scheme, s.tw_scale = int(self.scheme), float(self.tw_scale)
        s.wetdry = int(self.wetdry)
        return s

    @classmethod
    def from_spec(cls, spec, **kw):
        return cls(spec.ndim, spec.nx, spec.ny, spec.x_lo, spec.y_lo,
                   spec.dx, spec.dy, **kw)


_lib = None
_D = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _bind(ctypes.CDLL(_LIB))
    return _lib


def _bind(lib):
    G = ctypes.POINTER(_Grid)
    lib.orc_fwd_riemann.argtypes = [ctypes.c_double] * 9 + [_D]
    lib.orc_fwd_riemann.restype = None
    lib.orc_fwd_step.argtypes = [G, _D, _D, _D, _D, ctypes.c_double]
    lib.orc_fwd_step.restype = ctypes.c_int
    lib.orc_fwd_step_flux.argtypes = [G, _D, _D, _D, _D, ctypes.c_double, _D, _D, _D, _D]
    lib.orc_fwd_step_flux.restype = ctypes.c_int
    lib.orc_fwd_step_ctu.argtypes = [G, _D, _D, _D, _D, ctypes.c_double]
    lib.orc_fwd_step_ctu.restype = ctypes.c_int
    lib.orc_ctu_tsplit.argtypes = [ctypes.c_double] * 3 + [_D, _D, _D]
    lib.orc_ctu_tsplit.restype = None
    lib.orc_fwd_smax.argtypes = [G, _D, _D, _D]
    lib.orc_fwd_smax.restype = ctypes.c_double
    lib.orc_fwd_run.argtypes = [G, _D, _D, _D, _D, ctypes.c_long,
                                ctypes.c_double, _D]
    lib.orc_fwd_run.restype = ctypes.c_long
    lib.orc_lin_step.argtypes = [G, _D, _D, _D, _D, ctypes.c_double]
    lib.orc_lin_step.restype = ctypes.c_int
    lib.orc_adj_step.argtypes = [G, _D, _D, _D, _D, ctypes.c_double]
    lib.orc_adj_step.restype = ctypes.c_int
    lib.orc_adj_smax.argtypes = [G, _D]
    lib.orc_adj_smax.restype = ctypes.c_double
    lib.orc_adj_run.argtypes = [G, _D, _D, ctypes.c_double, ctypes.c_int,
                                ctypes.c_long, _D, _D,
                                ctypes.POINTER(ctypes.c_long), _D]
    lib.orc_adj_run.restype = ctypes.c_long
    lib.orc_flag.argtypes = [G, _D, _D, _D, _D, ctypes.c_double, G, _D, _D,
                             _D, ctypes.c_long, ctypes.c_double,
                             ctypes.c_double, ctypes.c_double, ctypes.c_int,
                             ctypes.POINTER(ctypes.c_uint8), _D]
    lib.orc_flag.restype = ctypes.c_long
    lib.orc_flag_surface.argtypes = [G, _D, _D, ctypes.c_double,
                                     ctypes.POINTER(ctypes.c_uint8)]
    lib.orc_flag_surface.restype = ctypes.c_long
    lib.orc_gauge.argtypes = [G, _D, _D, ctypes.c_long, _D, _D]
    lib.orc_gauge.restype = None
    lib.orc_num_threads.restype = ctypes.c_int
    lib.orc_set_threads.argtypes = [ctypes.c_int]
    return lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n: int):
    _load().orc_set_threads(int(n))


def num_threads() -> int:
    return int(_load().orc_num_threads())


# ---------------------------------------------------------------- forward
def fwd_step(grid: Grid, h, hu, hv, B, dt):
    """One forward step (in place on copies; returns new h, hu, hv)."""
    h, hu, B = _f64(h).copy(), _f64(hu).copy(), _f64(B)
    hv = None if hv is None else _f64(hv).copy()
    g = grid.c()
    rc = _load().orc_fwd_step(ctypes.byref(g), _p(h), _p(hu), _p(hv), _p(B), dt)
    if rc:
        raise FloatingPointError(f"oracle forward step unstable ({rc})")
    return h, hu, hv


def fwd_riemann(g, left, right):
    """One forward Riemann solve (test-only view).  left/right = (h, normal
    momentum, tangential momentum, B).  Returns dict(s [3], Z [3, 3] (wave p,
    component m), uhat, vhat, chat)."""
    out = np.zeros(15)
    _load().orc_fwd_riemann(float(g), *[float(x) for x in left],
                            *[float(x) for x in right], _p(out))
    return dict(s=out[0:3].copy(), Z=out[3:12].reshape(3, 3).copy(),
                uhat=out[12], vhat=out[13], chat=out[14])


def fwd_step_flux(grid: Grid, h, hu, hv, B, dt):
    """One 2D split forward step that also returns the mass fluxes per cell:
    (h, hu, hv, phi) with phi[0..3] = x low, x high, y low, y high edge flux
    as the cell's update uses them (dh = -nu (phi_hi - phi_lo) per sweep)."""
    h, hu, hv, B = _f64(h).copy(), _f64(hu).copy(), _f64(hv).copy(), _f64(B)
    phi = np.zeros((4, h.size))
    g = grid.c()
    rc = _load().orc_fwd_step_flux(ctypes.byref(g), _p(h), _p(hu), _p(hv), _p(B), dt,
                                   *[phi[k].ctypes.data_as(_D) for k in range(4)])
    if rc:
        raise FloatingPointError(f"oracle forward step failed ({rc})")
    return h, hu, hv, phi


def ctu_tsplit(uhat, vhat, chat, a):
    """Transverse split of a fluctuation a (edge frame) -> (bm, bp)."""
    a = _f64(a).copy()
    bm, bp = np.zeros(3), np.zeros(3)
    _load().orc_ctu_tsplit(float(uhat), float(vhat), float(chat), _p(a), _p(bm), _p(bp))
    return bm, bp


def fwd_smax(grid: Grid, h, hu, hv):
    hv = np.zeros_like(_f64(h)) if hv is None else _f64(hv)
    g = grid.c()
    return _load().orc_fwd_smax(ctypes.byref(g), _p(_f64(h)), _p(_f64(hu)), _p(hv))


def fwd_run(grid: Grid, h, hu, hv, B, max_steps, t_end, t=0.0):
    """CFL-limited steps up to t_end; returns (h, hu, hv, t, steps)."""
    h, hu, B = _f64(h).copy(), _f64(hu).copy(), _f64(B)
    hv = np.zeros_like(h) if hv is None else _f64(hv).copy()
    tt = ctypes.c_double(t)
    g = grid.c()
    k = _load().orc_fwd_run(ctypes.byref(g), _p(h), _p(hu), _p(hv), _p(B),
                            int(max_steps), float(t_end), ctypes.byref(tt))
    if k < 0:
        raise FloatingPointError(f"oracle forward run unstable ({k})")
    return h, hu, hv, tt.value, int(k)


# ----------------------------------------------------------------- linear
def lin_step(grid: Grid, eta, mu, gam, hbar, dt):
    eta, mu = _f64(eta).copy(), _f64(mu).copy()
    gam = None if gam is None else _f64(gam).copy()
    g = grid.c()
    _load().orc_lin_step(ctypes.byref(g), _p(eta), _p(mu), _p(gam), _p(_f64(hbar)), dt)
    return eta, mu, gam


# ---------------------------------------------------------------- adjoint
def adj_step(grid: Grid, eta, mu, gam, hbar, dt):
    eta, mu = _f64(eta).copy(), _f64(mu).copy()
    gam = None if gam is None else _f64(gam).copy()
    g = grid.c()
    _load().orc_adj_step(ctypes.byref(g), _p(eta), _p(mu), _p(gam), _p(_f64(hbar)), dt)
    return eta, mu, gam


def adj_smax(grid: Grid, hbar):
    g = grid.c()
    return _load().orc_adj_smax(ctypes.byref(g), _p(_f64(hbar)))


def adj_run(grid: Grid, hbar, phi, t_f, every, max_snaps=None):
    """Returns (snaps [K, ncomp, n], tau [K], n_steps, dt)."""
    nc = grid.ndim + 1
    phi = _f64(phi).reshape(nc, grid.n)
    if max_snaps is None:
        smax = adj_smax(grid, hbar)
        N = max(1, int(np.ceil(t_f * smax / grid.cfl)))
        max_snaps = N // every + 3
    snaps = np.zeros((max_snaps, nc, grid.n))
    tau = np.zeros(max_snaps)
    ns = ctypes.c_long(0)
    dt = ctypes.c_double(0.0)
    g = grid.c()
    k = _load().orc_adj_run(ctypes.byref(g), _p(_f64(hbar)), _p(phi), float(t_f),
                            int(every), int(max_snaps), _p(snaps), _p(tau),
                            ctypes.byref(ns), ctypes.byref(dt))
    if k < 0:
        raise RuntimeError(f"oracle adjoint run failed ({k})")
    return snaps[:k].copy(), tau[:k].copy(), int(ns.value), float(dt.value)


# ------------------------------------------------------------------- flag
def flag(fgrid: Grid, h, hu, hv, B, t, agrid: Grid, hbar_adj, snaps, tau,
         t_s, t_f, tol, mode=FLAG_INTERP):
    """Returns (flags uint8 [n], m float64 [n], count)."""
    n = fgrid.n
    snaps = _f64(snaps)
    K = snaps.shape[0]
    flags = np.zeros(n, dtype=np.uint8)
    m = np.zeros(n)
    hv = np.zeros(n) if hv is None else _f64(hv)
    fg, ag = fgrid.c(), agrid.c()
    cnt = _load().orc_flag(ctypes.byref(fg), _p(_f64(h)), _p(_f64(hu)), _p(hv),
                           _p(_f64(B)), float(t), ctypes.byref(ag),
                           _p(_f64(hbar_adj)), _p(snaps), _p(_f64(tau)), int(K),
                           float(t_s), float(t_f), float(tol), int(mode),
                           flags.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                           _p(m))
    return flags, m, int(cnt)


def flag_surface(grid: Grid, h, B, tol):
    """Surface flags |eta| > tol (uint8 [n]) and their count."""
    flags = np.zeros(grid.n, dtype=np.uint8)
    g = grid.c()
    c = _load().orc_flag_surface(ctypes.byref(g), _p(_f64(h)), _p(_f64(B)), float(tol),
                                 flags.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return flags, int(c)


def gauge(grid: Grid, h, B, xy):
    xy = _f64(xy).reshape(-1, 2)
    out = np.zeros(xy.shape[0])
    g = grid.c()
    _load().orc_gauge(ctypes.byref(g), _p(_f64(h)), _p(_f64(B)), xy.shape[0],
                      _p(xy), _p(out))
    return out
