"""Seeded synthetic inputs for the adjoint-guided shallow-water path.

This module holds only input generation: grid geometry, bathymetry, initial
surface displacement, the adjoint's functional data phi, gauge positions and
patch/request layouts.  It contains none of the method's arithmetic (no
Riemann solve, no update, no inner product), so both the CUDA path and the
FP64 oracle can consume its arrays without sharing any of the method.

The paper's workload (a Pacific tsunami over ETOPO1 and Crescent City DEMs,
Sec. 6) needs datasets that are not available; these generators stand in for
it with the paper's scales: a 4000 m deep basin, a shallow continental shelf
(Sec. 3 example: 4000 m ocean, 200 m shelf), decimetre to metre surface waves
and hours-long runs.  Every random draw comes from
``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Gravitational constant used throughout (the paper leaves its value open).
G = 9.81


@dataclass(frozen=True)
class GridSpec:
    """Uniform Cartesian grid, cell-centred, row-major with x fastest."""
    ndim: int
    nx: int
    ny: int
    x_lo: float
    y_lo: float
    dx: float
    dy: float

    @property
    def n(self) -> int:
        return self.nx * self.ny

    def centres(self):
        xc = self.x_lo + (np.arange(self.nx) + 0.5) * self.dx
        yc = self.y_lo + (np.arange(self.ny) + 0.5) * self.dy
        return xc, yc


@dataclass
class Scenario:
    """A forward scenario plus its adjoint target (all arrays FP64, row-major)."""
    grid: GridSpec
    B: np.ndarray            # bottom elevation, negative offshore
    eta0: np.ndarray         # initial surface elevation eta = h + B
    hu0: np.ndarray
    hv0: np.ndarray
    adj_grid: GridSpec
    B_adj: np.ndarray
    phi: np.ndarray          # (ncomp, n_adj): adjoint data at t_f
    t_f: float
    t_s: float
    tol: float
    gauges: np.ndarray       # (ngauge, 2) x, y
    meta: dict = field(default_factory=dict)


# --------------------------------------------------------------------------
# Config 1: 1D ocean with a step shelf
# --------------------------------------------------------------------------
def config1(nx: int = 2000) -> Scenario:
    """1D grid on [-400 km, 400 km]; 4000 m ocean stepping to a 200 m shelf at
    x = 300 km; Gaussian hump 0.5 m exp(-(x/20 km)^2) at rest; adjoint data a
    Gaussian of 10 km width centred at x = 350 km; t_f = 3 h."""
    L = 800e3
    g = GridSpec(1, nx, 1, -400e3, 0.0, L / nx, 1.0)
    xc, _ = g.centres()
    B = np.where(xc < 300e3, -4000.0, -200.0)
    eta0 = 0.5 * np.exp(-(xc / 20e3) ** 2)
    hu0 = np.zeros(nx)
    hv0 = np.zeros(nx)
    phi = np.zeros((2, nx))
    phi[0] = np.exp(-((xc - 350e3) / 10e3) ** 2)
    gauges = np.array([[150e3, 0.0], [340e3, 0.0]])
    return Scenario(g, B, eta0, hu0, hv0, g, B.copy(), phi, t_f=10800.0,
                    t_s=10800.0, tol=1e-3, gauges=gauges,
                    meta={"snap_every": 10})


# --------------------------------------------------------------------------
# Paper Sec. 3 example: 1D, walls, 200 m shelf on 0-50 km, 0.4 m hump at 125 km
# --------------------------------------------------------------------------
def paper_1d_example(nx: int = 800) -> Scenario:
    """Sec. 3: domain 0-400 km, depth 200 m on 0-50 km and 4000 m beyond,
    reflecting walls, a 0.4 m stationary hump at 125 km, target interval
    10-25 km (indicator functional), t_f = 4200 s, t_s = 3800 s."""
    L = 400e3
    g = GridSpec(1, nx, 1, 0.0, 0.0, L / nx, 1.0)
    xc, _ = g.centres()
    B = np.where(xc < 50e3, -200.0, -4000.0)
    eta0 = 0.4 * np.exp(-((xc - 125e3) / 10e3) ** 2)
    phi = np.zeros((2, nx))
    phi[0] = ((xc > 10e3) & (xc < 25e3)).astype(np.float64)
    return Scenario(g, B, eta0, np.zeros(nx), np.zeros(nx), g, B.copy(), phi,
                    t_f=4200.0, t_s=3800.0, tol=0.1,
                    gauges=np.array([[17.5e3, 0.0]]), meta={"snap_every": 5})


# --------------------------------------------------------------------------
# 2D basin with shelf and seamounts (configs 2-5)
# --------------------------------------------------------------------------
def basin_bathymetry(grid: GridSpec, L: float, seed: int, n_seamounts: int,
                     shelf_frac: float = 1740.0 / 2048.0,
                     basin_frac: float = 1600.0 / 2048.0,
                     seamount_params=None) -> np.ndarray:
    """4000 m basin, tanh shelf rising to 100 m depth on the +x side, Gaussian
    seamounts (height 500-2000 m, width 10-50 km) over the basin, depth
    clamped to at least 50 m so no cell is dry."""
    xc, yc = grid.centres()
    X, Y = np.meshgrid(xc, yc)
    if seamount_params is None:
        seamount_params = seamounts(L, seed, n_seamounts, basin_frac)
    B = -4000.0 + 3900.0 * 0.5 * (1.0 + np.tanh((X - shelf_frac * L) / 30e3))
    for (cx, cy, a, w) in seamount_params:
        B = B + a * np.exp(-(((X - cx) ** 2 + (Y - cy) ** 2) / (w * w)))
    return np.minimum(B, -50.0).ravel()


def seamounts(L: float, seed: int, n: int, basin_frac: float):
    rng = np.random.default_rng(seed)
    cx = rng.uniform(0.0, basin_frac * L, n)
    cy = rng.uniform(0.0, L, n)
    a = rng.uniform(500.0, 2000.0, n)
    w = rng.uniform(10e3, 50e3, n)
    return list(zip(cx, cy, a, w))


def gaussian_field(grid: GridSpec, cx: float, cy: float, amp: float,
                   width: float) -> np.ndarray:
    xc, yc = grid.centres()
    X, Y = np.meshgrid(xc, yc)
    return (amp * np.exp(-(((X - cx) ** 2 + (Y - cy) ** 2) / (width * width)))).ravel()


def disc_indicator(grid: GridSpec, cx: float, cy: float, radius: float) -> np.ndarray:
    """1 at cell centres within `radius` of (cx, cy), else 0: an indicator
    target region, as the paper's examples use for the adjoint data."""
    xc, yc = grid.centres()
    X, Y = np.meshgrid(xc, yc)
    return (((X - cx) ** 2 + (Y - cy) ** 2) <= radius * radius).astype(np.float64).ravel()


def source_point(rng, target, L, rmin=300e3, rmax=700e3, basin_frac=1600.0 / 2048.0):
    """A seeded basin point between rmin and rmax from the target."""
    for _ in range(10000):
        r = rng.uniform(rmin, rmax)
        a = rng.uniform(0.0, 2.0 * np.pi)
        x = target[0] + r * np.cos(a)
        y = target[1] + r * np.sin(a)
        if 0.05 * L < x < basin_frac * L and 0.05 * L < y < 0.95 * L:
            return x, y
    raise RuntimeError("no source point found")


def config2(n: int = 2048, L: float = 2048e3, seed: int = 1605,
            n_seamounts: int = 20, amp: float = 1.0, src_width: float = 30e3,
            adj_n: int | None = None, n_gauges: int = 2,
            shelf_frac: float = 1740.0 / 2048.0,
            src_r: tuple = (300e3, 700e3)) -> Scenario:
    """2D n x n grid on [0, L]^2 (1 km cells at n = 2048).  Gaussian source of
    amplitude `amp` and width 30 km at a seeded basin point 300-700 km from the
    target; adjoint data a 10 km Gaussian in eta at the shelf break; t_s / t_f
    set to the paper's ratio 3.5 h / 11 h."""
    rng = np.random.default_rng(seed)
    grid = GridSpec(2, n, n, 0.0, 0.0, L / n, L / n)
    sm = seamounts(L, seed + 1, n_seamounts, 1600.0 / 2048.0)
    B = basin_bathymetry(grid, L, seed, n_seamounts, shelf_frac=shelf_frac,
                         seamount_params=sm)
    # target at the shelf break: waves from 300-700 km away reach it within
    # the time window [t_s, t_f]
    target = (shelf_frac * L, 0.5 * L)
    sx, sy = source_point(rng, target, L, rmin=src_r[0], rmax=src_r[1])
    eta0 = gaussian_field(grid, sx, sy, amp, src_width)
    eta0 = np.where(eta0 < 1e-12, 0.0, eta0)
    if adj_n is None:
        adj_n = n
    adj_grid = GridSpec(2, adj_n, adj_n, 0.0, 0.0, L / adj_n, L / adj_n)
    B_adj = basin_bathymetry(adj_grid, L, seed, n_seamounts,
                             shelf_frac=shelf_frac, seamount_params=sm)
    phi = np.zeros((3, adj_grid.n))
    phi[0] = gaussian_field(adj_grid, target[0], target[1], 1.0, 10e3)
    # dt0 ~ 0.75 / (sqrt(g 4000) / dx) is the first CFL step in the basin
    # (per-direction Courant number of the split step); t_f spans 2000 such
    # steps, so the forward run to t_f is ~2000 steps.
    dt0 = 0.75 / (np.sqrt(G * 4000.0) / grid.dx)
    t_f = 2000.0 * dt0
    gx = np.concatenate([rng.uniform(0.1 * L, 0.7 * L, n_gauges // 2),
                         target[0] - rng.uniform(5e3, 100e3, n_gauges - n_gauges // 2)])
    gy = np.concatenate([rng.uniform(0.1 * L, 0.9 * L, n_gauges // 2),
                         target[1] + rng.uniform(-100e3, 100e3, n_gauges - n_gauges // 2)])
    gauges = np.stack([gx, gy], axis=1)
    return Scenario(grid, B, eta0, np.zeros(grid.n), np.zeros(grid.n),
                    adj_grid, B_adj, phi, t_f=t_f, t_s=0.32 * t_f, tol=1e-3,
                    gauges=gauges,
                    meta={"seed": seed, "source": (sx, sy), "target": target,
                          "snap_every": 20, "flag_every": 10, "steps": 2000})


def config4(n: int = 4096, adj_n: int = 1024, steps: int = 5000) -> Scenario:
    """Precision study: n^2 on [0, n km]^2, 40 seamounts, shelf at 0.85 L,
    source amplitude 0.2 m, adjoint on a coarser adj_n^2 grid, 16 gauges,
    t_f spanning `steps` basin CFL steps.  The source sits at the distance a
    4000 m-deep wave covers in 0.55-0.75 t_f, so the first arrival at the
    target falls inside the window [t_s, t_f] and the flag sets are not
    empty."""
    L = n * 1e3
    dt0 = 0.75 / (np.sqrt(G * 4000.0) / (L / n))
    t_f = steps * dt0 * 1.001
    c = np.sqrt(G * 4000.0)
    sc = config2(n=n, L=L, seed=4096, n_seamounts=40, amp=0.2, adj_n=adj_n,
                 n_gauges=16, shelf_frac=0.85,
                 src_r=(0.55 * c * t_f, 0.75 * c * t_f))
    sc.t_f = t_f
    sc.t_s = 0.32 * t_f
    sc.meta["steps"] = steps
    return sc


def small_2d(nx: int, ny: int, seed: int = 7, L: float | None = None,
             amp: float = 0.5) -> Scenario:
    """A small 2D basin used by the parity tests: same generator, rectangular."""
    if L is None:
        L = 1000e3
    dx = L / nx
    grid = GridSpec(2, nx, ny, 0.0, 0.0, dx, dx)
    rng = np.random.default_rng(seed)
    Ly = ny * dx
    sm = [(rng.uniform(0, 0.7 * L), rng.uniform(0, Ly), rng.uniform(500, 2000),
           rng.uniform(3 * dx, 10 * dx)) for _ in range(6)]
    xc, yc = grid.centres()
    X, Y = np.meshgrid(xc, yc)
    B = -4000.0 + 3900.0 * 0.5 * (1.0 + np.tanh((X - 0.85 * L) / (4 * dx)))
    for (cx, cy, a, w) in sm:
        B = B + a * np.exp(-(((X - cx) ** 2 + (Y - cy) ** 2) / (w * w)))
    B = np.minimum(B, -50.0).ravel()
    sx, sy = rng.uniform(0.2 * L, 0.5 * L), rng.uniform(0.3 * Ly, 0.7 * Ly)
    eta0 = gaussian_field(grid, sx, sy, amp, 6 * dx)
    hu0 = rng.uniform(-1.0, 1.0, grid.n) * 5.0
    hv0 = rng.uniform(-1.0, 1.0, grid.n) * 5.0
    target = (0.9 * L, 0.5 * Ly)
    phi = np.zeros((3, grid.n))
    phi[0] = gaussian_field(grid, target[0], target[1], 1.0, 4 * dx)
    t_f = 400.0 * 0.75 / (2.0 * np.sqrt(G * 4000.0) / dx)
    gauges = np.array([[0.3 * L, 0.5 * Ly], [0.88 * L, 0.45 * Ly]])
    return Scenario(grid, B, eta0, hu0, hv0, grid, B.copy(), phi, t_f=t_f,
                    t_s=0.32 * t_f, tol=1e-3, gauges=gauges,
                    meta={"target": target, "snap_every": 5})


# --------------------------------------------------------------------------
# Config 3: uneven patches on three levels
# --------------------------------------------------------------------------
def config3_patches(seed: int = 5320, n_patches: int = 1500, L: float = 2048e3,
                    smin: int = 16, smax: int = 256):
    """1500 patches, level uniform in {1,2,3}, sides uniform in [16, 256],
    cell size 1 km / 4^(level-1), origins uniform inside the domain."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_patches):
        lev = int(rng.integers(1, 4))
        nx = int(rng.integers(smin, smax + 1))
        ny = int(rng.integers(smin, smax + 1))
        d = 1e3 / 4 ** (lev - 1)
        x0 = rng.uniform(0.0, L - nx * d)
        y0 = rng.uniform(0.0, L - ny * d)
        out.append((lev, x0, y0, nx, ny, d))
    return out


# --------------------------------------------------------------------------
# Config 5: request trace for the serving loop
# --------------------------------------------------------------------------
def config5_requests(seed: int = 2026, n: int = 512, rate: float = 20.0,
                     sizes=(512, 1024, 2048, 4096)):
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n))
    out = []
    for i in range(n):
        out.append({"id": i, "arrival": float(arrivals[i]),
                    "n": int(rng.choice(sizes)),
                    "amp": float(rng.uniform(0.1, 2.0)),
                    "width": float(rng.uniform(10e3, 60e3)),
                    "src_u": float(rng.uniform()), "src_v": float(rng.uniform())})
    return out


def patch_fields(patch, L: float = 2048e3, seed: int = 1605, n_seamounts: int = 20,
                 src=(700e3, 1024e3), amp: float = 1.0, width: float = 30e3):
    """Bathymetry and initial surface of one patch (level, x_lo, y_lo, nx, ny,
    dx, dy) sampled from the basin fields of the 2D configurations."""
    lev, x0, y0, nx, ny, dx, dy = patch
    g = GridSpec(2, nx, ny, x0, y0, dx, dy)
    sm = seamounts(L, seed + 1, n_seamounts, 1600.0 / 2048.0)
    B = basin_bathymetry(g, L, seed, n_seamounts, seamount_params=sm)
    eta = gaussian_field(g, src[0], src[1], amp, width)
    return B, eta


# ------------------------------------------------------------- AMR cases
def amr_basin(nc: int, r: int, boxes, dx: float = 10e3, rest: bool = False,
              seed: int | None = None, mean_coarse: bool = False):
    """A walled nc x nc coarse basin (cell dx) with fine patches refined by r.

    boxes: patch interiors in coarse cells, (i0, j0, mx, my); each patch is
    returned with its 2-cell ring.  Bottom and surface are analytic (a
    sinusoidal 80-120 m bottom, a 0.5 m Gaussian hump of width 3 dx at the
    centre, or the ocean at rest), sampled at coarse centres and once on the
    global fine grid, so patches agree wherever they overlap.  seed: uniform
    random momenta in [-5, 5] (r = 1 only, where the levels share cells).
    mean_coarse: the coarse bottom and surface are the means of the fine
    samples over each coarse cell instead (a hierarchy whose covered coarse
    cells already hold the fine means).
    Returns a dict with the coarse fields (B, eta, hu, hv), per patch the
    descriptor (level 1, x_lo, y_lo, nx, ny, dx, dy) and fields (B, eta, hu,
    hv, ring included)."""
    def bottom(x, y):
        return -100.0 - 20.0 * np.sin(x / 7e4) * np.cos(y / 9e4)

    L = nc * dx

    def hump(x, y):
        return 0.5 * np.exp(-((x - 0.5 * L) ** 2 + (y - 0.5 * L) ** 2) / (3 * dx) ** 2)

    xc = (np.arange(nc) + 0.5) * dx
    X, Y = np.meshgrid(xc, xc)
    xf = (np.arange(nc * r) + 0.5) * (dx / r)
    XF, YF = np.meshgrid(xf, xf)
    Bc, BF = bottom(X, Y), bottom(XF, YF)
    ec = np.zeros_like(X) if rest else hump(X, Y)
    EF = np.zeros_like(XF) if rest else hump(XF, YF)
    if mean_coarse:
        Bc = BF.reshape(nc, r, nc, r).mean(axis=(1, 3))
        ec = EF.reshape(nc, r, nc, r).mean(axis=(1, 3))
    uc = np.zeros_like(X)
    UF = np.zeros_like(XF)
    if seed is not None:
        assert r == 1
        uc = np.random.default_rng(seed).uniform(-5.0, 5.0, X.shape)
        UF = uc
    out = {"coarse": {"B": Bc.ravel(), "eta": ec.ravel(), "hu": uc.ravel(), "hv": -uc.ravel()},
           "patches": [], "dx": dx, "nc": nc, "r": r}
    dxf = dx / r
    for (i0, j0, mx, my) in boxes:
        nx, ny = mx * r + 4, my * r + 4
        I0, J0 = i0 * r - 2, j0 * r - 2
        sl = lambda a: a[J0:J0 + ny, I0:I0 + nx].ravel().copy()
        desc = (1, i0 * dx - 2 * dxf, j0 * dx - 2 * dxf, nx, ny, dxf, dxf)
        out["patches"].append({"box": (i0, j0, mx, my), "desc": desc, "B": sl(BF),
                               "eta": sl(EF), "hu": sl(UF), "hv": -sl(UF)})
    return out


def amr_levels_basin(nc: int, levels, dx: float = 10e3, rest: bool = False,
                     seed: int | None = None, mean_coarse: bool = False):
    """The walled basin of amr_basin with nested levels.

    levels: [(r, boxes), ...], level l's boxes (i0, j0, mx, my) in global
    level-(l - 1) cells (the uniform grid of that level's cell size over the
    whole domain).  Every level samples the bottom and surface at its own
    centres, or (mean_coarse) the finest level samples them and every other
    level holds the means of the level below.  seed: uniform random momenta
    in [-5, 5] (all ratios 1).  Returns a dict with the coarse fields (B, eta,
    hu, hv), per level "r" and "patches" (descriptor (l, x_lo, y_lo, nx, ny,
    dx, dy) and fields B, eta, hu, hv, ring included)."""
    def bottom(x, y):
        return -100.0 - 20.0 * np.sin(x / 7e4) * np.cos(y / 9e4)

    L = nc * dx

    def hump(x, y):
        return 0.5 * np.exp(-((x - 0.5 * L) ** 2 + (y - 0.5 * L) ** 2) / (3 * dx) ** 2)

    ratios = [lv[0] for lv in levels]
    F, n, d = [], nc, dx
    for l in range(len(levels) + 1):
        if l > 0:
            n, d = n * ratios[l - 1], d / ratios[l - 1]
        xc = (np.arange(n) + 0.5) * d
        X, Y = np.meshgrid(xc, xc)
        F.append([bottom(X, Y), np.zeros_like(X) if rest else hump(X, Y)])
    if mean_coarse:
        for l in range(len(levels) - 1, -1, -1):
            r = ratios[l]
            m = F[l + 1][0].shape[0] // r
            F[l] = [a.reshape(m, r, m, r).mean(axis=(1, 3)) for a in F[l + 1]]
    U = None
    if seed is not None:
        assert all(r == 1 for r in ratios)
        U = np.random.default_rng(seed).uniform(-5.0, 5.0, (nc, nc))
    uc = np.zeros((nc, nc)) if U is None else U
    out = {"coarse": {"B": F[0][0].ravel(), "eta": F[0][1].ravel(), "hu": uc.ravel(),
                      "hv": -uc.ravel()}, "levels": [], "dx": dx, "nc": nc}
    dp = dx
    for l, (r, boxes) in enumerate(levels, start=1):
        BF, EF = F[l]
        UF = np.zeros_like(BF) if U is None else U
        df = dp / r
        pats = []
        for (i0, j0, mx, my) in boxes:
            nx, ny = mx * r + 4, my * r + 4
            I0, J0 = i0 * r - 2, j0 * r - 2
            sl = lambda a: a[J0:J0 + ny, I0:I0 + nx].ravel().copy()
            desc = (l, i0 * dp - 2 * df, j0 * dp - 2 * df, nx, ny, df, df)
            pats.append({"box": (i0, j0, mx, my), "desc": desc, "B": sl(BF), "eta": sl(EF),
                         "hu": sl(UF), "hv": -sl(UF)})
        out["levels"].append({"r": r, "patches": pats})
        dp = df
    return out


def amr_basin_2048(ratio: int = 4, side: int = 32, tiles: int = 8):
    """The basin of the 2D configurations as a two-level hierarchy: the
    2048^2 coarse grid (1 km cells) and tiles x tiles fine patches of
    side x side coarse cells refined by `ratio`, tiling a square centred on
    the source of the basin fields (700 km, 1024 km), each with its 2-cell
    ring, fields sampled at the fine cell centres.  Returns (B, eta, n, dx,
    descs, fields) with fields[k] = (B, eta) of patch k."""
    n, dx = 2048, 1e3
    B, eta = patch_fields((1, 0.0, 0.0, n, n, dx, dx))
    i0, j0 = 700 - tiles * side // 2, 1024 - tiles * side // 2
    dxf = dx / ratio
    descs = []
    for b in range(tiles):
        for a in range(tiles):
            pi, pj = i0 + a * side, j0 + b * side
            descs.append((1, pi * dx - 2 * dxf, pj * dx - 2 * dxf, side * ratio + 4,
                          side * ratio + 4, dxf, dxf))
    fields = [patch_fields(q) for q in descs]
    return B, eta, n, dx, descs, fields


def amr_basin_2048_nested(ratio: int = 4, side: int = 32, tiles: int = 8, side2: int = 32,
                          tiles2: int = 4):
    """amr_basin_2048 with a second level: tiles2 x tiles2 patches of side2 x
    side2 level-1 cells refined by `ratio` again, tiling a square centred on
    the source inside the level-1 square (level 2 of the patch set).
    Returns (B, eta, n, dx, descs, fields) with the level-1 descriptors
    first, then level 2's."""
    B, eta, n, dx, descs, fields = amr_basin_2048(ratio, side, tiles)
    dx1 = dx / ratio
    dx2 = dx1 / ratio
    # the source (700 km, 1024 km) in level-1 cells
    c1, c2 = int(round(700e3 / dx1)), int(round(1024e3 / dx1))
    i0, j0 = c1 - tiles2 * side2 // 2, c2 - tiles2 * side2 // 2
    d2 = []
    for b in range(tiles2):
        for a in range(tiles2):
            pi, pj = i0 + a * side2, j0 + b * side2
            d2.append((2, pi * dx1 - 2 * dx2, pj * dx1 - 2 * dx2, side2 * ratio + 4,
                       side2 * ratio + 4, dx2, dx2))
    return B, eta, n, dx, descs + d2, fields + [patch_fields(q) for q in d2]

