"""Pins of the oracle's adjoint-weighted flagging (Sec. 4.1, 4.2, 6) and gauge
sampling against brute force and closed forms.

  * INTERP: m equals the maximum of |q^(tau).q| over a dense uniform sampling
    of the window, q^(tau) the piecewise-linear interpolant (brute force)
  * INTERP flags are a subset of BRACKET flags (Eq. ip_timepoint is the more
    conservative rule)
  * t_s = t_f reduces the time-range rule to a single time: INTERP gives
    |q^(t).q|, BRACKET gives Eq. ip_timepoint over the two bracketing snapshots
  * lowering t_s widens the window: flags form a superset
  * t > t_f: empty window, no flags
  * a dry forward cell or a dry adjoint stencil cell gives m = 0 (Sec. 6)
  * bilinear spatial interpolation is exact for fields linear in x and y and
    the identity when the grids coincide (Sec. 4)
  * gauges reproduce bilinear fields exactly and clamp outside the centres
"""
import numpy as np
import pytest

import oracle as O


def _setup(seed=31, nx=12, ny=9, K=9):
    rng = np.random.default_rng(seed)
    fg = O.Grid(2, nx, ny, 0.0, 0.0, 1000.0, 1000.0)
    B = -rng.uniform(100.0, 4000.0, fg.n)
    h = -B + rng.uniform(-1, 1, fg.n)
    hu = rng.uniform(-5, 5, fg.n)
    hv = rng.uniform(-5, 5, fg.n)
    tau = np.sort(rng.uniform(0.0, 1000.0, K))[::-1].copy()
    tau[0], tau[-1] = 1000.0, 0.0
    snaps = rng.uniform(-1, 1, (K, 3, fg.n)) * 1e-3
    hbar = -B
    return fg, B, h, hu, hv, tau, snaps, hbar


def _interp_dot(tau, snaps, q, cell, s):
    """q^(s).q for the piecewise-linear interpolant, by direct evaluation."""
    k = np.searchsorted(-tau, -s, side="right") - 1
    k = min(max(k, 0), len(tau) - 2)
    a = (s - tau[k + 1]) / (tau[k] - tau[k + 1])
    qh = a * snaps[k, :, cell] + (1 - a) * snaps[k + 1, :, cell]
    return float(np.dot(qh, q))


def test_interp_matches_dense_brute_force():
    fg, B, h, hu, hv, tau, snaps, hbar = _setup()
    t, t_s, t_f = 230.0, 400.0, 1000.0
    T = min(t + t_f - t_s, t_f)
    _, m, _ = O.flag(fg, h, hu, hv, B, t, fg, hbar, snaps, tau, t_s, t_f, 0.0,
                     O.FLAG_INTERP)
    ss = np.linspace(t, T, 10001)
    for cell in range(0, fg.n, 7):
        q = np.array([h[cell] + B[cell], hu[cell], hv[cell]])
        brute = max(abs(_interp_dot(tau, snaps, q, cell, s)) for s in ss)
        assert brute <= m[cell] * (1 + 1e-12)
        assert m[cell] - brute <= 1e-3 * m[cell]


def test_interp_subset_of_bracket_and_monotone_in_ts():
    fg, B, h, hu, hv, tau, snaps, hbar = _setup(seed=32)
    args = (fg, h, hu, hv, B, 300.0, fg, hbar, snaps, tau)
    tol = 0.5 * 1e-3 * 2.0
    fi, mi, ci = O.flag(*args, 500.0, 1000.0, tol, O.FLAG_INTERP)
    fb, mb, cb = O.flag(*args, 500.0, 1000.0, tol, O.FLAG_BRACKET)
    assert np.all(mi <= mb * (1 + 1e-15))
    assert np.all(fb[fi == 1] == 1)
    assert 0 < ci <= cb
    prev = None
    for t_s in (900.0, 700.0, 500.0, 200.0, 0.0):
        f, m, c = O.flag(*args, t_s, 1000.0, tol, O.FLAG_INTERP)
        if prev is not None:
            assert np.all(f[prev == 1] == 1)
        prev = f
    assert c == fg.n or c > ci


def test_single_time_reduction():
    fg, B, h, hu, hv, tau, snaps, hbar = _setup(seed=33)
    t = 0.5 * (tau[3] + tau[4])
    _, mi, _ = O.flag(fg, h, hu, hv, B, t, fg, hbar, snaps, tau, 1000.0, 1000.0,
                      0.0, O.FLAG_INTERP)
    _, mb, _ = O.flag(fg, h, hu, hv, B, t, fg, hbar, snaps, tau, 1000.0, 1000.0,
                      0.0, O.FLAG_BRACKET)
    for cell in range(fg.n):
        q = np.array([h[cell] + B[cell], hu[cell], hv[cell]])
        d3 = float(np.dot(snaps[3, :, cell], q))
        d4 = float(np.dot(snaps[4, :, cell], q))
        scale = np.abs(snaps[3:5, :, cell] * q).sum()
        assert abs(mb[cell] - max(abs(d3), abs(d4))) <= 1e-15 * scale
        assert abs(mi[cell] - abs(_interp_dot(tau, snaps, q, cell, t))) <= 1e-15 + 1e-12 * mi[cell]
    # exactly at a snapshot time both modes give that snapshot's |q^.q|
    _, mi, _ = O.flag(fg, h, hu, hv, B, tau[5], fg, hbar, snaps, tau, 1000.0,
                      1000.0, 0.0, O.FLAG_INTERP)
    _, mb, _ = O.flag(fg, h, hu, hv, B, tau[5], fg, hbar, snaps, tau, 1000.0,
                      1000.0, 0.0, O.FLAG_BRACKET)
    for cell in range(fg.n):
        q = np.array([h[cell] + B[cell], hu[cell], hv[cell]])
        d5 = abs(float(np.dot(snaps[5, :, cell], q)))
        scale = np.abs(snaps[5, :, cell] * q).sum()
        assert abs(mi[cell] - d5) <= 1e-15 * scale and mb[cell] == mi[cell]


def test_after_final_time_no_flags():
    fg, B, h, hu, hv, tau, snaps, hbar = _setup(seed=34)
    f, m, c = O.flag(fg, h, hu, hv, B, 1000.5, fg, hbar, snaps, tau, 0.0, 1000.0,
                     0.0, O.FLAG_INTERP)
    assert c == 0 and np.all(m == 0) and np.all(f == 0)


def test_dry_cells_give_zero():
    fg, B, h, hu, hv, tau, snaps, hbar = _setup(seed=35)
    hbar = hbar.copy()
    h = h.copy()
    hbar[17] = 0.0       # adjoint dry
    h[40] = 0.0005       # forward dry (below dry_tol = 1e-3)
    f, m, c = O.flag(fg, h, hu, hv, B, 100.0, fg, hbar, snaps, tau, 0.0, 1000.0,
                     0.0, O.FLAG_INTERP)
    assert m[17] == 0.0 and f[17] == 0
    assert m[40] == 0.0 and f[40] == 0
    assert np.all(m[np.r_[0:17, 18:40, 41:fg.n]] > 0)


def test_bilinear_exact_for_linear_fields_on_coarse_adjoint_grid():
    fg = O.Grid(2, 16, 12, 0.0, 0.0, 1000.0, 1000.0)
    ag = O.Grid(2, 6, 5, 0.0, 0.0, 16000.0 / 6, 12000.0 / 5)
    xa = (np.arange(6) + 0.5) * ag.dx
    ya = (np.arange(5) + 0.5) * ag.dy
    XA, YA = np.meshgrid(xa, ya)
    lin = lambda X, Y, a, b, c: a + b * X * 1e-5 + c * Y * 1e-5
    snaps = np.stack([np.stack([lin(XA, YA, 1, 2, -1).ravel(),
                                lin(XA, YA, -0.5, 1, 3).ravel(),
                                lin(XA, YA, 2, -1, 0.5).ravel()])])
    tau = np.array([500.0])
    B = np.full(fg.n, -1000.0)
    h = np.full(fg.n, 1001.0)  # eta = 1
    hu = np.full(fg.n, 2.0)
    hv = np.full(fg.n, -3.0)
    _, m, _ = O.flag(fg, h, hu, hv, B, 500.0, ag, np.full(ag.n, 100.0), snaps,
                     tau, 500.0, 500.0, 0.0, O.FLAG_INTERP)
    xf = (np.arange(16) + 0.5) * 1000.0
    yf = (np.arange(12) + 0.5) * 1000.0
    XF, YF = np.meshgrid(xf, yf)
    XC = np.clip(XF, xa[0], xa[-1])
    YC = np.clip(YF, ya[0], ya[-1])
    want = np.abs(1.0 * lin(XC, YC, 1, 2, -1) + 2.0 * lin(XC, YC, -0.5, 1, 3)
                  - 3.0 * lin(XC, YC, 2, -1, 0.5)).ravel()
    assert np.abs(m - want).max() <= 1e-13 * want.max()


def test_gauge_bilinear_and_clamp():
    g = O.Grid(2, 7, 5, 100.0, -50.0, 20.0, 30.0)
    xc = 100.0 + (np.arange(7) + 0.5) * 20.0
    yc = -50.0 + (np.arange(5) + 0.5) * 30.0
    X, Y = np.meshgrid(xc, yc)
    f = lambda x, y: 0.3 + 0.01 * x - 0.02 * y + 1e-4 * x * y
    B = np.full(35, -10.0)
    h = (f(X, Y) - B.reshape(5, 7)).ravel()
    xy = np.array([[130.0, -20.0], [181.3, 41.0], [0.0, 0.0], [500.0, 500.0]])
    got = O.gauge(g, h, B, xy)
    xcl = np.clip(xy[:, 0], xc[0], xc[-1])
    ycl = np.clip(xy[:, 1], yc[0], yc[-1])
    assert np.allclose(got, f(xcl, ycl), rtol=0, atol=1e-12)


def test_surface_flags_are_the_disc_of_a_gaussian_hump():
    """|eta| > tol for eta = A exp(-r^2/w^2) is the disc r < w sqrt(ln(A/tol)):
    the flagged cells are exactly the cell centres inside it; a dry cell is
    never flagged, and a trough flags like a crest."""
    n, d = 80, 1000.0
    g = O.Grid(2, n, n, 0.0, 0.0, d, d)
    xc = (np.arange(n) + 0.5) * d
    X, Y = np.meshgrid(xc, xc)
    A, w, tol = 0.5, 12e3, 0.14
    r2 = (X - 37.3e3) ** 2 + (Y - 41.9e3) ** 2
    eta = A * np.exp(-r2 / w ** 2)
    B = np.full(n * n, -3000.0)
    f, c = O.flag_surface(g, eta.ravel() - B, B, tol)
    inside = (r2 < w ** 2 * np.log(A / tol)).ravel()
    assert np.array_equal(f.astype(bool), inside) and c == inside.sum() > 0
    f2, c2 = O.flag_surface(g, -eta.ravel() - B, B, tol)
    assert np.array_equal(f2, f)
    h = eta.ravel() - B
    k = int(np.argmax(inside))
    h[k] = 0.0005
    f3, c3 = O.flag_surface(g, h, B, tol)
    assert f3[k] == 0 and c3 == c - 1
