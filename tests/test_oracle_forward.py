"""Pins of the oracle's forward shallow-water step against facts fixed by the
paper and by the mathematics (no GPU).

  * ocean at rest stays at rest bit-exactly (well-balanced source, Eq. swe_1d)
  * mass is conserved on closed domains (conservation form of Eq. swe_1d/swe)
  * small waves travel at sqrt(g hbar) (Sec. 1 / Sec. 3 linear wave speed)
  * small waves match the d'Alembert solution of the linearisation
    (Eq. swe_1d_linearized) with first order (order 1) and better than
    first order (order 2, limited corrections) convergence
  * the 1D wet dam break converges to the exact Riemann solution (Stoker)
  * 2D reduces to 1D for y-uniform and for x-uniform data, bit for bit; the
    x -> -x mirror holds to roundoff
  * the split order-2 scheme is stable at cfl 0.75 (noise does not grow)
"""
import numpy as np
import pytest

import oracle as O

G = 9.81


def flat_1d(nx, L, depth, bc=(0, 0, 0, 0), order=2):
    g = O.Grid(1, nx, 1, -L / 2, 0.0, L / nx, 1.0, order=order, bc=bc)
    xc = g.x_lo + (np.arange(nx) + 0.5) * g.dx
    B = np.full(nx, -depth)
    return g, xc, B


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 1, 1, 1), (1, 0, 0, 1)])
def test_lake_at_rest_bit_exact(order, bc):
    rng = np.random.default_rng(11)
    nx, ny = 24, 17
    g = O.Grid(2, nx, ny, 0.0, 0.0, 1000.0, 1300.0, order=order, bc=bc)
    B = -rng.uniform(50.0, 4000.0, nx * ny)
    h = -B
    hu = np.zeros_like(h)
    hv = np.zeros_like(h)
    h2, hu2, hv2, t, k = O.fwd_run(g, h, hu, hv, B, 1000, 1e12)
    assert k == 1000
    assert np.array_equal(h2, h) and np.all(hu2 == 0) and np.all(hv2 == 0)


@pytest.mark.parametrize("order", [1, 2])
def test_mass_conservation_walls(order):
    rng = np.random.default_rng(12)
    nx, ny = 30, 22
    g = O.Grid(2, nx, ny, 0.0, 0.0, 1000.0, 1000.0, order=order, bc=(1, 1, 1, 1))
    xc = (np.arange(nx) + 0.5) * 1000.0
    yc = (np.arange(ny) + 0.5) * 1000.0
    X, Y = np.meshgrid(xc, yc)
    # smooth random bathymetry between ~200 m and 4000 m
    B = -4000.0 + np.zeros_like(X)
    for _ in range(6):
        cx, cy = rng.uniform(0, 30e3), rng.uniform(0, 22e3)
        B += rng.uniform(500, 1900) * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (4e3) ** 2)
    B = np.minimum(B, -200.0).ravel()
    eta = 2.0 * np.exp(-((X - 12e3) ** 2 + (Y - 9e3) ** 2) / (4e3) ** 2).ravel()
    h = eta - B
    hu = rng.uniform(-3, 3, h.size)
    hv = rng.uniform(-3, 3, h.size)
    m0 = h.sum()
    h2, hu2, hv2, t, k = O.fwd_run(g, h, hu, hv, B, 1000, 1e12)
    assert k == 1000
    assert abs(h2.sum() - m0) / m0 <= 1e-13
    assert np.abs(h2 - h).max() > 1e-3  # the state did evolve


def test_mass_conservation_detects_open_boundary():
    """Control: with extrapolation the same run does exchange mass."""
    nx = 60
    g, xc, B = flat_1d(nx, 60e3, 100.0, bc=(0, 0, 0, 0))
    h = -B + 1.0 * np.exp(-(xc / 5e3) ** 2)
    h2, hu2, _, _, _ = O.fwd_run(g, h, np.zeros(nx), None, B, 400, 1e12)
    assert abs(h2.sum() - h.sum()) / h.sum() > 1e-6


def _centroid(x, f):
    return (x * f).sum() / f.sum()


@pytest.mark.parametrize("order", [1, 2])
def test_linear_wave_speed_forward(order):
    """Each half of a small hump travels at sqrt(g hbar): the centroid of the
    right-going pulse sits at c t (within dx/10), the left one at -c t."""
    nx, L, depth = 2000, 800e3, 4000.0
    g, xc, B = flat_1d(nx, L, depth, order=order)
    eta0 = 1e-3 * np.exp(-(xc / 20e3) ** 2)
    h, hu, _, t, k = O.fwd_run(g, -B + eta0, np.zeros(nx), None, B, 100000, 1500.0)
    assert abs(t - 1500.0) < 1e-9
    eta = h + B
    c = np.sqrt(G * depth)
    right = xc > 0
    xr = _centroid(xc[right], eta[right])
    xl = _centroid(xc[~right], eta[~right])
    assert abs(xr - c * t) < 0.1 * g.dx, (xr, c * t)
    assert abs(xl + c * t) < 0.1 * g.dx, (xl, -c * t)
    # each half carries half the mass, and momentum = c * eta in it
    assert abs(eta[right].sum() - 0.5 * eta0.sum()) < 1e-3 * eta0.sum()
    assert abs(hu[right].sum() - c * eta[right].sum()) < 1e-2 * c * eta[right].sum()


def _dalembert_error(nx, order):
    L, depth = 400e3, 4000.0
    g, xc, B = flat_1d(nx, L, depth, order=order)
    f = lambda x: 1e-3 * np.exp(-(x / 25e3) ** 2)
    T = 500.0  # pulses travel ~99 km, well inside the 400 km domain
    h, hu, _, t, _ = O.fwd_run(g, -B + f(xc), np.zeros(nx), None, B, 10 ** 6, T)
    c = np.sqrt(G * depth)
    # cell averages of the exact solution by 5-point Gauss quadrature
    gp = np.array([-0.9061798459, -0.5384693101, 0.0, 0.5384693101, 0.9061798459])
    gw = np.array([0.2369268851, 0.4786286705, 0.5688888889, 0.4786286705, 0.2369268851])
    ex = np.zeros(nx)
    for p, w in zip(gp, gw):
        x = xc + 0.5 * g.dx * p
        ex += 0.5 * w * 0.5 * (f(x - c * t) + f(x + c * t))
    return np.abs((h + B) - ex).sum() * g.dx


def test_smooth_convergence_order1_and_order2():
    e1 = [_dalembert_error(n, 1) for n in (200, 400)]
    e2 = [_dalembert_error(n, 2) for n in (200, 400)]
    p1 = np.log2(e1[0] / e1[1])
    p2 = np.log2(e2[0] / e2[1])
    assert 0.7 < p1 < 1.3, p1
    assert p2 > 1.5, p2
    assert e2[1] < 0.2 * e1[1]


def stoker_exact(x, t, hl, hr):
    """Exact solution of the wet dam break (rarefaction + shock)."""
    cl = np.sqrt(G * hl)

    def fres(hm):
        um_r = 2.0 * (cl - np.sqrt(G * hm))
        um_s = (hm - hr) * np.sqrt(0.5 * G * (1.0 / hm + 1.0 / hr))
        return um_r - um_s
    a, b = hr, hl
    for _ in range(200):
        m = 0.5 * (a + b)
        if fres(a) * fres(m) <= 0:
            b = m
        else:
            a = m
    hm = 0.5 * (a + b)
    um = 2.0 * (cl - np.sqrt(G * hm))
    s = hm * um / (hm - hr)
    xi = x / t
    h = np.empty_like(x)
    u = np.empty_like(x)
    cm = np.sqrt(G * hm)
    for k, z in enumerate(xi):
        if z <= -cl:
            h[k], u[k] = hl, 0.0
        elif z <= um - cm:
            c = (2.0 * cl - z) / 3.0
            h[k], u[k] = c * c / G, (2.0 * cl + 2.0 * z) / 3.0
        elif z < s:
            h[k], u[k] = hm, um
        else:
            h[k], u[k] = hr, 0.0
    return h, u


def _dam_break_l1(nx, order=2, t_end=0.1):
    g = O.Grid(1, nx, 1, -1.0, 0.0, 2.0 / nx, 1.0, order=order)
    xc = -1.0 + (np.arange(nx) + 0.5) * g.dx
    B = np.zeros(nx)
    h0 = np.where(xc < 0.0, 2.0, 1.0)
    h, hu, _, t, _ = O.fwd_run(g, h0, np.zeros(nx), None, B, 10 ** 6, t_end)
    he, ue = stoker_exact(xc, t, 2.0, 1.0)
    return np.abs(h - he).sum() * g.dx, np.abs(hu - he * ue).sum() * g.dx


def test_dam_break_exact_solution():
    e = {n: _dam_break_l1(n) for n in (500, 1000, 2000)}
    assert e[2000][0] < 2e-3 and e[2000][1] < 6e-3, e[2000]
    ph = np.log2(e[500][0] / e[2000][0]) / 2.0
    pm = np.log2(e[500][1] / e[2000][1]) / 2.0
    assert ph >= 0.5 and pm >= 0.5, (ph, pm)


def test_2d_reduces_to_1d_for_y_uniform_data():
    nx, ny = 80, 5
    rng = np.random.default_rng(3)
    B1 = -rng.uniform(200.0, 4000.0, nx)
    eta1 = 0.5 * np.exp(-((np.arange(nx) - 30.0) / 6.0) ** 2)
    hu1 = rng.uniform(-2, 2, nx)
    g1 = O.Grid(1, nx, 1, 0.0, 0.0, 2000.0, 1.0, order=2, bc=(1, 0, 0, 0))
    g2 = O.Grid(2, nx, ny, 0.0, 0.0, 2000.0, 1500.0, order=2, bc=(1, 0, 0, 0))
    dt = 2.0
    h1, u1 = eta1 - B1, hu1.copy()
    h2, u2, v2 = np.tile(h1, ny), np.tile(u1, ny), np.zeros(nx * ny)
    B2 = np.tile(B1, ny)
    for _ in range(50):
        h1, u1, _ = O.fwd_step(g1, h1, u1, None, B1, dt)
        h2, u2, v2 = O.fwd_step(g2, h2, u2, v2, B2, dt)
    for j in range(ny):
        assert np.array_equal(h2[j * nx:(j + 1) * nx], h1)
        assert np.array_equal(u2[j * nx:(j + 1) * nx], u1)
    assert np.all(v2 == 0)


def test_y_sweep_reduces_to_1d_and_mirror():
    """x-uniform data with hu = 0: the x-sweep changes nothing and the y-sweep
    is the 1D solver along y, bit for bit.  The x -> -x mirror holds to
    roundoff."""
    nx, ny = 5, 80
    rng = np.random.default_rng(3)
    B1 = -rng.uniform(200.0, 4000.0, ny)
    eta1 = 0.5 * np.exp(-((np.arange(ny) - 30.0) / 6.0) ** 2)
    hv1 = rng.uniform(-2, 2, ny)
    g1 = O.Grid(1, ny, 1, 0.0, 0.0, 1500.0, 1.0, order=2, bc=(1, 0, 0, 0))
    g2 = O.Grid(2, nx, ny, 0.0, 0.0, 2000.0, 1500.0, order=2, bc=(0, 0, 1, 0))
    h1, v1 = eta1 - B1, hv1.copy()
    h2 = np.repeat(h1, nx)
    v2 = np.repeat(v1, nx)
    u2 = np.zeros(nx * ny)
    B2 = np.repeat(B1, nx)
    for _ in range(50):
        h1, v1, _ = O.fwd_step(g1, h1, v1, None, B1, 2.0)
        h2, u2, v2 = O.fwd_step(g2, h2, u2, v2, B2, 2.0)
    for i in range(nx):
        assert np.array_equal(h2[i::nx], h1)
        assert np.array_equal(v2[i::nx], v1)
    assert np.all(u2 == 0)
    # mirror x -> -x: h even, hu odd
    nx, ny = 23, 31
    B = -rng.uniform(100.0, 4000.0, (ny, nx))
    eta = rng.uniform(-1, 1, (ny, nx))
    hu = rng.uniform(-5, 5, (ny, nx))
    hv = rng.uniform(-5, 5, (ny, nx))
    ga = O.Grid(2, nx, ny, 0.0, 0.0, 1000.0, 1000.0, order=2, bc=(1, 0, 0, 1))
    gm = O.Grid(2, nx, ny, 0.0, 0.0, 1000.0, 1000.0, order=2, bc=(0, 1, 0, 1))
    a = ((eta - B).ravel(), hu.ravel(), hv.ravel())
    c = ((eta - B)[:, ::-1].ravel(), -hu[:, ::-1].ravel(), hv[:, ::-1].ravel())
    for _ in range(20):
        a = O.fwd_step(ga, *a, B.ravel(), 3.0)
        c = O.fwd_step(gm, *c, B[:, ::-1].ravel(), 3.0)
    scale = np.abs(a[0]).max()
    assert np.abs(a[0].reshape(ny, nx)[:, ::-1] - c[0].reshape(ny, nx)).max() <= 1e-12 * scale
    assert np.abs(a[1].reshape(ny, nx)[:, ::-1] + c[1].reshape(ny, nx)).max() <= 1e-9


def test_split_scheme_is_stable_at_cfl_075():
    """Dimensional splitting keeps the order-2 scheme stable at cfl 0.75:
    grid-scale noise of 1e-8 m on a flat 4000 m basin with a smooth 5 cm wave
    stays bounded over 3000 steps, and a 1e-9 perturbation does not grow.
    (Without splitting or transverse corrections, the unsplit second-order
    update lacks the cross-derivative term and this noise grows by orders of
    magnitude.)"""
    rng = np.random.default_rng(0)
    n = 64
    g = O.Grid(2, n, n, 0, 0, 1000., 1000., order=2, cfl=0.75, bc=(1, 1, 1, 1))
    B = np.full(n * n, -4000.0)
    x = (np.arange(n) + 0.5) * 1000.
    X, Y = np.meshgrid(x, x)
    eta = 0.05 * np.exp(-((X - 20e3) ** 2 + (Y - 30e3) ** 2) / (6e3) ** 2).ravel()
    eta = eta + 1e-8 * rng.standard_normal(n * n)
    z = np.zeros(n * n)
    h2, _, _, _, _ = O.fwd_run(g, eta - B, z, z, B, 3000, 1e12)
    e2 = eta + 1e-9 * rng.standard_normal(n * n)
    h3, _, _, _, _ = O.fwd_run(g, e2 - B, z, z, B, 3000, 1e12)
    assert np.abs(h2 + B).max() < 0.05
    assert np.abs(h2 - h3).max() < 1e-8


def test_cfl_number_closed_form():
    g = O.Grid(2, 3, 2, 0.0, 0.0, 1000.0, 500.0)
    h = np.array([100.0, 400.0, 900.0, 100.0, 100.0, 100.0])
    hu = np.array([100.0, -400.0, 0.0, 0.0, 0.0, 0.0])
    hv = np.array([0.0, 800.0, 0.0, 0.0, 0.0, 0.0])
    s = [max((abs(hu[k] / h[k]) + np.sqrt(G * h[k])) / 1000.0,
             (abs(hv[k] / h[k]) + np.sqrt(G * h[k])) / 500.0) for k in range(6)]
    assert O.fwd_smax(g, h, hu, hv) == max(s)
