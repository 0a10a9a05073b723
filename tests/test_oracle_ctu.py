"""Pins of the oracle's unsplit 2D step with transverse waves (scheme 1).

The paper defers the general theory of its finite volume methods to
LeVeque (2002) (Sec. 6); the unsplit wave-propagation update with transverse
Riemann solves is that book's multidimensional method.  The oracle's version
is pinned here against things other than itself:

- the transverse split against the flux Jacobian, by finite differences of
  the tangential flux, and against numpy's eigen-decomposition of it;
- data constant in y: the step must equal the (pinned) 1D step row by row,
  bit for bit;
- transposition symmetry, mass conservation with walls, the ocean at rest;
- second-order convergence to the exact linear standing wave of a walled
  basin, and stability at Courant number 0.9.  The same runs with the
  transverse terms dropped, halved, doubled or sign-flipped (planted in the
  oracle through tw_scale) must fail these pins.
"""
import numpy as np
import pytest

import oracle as O

G = 9.81


def tangential_flux(q):
    """Flux along the tangential direction, edge frame (h, m_n, m_t)."""
    h, mn, mt = q
    return np.array([mt, mn * mt / h, mt * mt / h + 0.5 * G * h * h])


def fd_jacobian(q, eps=1e-6):
    J = np.zeros((3, 3))
    for k in range(3):
        d = np.zeros(3)
        d[k] = eps * max(1.0, abs(q[k]))
        J[:, k] = (tangential_flux(q + d) - tangential_flux(q - d)) / (2 * d[k])
    return J


@pytest.mark.parametrize("seed", range(6))
def test_transverse_split_against_the_flux_jacobian(seed):
    rng = np.random.default_rng(seed)
    h = 5.0 + 100 * rng.random()
    c = np.sqrt(G * h)
    u, v = rng.uniform(-0.8, 0.8, 2) * c
    if seed == 5:
        v = 1.3 * c   # supersonic across: everything moves in +t
    a = rng.standard_normal(3) * np.array([1.0, c, c])
    bm, bp = O.ctu_tsplit(u, v, c, a)
    J = fd_jacobian(np.array([h, h * u, h * v]))
    scale = np.abs(J @ a).max()
    np.testing.assert_allclose(bm + bp, J @ a, rtol=0, atol=1e-6 * scale)
    lam, R = np.linalg.eig(J)
    lam, R = lam.real, R.real
    beta = np.linalg.solve(R, a)
    want_p = R @ (np.maximum(lam, 0) * beta)
    want_m = R @ (np.minimum(lam, 0) * beta)
    np.testing.assert_allclose(bp, want_p, rtol=0, atol=1e-6 * scale)
    np.testing.assert_allclose(bm, want_m, rtol=0, atol=1e-6 * scale)
    if seed == 5:
        assert np.all(bm == 0.0)


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("bcx", [O.BC_EXTRAP, O.BC_WALL])
def test_data_constant_in_y_reduces_to_the_1d_step(order, bcx):
    rng = np.random.default_rng(10 + order + 2 * bcx)
    nx, ny = 37, 5
    B1 = -100 + 20 * rng.random(nx)
    h1 = -B1 + 0.5 * rng.standard_normal(nx)
    hu1 = 3 * rng.standard_normal(nx)
    g1 = O.Grid(1, nx, 1, dx=1000.0, order=order, bc=(bcx, bcx, 0, 0))
    r1 = O.fwd_step(g1, h1, hu1, None, B1, 5.0)
    g2 = O.Grid(2, nx, ny, dx=1000.0, dy=700.0, order=order,
                bc=(bcx, bcx, O.BC_WALL, O.BC_EXTRAP), scheme=O.SCHEME_CTU)
    rep = lambda a: np.tile(a, ny)
    r2 = O.fwd_step(g2, rep(h1), rep(hu1), np.zeros(nx * ny), rep(B1), 5.0)
    assert np.array_equal(r2[0], rep(r1[0]))
    assert np.array_equal(r2[1], rep(r1[1]))
    assert np.all(r2[2] == 0.0)


def _random_state(rng, nx, ny):
    B = -100 + 20 * rng.random((ny, nx))
    h = -B + 0.5 * rng.standard_normal((ny, nx))
    hu = 3 * rng.standard_normal((ny, nx))
    hv = 3 * rng.standard_normal((ny, nx))
    return B, h, hu, hv


def test_transposition_symmetry():
    rng = np.random.default_rng(3)
    nx, ny = 23, 17
    B, h, hu, hv = _random_state(rng, nx, ny)
    g = O.Grid(2, nx, ny, dx=1000.0, dy=800.0, bc=(0, 1, 1, 0), scheme=O.SCHEME_CTU)
    gt = O.Grid(2, ny, nx, dx=800.0, dy=1000.0, bc=(1, 0, 0, 1), scheme=O.SCHEME_CTU)
    a = O.fwd_step(g, h.ravel(), hu.ravel(), hv.ravel(), B.ravel(), 6.0)
    b = O.fwd_step(gt, h.T.ravel(), hv.T.ravel(), hu.T.ravel(), B.T.ravel(), 6.0)
    # only the order of the final x and y additions differs
    np.testing.assert_allclose(a[0].reshape(ny, nx), b[0].reshape(nx, ny).T, rtol=0, atol=1e-12)
    np.testing.assert_allclose(a[1].reshape(ny, nx), b[2].reshape(nx, ny).T, rtol=0, atol=1e-12)
    np.testing.assert_allclose(a[2].reshape(ny, nx), b[1].reshape(nx, ny).T, rtol=0, atol=1e-12)
    assert np.abs(a[1] - hu.ravel()).max() > 1.0   # the step did something


def test_mass_with_walls_and_the_ocean_at_rest():
    rng = np.random.default_rng(4)
    nx, ny = 23, 17
    B, h, hu, hv = _random_state(rng, nx, ny)
    g = O.Grid(2, nx, ny, dx=1000.0, dy=800.0, bc=(1, 1, 1, 1), scheme=O.SCHEME_CTU)
    m0 = h.sum()
    for _ in range(5):
        h, hu, hv = (a.reshape(ny, nx) for a in
                     O.fwd_step(g, h.ravel(), hu.ravel(), hv.ravel(), B.ravel(), 6.0))
    assert abs(h.sum() - m0) < 1e-12 * m0
    h0 = -B.ravel()
    r = O.fwd_step(g, h0, 0 * h0, 0 * h0, B.ravel(), 6.0)
    assert np.array_equal(r[0], h0) and np.all(r[1] == 0) and np.all(r[2] == 0)


def standing_wave_error(N, tw=1.0, cfl=0.9, scheme=O.SCHEME_CTU, eps=1e-3):
    """Mean |eta - exact| / eps after one period of the (1,1) mode of the
    linearised SWE in a walled square basin (flat bottom, depth 10 m):
    eta = eps cos(kx) cos(ky) cos(wt), w = c k sqrt(2), k = pi / L."""
    L, h0 = 1e5, 10.0
    c = np.sqrt(G * h0)
    k = np.pi / L
    om = c * k * np.sqrt(2)
    dx = L / N
    x = (np.arange(N) + 0.5) * dx
    X, Y = np.meshgrid(x, x)
    eta = eps * np.cos(k * X) * np.cos(k * Y)
    B = -h0 * np.ones_like(X)
    g = O.Grid(2, N, N, dx=dx, dy=dx, order=2, bc=(1, 1, 1, 1), cfl=cfl, scheme=scheme,
               tw_scale=tw)
    T = 2 * np.pi / om
    try:
        h, _, _, _, _ = O.fwd_run(g, (eta + h0).ravel(), 0 * X.ravel(), 0 * X.ravel(),
                                  B.ravel(), 100000, T)
    except FloatingPointError:
        return np.inf
    ex = eps * np.cos(k * X) * np.cos(k * Y) * np.cos(om * T)
    e = np.abs((h - h0).reshape(N, N) - ex).mean() / eps
    return e if np.isfinite(e) else np.inf


@pytest.mark.parametrize("cfl", [0.45, 0.9])
def test_second_order_convergence_to_the_standing_wave(cfl):
    e = [standing_wave_error(N, cfl=cfl) for N in (16, 32, 64)]
    rates = [np.log2(e[i] / e[i + 1]) for i in range(2)]
    assert min(rates) > 1.7, (e, rates)
    assert e[-1] < 1e-3


@pytest.mark.parametrize("tw", [0.0, -1.0, 0.5, 2.0])
def test_planted_transverse_mistakes_fail_the_pins(tw):
    # a dropped, sign-flipped, halved or doubled transverse term is first
    # order at best at Courant number 0.45 and unstable or first order at 0.9
    for cfl in (0.45, 0.9):
        e = [standing_wave_error(N, tw=tw, cfl=cfl) for N in (16, 32, 64)]
        if all(np.isfinite(e)) and e[-1] < 1.0:
            assert np.log2(e[1] / e[2]) < 1.3, (tw, cfl, e)
            assert e[-1] > 2e-3, (tw, cfl, e)
