"""Pins of the oracle's adjoint step (Sec. 3-5) against facts that do not come
from the oracle itself.

  * discrete duality: with walls, one step of the time-reversed adjoint is the
    exact transpose of one step of the linear forward problem
    (Eq. q_equality / reduced2d in discrete form), 1D and 2D
  * hence J_n = sum q^(t_n).q(t_n) dx is constant to roundoff (Eq. J)
  * with limited second-order corrections the drift of J vanishes under
    refinement
  * adjoint waves travel at sqrt(g hbar) along the eigenvectors [c,1],[-c,1]
    of the time-reversed flux (Sec. 3.1)
  * crossing forward and adjoint waves have zero inner product, aligned ones
    do not (Sec. 3.1)
  * wet/dry edges act as walls (Sec. 5): a dry cell never changes and the
    wet side is closed
"""
import numpy as np
import pytest

import oracle as O

G = 9.81


def _matrices(grid, hbar, dt):
    nc = grid.ndim + 1
    n = grid.n
    Mf = np.zeros((nc * n, nc * n))
    Ma = np.zeros((nc * n, nc * n))
    for col in range(nc * n):
        v = np.zeros(nc * n)
        v[col] = 1.0
        parts = [v[k * n:(k + 1) * n] for k in range(nc)]
        gam = parts[2] if nc == 3 else None
        e, m, gg = O.lin_step(grid, parts[0], parts[1], gam, hbar, dt)
        Mf[:, col] = np.concatenate([e, m] + ([gg] if nc == 3 else []))
        e, m, gg = O.adj_step(grid, parts[0], parts[1], gam, hbar, dt)
        Ma[:, col] = np.concatenate([e, m] + ([gg] if nc == 3 else []))
    return Mf, Ma


@pytest.mark.parametrize("dims", [(16, 1, 1), (5, 4, 2)])
def test_adjoint_step_is_transpose_of_linear_step_with_walls(dims):
    nx, ny, ndim = dims
    rng = np.random.default_rng(21)
    hbar = rng.uniform(100.0, 4000.0, nx * ny)
    grid = O.Grid(ndim, nx, ny, 0.0, 0.0, 1000.0, 1200.0, order=1, bc=(1, 1, 1, 1))
    dt = 0.4 * 1000.0 / np.sqrt(G * hbar.max())
    Mf, Ma = _matrices(grid, hbar, dt)
    assert np.abs(Ma - Mf.T).max() <= 1e-13 * np.abs(Mf).max()
    assert np.abs(Mf - np.eye(Mf.shape[0])).max() > 1e-3


def test_transpose_fails_with_open_boundaries():
    """Control: extrapolation leaves boundary terms, so duality must break."""
    rng = np.random.default_rng(22)
    hbar = rng.uniform(100.0, 4000.0, 16)
    grid = O.Grid(1, 16, 1, 0.0, 0.0, 1000.0, 1.0, order=1, bc=(0, 0, 0, 0))
    Mf, Ma = _matrices(grid, hbar, 1.0)
    assert np.abs(Ma - Mf.T).max() > 1e-3 * np.abs(Mf).max()


def _j_series(grid, hbar, q0, phi, dt, nsteps):
    nc = grid.ndim + 1
    n = grid.n
    adj = [tuple(phi[k] for k in range(nc))]
    s = adj[0]
    for _ in range(nsteps):
        s = O.adj_step(grid, s[0], s[1], s[2] if nc == 3 else None, hbar, dt)
        adj.append(s)
    q = tuple(q0[k] for k in range(nc))
    J = []
    for k in range(nsteps + 1):
        qh = adj[nsteps - k]  # q^(t_k) = q~(t_f - t_k)
        J.append(sum(float(np.dot(qh[c], q[c])) for c in range(nc)) * grid.dx * grid.dy)
        if k < nsteps:
            q = O.lin_step(grid, q[0], q[1], q[2] if nc == 3 else None, hbar, dt)
    return np.array(J)


def test_adjoint_identity_J_constant_order1_walls():
    nx, ny = 24, 18
    rng = np.random.default_rng(23)
    grid = O.Grid(2, nx, ny, 0.0, 0.0, 1000.0, 1000.0, order=1, bc=(1, 1, 1, 1))
    hbar = rng.uniform(200.0, 4000.0, nx * ny)
    dt = 0.4 / (2.0 * np.sqrt(G * hbar.max()) / 1000.0)
    q0 = rng.uniform(-1, 1, (3, nx * ny))
    phi = rng.uniform(-1, 1, (3, nx * ny))
    J = _j_series(grid, hbar, q0, phi, dt, 1000)
    assert np.abs(J - J[0]).max() <= 1e-12 * np.abs(q0).max() * np.abs(phi).max() * grid.n * 1e6
    assert np.abs(J - J[0]).max() / abs(J[0]) <= 1e-12 * 10  # J[0] is O(sum)


def test_adjoint_identity_order2_drift_vanishes_under_refinement():
    drifts = []
    for nx in (50, 100, 200):
        L = 200e3
        grid = O.Grid(1, nx, 1, 0.0, 0.0, L / nx, 1.0, order=2, bc=(1, 1, 1, 1))
        xc = (np.arange(nx) + 0.5) * grid.dx
        hbar = 2000.0 + 1500.0 * np.tanh((xc - 100e3) / 20e3)
        dt = 0.5 * grid.dx / np.sqrt(G * hbar.max())
        q0 = np.stack([np.exp(-((xc - 60e3) / 15e3) ** 2), np.zeros(nx)])
        phi = np.stack([np.exp(-((xc - 150e3) / 15e3) ** 2), np.zeros(nx)])
        T = 600.0
        n = int(round(T / dt))
        dt = T / n
        J = _j_series(grid, hbar, q0, phi, dt, n)
        drifts.append(np.abs(J - J[0]).max() / np.abs(J).max())
    assert drifts[2] < drifts[1] < drifts[0], drifts


def test_adjoint_wave_speed_and_eigenvectors():
    nx, L, depth = 2000, 800e3, 4000.0
    grid = O.Grid(1, nx, 1, -L / 2, 0.0, L / nx, 1.0, order=2)
    xc = -L / 2 + (np.arange(nx) + 0.5) * grid.dx
    hbar = np.full(nx, depth)
    c = np.sqrt(G * depth)
    dt = 0.75 * grid.dx / c
    e, m = np.exp(-(xc / 20e3) ** 2), np.zeros(nx)
    nsteps = 800
    for _ in range(nsteps):
        e, m, _ = O.adj_step(grid, e, m, None, hbar, dt)
    t = nsteps * dt
    r = xc > 0
    xr = (xc[r] * e[r]).sum() / e[r].sum()
    xl = (xc[~r] * e[~r]).sum() / e[~r].sum()
    assert abs(xr - c * t) < 0.1 * grid.dx and abs(xl + c * t) < 0.1 * grid.dx
    # right-moving (speed +c) part lies along [-c, 1]: mu~ = -eta~/c
    assert abs(m[r].sum() + e[r].sum() / c) < 1e-2 * e[r].sum() / c
    assert abs(m[~r].sum() - e[~r].sum() / c) < 1e-2 * e[~r].sum() / c


def test_crossing_waves_are_orthogonal_aligned_are_not():
    nx, L, depth = 2000, 400e3, 4000.0
    grid = O.Grid(1, nx, 1, -L / 2, 0.0, L / nx, 1.0, order=2)
    xc = -L / 2 + (np.arange(nx) + 0.5) * grid.dx
    hbar = np.full(nx, depth)
    B = -hbar
    c = np.sqrt(G * depth)
    tstar = 50e3 / c
    nsteps = 500  # dt c / dx = 0.5
    dt = tstar / nsteps
    f = lambda x0: 1e-2 * np.exp(-((xc - x0) / 10e3) ** 2)

    def forward(eta0, mu0):
        h, hu = -B + eta0, mu0
        for _ in range(nsteps):
            h, hu, _ = O.fwd_step(grid, h, hu, None, B, dt)
        return h + B, hu

    def adjoint(e0, m0):
        e, m = e0, m0
        for _ in range(nsteps):
            e, m, _ = O.adj_step(grid, e, m, None, hbar, dt)
        return e, m

    # adjoint left-going in forward time: data along [-c, 1] at x = 50 km
    g0 = np.exp(-((xc - 50e3) / 10e3) ** 2)
    ea, ma = adjoint(-c * g0, g0)
    # forward right-going from -50 km (crosses at 0) vs left-going from 100 km
    e1, m1 = forward(f(-50e3), c * f(-50e3))
    e2, m2 = forward(f(100e3), -c * f(100e3))
    J_cross = np.sum(ea * e1 + ma * m1)
    J_align = np.sum(ea * e2 + ma * m2)
    assert abs(J_align) > 0.5 * 2 * c * np.sum(g0 * f(0.0))
    assert abs(J_cross) <= 1e-3 * abs(J_align)


@pytest.mark.parametrize("order", [1, 2])
def test_dry_cells_act_as_walls(order):
    nx = 80
    grid = O.Grid(1, nx, 1, 0.0, 0.0, 1000.0, 1.0, order=order, bc=(0, 0, 0, 0))
    hbar = np.full(nx, 3000.0)
    hbar[60:] = 0.0  # dry to the right of cell 59
    e = np.exp(-((np.arange(nx) - 50.0) / 3.0) ** 2)
    e[60:] = 0.0
    m = np.zeros(nx)
    tot0 = e[:60].sum()
    dt = 0.5 * 1000.0 / np.sqrt(G * 3000.0)
    for _ in range(30):
        e, m, _ = O.adj_step(grid, e, m, None, hbar, dt)
        assert np.all(e[60:] == 0.0) and np.all(m[60:] == 0.0)
    # the pulse has reflected off the wet/dry edge; the adjoint eta~ is in
    # conservation form, so its sum is unchanged while the open left boundary
    # stays quiet
    assert e[:60].max() > 0.1
    assert abs(e[:60].sum() - tot0) <= 1e-12 * tot0
    assert abs(e[0]) < 1e-12


def test_dry_wall_matches_domain_wall():
    """A wet/dry edge and a domain wall at the same place give the same
    first-order solution."""
    nx = 60
    hb = np.full(nx, 2500.0)
    e0 = np.exp(-((np.arange(nx) - 30.0) / 4.0) ** 2)
    g1 = O.Grid(1, nx, 1, 0.0, 0.0, 1000.0, 1.0, order=1, bc=(1, 1, 0, 0))
    g2 = O.Grid(1, nx + 5, 1, 0.0, 0.0, 1000.0, 1.0, order=1, bc=(1, 0, 0, 0))
    hb2 = np.concatenate([hb, np.zeros(5)])
    a = (e0, np.zeros(nx))
    b = (np.concatenate([e0, np.zeros(5)]), np.zeros(nx + 5))
    dt = 0.5 * 1000.0 / np.sqrt(G * 2500.0)
    for _ in range(80):
        a = O.adj_step(g1, a[0], a[1], None, hb, dt)[:2]
        b = O.adj_step(g2, b[0], b[1], None, hb2, dt)[:2]
    assert np.abs(a[0] - b[0][:nx]).max() <= 1e-14
    assert np.abs(a[1] - b[1][:nx]).max() <= 1e-14
