"""Pins for the oracle parts that the conservation, symmetry and
exact-solution pins leave open, each shown to catch a plausible mistake
planted in a separately compiled copy of the oracle (ORC_PLANT in
swe_oracle.c; no GPU).

  * Roe property of the forward Riemann solver (Sec. 6, the Roe solver for
    the shallow water equations).  Over a flat bottom the f-waves must be
    the eigen-decomposition of the jump in Q on the Roe matrix's
    eigenvectors, Z^p = s^p alpha^p r^p with dQ = sum alpha^p r^p, and
    sum Z^p must be the jump in the physical flux.  This holds only when
    uhat and vhat are the sqrt(h)-weighted averages and chat^2 = g hbar_avg,
    so it fixes the tangential (shear) wave and its vhat weighting, which
    every earlier pin left open.
  * Tangential momentum.  For data uniform in y with walls in x, the
    x-flux of hv is hu v in conservation form, so sum hv stays constant.
  * Time autonomy of the adjoint (Sec. 3.2: adjoint solutions for a later
    target time are translates in time).  An adjoint solved for t_f - Delta,
    Delta a whole number of snapshot intervals, holds the same snapshots as
    the one for t_f, each recorded Delta earlier, bit for bit.  This fixes
    the step count N = ceil(t_f s_max / cfl) and dt = t_f / N.
  * Snapshot times.  Adjoint pulses stored at tau_k sit at x0 +- c (t_f -
    tau_k) on a flat bottom (the relation q^(x, tau) = q~(x, t_f - tau) of
    Sec. 4 and the wave speed sqrt(g hbar)), which fixes the tau recorded
    with each snapshot.
"""
import numpy as np
import pytest

import oracle as O

G = 9.81


# ------------------------------------------------------------ Roe property
def roe_property_error(n=300, seed=31):
    """Largest relative violation over random wet edge states on a flat
    bottom of (i) Z^p = s^p alpha^p r^p and (ii) sum_p Z^p = df."""
    rng = np.random.default_rng(seed)
    worst = 0.0
    for _ in range(n):
        hL, hR = rng.uniform(5.0, 4000.0, 2)
        uL, uR, vL, vR = rng.uniform(-8.0, 8.0, 4)
        B = -4500.0
        w = O.fwd_riemann(G, (hL, hL * uL, hL * vL, B), (hR, hR * uR, hR * vR, B))
        uh, vh, ch, s, Z = w["uhat"], w["vhat"], w["chat"], w["s"], w["Z"]
        # eigenvectors of the Roe matrix, one per column
        R = np.array([[1.0, 0.0, 1.0], [uh - ch, 0.0, uh + ch], [vh, 1.0, vh]])
        dQ = np.array([hR - hL, hR * uR - hL * uL, hR * vR - hL * vL])
        alpha = np.linalg.solve(R, dQ)
        Z_eig = np.array([s[p] * alpha[p] * R[:, p] for p in range(3)])

        def flux(h, u, v):
            return np.array([h * u, h * u * u + 0.5 * G * h * h, h * u * v])

        df = flux(hR, uR, vR) - flux(hL, uL, vL)
        scale = max(np.abs(Z).max(), np.abs(df).max())
        worst = max(worst, np.abs(Z - Z_eig).max() / scale,
                    np.abs(Z.sum(axis=0) - df).max() / scale)
        # the speeds are the Roe matrix's eigenvalues for those vectors
        worst = max(worst, np.abs(s - [uh - ch, uh, uh + ch]).max() / ch)
    return worst


def test_forward_riemann_has_the_roe_property():
    assert roe_property_error() <= 1e-10


def test_roe_property_fails_for_other_averages():
    """Control: the same decomposition at the arithmetic-mean state (a
    state a wrong solver might use) violates the property on these data, so
    the pin above can tell the averages apart."""
    rng = np.random.default_rng(32)
    hL, hR = 300.0, 2500.0
    uL, uR, vL, vR = 3.0, -5.0, 6.0, -2.0
    dQ = np.array([hR - hL, hR * uR - hL * uL, hR * vR - hL * vL])
    uh, vh = 0.5 * (uL + uR), 0.5 * (vL + vR)
    ch = np.sqrt(G * 0.5 * (hL + hR))
    R = np.array([[1.0, 0.0, 1.0], [uh - ch, 0.0, uh + ch], [vh, 1.0, vh]])
    s = np.array([uh - ch, uh, uh + ch])
    A_dQ = R @ (s * np.linalg.solve(R, dQ))
    df = (np.array([hR * uR, hR * uR * uR + 0.5 * G * hR * hR, hR * uR * vR])
          - np.array([hL * uL, hL * uL * uL + 0.5 * G * hL * hL, hL * uL * vL]))
    assert np.abs(A_dQ - df).max() > 1e-3 * np.abs(df).max()
    del rng


# ---------------------------------------------------- tangential momentum
def tangential_momentum_drift(order, steps=1000, seed=33):
    """Relative change of sum hv over `steps` steps on data uniform in y,
    walls in x, extrapolation in y, variable bottom, random hu and hv."""
    rng = np.random.default_rng(seed)
    nx, ny, dx = 48, 4, 2000.0
    grid = O.Grid(2, nx, ny, 0.0, 0.0, dx, dx, order=order, bc=(1, 1, 0, 0))
    x = (np.arange(nx) + 0.5) * dx
    Brow = -4000.0 + 3000.0 * np.exp(-((x - 50e3) / 15e3) ** 2)
    eta = 0.5 * np.exp(-((x - 30e3) / 8e3) ** 2)
    hu_row = rng.uniform(-300.0, 300.0, nx)
    hv_row = rng.uniform(-300.0, 300.0, nx)
    B = np.tile(Brow, ny)
    h = np.tile(eta - Brow, ny)
    hu, hv = np.tile(hu_row, ny), np.tile(hv_row, ny)
    h2, hu2, hv2, _, k = O.fwd_run(grid, h, hu, hv, B, steps, 1e12)
    assert k == steps
    assert np.abs(hv2 - hv).max() > 1.0   # hv did change locally
    return abs(hv2.sum() - hv.sum()) / np.abs(hv).sum()


@pytest.mark.parametrize("order", [1, 2])
def test_tangential_momentum_is_conserved(order):
    assert tangential_momentum_drift(order) <= 1e-13


# --------------------------------------------------- adjoint time autonomy
def _adjoint_case(nx=200, dx=2000.0):
    x = (np.arange(nx) + 0.5) * dx
    hbar = np.where(x < 0.7 * nx * dx, 4000.0, 300.0)
    grid = O.Grid(1, nx, 1, 0.0, 0.0, dx, 1.0, order=2)
    phi = np.zeros((2, nx))
    phi[0] = np.exp(-((x - 0.8 * nx * dx) / (5 * dx)) ** 2)
    return grid, hbar, phi


def autonomy_mismatch(N=60, every=5, shift=3):
    """Solve the adjoint for t_f = N dt and for t_f - shift * every * dt, with
    dt an exactly representable step just under the CFL limit, so that both
    t_f are exact multiples of it.  Returns a list of violated facts (empty
    when the translate property holds bit for bit)."""
    grid, hbar, phi = _adjoint_case()
    smax = O.adj_smax(grid, hbar)
    dt = np.floor(grid.cfl / smax * 256.0) / 256.0      # dt smax / cfl just below 1
    t_f = N * dt
    delta = shift * every * dt
    snaps, tau, N1, dt1 = O.adj_run(grid, hbar, phi, t_f, every)
    snaps2, tau2, N2, dt2 = O.adj_run(grid, hbar, phi, t_f - delta, every)
    bad = []
    if N1 != N or dt1 != dt:
        bad.append(f"N {N1} dt {dt1!r}: expected N {N}, dt {dt!r}")
    if N2 != N - shift * every or dt2 != dt1:
        bad.append(f"shifted run: N {N2} dt {dt2!r}")
    K2 = snaps2.shape[0]
    if K2 > snaps.shape[0] or not np.array_equal(snaps2, snaps[:K2]):
        bad.append("shifted snapshots differ from the original ones")
    if K2 <= snaps.shape[0] and not np.array_equal(tau2 + delta, tau[:K2]):
        bad.append("shifted snapshot times are not the original ones minus Delta")
    return bad


def test_adjoint_is_autonomous_in_time():
    assert autonomy_mismatch() == []


# ------------------------------------------------------- snapshot times
def snapshot_position_error(every=20):
    """Largest distance, in cells, between the centroid of each adjoint
    pulse half in a stored snapshot and x0 +- c (t_f - tau_k)."""
    nx, L, depth = 1600, 640e3, 4000.0
    grid = O.Grid(1, nx, 1, -L / 2, 0.0, L / nx, 1.0, order=2)
    xc = -L / 2 + (np.arange(nx) + 0.5) * grid.dx
    hbar = np.full(nx, depth)
    c = np.sqrt(G * depth)
    phi = np.zeros((2, nx))
    phi[0] = np.exp(-(xc / 15e3) ** 2)
    t_f = 1200.0
    snaps, tau, N, dt = O.adj_run(grid, hbar, phi, t_f, every)
    worst = 0.0
    for k in range(1, snaps.shape[0]):
        s = t_f - tau[k]
        if c * s < 60e3:       # halves not yet apart
            continue
        e = snaps[k, 0]
        r = xc > 0
        xr = (xc[r] * e[r]).sum() / e[r].sum()
        xl = (xc[~r] * e[~r]).sum() / e[~r].sum()
        worst = max(worst, abs(xr - c * s) / grid.dx, abs(xl + c * s) / grid.dx)
    return worst


def test_snapshot_times_match_the_wave_position():
    assert snapshot_position_error() <= 0.1


# --------------------------------------------------- planted mistakes
@pytest.mark.parametrize("plant,what", [
    (1, "roe"), (2, "roe"), (3, "roe"), (1, "tangential"),
    (4, "autonomy"), (5, "snapshot_times")])
def test_planted_mistake_fails_its_pin(tmp_path, plant, what):
    """Each ORC_PLANT variant of the oracle must fail the pin meant to catch
    it: 1 beta2 with uhat, 2 arithmetic vhat, 3 arithmetic uhat, 4 N one too
    many, 5 tau one snapshot late."""
    with O.planted(plant, str(tmp_path)):
        if what == "roe":
            assert roe_property_error() > 1e-4
        elif what == "tangential":
            assert tangential_momentum_drift(2, steps=300) > 1e-8
        elif what == "autonomy":
            assert autonomy_mismatch() != []
        else:
            assert snapshot_position_error() > 5.0
