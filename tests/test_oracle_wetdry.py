"""Pins of the oracle's shore solver (wetdry = 1, oracle/swe_oracle.c): the
forward step at dry cells and transonic edges (Sec. 6: the solver reduces to
Roe away from the shore and handles inundation).

- Ritter's dam break over a dry bed (the exact solution): the L1 error falls
  under refinement, and the depth at the dam tends to 4 h0 / 9;
- the ocean at rest against dry land (a 1D beach, a 2D island) stays exactly
  at rest: the fluxes of the unreconstructed states and the dropped
  reconstruction pressure terms (planted) do not;
- mass between walls is conserved exactly while a wave runs up a beach and
  back (CFL 1/2, the positivity bound of the reconstruction); without the
  shore solver at transonic edges, or with the unreconstructed states
  (planted), depths go negative, the dry reset adds mass and the pin fails;
- depths stay non-negative and dry cells hold no momentum;
- with no dry cell and no transonic edge the step is the Roe step bit for
  bit.
"""
import numpy as np
import pytest

import oracle as O
from paper_1605_05320_gb300 import synth

G = 9.81


def ritter(x, t, h0):
    """Dry-bed dam break at x = 0 (Ritter): depth at time t."""
    c0 = np.sqrt(G * h0)
    return np.where(x < -c0 * t, h0,
                    np.where(x < 2 * c0 * t, (2 * c0 - x / t) ** 2 / (9 * G), 0.0))


def ritter_run(n, T=6.0, h0=1.0, L=100.0):
    g = O.Grid(1, n, 1, -L, 0.0, 2 * L / n, 1.0, order=2, bc=(1, 1, 1, 1), wetdry=1)
    x = -L + (np.arange(n) + 0.5) * 2 * L / n
    h = np.where(x < 0, h0, 0.0)
    h, hu, _, t, k = O.fwd_run(g, h, np.zeros(n), None, np.zeros(n), 100000, T)
    assert t == T
    return x, h, hu


def test_ritter_dam_break_converges_to_the_exact_solution():
    errs, dam = [], []
    for n in (200, 400, 800):
        x, h, hu = ritter_run(n)
        errs.append(np.abs(h - ritter(x, 6.0, 1.0)).sum() * 200.0 / n)
        dam.append(np.interp(0.0, x, h))
        assert h.min() >= 0.0
        assert np.all(hu[h <= 1e-3] == 0.0)
    # measured 0.600, 0.319, 0.196
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.25 and errs[1] / errs[2] > 1.4
    # the dam depth 4 h0 / 9 = 0.444 (measured 0.456, 0.450, 0.447)
    assert abs(dam[2] - 4.0 / 9.0) < 0.015 * (4.0 / 9.0), dam


def beach_1d(n=200):
    L = 1000.0
    g = O.Grid(1, n, 1, 0.0, 0.0, L / n, 1.0, order=2, bc=(1, 1, 1, 1), wetdry=1)
    x = (np.arange(n) + 0.5) * L / n
    B = -1.0 + 2.0 * x / L + 0.3 * np.sin(x / 40)
    return g, B


def island_2d(n=48):
    L = 1000.0
    g = O.Grid(2, n, n, 0.0, 0.0, L / n, L / n, order=2, bc=(1, 1, 1, 1), wetdry=1)
    xc = (np.arange(n) + 0.5) * L / n
    X, Y = np.meshgrid(xc, xc)
    B = (-2.0 + 3.0 * np.exp(-((X - 500) ** 2 + (Y - 450) ** 2) / 150 ** 2) + 0.002 * X).ravel()
    return g, B


def rest_error(case):
    g, B = case()
    h0 = np.maximum(0.0, -B)
    assert (h0 == 0).sum() > 10 and (h0 > 0).sum() > 10
    hv = None if g.ndim == 1 else np.zeros(g.n)
    h, hu, hv, _, k = O.fwd_run(g, h0, np.zeros(g.n), hv, B, 150, 1e9)
    assert k == 150
    err = np.abs(h - h0).max() + np.abs(hu).max()
    if hv is not None:
        err += np.abs(hv).max()
    return err


@pytest.mark.parametrize("case", [beach_1d, island_2d])
def test_ocean_at_rest_against_dry_land_stays_at_rest(case):
    assert rest_error(case) == 0.0


def runup(cfl=0.5, n=48, steps=150):
    """A 0.4 m hump in 2 m of water running up a wavy beach that rises above
    the surface, walls all round."""
    L = 1000.0
    g = O.Grid(2, n, n, 0.0, 0.0, L / n, L / n, order=2, bc=(1, 1, 1, 1), wetdry=1, cfl=cfl)
    xc = (np.arange(n) + 0.5) * L / n
    X, Y = np.meshgrid(xc, xc)
    B = (-2.0 + 3.0 * X / L + 0.2 * np.cos(Y / 90)).ravel()
    eta = (0.4 * np.exp(-((X - 250) ** 2 + (Y - 500) ** 2) / 80 ** 2)).ravel()
    h0 = np.maximum(0.0, eta - B)
    h, hu, hv, _, k = O.fwd_run(g, h0, np.zeros(g.n), np.zeros(g.n), B, steps, 1e9)
    assert k == steps
    return h0, h, hu, hv


def test_mass_is_conserved_while_a_wave_runs_up_a_beach():
    h0, h, hu, hv = runup()
    wet0, wet1 = (h0 > 1e-3).sum(), (h > 1e-3).sum()
    assert wet1 > wet0 + 20           # the shoreline moved (measured 1548 -> 1607 cells)
    assert abs(h.sum() - h0.sum()) <= 1e-13 * h0.sum()
    assert h.min() >= 0.0
    dry = h <= 1e-3
    assert np.all(hu[dry] == 0.0) and np.all(hv[dry] == 0.0)


@pytest.mark.parametrize("plant,pin", [(6, "rest"), (8, "rest"), (6, "mass"), (7, "mass")])
def test_planted_shore_mistakes_fail_their_pins(plant, pin, tmp_path):
    with O.planted(plant, str(tmp_path)):
        if pin == "rest":
            assert rest_error(beach_1d) > 1e-4 and rest_error(island_2d) > 1e-3
        else:
            h0, h, *_ = runup()
            assert abs(h.sum() - h0.sum()) > 1e-8 * h0.sum()   # measured 6.6e-7, 7.0e-6


def test_without_dry_cells_the_step_is_the_roe_step():
    sc = synth.small_2d(60, 44, seed=3)
    h0 = sc.eta0 - sc.B
    out = []
    for wd in (0, 1):
        g = O.Grid.from_spec(sc.grid, bc=(1, 0, 0, 1), wetdry=wd)
        out.append(O.fwd_run(g, h0, sc.hu0, sc.hv0, sc.B, 40, 1e9)[:3])
    for a, b in zip(*out):
        assert np.array_equal(a, b)
