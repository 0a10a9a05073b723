"""Pins of the oracle's two-level AMR glue (oracle/amr.py): ring fills from
siblings and from the coarse level (linear in time, limited-linear in space),
r fine substeps per coarse step, averaging down.

- r = 1: the hierarchy is the single grid, whatever the patches (overlapping,
  adjacent, apart);
- the ocean at rest stays exactly at rest for r = 2 and 4 over a bottom
  sampled separately on each level;
- a patch cut in two (the cut filled from the sibling) gives the patch;
- a field linear in x and y is filled exactly at the ring cells' centres
  (pins the fine cell's offset inside its coarse cell and the slopes); the
  offset taken at the fine cell's corner (planted) misses by half a cell;
- refining a patch brings its region closer to a uniformly fine run than the
  coarse grid alone; piecewise-constant coarse fills, fills frozen at the
  coarse step's start or end, slopes of the wrong sign, or an average over r
  instead of r^2 cells (mistakes planted in subclasses) do not.
- refluxing: with coarse bottoms that are the means of the fine ones, the
  total mass is conserved between walls (without refluxing it drifts); the
  ocean stays at rest; r = 1 stays the single grid to rounding; refluxing
  with a flipped sign or without the 1/r weight of a fine edge (planted)
  does not conserve mass.

The pins of the fills and of the average run with refluxing off: refluxing
changes only the uncovered coarse cells beside a patch, and those pins were
chosen to fix the fill and average rules.
"""
import numpy as np
import pytest

import oracle as O
from oracle.amr import RING, Hierarchy, Patch, fine_grid, minmod

DX = 10e3
H0 = 130.0


def bottom(x, y):
    return -100.0 - 20.0 * np.sin(x / 7e4) * np.cos(y / 9e4)


def hump(x, y, L):
    return 0.5 * np.exp(-((x - 0.5 * L) ** 2 + (y - 0.5 * L) ** 2) / (3 * DX) ** 2)


def fields(n, d):
    x = (np.arange(n) + 0.5) * d
    X, Y = np.meshgrid(x, x)
    return X, Y


def build(nc, r, patches, cls=Hierarchy, rest=False, seed=None, reflux=False,
          mean_bottom=False):
    """Coarse nc^2 basin with walls, fine patches sampled on the global fine
    grid (so patches agree wherever they overlap), a hump at the centre.
    mean_bottom: the coarse bottom and surface are the means of the fine
    ones over each coarse cell (else sampled at the coarse centres)."""
    cg = O.Grid(2, nc, nc, 0.0, 0.0, DX, DX, order=2, bc=(1, 1, 1, 1))
    L = nc * DX
    X, Y = fields(nc, DX)
    Bc = bottom(X, Y).ravel()
    ec = np.zeros(nc * nc) if rest else hump(X, Y, L).ravel()
    XF, YF = fields(nc * r, DX / r)
    BF, EF = bottom(XF, YF), (np.zeros_like(XF) if rest else hump(XF, YF, L))
    if mean_bottom:
        Bc = BF.reshape(nc, r, nc, r).mean(axis=(1, 3)).ravel()
        ec = EF.reshape(nc, r, nc, r).mean(axis=(1, 3)).ravel()
    uc = np.zeros(nc * nc)
    UF = np.zeros_like(XF)
    if seed is not None:
        rng = np.random.default_rng(seed)
        uc = rng.uniform(-5, 5, nc * nc)
        assert r == 1
        UF = uc.reshape(nc, nc)
    Bf, fine = [], []
    for p in patches:
        g = fine_grid(cg, p, r)
        I0, J0 = p.i0 * r - RING, p.j0 * r - RING
        sl = lambda a: a[J0:J0 + g.ny, I0:I0 + g.nx].ravel().copy()
        Bf.append(sl(BF))
        fine.append((sl(EF) - sl(BF), sl(UF), -sl(UF)))
    H = cls(cg, Bc, patches, r, Bf, reflux=reflux)
    H.set_state(ec - Bc, uc, -uc, fine, 0.0)
    return H, cg, Bc, ec, BF, EF, uc


def dt_coarse(cg):
    return 0.6 * cg.cfl * cg.dx / np.sqrt(9.81 * H0)


def test_ratio_one_is_the_single_grid():
    patches = [Patch(5, 6, 6, 5), Patch(9, 8, 5, 7), Patch(14, 3, 4, 4)]
    H, cg, Bc, ec, _, _, uc = build(24, 1, patches, seed=1)
    h, hu, hv = ec - Bc, uc.copy(), -uc
    dt, t = dt_coarse(cg), 0.0
    for _ in range(10):
        assert H.step(t, dt)
        h, hu, hv = O.fwd_step(cg, h, hu, hv, Bc, (t + dt) - t)
        t = t + dt
    for a, b in ((H.h, h), (H.hu, hu), (H.hv, hv)):
        assert np.abs(a - b).max() <= 1e-14 * np.abs(b).max()
    assert H.t_c == H.t_f == t


@pytest.mark.parametrize("r", [2, 4])
def test_ocean_at_rest_stays_at_rest(r):
    H, cg, Bc, *_ = build(16, r, [Patch(4, 4, 5, 6), Patch(7, 8, 4, 4)], rest=True)
    dt, t = dt_coarse(cg), 0.0
    for _ in range(4):
        assert H.step(t, dt)
        t = t + dt
    assert np.all(H.h + Bc == 0.0) and np.all(H.hu == 0) and np.all(H.hv == 0)
    for f, b in zip(H.fine, H.Bf):
        assert np.all(f[0] + b == 0.0) and np.all(f[1] == 0) and np.all(f[2] == 0)


def test_a_patch_cut_in_two_gives_the_patch():
    one, cg, *_ = build(24, 2, [Patch(8, 8, 8, 8)])
    two, *_ = build(24, 2, [Patch(8, 8, 3, 8), Patch(11, 8, 5, 8)])
    dt, t = dt_coarse(cg), 0.0
    for _ in range(6):
        assert one.step(t, dt) and two.step(t, dt)
        t = t + dt
    scale = np.abs(one.h + one.B).max()
    assert np.abs((one.h - two.h)).max() <= 1e-12 * scale
    assert np.abs(one.hu - two.hu).max() <= 1e-12 * np.abs(one.hu).max()
    # the fine cells of the halves equal the whole patch's
    g1 = one.grids[0]
    for k, p in enumerate(two.patches):
        g = two.grids[k]
        for j in range(RING, g.ny - RING):
            row1 = (j * g1.nx) + (p.i0 - 8) * 2
            a = two.fine[k][0][j * g.nx + RING:(j + 1) * g.nx - RING]
            b = one.fine[0][0][row1 + RING:row1 + RING + g.nx - 2 * RING]
            assert np.abs(a - b).max() <= 1e-12 * 130.0


def region_errors(r, steps, cls=Hierarchy, p=Patch(8, 8, 8, 8)):
    """Max |eta - eta_fine| over the patch's coarse cells for the hierarchy
    and for the coarse grid alone; eta_fine is a uniformly fine run averaged
    to coarse cells."""
    nc = 24
    H, cg, Bc, ec, BF, EF, _ = build(nc, r, [p], cls=cls)
    dt, t = dt_coarse(cg), 0.0
    h, hu, hv = ec - Bc, 0 * ec, 0 * ec
    for _ in range(steps):
        assert H.step(t, dt)
        h, hu, hv = O.fwd_step(cg, h, hu, hv, Bc, (t + dt) - t)
        t = t + dt
    fg = O.Grid(2, nc * r, nc * r, 0.0, 0.0, DX / r, DX / r, order=2, bc=(1, 1, 1, 1))
    fh, fu, fv = (EF - BF).ravel(), 0 * EF.ravel(), 0 * EF.ravel()
    for _ in range(steps * r):
        fh, fu, fv = O.fwd_step(fg, fh, fu, fv, BF.ravel(), dt / r)
    ref = (fh + BF.ravel()).reshape(nc, r, nc, r).mean(axis=(1, 3)).ravel()
    m = np.zeros((nc, nc), bool)
    m[p.j0:p.j0 + p.my, p.i0:p.i0 + p.mx] = True
    m = m.ravel()
    return np.abs(H.h + Bc - ref)[m].max(), np.abs(h + Bc - ref)[m].max()


@pytest.mark.parametrize("r,steps,factor", [(2, 4, 0.3), (2, 12, 0.7), (4, 4, 0.5)])
def test_refinement_moves_the_patch_towards_the_fine_solution(r, steps, factor):
    amr, coarse = region_errors(r, steps)
    assert amr < factor * coarse, (amr, coarse)


class ConstantFill(Hierarchy):
    """Planted mistake: coarse fills without the limited slopes."""

    def fill(self, old, t_n, dt_c):
        r, nxc = self.r, self.coarse.nx
        a = min(max((self.t_f - t_n) / dt_c, 0.0), 1.0)
        for k, (p, g) in enumerate(zip(self.patches, self.grids)):
            fh, fu, fv = self.fine[k]
            for j in range(g.ny):
                for i in range(g.nx):
                    if RING <= i < g.nx - RING and RING <= j < g.ny - RING:
                        continue
                    c = ((p.j0 * r - RING + j) // r) * nxc + (p.i0 * r - RING + i) // r
                    o = j * g.nx + i
                    eo, en = old[0][c] + self.B[c], self.h[c] + self.B[c]
                    fh[o] = eo + a * (en - eo) - self.Bf[k][o]
                    fu[o] = old[1][c] + a * (self.hu[c] - old[1][c])
                    fv[o] = old[2][c] + a * (self.hv[c] - old[2][c])


class FrozenStart(Hierarchy):
    """Planted mistake: coarse fills always from the coarse step's start."""

    def fill(self, old, t_n, dt_c):
        t = self.t_f
        self.t_f = t_n
        super().fill(old, t_n, dt_c)
        self.t_f = t


class FrozenEnd(Hierarchy):
    """Planted mistake: coarse fills always from the coarse step's end."""

    def fill(self, old, t_n, dt_c):
        t = self.t_f
        self.t_f = t_n + dt_c
        super().fill(old, t_n, dt_c)
        self.t_f = t


@pytest.mark.parametrize("cls", [ConstantFill, FrozenStart, FrozenEnd])
def test_planted_fill_mistakes_lose_accuracy(cls):
    # a small patch around the hump, which the waves leave within the run:
    # what crosses its ring decides its accuracy
    p = Patch(10, 10, 4, 4)
    good, coarse = region_errors(4, 6, p=p)
    bad = region_errors(4, 6, cls=cls, p=p)[0]
    assert good < 0.5 * coarse, (good, coarse)
    assert bad > 1.5 * good, (good, bad)


def test_time_interpolation_at_mid_step():
    """Halfway through a coarse step, a coarse-filled ring cell on a flat
    field holds the mean of the coarse cell's old and new values."""
    H, cg, Bc, *_ = build(12, 2, [Patch(4, 4, 4, 4)], rest=True)
    old = (H.h.copy(), H.hu.copy(), H.hv.copy())
    H.h = H.h + 0.25      # eta rises by 0.25 m everywhere
    H.hu = H.hu + 3.0
    H.t_f = 50.0
    H.fill(old, 0.0, 100.0)
    f, b = H.fine[0], H.Bf[0]
    ring = np.ones(H.grids[0].n, bool)
    g = H.grids[0]
    ring.reshape(g.ny, g.nx)[RING:-RING, RING:-RING] = False
    np.testing.assert_allclose((f[0] + b)[ring], 0.125, rtol=0, atol=1e-12)
    np.testing.assert_allclose(f[1][ring], 1.5, rtol=0, atol=1e-12)


def linear_fill_error(cls=Hierarchy, r=3):
    """A surface and momenta linear in x and y on the coarse grid: minmod
    slopes of a linear field are its exact differences, so every
    coarse-filled ring cell must hold the field at its own centre."""
    nc = 16
    H, cg, Bc, *_ = build(nc, r, [Patch(5, 6, 4, 3)], cls=cls, rest=True)
    xc = (np.arange(nc) + 0.5) * DX
    X, Y = np.meshgrid(xc, xc)
    eta = (1e-3 * X / DX + 2e-3 * Y / DX).ravel()
    H.h = eta - Bc
    H.hu = (0.5 * X / DX - 0.25 * Y / DX).ravel()
    H.hv = (0.1 * Y / DX).ravel()
    H.fill((H.h.copy(), H.hu.copy(), H.hv.copy()), 0.0, 100.0)
    g, p = H.grids[0], H.patches[0]
    xf = g.x_lo + (np.arange(g.nx) + 0.5) * g.dx
    yf = g.y_lo + (np.arange(g.ny) + 0.5) * g.dy
    XF, YF = np.meshgrid(xf, yf)
    ring = np.ones((g.ny, g.nx), bool)
    ring[RING:-RING, RING:-RING] = False
    f, b = H.fine[0], H.Bf[0]
    want = [(1e-3 * XF / DX + 2e-3 * YF / DX), 0.5 * XF / DX - 0.25 * YF / DX, 0.1 * YF / DX]
    got = [(f[0] + b).reshape(g.ny, g.nx), f[1].reshape(g.ny, g.nx), f[2].reshape(g.ny, g.nx)]
    return max(float(np.abs(a - w)[ring].max()) for a, w in zip(got, want))


class HalfCellOffset(Hierarchy):
    """Planted mistake: the fine cell's offset inside its coarse cell taken
    at its lower corner instead of its centre."""

    @staticmethod
    def sub_offset(I, ic, r):
        return (I - ic * r) / r - 0.5


def test_a_linear_field_is_filled_exactly_at_the_fine_centres():
    """Pins the fine cell's position inside its coarse cell (xi, zeta) and the
    slopes: exact to rounding for r = 2, 3, 4."""
    for r in (2, 3, 4):
        assert linear_fill_error(r=r) <= 1e-12
        assert linear_fill_error(HalfCellOffset, r=r) > 1e-4   # half a fine cell of slope


class AverageByR(Hierarchy):
    """Planted mistake: the average divides by r instead of r^2."""

    def average(self):
        r, nxc = self.r, self.coarse.nx
        for jc in range(self.coarse.ny):
            for ic in range(nxc):
                src = self.owner(ic * r, jc * r)
                if src is None:
                    continue
                q, base = src
                g = self.grids[q]
                fh, fu, fv = self.fine[q]
                se = su = sv = 0.0
                for jj in range(r):
                    for ii in range(r):
                        s = base + jj * g.nx + ii
                        se += fh[s] + self.Bf[q][s]
                        su += fu[s]
                        sv += fv[s]
                c = jc * nxc + ic
                self.h[c] = se / r - self.B[c]
                self.hu[c] = su / r
                self.hv[c] = sv / r


class FlippedSlopes(Hierarchy):
    """Planted mistake: the coarse fill's limited slopes enter with the wrong
    sign (the ring leans away from the coarse gradient)."""

    def fill(self, old, t_n, dt_c):
        r, nxc = self.r, self.coarse.nx
        a = min(max((self.t_f - t_n) / dt_c, 0.0), 1.0)
        eta_o, eta_n = old[0] + self.B, self.h + self.B
        for k, (p, g) in enumerate(zip(self.patches, self.grids)):
            fh, fu, fv = self.fine[k]
            for j in range(g.ny):
                for i in range(g.nx):
                    if RING <= i < g.nx - RING and RING <= j < g.ny - RING:
                        continue
                    I, J = p.i0 * r - RING + i, p.j0 * r - RING + j
                    o = j * g.nx + i
                    src = self.owner(I, J, skip=k)
                    if src is not None:
                        q, s = src
                        sh, su, sv = self.fine[q]
                        fh[o] = sh[s] + self.Bf[q][s] - self.Bf[k][o]
                        fu[o], fv[o] = su[s], sv[s]
                        continue
                    ic, jc = I // r, J // r
                    xi = ((I - ic * r) + 0.5) / r - 0.5
                    zeta = ((J - jc * r) + 0.5) / r - 0.5
                    v = []
                    for qo, qn in ((eta_o, eta_n), (old[1], self.hu), (old[2], self.hv)):
                        at = lambda ii, jj: qo[jj * nxc + ii] + a * (qn[jj * nxc + ii] - qo[jj * nxc + ii])
                        qc = at(ic, jc)
                        sx = sy = 0.0
                        if 0 < ic < nxc - 1:
                            sx = minmod(qc - at(ic - 1, jc), at(ic + 1, jc) - qc)
                        if 0 < jc < self.coarse.ny - 1:
                            sy = minmod(qc - at(ic, jc - 1), at(ic, jc + 1) - qc)
                        v.append(qc - sx * xi - sy * zeta)
                    fh[o] = v[0] - self.Bf[k][o]
                    fu[o], fv[o] = v[1], v[2]



@pytest.mark.parametrize("cls", [AverageByR, FlippedSlopes])
def test_planted_glue_mistakes_fail_the_accuracy_pins(cls):
    fails = 0
    for (r, steps, factor) in [(2, 4, 0.3), (2, 12, 0.7), (4, 4, 0.5)]:
        amr, coarse = region_errors(r, steps, cls=cls)
        fails += not (amr < factor * coarse)
    assert fails >= 2


# ----------------------------------------------------------------- refluxing
PATCH_SETS = [(2, [Patch(8, 8, 8, 8)]),
              (4, [Patch(6, 6, 5, 7), Patch(11, 9, 6, 4)]),
              (3, [Patch(4, 4, 6, 6), Patch(10, 4, 4, 6), Patch(12, 7, 5, 5)])]


def mass_drift(r, patches, cls=Hierarchy, reflux=True, steps=10):
    H, cg, *_ = build(24, r, patches, cls=cls, reflux=reflux, mean_bottom=True)
    dt, t = dt_coarse(cg), 0.0
    m0 = H.h.sum()
    for _ in range(steps):
        assert H.step(t, dt)
        t = t + dt
    return abs(H.h.sum() - m0) / m0


@pytest.mark.parametrize("r,patches", PATCH_SETS)
def test_refluxing_conserves_mass(r, patches):
    """Walls all round, coarse bottoms the means of the fine ones: the mass
    of the hierarchy (uncovered coarse cells plus the covered ones, which
    hold the fine means) stays constant with refluxing, and drifts without."""
    assert mass_drift(r, patches) <= 1e-13
    assert mass_drift(r, patches, reflux=False) > 1e-8


class RefluxSign(Hierarchy):
    """Planted mistake: the reflux correction applied with a flipped sign."""
    reflux_sign = -1.0


class RefluxWeight(Hierarchy):
    """Planted mistake: each fine edge weighted as a whole coarse edge."""
    fine_weight_is_one = True


@pytest.mark.parametrize("cls", [RefluxSign, RefluxWeight])
def test_planted_reflux_mistakes_break_conservation(cls):
    r, patches = PATCH_SETS[1]
    assert mass_drift(r, patches, cls=cls) > 1e-8


def test_refluxing_keeps_the_ocean_at_rest_and_r1_the_single_grid():
    H, cg, Bc, *_ = build(16, 4, [Patch(4, 4, 5, 6), Patch(7, 8, 4, 4)], rest=True,
                          reflux=True)
    dt, t = dt_coarse(cg), 0.0
    for _ in range(4):
        assert H.step(t, dt)
        t = t + dt
    assert np.all(H.h + Bc == 0.0) and np.all(H.hu == 0) and np.all(H.hv == 0)
    patches = [Patch(5, 6, 6, 5), Patch(9, 8, 5, 7), Patch(14, 3, 4, 4)]
    H, cg, Bc, ec, _, _, uc = build(24, 1, patches, seed=1, reflux=True)
    h, hu, hv = ec - Bc, uc.copy(), -uc
    t = 0.0
    for _ in range(10):
        assert H.step(t, dt)
        h, hu, hv = O.fwd_step(cg, h, hu, hv, Bc, (t + dt) - t)
        t = t + dt
    for a, b in ((H.h, h), (H.hu, hu), (H.hv, hv)):
        assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()


def test_refluxing_a_patch_cut_in_two_gives_the_patch():
    one, cg, *_ = build(24, 2, [Patch(8, 8, 8, 8)], reflux=True)
    two, *_ = build(24, 2, [Patch(8, 8, 3, 8), Patch(11, 8, 5, 8)], reflux=True)
    dt, t = dt_coarse(cg), 0.0
    for _ in range(6):
        assert one.step(t, dt) and two.step(t, dt)
        t = t + dt
    assert np.abs(one.h - two.h).max() <= 1e-12 * np.abs(one.h + one.B).max()
