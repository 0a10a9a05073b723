"""AMR glue over several nested patch levels: the oracle (FP64, plain loops).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the bench's
CPU leg are the only callers; nothing here is shared with the CUDA library.

The paper's runs nest patches several levels deep, each level refined from
the one above it by an integer ratio in space and in time (Sec. 1, Sec. 6:
four levels in its Crescent City run).  Level 0 is a coarse grid; level l
(1 <= l <= L) holds patches whose interiors are whole cells of level l - 1,
refined by r_l.  Level l's cells have width dx_l = dx_{l-1} / r_l and are
numbered on a virtual uniform grid over the whole domain ("global" level-l
cells).  A patch is given by its interior in global level-(l - 1) cells,
(i0, j0, mx, my), and stored with a 2-cell ring as ordinary cells.

One coarse step of dt_c from t_n (Berger-Oliger subcycling):

  advance(0): the coarse grid steps once, to t_n + dt_c; then run(1) over
  that step; then average(1) and the refluxing of level 0.

  run(l) over a parent step [t_p, t_p + dt_p]: r_l substeps, the k-th ending
  at t_k = t_p + dt_p k / r_l (exactly t_p + dt_p for k = r_l).  A level
  with children takes exactly one launch per substep (so that its states
  before and after bracket the substep); the finest level takes up to m.
  Before every launch every ring of the level is filled; each patch steps
  with the level's common dt = min(cfl / s_max(level, ring included),
  t_k - t).  After each substep of a level l < L: run(l + 1) over it, then
  average(l + 1) and the refluxing of level l.

  fill(l): a ring cell inside the interior of another level-l patch copies
  that patch's cell (lowest patch index wins).  Otherwise it interpolates its
  parent: the level-(l - 1) cell P holding it, in the lowest-index patch
  whose interior holds P (or the coarse grid at l = 1).  First linearly in
  time between the parent's states at the start and end of its step (the
  state its step read, rings as filled for it, and the state it wrote; eta
  and both momenta, alpha = (t - t_p) / dt_p clamped to [0, 1]); then
  within P, q = q_P + s_x xi + s_y zeta with xi, zeta in (-1/2, 1/2) the
  fine centre's offset from P's centre in parent cells and minmod slopes
  from P's neighbours in the parent's array (zero where a neighbour lies
  outside that array: the domain edge for the coarse grid).  Its depth is
  eta - B of the ring cell.

  average(l): every level-(l - 1) cell under a level-l interior (lowest
  patch index), in every copy of it (the coarse grid, or each level-(l - 1)
  patch whose interior holds it), becomes the mean of its r_l^2 cells: eta
  and both momenta, summed row by row.

  refluxing of level l - 1 (optional, on by default): every copy of a
  level-(l - 1) interior cell U that is not under a level-l interior, beside
  a cell V that is, corrects its depth by the mass its own updates moved
  through the edge U|V minus the mass level l moved through it over the
  parent step: dh_U = sum (dt / d) phi_U - sum sum (dt_l / d) (1 / r_l)
  phi_f, phi the split step's mass flux through the edge (the fine fluxes
  of the r_l cells of V's lowest-index level-l patch along the edge, over
  every level-l launch of the parent step; signs flipped when V lies on U's
  low side), d the level-(l - 1) cell width across the edge.

With one level this is the two-level glue of oracle/amr.py, step for step.
Every ring of a level l >= 2 must lie inside the interiors of level l - 1
(proper nesting); level-1 rings must lie inside the domain.
"""
from __future__ import annotations

import numpy as np

from . import BC_EXTRAP, Grid, fwd_smax, fwd_step_flux
from .amr import RING, Patch, minmod

__all__ = ["LevelHierarchy", "Patch", "RING"]


class LevelHierarchy:
    """Coarse grid (h, hu, hv) with bottom B and levels [(patches, r, Bf)]
    (Bf[k]: bottom of patch k, ring included)."""

    # planted-mistake hooks for the tests
    reflux_sign = 1.0
    skip_level_in_fill = False   # fill level l >= 2 from the coarse grid
    alpha_from_coarse_step = False   # time-interpolate against the coarse step

    def __init__(self, coarse: Grid, B, levels, reflux=True):
        self.coarse = coarse
        self.B = np.asarray(B, dtype=np.float64)
        self.L = len(levels)
        self.r = [1] + [int(lv[1]) for lv in levels]
        self.P = [None] + [list(lv[0]) for lv in levels]
        self.Bf = [None] + [[np.asarray(b, dtype=np.float64) for b in lv[2]] for lv in levels]
        self.dx = [coarse.dx]
        self.dy = [coarse.dy]
        for l in range(1, self.L + 1):
            self.dx.append(self.dx[l - 1] / self.r[l])
            self.dy.append(self.dy[l - 1] / self.r[l])
        self.G = [None]
        for l in range(1, self.L + 1):
            self.G.append([self._grid(l, p) for p in self.P[l]])
        self.reflux = bool(reflux)
        self._check_nesting()
        self.edges = [None] + [self._edges(l) for l in range(1, self.L + 1)]
        self.t = [0.0] * (self.L + 1)

    # ------------------------------------------------------------ geometry
    def _grid(self, l, p):
        c = self.coarse
        dxp, dyp = self.dx[l - 1], self.dy[l - 1]
        return Grid(2, p.mx * self.r[l] + 2 * RING, p.my * self.r[l] + 2 * RING,
                    c.x_lo + p.i0 * dxp - RING * self.dx[l],
                    c.y_lo + p.j0 * dyp - RING * self.dy[l], self.dx[l], self.dy[l],
                    order=c.order, bc=(BC_EXTRAP,) * 4, g=c.g, cfl=c.cfl, dry_tol=c.dry_tol)

    def global_size(self, l):
        n = 1
        for k in range(1, l + 1):
            n *= self.r[k]
        return self.coarse.nx * n, self.coarse.ny * n

    def origin(self, l, q):
        """Global level-l index of patch q's array column 0 and row 0."""
        p, r = self.P[l][q], self.r[l]
        return p.i0 * r - RING, p.j0 * r - RING

    def owner(self, l, I, J, skip=-1):
        """At level 0: the coarse cell (None, index) if (I, J) is in the
        domain.  At level l >= 1: the lowest-index level-l patch (other than
        skip) whose interior holds global cell (I, J), and its local index
        there.  None if none."""
        if l == 0:
            c = self.coarse
            if 0 <= I < c.nx and 0 <= J < c.ny:
                return None, J * c.nx + I
            return None
        r = self.r[l]
        for q, p in enumerate(self.P[l]):
            if q == skip:
                continue
            if p.i0 * r <= I < (p.i0 + p.mx) * r and p.j0 * r <= J < (p.j0 + p.my) * r:
                I0, J0 = self.origin(l, q)
                return q, (J - J0) * self.G[l][q].nx + (I - I0)
        return None

    def _check_nesting(self):
        for l in range(1, self.L + 1):
            nxg, nyg = self.global_size(l)
            for q, g in enumerate(self.G[l]):
                I0, J0 = self.origin(l, q)
                if I0 < 0 or J0 < 0 or I0 + g.nx > nxg or J0 + g.ny > nyg:
                    raise ValueError(f"level {l} patch {q}: ring outside the domain")
                if l == 1:
                    continue
                r = self.r[l]
                for j in range(g.ny):
                    for i in range(g.nx):
                        if self.owner(l - 1, (I0 + i) // r, (J0 + j) // r) is None:
                            raise ValueError(f"level {l} patch {q}: not nested in level {l - 1}")

    def copies(self, l):
        """Every copy of a level-l interior cell: (patch or None, local index,
        global I, J).  Level 0: the coarse cells."""
        out = []
        if l == 0:
            c = self.coarse
            for J in range(c.ny):
                for I in range(c.nx):
                    out.append((None, J * c.nx + I, I, J))
            return out
        for q, g in enumerate(self.G[l]):
            I0, J0 = self.origin(l, q)
            for j in range(RING, g.ny - RING):
                for i in range(RING, g.nx - RING):
                    out.append((q, j * g.nx + i, I0 + i, J0 + j))
        return out

    def _edges(self, l):
        """Edges between a copy of an uncovered level-(l - 1) cell U and a
        neighbour V under a level-l interior: (U patch or None, U local
        index, axis, side, level-l owner q of V, V's r_l cells of q along
        the edge), U in the order of copies(l - 1), then +x, -x, +y, -y."""
        r = self.r[l]
        nxg, nyg = self.global_size(l - 1)
        edges = []
        for (pu, u, I, J) in self.copies(l - 1):
            if self.owner(l, I * r, J * r) is not None:
                continue
            for axis, side in ((0, 1), (0, -1), (1, 1), (1, -1)):
                Iv, Jv = (I + side, J) if axis == 0 else (I, J + side)
                if not (0 <= Iv < nxg and 0 <= Jv < nyg):
                    continue
                own = self.owner(l, Iv * r, Jv * r)
                if own is None:
                    continue
                q = own[0]
                I0, J0 = self.origin(l, q)
                nx = self.G[l][q].nx
                cells = []
                for k in range(r):
                    if axis == 0:
                        If, Jf = Iv * r + (0 if side > 0 else r - 1), Jv * r + k
                    else:
                        If, Jf = Iv * r + k, Jv * r + (0 if side > 0 else r - 1)
                    cells.append((Jf - J0) * nx + (If - I0))
                edges.append((pu, u, axis, side, q, cells))
        return edges

    # -------------------------------------------------------------- state
    def set_state(self, h, hu, hv, fine, t):
        """fine[l - 1][k] = (h, hu, hv) of level-l patch k, ring included."""
        self.h, self.hu, self.hv = (np.array(a, dtype=np.float64) for a in (h, hu, hv))
        self.q = [None] + [[[np.array(a, dtype=np.float64) for a in f] for f in lv]
                           for lv in fine]
        self.t = [float(t)] * (self.L + 1)

    def level_arrays(self, l, q):
        """(h, hu, hv, B, nx, ny) of the coarse grid (l = 0) or patch q."""
        if l == 0:
            c = self.coarse
            return self.h, self.hu, self.hv, self.B, c.nx, c.ny
        g = self.G[l][q]
        f = self.q[l][q]
        return f[0], f[1], f[2], self.Bf[l][q], g.nx, g.ny

    def snapshot(self, l):
        """Copies of level l's state arrays (h, hu, hv) per patch (or the
        coarse grid's, as a one-element list)."""
        if l == 0:
            return [(self.h.copy(), self.hu.copy(), self.hv.copy())]
        return [tuple(a.copy() for a in f) for f in self.q[l]]

    def level_smax(self, l):
        return max(fwd_smax(g, f[0], f[1], f[2]) for g, f in zip(self.G[l], self.q[l]))

    # ------------------------------------------------------------ pieces
    def fill(self, l, old, t_p, dt_p):
        """Fill the rings of level l at its time t[l]: from siblings, else
        from the parent level between its states old (t_p) and current
        (t_p + dt_p)."""
        r = self.r[l]
        a = (self.t[l] - t_p) / dt_p
        a = 0.0 if a < 0.0 else (1.0 if a > 1.0 else a)
        lp = l - 1
        for k, g in enumerate(self.G[l]):
            fh, fu, fv = self.q[l][k]
            I0, J0 = self.origin(l, k)
            for j in range(g.ny):
                for i in range(g.nx):
                    if RING <= i < g.nx - RING and RING <= j < g.ny - RING:
                        continue
                    I, J = I0 + i, J0 + j
                    o = j * g.nx + i
                    src = self.owner(l, I, J, skip=k)
                    if src is not None:
                        q, s = src
                        sh, su, sv = self.q[l][q]
                        fh[o] = sh[s] + self.Bf[l][q][s] - self.Bf[l][k][o]
                        fu[o], fv[o] = su[s], sv[s]
                        continue
                    if self.skip_level_in_fill and l >= 2:
                        v = self._interp_coarse(l, I, J)
                    else:
                        v = self._interp_parent(lp, I // r, J // r, I, J, r, old, a)
                    fh[o] = v[0] - self.Bf[l][k][o]
                    fu[o], fv[o] = v[1], v[2]

    @staticmethod
    def sub_offset(I, Ip, r):
        """Offset of cell I's centre from its parent cell Ip's centre, in
        parent cells (in (-1/2, 1/2))."""
        return ((I - Ip * r) + 0.5) / r - 0.5

    def _interp_parent(self, lp, Ip, Jp, I, J, r, old, a):
        qp, c = self.owner(lp, Ip, Jp)
        h, hu, hv, Bp, nx, ny = self.level_arrays(lp, 0 if qp is None else qp)
        oh, ou, ov = old[0 if qp is None else qp]
        ic, jc = c % nx, c // nx
        xi = self.sub_offset(I, Ip, r)
        zeta = self.sub_offset(J, Jp, r)
        v = []
        for qo, qn, add in ((oh, h, Bp), (ou, hu, None), (ov, hv, None)):
            def at(ii, jj):
                cc = jj * nx + ii
                o_ = qo[cc] + (add[cc] if add is not None else 0.0)
                n_ = qn[cc] + (add[cc] if add is not None else 0.0)
                return o_ + a * (n_ - o_)
            qc = at(ic, jc)
            sx = sy = 0.0
            if 0 < ic < nx - 1:
                sx = minmod(qc - at(ic - 1, jc), at(ic + 1, jc) - qc)
            if 0 < jc < ny - 1:
                sy = minmod(qc - at(ic, jc - 1), at(ic, jc + 1) - qc)
            v.append(qc + sx * xi + sy * zeta)
        return v

    def _interp_coarse(self, l, I, J):
        """Planted mistake: the coarse cell holding the fine cell, no time or
        space interpolation."""
        n = 1
        for k in range(1, l + 1):
            n *= self.r[k]
        c = (J // n) * self.coarse.nx + (I // n)
        return [self.h[c] + self.B[c], self.hu[c], self.hv[c]]

    def average(self, l):
        """Every copy of a level-(l - 1) cell under a level-l interior := the
        mean of its r_l^2 cells (lowest-index level-l patch)."""
        r = self.r[l]
        for (pu, u, I, J) in self.copies(l - 1):
            src = self.owner(l, I * r, J * r)
            if src is None:
                continue
            q, base = src
            g = self.G[l][q]
            fh, fu, fv = self.q[l][q]
            se = su = sv = 0.0
            for jj in range(r):
                for ii in range(r):
                    s = base + jj * g.nx + ii
                    se += fh[s] + self.Bf[l][q][s]
                    su += fu[s]
                    sv += fv[s]
            h, hu, hv, Bp, _, _ = self.level_arrays(l - 1, 0 if pu is None else pu)
            h[u] = se / (r * r) - Bp[u]
            hu[u] = su / (r * r)
            hv[u] = sv / (r * r)

    def _apply_reflux(self, l, dh):
        """Refluxing of level l - 1 from the per-edge corrections dh."""
        if not self.reflux:
            return
        for e, (pu, u, axis, side, q, cells) in enumerate(self.edges[l]):
            h = self.level_arrays(l - 1, 0 if pu is None else pu)[0]
            h[u] += self.reflux_sign * dh[e]

    def _add_coarse_part(self, l, dh, dt, phis):
        """Level l - 1's own fluxes through the edges of level l over a step
        of dt; phis[patch or 0] the flux arrays of level l - 1."""
        for e, (pu, u, axis, side, q, cells) in enumerate(self.edges[l]):
            d = self.dx[l - 1] if axis == 0 else self.dy[l - 1]
            ph = phis[0 if pu is None else pu]
            f = ph[2 * axis + 1][u] if side > 0 else -ph[2 * axis][u]
            dh[e] += dt / d * f

    def _add_fine_part(self, l, dh, dt, phis):
        """Level l's fluxes into its region across the edges of level l over
        a launch of dt."""
        r = self.r[l]
        for e, (pu, u, axis, side, q, cells) in enumerate(self.edges[l]):
            d = self.dx[l - 1] if axis == 0 else self.dy[l - 1]
            ph = phis[q][2 * axis] if side > 0 else -phis[q][2 * axis + 1]
            w = 1.0 / r
            dh[e] -= dt / d * w * sum(ph[c] for c in cells)

    # -------------------------------------------------------------- step
    def step(self, t_n, dt_c, m=1):
        """One coarse step of dt_c from t_n.  Returns False if a level did
        not reach t_n + dt_c."""
        cg = self.coarse
        t_end = t_n + dt_c
        dt = cg.cfl / fwd_smax(cg, self.h, self.hu, self.hv)
        if t_end - self.t[0] < dt:
            dt = t_end - self.t[0]
        old = self.snapshot(0)
        self._coarse_step = (t_n, dt_c)
        dh = np.zeros(len(self.edges[1])) if self.L >= 1 else None
        if dt > 0.0:
            self.h, self.hu, self.hv, phi = fwd_step_flux(cg, self.h, self.hu, self.hv, self.B, dt)
            self.t[0] = self.t[0] + dt
            if self.L >= 1:
                self._add_coarse_part(1, dh, dt, [phi])
        ok = self.t[0] == t_end
        if self.L >= 1:
            ok = self._run(1, t_n, dt_c, old, dh, m) and ok
            self.average(1)
            self._apply_reflux(1, dh)
        return ok

    def _run(self, l, t_p, dt_p, old_parent, dh_l, m):
        """Level l over the parent step [t_p, t_p + dt_p]; dh_l collects the
        fine parts of the edges of level l."""
        r = self.r[l]
        t_end = t_p + dt_p
        launches = m if l == self.L else 1
        ok = True
        for k in range(1, r + 1):
            t_k = t_end if k == r else t_p + dt_p * k / r
            t_km1 = t_p if k == 1 else t_p + dt_p * (k - 1) / r
            old_l = None
            dh_c = np.zeros(len(self.edges[l + 1])) if l < self.L else None
            for _ in range(launches):
                dt = self.G[l][0].cfl / self.level_smax(l)
                if t_k - self.t[l] < dt:
                    dt = t_k - self.t[l]
                if self.alpha_from_coarse_step:
                    self.fill(l, old_parent, *self._coarse_step)
                else:
                    self.fill(l, old_parent, t_p, dt_p)
                if old_l is None:
                    # the state this level's step reads, rings as filled
                    # for it: its children's start state
                    old_l = self.snapshot(l)
                if dt > 0.0:
                    phis = []
                    for q, g in enumerate(self.G[l]):
                        f = self.q[l][q]
                        nh, nu, nv, ph = fwd_step_flux(g, f[0], f[1], f[2], self.Bf[l][q], dt)
                        self.q[l][q] = [nh, nu, nv]
                        phis.append(ph)
                    self.t[l] = self.t[l] + dt
                    self._add_fine_part(l, dh_l, dt, phis)
                    if l < self.L:
                        self._add_coarse_part(l + 1, dh_c, dt, phis)
            ok = ok and self.t[l] == t_k
            if l < self.L:
                ok = self._run(l + 1, t_km1, t_k - t_km1, old_l, dh_c, m) and ok
                self.average(l + 1)
                self._apply_reflux(l + 1, dh_c)
        return ok
