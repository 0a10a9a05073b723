"""Two-level AMR glue around the forward step: the oracle (FP64, plain loops).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the bench's
CPU leg are the only callers; nothing here is shared with the CUDA library.

The paper's runs hold patches on finer levels, refined by an integer ratio
in space and in time (Sec. 1, Sec. 6).  This is the glue between one coarse
grid and one level of fine patches, one coarse step at a time:

  1. the coarse grid steps from t_n to t_n + dt_c;
  2. the fine level takes r substeps, the k-th ending at
     t_k = t_n + dt_c k / r (t_r = t_n + dt_c), with at most m launches each.
     Before every launch the 2-cell ring of every fine patch is filled.  A
     ring cell that lies in the interior of another patch copies that patch's
     cell (the lowest patch index wins).  Otherwise it interpolates the
     coarse level: first linearly in time, per coarse cell, between the
     states at t_n and t_n + dt_c (eta = h + B and both momenta,
     alpha = (t - t_n) / dt_c clamped to [0, 1], q = q_old + alpha
     (q_new - q_old)); then in space, piecewise linearly within the coarse
     cell C containing the ring cell, q = q_C + s_x xi + s_y zeta, where
     xi, zeta in (-1/2, 1/2) is the fine centre's offset from C's centre in
     coarse cells and s_x = minmod(q_C - q_W, q_E - q_C) (zero if a
     neighbour lies outside the domain), s_y likewise.  Its depth is
     eta - B_fine;
  3. every coarse cell under a patch interior (the lowest patch index wins)
     becomes the mean of its r x r fine cells: eta and both momenta, summed
     row by row, divided by r^2; its depth is eta - B_coarse;
  4. refluxing (optional, on by default): every uncovered coarse cell U
     beside a covered coarse cell V had its mass updated with the coarse
     mass flux through the edge U|V, while the fine level moved mass across
     the same edge with its own fluxes.  U's depth is corrected by the
     difference, per sweep (x-edges in the x-sweep, y-edges in the y-sweep):
       dh_U = (dt_c / dx_c) phi_c - sum_s sum_J (dt_s / dx_c) (1 / r) phi_f,
     phi_c the coarse flux through the edge as U's update used it, phi_f the
     flux through each of the r fine edges along it as the fine interior
     cell's update used it, over the r fine substeps s (signs flipped when U
     lies on the high side).  The total mass (uncovered coarse cells plus
     the covered ones, which hold the fine means) is then conserved between
     walls.

Patches are aligned with the coarse grid (interior on whole coarse cells)
and their rings lie inside the coarse domain.  A fine patch is stored with
its ring as ordinary cells: the fine step updates the ring too (with
extrapolation beyond it), which matters only through the level's CFL
maximum, and the next fill overwrites it.  Every time step is
dt = min(cfl / s_max, t_end - t) on the current state, as for a single grid;
all patches of the level share one dt.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import BC_EXTRAP, Grid, fwd_smax, fwd_step, fwd_step_flux

RING = 2


@dataclass
class Patch:
    """Interior of a fine patch in coarse cells: lower-left (i0, j0), size
    mx x my."""
    i0: int
    j0: int
    mx: int
    my: int


def fine_grid(coarse: Grid, p: Patch, r: int) -> Grid:
    """The fine patch as a grid of its own, ring included."""
    dxf, dyf = coarse.dx / r, coarse.dy / r
    return Grid(2, p.mx * r + 2 * RING, p.my * r + 2 * RING,
                coarse.x_lo + p.i0 * coarse.dx - RING * dxf,
                coarse.y_lo + p.j0 * coarse.dy - RING * dyf, dxf, dyf,
                order=coarse.order, bc=(BC_EXTRAP,) * 4, g=coarse.g, cfl=coarse.cfl,
                dry_tol=coarse.dry_tol)


def minmod(a, b):
    """The smaller in magnitude of a and b if they have the same sign, else 0."""
    if a * b <= 0.0:
        return 0.0
    return a if abs(a) < abs(b) else b


class Hierarchy:
    """Coarse grid state (h, hu, hv) with bottom B, fine patches with their
    own bottoms Bf[k] (ring included), refinement ratio r."""

    # the method's refluxing sign and fine-edge weight divisor (r); tests
    # override them in subclasses to plant mistakes
    reflux_sign = 1.0
    fine_weight_is_one = False

    def __init__(self, coarse: Grid, B, patches, r, Bf, reflux=True):
        self.coarse, self.r, self.patches = coarse, int(r), list(patches)
        self.B = np.asarray(B, dtype=np.float64)
        self.Bf = [np.asarray(b, dtype=np.float64) for b in Bf]
        self.grids = [fine_grid(coarse, p, r) for p in self.patches]
        for p, g in zip(self.patches, self.grids):
            if not (p.i0 * r - RING >= 0 and p.j0 * r - RING >= 0
                    and (p.i0 + p.mx) * r + RING <= coarse.nx * r
                    and (p.j0 + p.my) * r + RING <= coarse.ny * r):
                raise ValueError("a patch ring leaves the coarse domain")
        self.t_c = self.t_f = 0.0
        self.reflux = bool(reflux)
        self.cf_edges = self._coarse_fine_edges()

    def _coarse_fine_edges(self):
        """Edges between an uncovered coarse cell U and a covered one V:
        (U, axis 0/1, side +1 if V lies on U's high side else -1, owner
        patch q of V, fine cells of q along the edge inside V)."""
        cg, r = self.coarse, self.r
        covered = {}
        for jc in range(cg.ny):
            for ic in range(cg.nx):
                src = self.owner(ic * r, jc * r)
                if src is not None:
                    covered[(ic, jc)] = src[0]
        edges = []
        for jc in range(cg.ny):
            for ic in range(cg.nx):
                if (ic, jc) in covered:
                    continue
                for axis, side in ((0, 1), (0, -1), (1, 1), (1, -1)):
                    iv, jv = (ic + side, jc) if axis == 0 else (ic, jc + side)
                    q = covered.get((iv, jv))
                    if q is None:
                        continue
                    p, g = self.patches[q], self.grids[q]
                    cells = []
                    for k in range(r):
                        if axis == 0:
                            I = iv * r + (0 if side > 0 else r - 1)
                            J = jv * r + k
                        else:
                            I = iv * r + k
                            J = jv * r + (0 if side > 0 else r - 1)
                        cells.append((J - p.j0 * r + RING) * g.nx + (I - p.i0 * r + RING))
                    edges.append((jc * cg.nx + ic, axis, side, q, cells))
        return edges

    def set_state(self, h, hu, hv, fine, t):
        """fine[k] = (h, hu, hv) of patch k, ring included."""
        self.h, self.hu, self.hv = (np.array(a, dtype=np.float64) for a in (h, hu, hv))
        self.fine = [[np.array(a, dtype=np.float64) for a in f] for f in fine]
        self.t_c = self.t_f = float(t)

    # ------------------------------------------------------------ pieces
    def owner(self, I, J, skip=-1):
        """Lowest-index patch (other than skip) whose interior holds global
        fine cell (I, J), and its local index there; None if none."""
        r = self.r
        for q, p in enumerate(self.patches):
            if q == skip:
                continue
            if p.i0 * r <= I < (p.i0 + p.mx) * r and p.j0 * r <= J < (p.j0 + p.my) * r:
                g = self.grids[q]
                return q, (J - p.j0 * r + RING) * g.nx + (I - p.i0 * r + RING)
        return None

    @staticmethod
    def sub_offset(I, ic, r):
        """Offset of fine cell I's centre from its coarse cell ic's centre,
        in coarse cells (in (-1/2, 1/2))."""
        return ((I - ic * r) + 0.5) / r - 0.5

    def fill(self, old, t_n, dt_c):
        """Fill every ring from siblings or from the coarse states old (t_n)
        and current (t_n + dt_c), at the fine level's time t_f."""
        r, nxc = self.r, self.coarse.nx
        a = (self.t_f - t_n) / dt_c
        a = 0.0 if a < 0.0 else (1.0 if a > 1.0 else a)
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
                    xi = self.sub_offset(I, ic, r)
                    zeta = self.sub_offset(J, jc, r)
                    v = []
                    for qo, qn in ((eta_o, eta_n), (old[1], self.hu), (old[2], self.hv)):
                        def at(ii, jj):
                            c = jj * nxc + ii
                            return qo[c] + a * (qn[c] - qo[c])
                        qc = at(ic, jc)
                        sx = sy = 0.0
                        if 0 < ic < nxc - 1:
                            sx = minmod(qc - at(ic - 1, jc), at(ic + 1, jc) - qc)
                        if 0 < jc < self.coarse.ny - 1:
                            sy = minmod(qc - at(ic, jc - 1), at(ic, jc + 1) - qc)
                        v.append(qc + sx * xi + sy * zeta)
                    fh[o] = v[0] - self.Bf[k][o]
                    fu[o], fv[o] = v[1], v[2]

    def average(self):
        """Coarse cells under a patch interior := mean of their fine cells."""
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
                self.h[c] = se / (r * r) - self.B[c]
                self.hu[c] = su / (r * r)
                self.hv[c] = sv / (r * r)

    def fine_smax(self):
        return max(fwd_smax(g, f[0], f[1], f[2]) for g, f in zip(self.grids, self.fine))

    # -------------------------------------------------------------- step
    def step(self, t_n, dt_c, m=1):
        """One coarse step of dt_c from t_n with r fine substeps.  Returns
        False if a level did not reach t_n + dt_c."""
        cg, r = self.coarse, self.r
        t_end = t_n + dt_c
        dt = cg.cfl / fwd_smax(cg, self.h, self.hu, self.hv)
        if t_end - self.t_c < dt:
            dt = t_end - self.t_c
        old = (self.h.copy(), self.hu.copy(), self.hv.copy())
        dh = np.zeros(len(self.cf_edges))   # reflux correction per edge
        if dt > 0.0:
            self.h, self.hu, self.hv, phi = fwd_step_flux(cg, self.h, self.hu, self.hv, self.B, dt)
            self.t_c = self.t_c + dt
            for e, (u, axis, side, q, cells) in enumerate(self.cf_edges):
                d = cg.dx if axis == 0 else cg.dy
                # U's update took -(dt/d) phi_hi for a high-side neighbour,
                # +(dt/d) phi_lo for a low-side one
                f = phi[2 * axis + 1][u] if side > 0 else -phi[2 * axis][u]
                dh[e] += dt / d * f
        for k in range(1, r + 1):
            t_k = t_end if k == r else t_n + dt_c * k / r
            for _ in range(m):
                dtf = cg.cfl / self.fine_smax()
                if t_k - self.t_f < dtf:
                    dtf = t_k - self.t_f
                self.fill(old, t_n, dt_c)
                if dtf > 0.0:
                    phis = []
                    for q, g in enumerate(self.grids):
                        f = self.fine[q]
                        nh, nu, nv, ph = fwd_step_flux(g, f[0], f[1], f[2], self.Bf[q], dtf)
                        self.fine[q] = [nh, nu, nv]
                        phis.append(ph)
                    self.t_f = self.t_f + dtf
                    for e, (u, axis, side, q, cells) in enumerate(self.cf_edges):
                        d = cg.dx if axis == 0 else cg.dy
                        # mass entering the fine region across the edge: the
                        # fine cells' low-edge flux (V on U's high side) or
                        # high-edge flux with its sign flipped
                        ph = phis[q][2 * axis] if side > 0 else -phis[q][2 * axis + 1]
                        w = 1.0 if self.fine_weight_is_one else 1.0 / r
                        dh[e] -= dtf / d * w * sum(ph[c] for c in cells)
        self.average()
        if self.reflux:
            for e, (u, axis, side, q, cells) in enumerate(self.cf_edges):
                self.h[u] += self.reflux_sign * dh[e]
        return self.t_c == t_end and self.t_f == t_end
