/*
 * swe_oracle.c -- plain FP64 CPU oracle for the adjoint-guided shallow-water
 * path (Davis & LeVeque, arXiv 1605.05320).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file; only the tests, the package smoke check and the bench's
 * CPU-baseline leg do.  It shares no source with the CUDA library.
 *
 * Compiled with -O2 -ffp-contract=off so every operation rounds as written.
 * Arrays are row-major with x fastest, index j*nx + i, no ghost cells; every
 * routine builds its own ghost-padded copies (2 ghost layers).
 *
 * What each routine follows:
 *   fwd_riemann      Sec. 6 (Roe solver for SWE plus bathymetry) applied to
 *                    Eq. (swe_1d)/(swe): f-wave form, source folded into the
 *                    momentum jump as g*hhat*(eta_R - eta_L).
 *   orc_fwd_step     Godunov-type wave-propagation update with MC-limited
 *                    second-order corrections (order 2); in 2D dimensionally
 *                    split: an x-sweep over every row, then a y-sweep over
 *                    every column of the x-swept state.
 *   orc_fwd_step_ctu the unsplit 2D alternative (scheme 1): the
 *                    wave-propagation update of the textbook the paper defers
 *                    to for its methods (LeVeque 2002, the multidimensional
 *                    chapters, cited in Sec. 6): x- and y-edge waves all from
 *                    Q^n, MC-limited corrections, and transverse propagation
 *                    of each fluctuation into the neighbouring edge fluxes.
 *                    One detail is parity unpinned: which Roe state splits a
 *                    fluctuation transversely (its own edge's here).  Any
 *                    neighbouring edge's state gives an equally consistent
 *                    scheme that passes the same pins.
 *   orc_fwd_smax     CFL number max over cells of max_dir (|u|+c)/d_dir.
 *   orc_lin_step     first-order update of Eq. (hyp_linear) (and its 2D form,
 *                    Sec. 5, x-sweep then y-sweep), used only by the
 *                    adjoint-identity pins.
 *   orc_adj_step     one step of the time-reversed adjoint of Sec. 4:
 *                    q~_t - (A^T q~)_x [- (A_2^T q~)_y] = 0, f-wave form, walls
 *                    at wet/dry edges (Sec. 5 boundary condition); in 2D a
 *                    y-sweep then an x-sweep (the transpose of the forward
 *                    order, so one adjoint step is the transpose of one
 *                    linear forward step).
 *   orc_flag         Eq. (ip_timepoint) (BRACKET) and Eq. (ip_timerange) with
 *                    linear interpolation in time (INTERP), bilinear spatial
 *                    interpolation of the adjoint (Sec. 4), zero where the
 *                    adjoint is dry (Sec. 6).
 *   orc_flag_surface surface flagging |eta| > tol (Sec. 6 comparator).
 *   orc_gauge        bilinear interpolation of cell-centre eta (Sec. 6 gauges).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define BC_EXTRAP 0
#define BC_WALL 1

#define FLAG_INTERP 0
#define FLAG_BRACKET 1

typedef struct {
    int ndim;           /* 1 or 2 */
    int nx, ny;         /* ny == 1 when ndim == 1 */
    double x_lo, y_lo, dx, dy;
    int order;          /* 1 or 2 */
    int bc[4];          /* x_lo, x_hi, y_lo, y_hi */
    double g, cfl, dry_tol;
    double lin_nu[2];   /* internal: dt/dx, dt/dy of the linear sweeps */
    int scheme;         /* 2D forward step: 0 split, 1 unsplit with transverse waves */
    double tw_scale;    /* factor on the transverse terms: 1 for the method; the
                           tests set 0 or -1 to show their pins catch a dropped
                           or sign-flipped term */
    int wetdry;         /* forward split step: 1 handles dry cells (h <= dry_tol)
                           and transonic edges by the shore solver below */
} orc_grid;

#define NG 2

/*
 * ORC_PLANT selects a deliberately wrong variant of one step, compiled only
 * by the tests that show a pin catches that mistake (0, the default, is the
 * method):
 *   1  tangential wave strength formed with the normal Roe average
 *      (beta2 = df3 - uhat df1)
 *   2  tangential Roe average taken as the arithmetic mean of vL and vR
 *   3  normal Roe average taken as the arithmetic mean of uL and uR
 *   4  adjoint step count one more than ceil(t_f smax / cfl)
 *   5  snapshot times recorded one snapshot interval late
 *   6  shore solver: HLL flux of the cell states instead of the
 *      hydrostatically reconstructed ones
 *   7  shore solver used only at dry edges (transonic wet edges keep Roe)
 *   8  shore solver: the hydrostatic-reconstruction pressure terms dropped
 */
#ifndef ORC_PLANT
#define ORC_PLANT 0
#endif

/* ---------------------------------------------------------------- helpers */

static double *padded(const orc_grid *G) {
    size_t px = (size_t)G->nx + 2 * NG;
    size_t py = (G->ndim == 2) ? (size_t)G->ny + 2 * NG : 1;
    return (double *)calloc(px * py, sizeof(double));
}

/* index into a padded array: i in [-NG, nx+NG), j in [-NG, ny+NG) (2D) */
static inline size_t pidx(const orc_grid *G, int i, int j) {
    size_t px = (size_t)G->nx + 2 * NG;
    if (G->ndim == 1) return (size_t)(i + NG);
    return (size_t)(j + NG) * px + (size_t)(i + NG);
}

/*
 * Copy an interior field into a padded array and fill its ghost cells.
 * sign_x / sign_y: factor applied to mirrored ghosts at x walls / y walls
 * (-1 for the momentum normal to that wall, +1 otherwise).  Extrapolation
 * copies the nearest interior cell into both ghost layers.
 */
static void fill_padded(const orc_grid *G, const double *a, double *p,
                        double sign_x, double sign_y) {
    int nx = G->nx, ny = G->ny;
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++)
            p[pidx(G, i, j)] = a[(size_t)j * nx + i];
    for (int j = 0; j < ny; j++) {
        for (int k = 1; k <= NG; k++) {
            /* low x */
            if (G->bc[0] == BC_WALL)
                p[pidx(G, -k, j)] = sign_x * a[(size_t)j * nx + (k - 1)];
            else
                p[pidx(G, -k, j)] = a[(size_t)j * nx + 0];
            /* high x */
            if (G->bc[1] == BC_WALL)
                p[pidx(G, nx - 1 + k, j)] = sign_x * a[(size_t)j * nx + (nx - k)];
            else
                p[pidx(G, nx - 1 + k, j)] = a[(size_t)j * nx + (nx - 1)];
        }
    }
    if (G->ndim == 2) {
        for (int i = 0; i < nx; i++) {
            for (int k = 1; k <= NG; k++) {
                if (G->bc[2] == BC_WALL)
                    p[pidx(G, i, -k)] = sign_y * a[(size_t)(k - 1) * nx + i];
                else
                    p[pidx(G, i, -k)] = a[i];
                if (G->bc[3] == BC_WALL)
                    p[pidx(G, i, ny - 1 + k)] = sign_y * a[(size_t)(ny - k) * nx + i];
                else
                    p[pidx(G, i, ny - 1 + k)] = a[(size_t)(ny - 1) * nx + i];
            }
        }
    }
}

/* MC limiter phi(theta) = max(0, min((1+theta)/2, 2, 2 theta)) */
static double mc_limiter(double theta) {
    double a = 0.5 * (1.0 + theta);
    double b = 2.0;
    double c = 2.0 * theta;
    double m = a;
    if (b < m) m = b;
    if (c < m) m = c;
    if (m < 0.0) m = 0.0;
    return m;
}

static double sgn(double s) { return (s > 0.0) ? 1.0 : ((s < 0.0) ? -1.0 : 0.0); }

static double dot3(const double *a, const double *b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/*
 * Generic 1D wave data at one edge: MW waves of 3 components each, speeds.
 */
typedef struct {
    double s[3];
    double Z[3][3];
    double uhat, vhat, chat;   /* Roe state of the forward solve (edge frame) */
    int shore;                 /* fluctuations given directly (shore solver) */
    double amdq[3], apdq[3];
} edge_waves;

/*
 * Fluctuations and second-order correction for edge e given waves at e and at
 * its neighbours em (edge to the left) and ep (edge to the right).
 * apdq: goes to the right cell, amdq: to the left cell, F: correction flux.
 * nu = dt/dx.  Order 1 leaves F = 0.
 */
static void edge_fluxes(int mw, const edge_waves *em, const edge_waves *e,
                        const edge_waves *ep, double nu, int order,
                        double amdq[3], double apdq[3], double F[3]) {
    for (int m = 0; m < 3; m++) { amdq[m] = 0.0; apdq[m] = 0.0; F[m] = 0.0; }
    if (e->shore) {
        /* first order at the shore; its waves are zero for the neighbours'
           limiters */
        for (int m = 0; m < 3; m++) { amdq[m] = e->amdq[m]; apdq[m] = e->apdq[m]; }
        return;
    }
    for (int p = 0; p < mw; p++) {
        double s = e->s[p];
        for (int m = 0; m < 3; m++) {
            if (s < 0.0) amdq[m] += e->Z[p][m];
            else if (s > 0.0) apdq[m] += e->Z[p][m];
            else { amdq[m] += 0.5 * e->Z[p][m]; apdq[m] += 0.5 * e->Z[p][m]; }
        }
    }
    if (order < 2) return;
    for (int p = 0; p < mw; p++) {
        double s = e->s[p];
        const edge_waves *up = (s > 0.0) ? em : ep;
        double zz = dot3(e->Z[p], e->Z[p]);
        double theta = 0.0;
        if (zz != 0.0) theta = dot3(up->Z[p], e->Z[p]) / zz;
        double phi = mc_limiter(theta);
        double coef = 0.5 * sgn(s) * (1.0 - nu * fabs(s)) * phi;
        for (int m = 0; m < 3; m++) F[m] += coef * e->Z[p][m];
    }
}

/* ------------------------------------------------------- forward Riemann */

/*
 * f-wave Roe solver for the nonlinear SWE with bathymetry.  State components
 * (h, normal momentum, tangential momentum); B is bottom elevation.
 * Roe averages: hhat = (hL+hR)/2, uhat/vhat sqrt(h)-weighted, chat =
 * sqrt(g hhat).  The flux jump includes the bathymetry source as
 * g*hhat*(eta_R - eta_L) in the normal momentum so that the ocean at rest has
 * zero jump (well balanced).  Eigenvectors (1, uhat-chat, vhat), (0,0,1),
 * (1, uhat+chat, vhat).
 */
static void fwd_riemann(double g,
                        double hL, double mnL, double mtL, double BL,
                        double hR, double mnR, double mtR, double BR,
                        edge_waves *w) {
    double uL = mnL / hL, vL = mtL / hL;
    double uR = mnR / hR, vR = mtR / hR;
    double hhat = 0.5 * (hL + hR);
    double sqL = sqrt(hL), sqR = sqrt(hR);
#if ORC_PLANT == 3
    double uhat = 0.5 * (uL + uR);
#else
    double uhat = (sqL * uL + sqR * uR) / (sqL + sqR);
#endif
#if ORC_PLANT == 2
    double vhat = 0.5 * (vL + vR);
#else
    double vhat = (sqL * vL + sqR * vR) / (sqL + sqR);
#endif
    double chat = sqrt(g * hhat);
    double s1 = uhat - chat, s2 = uhat, s3 = uhat + chat;
    double etaL = hL + BL, etaR = hR + BR;
    double df1 = mnR - mnL;
    double df2 = (mnR * uR - mnL * uL) + g * hhat * (etaR - etaL);
    double df3 = mnR * vR - mnL * vL;
    double b1 = (s3 * df1 - df2) / (s3 - s1);
    double b3 = (df2 - s1 * df1) / (s3 - s1);
#if ORC_PLANT == 1
    double b2 = df3 - uhat * df1;
#else
    double b2 = df3 - vhat * df1;
#endif
    w->s[0] = s1; w->s[1] = s2; w->s[2] = s3;
    w->uhat = uhat; w->vhat = vhat; w->chat = chat;
    w->shore = 0;
    w->Z[0][0] = b1;  w->Z[0][1] = b1 * s1;  w->Z[0][2] = b1 * vhat;
    w->Z[1][0] = 0.0; w->Z[1][1] = 0.0;      w->Z[1][2] = b2;
    w->Z[2][0] = b3;  w->Z[2][1] = b3 * s3;  w->Z[2][2] = b3 * vhat;
}

/*
 * Shore solver (the reading of Sec. 6's "robust near shore and inundation"):
 * at an edge with a dry cell (h <= dry_tol) or a transonic rarefaction the
 * fluctuations come from the hydrostatic reconstruction of Audusse et al.
 * (2004) with an HLL flux, first order.  Reconstructed depths h*_L =
 * max(0, h_L + B_L - max(B_L, B_R)), h*_R likewise, with the cell velocities
 * (zero in a dry cell); HLL speeds s_L = min(u_L - c_L, u_R - c_R), s_R =
 * max(u_L + c_L, u_R + c_R) over the reconstructed states (c = 0 on a dry
 * side, so no speed exceeds a wet cell's |u| + c and the cell CFL number
 * bounds them: positivity of the scheme for CFL <= 1/2); flux
 * F = (s_R F_L - s_L F_R + s_L s_R (Q_R - Q_L)) / (s_R - s_L) over the
 * reconstructed states (F_L if s_L >= 0, F_R if s_R <= 0, zero when both are
 * dry).  The cell beside the edge sees F plus the pressure difference
 * g/2 (h^2 - h*^2) of its own side, so
 *   amdq = F + (0, g/2 (h_L^2 - h*_L^2), 0) - f(Q_L),
 *   apdq = f(Q_R) - F - (0, g/2 (h_R^2 - h*_R^2), 0),
 * f the physical flux (hu, hu u + g/2 h^2, hu v): well balanced (the ocean
 * at rest against dry land above it has zero fluctuations) and the mass flux
 * is F's first component on both sides.
 */
static void shore_riemann(double g, double dry_tol,
                          double hL, double mnL, double mtL, double BL,
                          double hR, double mnR, double mtR, double BR, edge_waves *w) {
    double uL = hL > dry_tol ? mnL / hL : 0.0, vL = hL > dry_tol ? mtL / hL : 0.0;
    double uR = hR > dry_tol ? mnR / hR : 0.0, vR = hR > dry_tol ? mtR / hR : 0.0;
    double Bm = BL > BR ? BL : BR;
    double hLs = hL + BL - Bm, hRs = hR + BR - Bm;
    if (hLs < 0.0) hLs = 0.0;
    if (hRs < 0.0) hRs = 0.0;
    double pL = 0.5 * g * (hL * hL), pR = 0.5 * g * (hR * hR);
    double pLs = 0.5 * g * (hLs * hLs), pRs = 0.5 * g * (hRs * hRs);
#if ORC_PLANT == 8
    pLs = pL; pRs = pR;
#endif
#if ORC_PLANT == 6
    double hLf = hL, hRf = hR, pLf = pL, pRf = pR;
#else
    double hLf = hLs, hRf = hRs, pLf = pLs, pRf = pRs;
#endif
    double FL[3] = {hLf * uL, hLf * uL * uL + pLf, hLf * uL * vL};
    double FR[3] = {hRf * uR, hRf * uR * uR + pRf, hRf * uR * vR};
    double QL[3] = {hLf, hLf * uL, hLf * vL}, QR[3] = {hRf, hRf * uR, hRf * vR};
    double F[3] = {0.0, 0.0, 0.0};
    if (hLf > 0.0 || hRf > 0.0) {
        double cL = sqrt(g * hLf), cR = sqrt(g * hRf);
        double sL = uL - cL < uR - cR ? uL - cL : uR - cR;
        double sR = uL + cL > uR + cR ? uL + cL : uR + cR;
        if (sL >= 0.0) {
            for (int m = 0; m < 3; m++) F[m] = FL[m];
        } else if (sR <= 0.0) {
            for (int m = 0; m < 3; m++) F[m] = FR[m];
        } else {
            for (int m = 0; m < 3; m++)
                F[m] = (sR * FL[m] - sL * FR[m] + sL * sR * (QR[m] - QL[m])) / (sR - sL);
        }
    }
    double fL[3] = {mnL, mnL * uL + pL, mnL * vL}, fR[3] = {mnR, mnR * uR + pR, mnR * vR};
    double SL[3] = {0.0, pL - pLs, 0.0}, SR[3] = {0.0, pR - pRs, 0.0};
    for (int m = 0; m < 3; m++) {
        w->amdq[m] = (F[m] + SL[m]) - fL[m];
        w->apdq[m] = fR[m] - (F[m] + SR[m]);
    }
    w->shore = 1;
    for (int p = 0; p < 3; p++) {
        w->s[p] = 0.0;
        for (int m = 0; m < 3; m++) w->Z[p][m] = 0.0;
    }
    w->uhat = 0.0; w->vhat = 0.0; w->chat = 0.0;
}

/*
 * One forward edge: the Roe solver, or with wetdry the shore solver at an
 * edge with a dry cell or a transonic rarefaction (u - c or u + c rising
 * through zero from the left cell to the right one).
 */
static void fwd_edge(const orc_grid *G,
                     double hL, double mnL, double mtL, double BL,
                     double hR, double mnR, double mtR, double BR, edge_waves *w) {
    if (G->wetdry) {
        int shore = !(hL > G->dry_tol) || !(hR > G->dry_tol);
#if ORC_PLANT != 7
        if (!shore) {
            double uL = mnL / hL, uR = mnR / hR;
            double cL = sqrt(G->g * hL), cR = sqrt(G->g * hR);
            shore = (uL - cL < 0.0 && uR - cR > 0.0) || (uL + cL < 0.0 && uR + cR > 0.0);
        }
#endif
        if (shore) {
            shore_riemann(G->g, G->dry_tol, hL, mnL, mtL, BL, hR, mnR, mtR, BR, w);
            return;
        }
    }
    fwd_riemann(G->g, hL, mnL, mtL, BL, hR, mnR, mtR, BR, w);
}

/*
 * Test-only view of one forward Riemann solve: out[0..2] the speeds,
 * out[3..11] the f-waves Z[p][m] row by row, out[12..14] uhat, vhat, chat.
 */
void orc_fwd_riemann(double g, double hL, double mnL, double mtL, double BL,
                     double hR, double mnR, double mtR, double BR, double *out) {
    edge_waves w;
    memset(&w, 0, sizeof w);
    fwd_riemann(g, hL, mnL, mtL, BL, hR, mnR, mtR, BR, &w);
    for (int p = 0; p < 3; p++) out[p] = w.s[p];
    for (int p = 0; p < 3; p++)
        for (int m = 0; m < 3; m++) out[3 + 3 * p + m] = w.Z[p][m];
    out[12] = w.uhat; out[13] = w.vhat; out[14] = w.chat;
}

/* --------------------------------------------------------- forward step */

/*
 * One sweep of size dt along x (dir 0) or y (dir 1), in place on (h, hu, hv):
 * every cell gets the fluctuations and corrections of its two edges in that
 * direction.  Along y the edge frame is (h, hv, hu).
 */
static void fwd_sweep(const orc_grid *G, int dir, double *h, double *hu, double *hv,
                      const double *B, double dt, double *phi_lo, double *phi_hi) {
    int nx = G->nx, ny = G->ny;
    size_t n = (size_t)nx * ny;
    double *ph = padded(G), *pu = padded(G), *pv = padded(G), *pB = padded(G);
    fill_padded(G, h, ph, 1.0, 1.0);
    fill_padded(G, hu, pu, -1.0, 1.0);
    fill_padded(G, hv, pv, 1.0, -1.0);
    fill_padded(G, B, pB, 1.0, 1.0);
    double *nh = (double *)malloc(n * sizeof(double));
    double *nu_ = (double *)malloc(n * sizeof(double));
    double *nv = (double *)malloc(n * sizeof(double));
    double nu = dt / (dir == 0 ? G->dx : G->dy);

#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++) {
        for (int i = 0; i < nx; i++) {
            size_t c = pidx(G, i, j);
            /* edges k-3/2 .. k+3/2 around the cell along the sweep */
            edge_waves w[4];
            for (int e = 0; e < 4; e++) {
                size_t a, b;
                if (dir == 0) { a = pidx(G, i - 2 + e, j); b = pidx(G, i - 1 + e, j); }
                else { a = pidx(G, i, j - 2 + e); b = pidx(G, i, j - 1 + e); }
                if (dir == 0)
                    fwd_edge(G, ph[a], pu[a], pv[a], pB[a], ph[b], pu[b], pv[b], pB[b], &w[e]);
                else
                    fwd_edge(G, ph[a], pv[a], pu[a], pB[a], ph[b], pv[b], pu[b], pB[b], &w[e]);
            }
            double amL[3], apL[3], FL[3], amR[3], apR[3], FR[3];
            edge_fluxes(3, &w[0], &w[1], &w[2], nu, G->order, amL, apL, FL);
            edge_fluxes(3, &w[1], &w[2], &w[3], nu, G->order, amR, apR, FR);
            double dq[3];
            for (int m = 0; m < 3; m++)
                dq[m] = -nu * (apL[m] + amR[m]) - nu * (FR[m] - FL[m]);
            size_t o = (size_t)j * nx + i;
            nh[o] = ph[c] + dq[0];
            if (dir == 0) { nu_[o] = pu[c] + dq[1]; nv[o] = pv[c] + dq[2]; }
            else { nv[o] = pv[c] + dq[1]; nu_[o] = pu[c] + dq[2]; }
            if (G->wetdry && !(nh[o] > G->dry_tol)) {
                /* a dry cell keeps no momentum (and no negative depth) */
                if (nh[o] < 0.0) nh[o] = 0.0;
                nu_[o] = 0.0;
                nv[o] = 0.0;
            }
            if (phi_lo) {
                /* mass flux through the cell's low and high edge of this sweep
                   as the cell's update sees it: dh = -nu (phi_hi - phi_lo) */
                double mn = dir == 0 ? pu[c] : pv[c];
                phi_lo[o] = mn - (apL[0] - FL[0]);
                phi_hi[o] = mn + (amR[0] + FR[0]);
            }
        }
    }
    memcpy(h, nh, n * sizeof(double));
    memcpy(hu, nu_, n * sizeof(double));
    memcpy(hv, nv, n * sizeof(double));
    free(ph); free(pu); free(pv); free(pB); free(nh); free(nu_); free(nv);
}

/* ------------------------------------------ unsplit step (scheme 1, 2D) */

/*
 * Ghost-padded copy with the corner ghosts filled too: fill_padded sets the
 * interior and the side ghosts, then the x rule is applied to every ghost
 * row, so a corner ghost takes both mappings and both sign factors (the
 * unsplit update reads the corner cells through its transverse terms).
 */
static void fill_padded_corners(const orc_grid *G, const double *a, double *p,
                                double sign_x, double sign_y) {
    int nx = G->nx, ny = G->ny;
    fill_padded(G, a, p, sign_x, sign_y);
    for (int j = -NG; j < ny + NG; j++) {
        if (j >= 0 && j < ny) continue;
        for (int k = 1; k <= NG; k++) {
            if (G->bc[0] == BC_WALL) p[pidx(G, -k, j)] = sign_x * p[pidx(G, k - 1, j)];
            else p[pidx(G, -k, j)] = p[pidx(G, 0, j)];
            if (G->bc[1] == BC_WALL) p[pidx(G, nx - 1 + k, j)] = sign_x * p[pidx(G, nx - k, j)];
            else p[pidx(G, nx - 1 + k, j)] = p[pidx(G, nx - 1, j)];
        }
    }
}

/*
 * Transverse splitting of a fluctuation a (edge frame: h, normal momentum,
 * tangential momentum) into its parts moving with negative (bm) and positive
 * (bp) speed along the tangential direction.  It uses the eigenstructure of
 * the tangential flux Jacobian at the edge's Roe state (uhat normal and vhat
 * tangential velocity, chat = sqrt(g hhat)): speeds vhat - chat, vhat,
 * vhat + chat with vectors (1, uhat, vhat - chat), (0, 1, 0),
 * (1, uhat, vhat + chat).  a = sum_p beta_p r_p; bm/bp = sum of
 * speed_p beta_p r_p over the negative/positive speeds.
 */
void orc_ctu_tsplit(double uhat, double vhat, double chat, const double a[3],
                    double bm[3], double bp[3]) {
    double mu[3] = {vhat - chat, vhat, vhat + chat};
    double r[3][3] = {{1.0, uhat, vhat - chat}, {0.0, 1.0, 0.0}, {1.0, uhat, vhat + chat}};
    double beta[3];
    beta[0] = ((vhat + chat) * a[0] - a[2]) / (2.0 * chat);
    beta[1] = a[1] - uhat * a[0];
    beta[2] = (a[2] - (vhat - chat) * a[0]) / (2.0 * chat);
    for (int m = 0; m < 3; m++) { bm[m] = 0.0; bp[m] = 0.0; }
    for (int p = 0; p < 3; p++) {
        double c = mu[p] * beta[p];
        for (int m = 0; m < 3; m++) {
            if (mu[p] < 0.0) bm[m] += c * r[p][m];
            else if (mu[p] > 0.0) bp[m] += c * r[p][m];
        }
    }
}

/* waves of the edge between padded cells a and b, in the frame of dir */
static void ctu_edge(const orc_grid *G, int dir, const double *ph, const double *pu,
                     const double *pv, const double *pB, size_t a, size_t b,
                     edge_waves *w) {
    if (dir == 0)
        fwd_riemann(G->g, ph[a], pu[a], pv[a], pB[a], ph[b], pu[b], pv[b], pB[b], w);
    else
        fwd_riemann(G->g, ph[a], pv[a], pu[a], pB[a], ph[b], pv[b], pu[b], pB[b], w);
}

/* padded index of cell (i, j) shifted by s along dir and by t across it */
static size_t ctu_at(const orc_grid *G, int dir, int i, int j, int s, int t) {
    return dir == 0 ? pidx(G, i + s, j + t) : pidx(G, i + t, j + s);
}

/*
 * For cell (i, j) and direction dir (0: x, 1: y), in dir's edge frame:
 * the fluctuations entering the cell through its low edge (ap_lo) and its
 * high edge (am_hi), and the low/high edge fluxes: the limited correction
 * minus k times the transverse parts, coming from the other direction, of
 * the four fluctuations that enter the cells beside the edge and move
 * towards it.  k = tw_scale * nu_other / 2.
 */
static void ctu_dir(const orc_grid *G, int dir, const double *ph, const double *pu,
                    const double *pv, const double *pB, int i, int j, double nu,
                    double k, double ap_lo[3], double am_hi[3], double F_lo[3],
                    double F_hi[3]) {
    int o = 1 - dir;   /* the other direction */
    edge_waves w[4];
    for (int e = 0; e < 4; e++)
        ctu_edge(G, dir, ph, pu, pv, pB, ctu_at(G, dir, i, j, e - 2, 0),
                 ctu_at(G, dir, i, j, e - 1, 0), &w[e]);
    double am_lo[3], ap_hi[3];
    edge_fluxes(3, &w[0], &w[1], &w[2], nu, G->order, am_lo, ap_lo, F_lo);
    edge_fluxes(3, &w[1], &w[2], &w[3], nu, G->order, am_hi, ap_hi, F_hi);
    /*
     * Fluctuations of the other direction's edges of the cells at offsets
     * s = -1, 0, +1 along dir (frame of o): the one entering the cell at s
     * through its low o-edge and the one entering through its high o-edge.
     * Their transverse split (along dir) uses the o-edge's Roe state; per
     * cell, P sums the parts moving in +dir (they reach the cell's high
     * dir-edge) and M the parts moving in -dir (its low dir-edge), each in
     * dir's frame (components 1 and 2 exchanged).  An edge's transverse term
     * is P of the cell below it plus M of the cell above it.
     */
    double P[3][3], M[3][3];
    for (int s = -1; s <= 1; s++) {
        edge_waves a[3];
        for (int e = 0; e < 3; e++)
            ctu_edge(G, o, ph, pu, pv, pB, ctu_at(G, dir, i, j, s, e - 1),
                     ctu_at(G, dir, i, j, s, e), &a[e]);
        double amL[3], apL[3], FL[3], amH[3], apH[3], FH[3];
        edge_fluxes(3, &a[0], &a[0], &a[1], nu, 1, amL, apL, FL);   /* low o-edge */
        edge_fluxes(3, &a[1], &a[1], &a[2], nu, 1, amH, apH, FH);   /* high o-edge */
        double pm[2][3], pp[2][3];
        orc_ctu_tsplit(a[0].uhat, a[0].vhat, a[0].chat, apL, pm[0], pp[0]);
        orc_ctu_tsplit(a[1].uhat, a[1].vhat, a[1].chat, amH, pm[1], pp[1]);
        static const int sw[3] = {0, 2, 1};
        for (int m = 0; m < 3; m++) {
            P[s + 1][m] = pp[0][sw[m]] + pp[1][sw[m]];
            M[s + 1][m] = pm[0][sw[m]] + pm[1][sw[m]];
        }
    }
    double tr_lo[3], tr_hi[3];
    for (int m = 0; m < 3; m++) {
        tr_lo[m] = P[0][m] + M[1][m];
        tr_hi[m] = P[1][m] + M[2][m];
    }
    for (int m = 0; m < 3; m++) {
        F_lo[m] = F_lo[m] - k * tr_lo[m];
        F_hi[m] = F_hi[m] - k * tr_hi[m];
    }
}

/*
 * One unsplit forward step of size dt (2D), in place on (h, hu, hv).  Every
 * x- and y-edge Riemann problem is solved from Q^n; with nu_x = dt/dx and
 * nu_y = dt/dy,
 *   Q_ij += -nu_x (A+dQ_{i-1/2,j} + A-dQ_{i+1/2,j}) - nu_x (F_{i+1/2,j} - F_{i-1/2,j})
 *           -nu_y (B+dQ_{i,j-1/2} + B-dQ_{i,j+1/2}) - nu_y (G_{i,j+1/2} - G_{i,j-1/2})
 * where an edge flux is its MC-limited correction minus (nu_other / 2) times
 * the transverse parts of the fluctuations described at ctu_dir, e.g.
 *   G_{i,j-1/2} = C_{i,j-1/2} - (nu_x/2) [B+A+dQ_{i-1/2,j-1} + B+A-dQ_{i+1/2,j-1}
 *                                        + B-A+dQ_{i-1/2,j} + B-A-dQ_{i+1/2,j}].
 * The four transverse terms of an edge are summed as (the two from the cell
 * below) + (the two from the cell above), each pair low o-edge first.
 * Returns 0, or -5 on a non-positive or non-finite depth.
 */
int orc_fwd_step_ctu(const orc_grid *G, double *h, double *hu, double *hv,
                     const double *B, double dt) {
    int nx = G->nx, ny = G->ny;
    size_t n = (size_t)nx * ny;
    double *ph = padded(G), *pu = padded(G), *pv = padded(G), *pB = padded(G);
    fill_padded_corners(G, h, ph, 1.0, 1.0);
    fill_padded_corners(G, hu, pu, -1.0, 1.0);
    fill_padded_corners(G, hv, pv, 1.0, -1.0);
    fill_padded_corners(G, B, pB, 1.0, 1.0);
    double *nh = (double *)malloc(n * sizeof(double));
    double *nu_ = (double *)malloc(n * sizeof(double));
    double *nv = (double *)malloc(n * sizeof(double));
    double nux = dt / G->dx, nuy = dt / G->dy;
    double kx = G->tw_scale * (0.5 * nuy);   /* on F: transverse parts of y-fluctuations */
    double ky = G->tw_scale * (0.5 * nux);   /* on G: transverse parts of x-fluctuations */

#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++) {
        for (int i = 0; i < nx; i++) {
            size_t c = pidx(G, i, j);
            double apL[3], amR[3], FL[3], FR[3];
            double bpB[3], bmT[3], GB[3], GT[3];
            ctu_dir(G, 0, ph, pu, pv, pB, i, j, nux, kx, apL, amR, FL, FR);
            ctu_dir(G, 1, ph, pu, pv, pB, i, j, nuy, ky, bpB, bmT, GB, GT);
            double dx_[3], dy_[3];   /* x frame and y frame */
            for (int m = 0; m < 3; m++) {
                dx_[m] = -nux * (apL[m] + amR[m]) - nux * (FR[m] - FL[m]);
                dy_[m] = -nuy * (bpB[m] + bmT[m]) - nuy * (GT[m] - GB[m]);
            }
            size_t o = (size_t)j * nx + i;
            nh[o] = (ph[c] + dx_[0]) + dy_[0];
            nu_[o] = (pu[c] + dx_[1]) + dy_[2];
            nv[o] = (pv[c] + dx_[2]) + dy_[1];
        }
    }
    memcpy(h, nh, n * sizeof(double));
    memcpy(hu, nu_, n * sizeof(double));
    memcpy(hv, nv, n * sizeof(double));
    free(ph); free(pu); free(pv); free(pB); free(nh); free(nu_); free(nv);
    int bad = 0;
    for (size_t k = 0; k < n; k++)
        if (!(h[k] > 0.0) || !isfinite(hu[k]) || !isfinite(hv[k])) bad = 1;
    return bad ? -5 : 0;
}

/*
 * One forward step of size dt, in place on (h, hu, hv): in 1D a single
 * x-sweep; in 2D an x-sweep of the whole grid, then a y-sweep of the x-swept
 * state (dimensional splitting); with scheme 1 a 2D step is orc_fwd_step_ctu.
 * hv may be NULL for ndim == 1 (treated as zero and not written).  Returns 0, or -5 when a non-positive or
 * non-finite depth appears.
 */
int orc_fwd_step(const orc_grid *G, double *h, double *hu, double *hv,
                 const double *B, double dt) {
    size_t n = (size_t)G->nx * G->ny;
    if (G->ndim == 2 && G->scheme == 1 && hv) {
        if (G->wetdry) return -1;   /* the shore solver is defined for the split step */
        return orc_fwd_step_ctu(G, h, hu, hv, B, dt);
    }
    double *v = hv;
    if (!hv) v = (double *)calloc(n, sizeof(double));
    fwd_sweep(G, 0, h, hu, v, B, dt, NULL, NULL);
    if (G->ndim == 2) fwd_sweep(G, 1, h, hu, v, B, dt, NULL, NULL);
    int bad = 0;
    for (size_t k = 0; k < n; k++)
        if (!(G->wetdry ? h[k] >= 0.0 : h[k] > 0.0) || !isfinite(hu[k]) || !isfinite(v[k]))
            bad = 1;
    if (!hv) free(v);
    return bad ? -5 : 0;
}

/*
 * A 2D split forward step, as orc_fwd_step with scheme 0, that also returns
 * per cell the mass flux through its low and high x-edge (x-sweep, from Q^n)
 * and y-edge (y-sweep, from the x-swept state), as the cell's update uses
 * them: phi[0], phi[1] (x low, high) and phi[2], phi[3] (y low, high), n
 * values each.  The refluxing of the AMR glue takes its fluxes from here.
 */
int orc_fwd_step_flux(const orc_grid *G, double *h, double *hu, double *hv, const double *B,
                      double dt, double *phi_xlo, double *phi_xhi, double *phi_ylo,
                      double *phi_yhi) {
    size_t n = (size_t)G->nx * G->ny;
    if (G->ndim != 2 || G->scheme != 0) return -1;
    fwd_sweep(G, 0, h, hu, hv, B, dt, phi_xlo, phi_xhi);
    fwd_sweep(G, 1, h, hu, hv, B, dt, phi_ylo, phi_yhi);
    int bad = 0;
    for (size_t k = 0; k < n; k++)
        if (!(G->wetdry ? h[k] >= 0.0 : h[k] > 0.0) || !isfinite(hu[k]) || !isfinite(hv[k]))
            bad = 1;
    return bad ? -5 : 0;
}

/*
 * CFL number: max over cells of (|u|+c)/dx [and (|v|+c)/dy]; with dimensional
 * splitting each sweep is limited by its own Courant number.
 */
double orc_fwd_smax(const orc_grid *G, const double *h, const double *hu,
                    const double *hv) {
    double smax = 0.0;
    size_t n = (size_t)G->nx * G->ny;
    for (size_t k = 0; k < n; k++) {
        if (G->wetdry && !(h[k] > G->dry_tol)) continue;   /* dry: no waves */
        double c = sqrt(G->g * h[k]);
        double s = (fabs(hu[k] / h[k]) + c) / G->dx;
        if (G->ndim == 2) {
            double sy = (fabs(hv[k] / h[k]) + c) / G->dy;
            if (sy > s) s = sy;
        }
        if (s > smax) smax = s;
    }
    return smax;
}

/*
 * Run up to max_steps CFL-limited steps, stopping at t_end:
 * dt_n = min(cfl / smax(Q^n), t_end - t_n).  Updates *t; returns the number
 * of steps taken, or a negative status.
 */
long orc_fwd_run(const orc_grid *G, double *h, double *hu, double *hv,
                 const double *B, long max_steps, double t_end, double *t) {
    long k;
    for (k = 0; k < max_steps; k++) {
        if (!(*t < t_end)) break;
        double smax = orc_fwd_smax(G, h, hu, hv);
        double dt = G->cfl / smax;
        if (dt > t_end - *t) dt = t_end - *t;
        int rc = orc_fwd_step(G, h, hu, hv, B, dt);
        if (rc) return rc;
        *t = *t + dt;
    }
    return k;
}

/* ------------------------------------------------- linear forward (tests) */

/*
 * First-order wave-propagation sweep for q_t + A(x) q_x = 0 along x (dir 0,
 * components (eta, mu)) or the y analogue (dir 1, components (eta, gamma)),
 * A = [[0,1],[g hbar,0]] (Eq. SWE_Aq).  At an edge the jump (d_eta, d_m)
 * splits as a1 [1, -cL] + a2 [1, cR]; the left-going part moves at -cL, the
 * right-going at +cR.  Walls mirror with the normal momentum negated.
 */
static void lin_sweep(const orc_grid *G, int dir, double *eta, double *mu, double *gam,
                      const double *c) {
    (void)0;
    int nx = G->nx, ny = G->ny;
    size_t n = (size_t)nx * ny;
    double *pe = padded(G), *pm = padded(G), *pg = padded(G), *pc = padded(G);
    fill_padded(G, eta, pe, 1.0, 1.0);
    fill_padded(G, mu, pm, -1.0, 1.0);
    fill_padded(G, gam, pg, 1.0, -1.0);
    fill_padded(G, c, pc, 1.0, 1.0);
    double *ne = (double *)malloc(n * sizeof(double));
    double *nm = (double *)malloc(n * sizeof(double));
    double *ng = (double *)malloc(n * sizeof(double));
    double *pn = dir == 0 ? pm : pg;  /* normal component */
    for (int j = 0; j < ny; j++) {
        for (int i = 0; i < nx; i++) {
            size_t ci = pidx(G, i, j);
            size_t lo = dir == 0 ? pidx(G, i - 1, j) : pidx(G, i, j - 1);
            size_t hi = dir == 0 ? pidx(G, i + 1, j) : pidx(G, i, j + 1);
            double de = 0.0, dn = 0.0;
            {   /* edge below/left: right-going part enters the cell */
                double cL = pc[lo], cR = pc[ci];
                double dE = pe[ci] - pe[lo], dM = pn[ci] - pn[lo];
                double a2 = (dM + cL * dE) / (cL + cR);
                de -= G->lin_nu[dir] * (cR * a2);
                dn -= G->lin_nu[dir] * (cR * a2 * cR);
            }
            {   /* edge above/right: left-going part enters the cell */
                double cL = pc[ci], cR = pc[hi];
                double dE = pe[hi] - pe[ci], dM = pn[hi] - pn[ci];
                double a1 = (cR * dE - dM) / (cL + cR);
                de -= G->lin_nu[dir] * (-cL * a1);
                dn -= G->lin_nu[dir] * (-cL * a1 * (-cL));
            }
            size_t o = (size_t)j * nx + i;
            ne[o] = pe[ci] + de;
            if (dir == 0) { nm[o] = pm[ci] + dn; ng[o] = pg[ci]; }
            else { ng[o] = pg[ci] + dn; nm[o] = pm[ci]; }
        }
    }
    memcpy(eta, ne, n * sizeof(double));
    memcpy(mu, nm, n * sizeof(double));
    memcpy(gam, ng, n * sizeof(double));
    free(pe); free(pm); free(pg); free(pc); free(ne); free(nm); free(ng);
}

/* One linear step: x-sweep, then (2D) y-sweep.  Order 1 only. */
int orc_lin_step(const orc_grid *G0, double *eta, double *mu, double *gam,
                 const double *hbar, double dt) {
    orc_grid G = *G0;
    size_t n = (size_t)G.nx * G.ny;
    double *c = (double *)malloc(n * sizeof(double));
    for (size_t k = 0; k < n; k++) c[k] = sqrt(G.g * hbar[k]);
    double *gm = gam ? gam : (double *)calloc(n, sizeof(double));
    G.lin_nu[0] = dt / G.dx;
    G.lin_nu[1] = dt / G.dy;
    lin_sweep(&G, 0, eta, mu, gm, c);
    if (G.ndim == 2) lin_sweep(&G, 1, eta, mu, gm, c);
    if (!gam) free(gm);
    free(c);
    return 0;
}

/* ----------------------------------------------------------- adjoint step */

/*
 * Adjoint Riemann solve at an edge of the time-reversed adjoint
 * q~_t + F(q~, x)_x = 0, F = -A^T q~ = -(g hbar mu~, eta~) along the normal
 * direction (the tangential component has no flux).  The flux Jacobian has
 * eigenpairs (-c, [c, 1]) and (+c, [-c, 1]); with the left cell's left-going
 * and the right cell's right-going eigenvector the flux jump splits as
 *   dF = b1 [cL, 1] + b2 [-cR, 1].
 * Components here are (eta~, normal, tangential).
 */
static void adj_riemann(double g, double eL, double mL, double hbL,
                        double eR, double mR, double hbR, edge_waves *w) {
    double cL = sqrt(g * hbL), cR = sqrt(g * hbR);
    double FL1 = -(g * hbL * mL), FL2 = -eL;
    double FR1 = -(g * hbR * mR), FR2 = -eR;
    double dF1 = FR1 - FL1, dF2 = FR2 - FL2;
    double b1 = (dF1 + cR * dF2) / (cL + cR);
    double b2 = (cL * dF2 - dF1) / (cL + cR);
    w->s[0] = -cL; w->s[1] = cR; w->s[2] = 0.0;
    w->shore = 0;
    w->Z[0][0] = b1 * cL;  w->Z[0][1] = b1;  w->Z[0][2] = 0.0;
    w->Z[1][0] = -b2 * cR; w->Z[1][1] = b2;  w->Z[1][2] = 0.0;
    w->Z[2][0] = 0.0;      w->Z[2][1] = 0.0; w->Z[2][2] = 0.0;
}

/*
 * Adjoint waves at the edge between padded cells a (left) and b (right),
 * normal momentum array pm, with walls at wet/dry edges: a dry cell
 * (hbar <= dry_tol) is replaced by the mirror image of its wet neighbour
 * (same eta~ and hbar, normal momentum negated).  Both dry: no waves.
 * Returns 1 for a wet/dry edge (a wall), 0 otherwise.  A wall edge carries
 * no second-order correction, so nothing crosses it.
 */
static int adj_edge(const orc_grid *G, const double *pe, const double *pm,
                    const double *phb, size_t a, size_t b, edge_waves *w) {
    int dryL = !(phb[a] > G->dry_tol), dryR = !(phb[b] > G->dry_tol);
    if (dryL && dryR) { memset(w, 0, sizeof(*w)); return 1; }
    if (dryL) {
        adj_riemann(G->g, pe[b], -pm[b], phb[b], pe[b], pm[b], phb[b], w);
        return 1;
    }
    if (dryR) {
        adj_riemann(G->g, pe[a], pm[a], phb[a], pe[a], -pm[a], phb[a], w);
        return 1;
    }
    adj_riemann(G->g, pe[a], pm[a], phb[a], pe[b], pm[b], phb[b], w);
    return 0;
}

/*
 * One adjoint sweep along x (dir 0, components (eta~, mu~)) or y (dir 1,
 * (eta~, gamma~)), in place.  Dry cells are left unchanged.
 */
static void adj_sweep(const orc_grid *G, int dir, double *eta, double *mu, double *gam,
                      const double *hbar, double dt) {
    int nx = G->nx, ny = G->ny;
    size_t n = (size_t)nx * ny;
    double *pe = padded(G), *pm = padded(G), *pg = padded(G), *phb = padded(G);
    fill_padded(G, eta, pe, 1.0, 1.0);
    fill_padded(G, mu, pm, -1.0, 1.0);
    fill_padded(G, gam, pg, 1.0, -1.0);
    fill_padded(G, hbar, phb, 1.0, 1.0);
    double *ne = (double *)malloc(n * sizeof(double));
    double *nm = (double *)malloc(n * sizeof(double));
    double *ng = (double *)malloc(n * sizeof(double));
    double nu = dt / (dir == 0 ? G->dx : G->dy);
    const double *pn = dir == 0 ? pm : pg;

#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++) {
        for (int i = 0; i < nx; i++) {
            size_t ci = pidx(G, i, j);
            size_t o = (size_t)j * nx + i;
            ne[o] = pe[ci]; nm[o] = pm[ci]; ng[o] = pg[ci];
            if (!(phb[ci] > G->dry_tol)) continue;
            edge_waves w[4];
            int wall[4];
            for (int e = 0; e < 4; e++) {
                size_t a, b;
                if (dir == 0) { a = pidx(G, i - 2 + e, j); b = pidx(G, i - 1 + e, j); }
                else { a = pidx(G, i, j - 2 + e); b = pidx(G, i, j - 1 + e); }
                wall[e] = adj_edge(G, pe, pn, phb, a, b, &w[e]);
            }
            double amL[3], apL[3], FL[3], amR[3], apR[3], FR[3];
            edge_fluxes(2, &w[0], &w[1], &w[2], nu, wall[1] ? 1 : G->order, amL, apL, FL);
            edge_fluxes(2, &w[1], &w[2], &w[3], nu, wall[2] ? 1 : G->order, amR, apR, FR);
            double de = -nu * (apL[0] + amR[0]) - nu * (FR[0] - FL[0]);
            double dn = -nu * (apL[1] + amR[1]) - nu * (FR[1] - FL[1]);
            ne[o] = pe[ci] + de;
            if (dir == 0) nm[o] = pm[ci] + dn;
            else ng[o] = pg[ci] + dn;
        }
    }
    memcpy(eta, ne, n * sizeof(double));
    memcpy(mu, nm, n * sizeof(double));
    memcpy(gam, ng, n * sizeof(double));
    free(pe); free(pm); free(pg); free(phb); free(ne); free(nm); free(ng);
}

/*
 * One step of the time-reversed adjoint (Sec. 4) of size dt, in place on
 * (eta~, mu~, gamma~); hbar = max(-B, 0) of the adjoint grid.  2D: a y-sweep,
 * then an x-sweep (the reverse of the forward order).  gam may be NULL for
 * ndim == 1.
 */
int orc_adj_step(const orc_grid *G, double *eta, double *mu, double *gam,
                 const double *hbar, double dt) {
    size_t n = (size_t)G->nx * G->ny;
    double *gm = gam ? gam : (double *)calloc(n, sizeof(double));
    if (G->ndim == 2) adj_sweep(G, 1, eta, mu, gm, hbar, dt);
    adj_sweep(G, 0, eta, mu, gm, hbar, dt);
    if (!gam) free(gm);
    return 0;
}

/* Adjoint CFL number: max over wet cells of c/dx [and c/dy], c = sqrt(g hbar). */
double orc_adj_smax(const orc_grid *G, const double *hbar) {
    double smax = 0.0;
    size_t n = (size_t)G->nx * G->ny;
    for (size_t k = 0; k < n; k++) {
        if (!(hbar[k] > G->dry_tol)) continue;
        double c = sqrt(G->g * hbar[k]);
        double s = c / G->dx;
        if (G->ndim == 2 && c / G->dy > s) s = c / G->dy;
        if (s > smax) smax = s;
    }
    return smax;
}

/*
 * Solve the time-reversed adjoint from q~(0) = phi over [0, t_f] with a fixed
 * step dt = t_f / N, N = ceil(t_f * smax / cfl), saving a snapshot every
 * `every` steps and always the last one.  Snapshot k holds q^(tau_k) with
 * tau_k = t_f - (steps done) * dt (Sec. 4: q^(x, t_f - t) = q~(x, t)).
 * snaps: [max_snaps][ncomp][n] with ncomp = ndim + 1; tau: [max_snaps].
 * Returns the number of snapshots, or a negative status (-2 if max_snaps is
 * too small).  *n_steps receives N and *dt_out the step.
 */
long orc_adj_run(const orc_grid *G, const double *hbar, const double *phi,
                 double t_f, int every, long max_snaps, double *snaps,
                 double *tau, long *n_steps, double *dt_out) {
    size_t n = (size_t)G->nx * G->ny;
    int nc = G->ndim + 1;
    double smax = orc_adj_smax(G, hbar);
    long N = (long)ceil(t_f * smax / G->cfl);
#if ORC_PLANT == 4
    N = N + 1;
#endif
    if (N < 1) N = 1;
    double dt = t_f / (double)N;
    double *e = (double *)malloc(n * sizeof(double));
    double *m = (double *)malloc(n * sizeof(double));
    double *gm = (double *)calloc(n, sizeof(double));
    memcpy(e, phi, n * sizeof(double));
    memcpy(m, phi + n, n * sizeof(double));
    if (nc == 3) memcpy(gm, phi + 2 * n, n * sizeof(double));
    long k = 0;
    /* snapshot 0: tau = t_f */
    if (k >= max_snaps) { free(e); free(m); free(gm); return -2; }
    memcpy(snaps + (size_t)k * nc * n, e, n * sizeof(double));
    memcpy(snaps + (size_t)k * nc * n + n, m, n * sizeof(double));
    if (nc == 3) memcpy(snaps + (size_t)k * nc * n + 2 * n, gm, n * sizeof(double));
    tau[k++] = t_f;
    for (long s = 1; s <= N; s++) {
        orc_adj_step(G, e, m, nc == 3 ? gm : NULL, hbar, dt);
        if (s % every == 0 || s == N) {
            if (k >= max_snaps) { free(e); free(m); free(gm); return -2; }
            memcpy(snaps + (size_t)k * nc * n, e, n * sizeof(double));
            memcpy(snaps + (size_t)k * nc * n + n, m, n * sizeof(double));
            if (nc == 3) memcpy(snaps + (size_t)k * nc * n + 2 * n, gm, n * sizeof(double));
#if ORC_PLANT == 5
            tau[k++] = t_f - (double)(s - every) * dt;
#else
            tau[k++] = t_f - (double)s * dt;
#endif
        }
    }
    free(e); free(m); free(gm);
    if (n_steps) *n_steps = N;
    if (dt_out) *dt_out = dt;
    return k;
}

/* ------------------------------------------------------------------ flag */

/*
 * Bilinear interpolation stencil of point (x, y) on the cell centres of grid
 * A, the coordinate clamped to the outermost centres.  Returns the four cell
 * indices and weights (1D: two, the others weight 0).
 */
static void bilinear(const orc_grid *A, double x, double y, size_t idx[4],
                     double w[4]) {
    double fx = (x - A->x_lo) / A->dx - 0.5;
    if (fx < 0.0) fx = 0.0;
    if (fx > (double)(A->nx - 1)) fx = (double)(A->nx - 1);
    int i0 = (int)floor(fx);
    if (i0 > A->nx - 2) i0 = A->nx - 2;
    if (i0 < 0) i0 = 0;
    double ax = fx - (double)i0;
    int i1 = (A->nx > 1) ? i0 + 1 : i0;
    if (A->nx == 1) ax = 0.0;
    if (A->ndim == 1) {
        idx[0] = (size_t)i0; idx[1] = (size_t)i1; idx[2] = 0; idx[3] = 0;
        w[0] = 1.0 - ax; w[1] = ax; w[2] = 0.0; w[3] = 0.0;
        return;
    }
    double fy = (y - A->y_lo) / A->dy - 0.5;
    if (fy < 0.0) fy = 0.0;
    if (fy > (double)(A->ny - 1)) fy = (double)(A->ny - 1);
    int j0 = (int)floor(fy);
    if (j0 > A->ny - 2) j0 = A->ny - 2;
    if (j0 < 0) j0 = 0;
    double ay = fy - (double)j0;
    int j1 = (A->ny > 1) ? j0 + 1 : j0;
    if (A->ny == 1) ay = 0.0;
    idx[0] = (size_t)j0 * A->nx + i0; w[0] = (1.0 - ax) * (1.0 - ay);
    idx[1] = (size_t)j0 * A->nx + i1; w[1] = ax * (1.0 - ay);
    idx[2] = (size_t)j1 * A->nx + i0; w[2] = (1.0 - ax) * ay;
    idx[3] = (size_t)j1 * A->nx + i1; w[3] = ax * ay;
}

/*
 * Adjoint-weighted flagging of the forward state (h, hu, hv, B) at time t.
 * snaps [K][ncomp][n_adj] with tau strictly decreasing (tau[0] = latest).
 * Window (Eq. ip_timerange, read with tau running from t up to
 * T = min(t + t_f - t_s, t_f)), clipped to [tau[K-1], tau[0]]:
 *   INTERP : q^(tau) linear in tau between snapshots; the maximum of
 *            |q^(tau).q| over the window of this piecewise-linear function is
 *            taken at the window ends or at snapshot times inside it.
 *   BRACKET: max over the snapshots from the latest one at or before t to the
 *            earliest one at or after T (Eq. ip_timepoint when t_s = t_f).
 * q = (eta = h + B, hu, hv); m = 0 where the forward cell is dry or any
 * weighted adjoint stencil cell is dry.  flags[i] = (m >= tol).  m_out may be
 * NULL.  Returns the number of flagged cells.
 */
long orc_flag(const orc_grid *F, const double *h, const double *hu,
              const double *hv, const double *B, double t,
              const orc_grid *A, const double *hbar_adj, const double *snaps,
              const double *tau, long K, double t_s, double t_f, double tol,
              int mode, uint8_t *flags, double *m_out) {
    size_t n = (size_t)F->nx * F->ny;
    size_t na = (size_t)A->nx * A->ny;
    int nc = A->ndim + 1;
    long count = 0;
    /* t + (t_f - t_s): the window length is added to t, so that T >= t holds
       exactly whenever t_s <= t_f (t_s = t_f gives the single time t) */
    double T = t + (t_f - t_s);
    if (T > t_f) T = t_f;
    double lo = t, hi = T;
    if (lo < tau[K - 1]) lo = tau[K - 1];
    if (hi > tau[0]) hi = tau[0];
    int empty = (K < 1) || (lo > hi) || (t > t_f);
    /* cells are independent: rows are shared out among threads */
#pragma omp parallel for schedule(static) reduction(+ : count)
    for (int j = 0; j < F->ny; j++) {
        for (int i = 0; i < F->nx; i++) {
            size_t o = (size_t)j * F->nx + i;
            double m = 0.0;
            double q[3];
            q[0] = h[o] + B[o];
            q[1] = hu[o];
            q[2] = (F->ndim == 2 && hv) ? hv[o] : 0.0;
            int dry = !(h[o] > F->dry_tol);
            double x = F->x_lo + ((double)i + 0.5) * F->dx;
            double y = F->y_lo + ((double)j + 0.5) * F->dy;
            size_t st[4];
            double w[4];
            bilinear(A, x, y, st, w);
            for (int c = 0; c < 4; c++)
                if (w[c] > 0.0 && !(hbar_adj[st[c]] > A->dry_tol)) dry = 1;
            if (!empty && !dry) {
                /* qhat_k . q at every snapshot, interpolated in space first */
                double *d = (double *)malloc((size_t)K * sizeof(double));
                for (long k = 0; k < K; k++) {
                    double qh[3] = {0.0, 0.0, 0.0};
                    for (int comp = 0; comp < nc; comp++) {
                        const double *s = snaps + ((size_t)k * nc + comp) * na;
                        double v = 0.0;
                        for (int c = 0; c < 4; c++) v += w[c] * s[st[c]];
                        qh[comp] = v;
                    }
                    if (A->ndim == 1) d[k] = qh[0] * q[0] + qh[1] * q[1];
                    else d[k] = qh[0] * q[0] + qh[1] * q[1] + qh[2] * q[2];
                }
                if (mode == FLAG_BRACKET) {
                    /* latest snapshot with tau <= lo, earliest with tau >= hi */
                    long kb = K - 1, ke = 0;
                    for (long k = 0; k < K; k++) if (tau[k] <= lo) { kb = k; break; }
                    for (long k = K - 1; k >= 0; k--) if (tau[k] >= hi) { ke = k; break; }
                    for (long k = ke; k <= kb; k++)
                        if (fabs(d[k]) > m) m = fabs(d[k]);
                } else {
                    /* value of the time interpolant at lo and at hi */
                    double ends[2] = {lo, hi};
                    for (int e = 0; e < 2; e++) {
                        double s = ends[e];
                        long k = 0;
                        while (k + 1 < K && tau[k + 1] > s) k++;
                        /* tau[k] >= s >= tau[k+1] (or k == K-1) */
                        double v;
                        if (k + 1 >= K || tau[k] == s) v = d[k];
                        else {
                            double a = (s - tau[k + 1]) / (tau[k] - tau[k + 1]);
                            /* interpolate the components, then dot */
                            double qh[3];
                            for (int comp = 0; comp < 3; comp++) qh[comp] = 0.0;
                            for (int comp = 0; comp < nc; comp++) {
                                const double *s0 = snaps + ((size_t)k * nc + comp) * na;
                                const double *s1 = snaps + ((size_t)(k + 1) * nc + comp) * na;
                                double v0 = 0.0, v1 = 0.0;
                                for (int c = 0; c < 4; c++) {
                                    v0 += w[c] * s0[st[c]];
                                    v1 += w[c] * s1[st[c]];
                                }
                                qh[comp] = a * v0 + (1.0 - a) * v1;
                            }
                            v = qh[0] * q[0] + qh[1] * q[1] + qh[2] * q[2];
                        }
                        if (fabs(v) > m) m = fabs(v);
                    }
                    for (long k = 0; k < K; k++)
                        if (tau[k] > lo && tau[k] < hi && fabs(d[k]) > m) m = fabs(d[k]);
                }
                free(d);
            }
            if (m_out) m_out[o] = m;
            uint8_t f = (!empty && !dry && m >= tol) ? 1 : 0;
            flags[o] = f;
            count += f;
        }
    }
    return count;
}

/*
 * Surface flagging (the default refinement criterion the paper compares
 * against, Sec. 6): flag a wet cell when its surface elevation relative to sea
 * level exceeds the tolerance, |eta| > tol, eta = h + B.  Returns the count.
 */
long orc_flag_surface(const orc_grid *G, const double *h, const double *B, double tol,
                      uint8_t *flags) {
    size_t n = (size_t)G->nx * G->ny;
    long count = 0;
    for (size_t k = 0; k < n; k++) {
        double eta = h[k] + B[k];
        uint8_t f = (h[k] > G->dry_tol && fabs(eta) > tol) ? 1 : 0;
        flags[k] = f;
        count += f;
    }
    return count;
}

/* Gauges: eta = h + B at (x, y) by bilinear interpolation of cell centres. */
void orc_gauge(const orc_grid *G, const double *h, const double *B, long ng,
               const double *xy, double *out) {
    for (long k = 0; k < ng; k++) {
        size_t st[4];
        double w[4];
        bilinear(G, xy[2 * k], xy[2 * k + 1], st, w);
        double v = 0.0;
        for (int c = 0; c < 4; c++) v += w[c] * (h[st[c]] + B[st[c]]);
        out[k] = v;
    }
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
