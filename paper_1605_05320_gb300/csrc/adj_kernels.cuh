// adj_kernels.cuh -- time-reversed linear adjoint step (Sec. 4, Sec. 5).
//
// q~ = (eta~, mu~, gamma~) solves q~_t + F_x + G_y = 0 with F = -A_1^T q~ =
// -(g hbar mu~, eta~, 0) and G = -A_2^T q~ = -(g hbar gamma~, 0, eta~), the
// transposed linearisation about the ocean at rest run forward in reversed
// time (q^(x, t_f - t) = q~(x, t)).  At an edge the flux jump splits along
// the left cell's left-going eigenvector [cL, 1] (speed -cL) and the right
// cell's right-going one [-cR, 1] (speed +cR), c = sqrt(g hbar): an f-wave
// form for spatially varying coefficients.  A wet/dry edge is a wall (zero
// normal velocity, Sec. 5): the dry side is the mirror of the wet one, and
// the edge carries no second-order correction.
#pragma once
#include "adj.cuh"

namespace swadj {

// Division: IEEE in double (the FP64 path rounds like the reference), a
// fast reciprocal-multiply in float.
__device__ __forceinline__ double adj_div(double a, double b) { return a / b; }
__device__ __forceinline__ float adj_div(float a, float b) { return __fdividef(a, b); }

template <typename R>
struct AdjWave {
    R b1, b2, cL, cR;
    int wall;
};

// Waves at the edge between (eL, mL, cL, ghL) and (eR, mR, cR, ghR), normal
// component m, c = sqrt(g hbar), gh = g hbar (c = 0 marks a dry cell).
template <typename R>
__device__ __forceinline__ AdjWave<R> adj_riemann(R eL, R mL, R cL, R ghL, R eR,
                                                  R mR, R cR, R ghR) {
    AdjWave<R> w;
    const bool dL = !(cL > R(0)), dR = !(cR > R(0));
    w.wall = (dL || dR) ? 1 : 0;
    if (dL && dR) { w.b1 = R(0); w.b2 = R(0); w.cL = R(0); w.cR = R(0); return w; }
    if (dL) { eL = eR; mL = -mR; cL = cR; ghL = ghR; }
    if (dR) { eR = eL; mR = -mL; cR = cL; ghR = ghL; }
    const R F1L = -(ghL * mL), F2L = -eL;
    const R F1R = -(ghR * mR), F2R = -eR;
    const R d1 = F1R - F1L, d2 = F2R - F2L;
    const R s = cL + cR;
    w.b1 = adj_div(d1 + cR * d2, s);
    w.b2 = adj_div(cL * d2 - d1, s);
    w.cL = cL;
    w.cR = cR;
    return w;
}

// Fluctuations and correction at edge w with neighbours wm (left), wp (right).
// Wave 1: Z = b1 (cL, 1), speed -cL (to the left cell);
// wave 2: Z = b2 (-cR, 1), speed +cR (to the right cell).
template <typename R>
__device__ __forceinline__ void adj_flux(const AdjWave<R> &wm, const AdjWave<R> &w,
                                         const AdjWave<R> &wp, R nu, int order,
                                         R am[2], R ap[2], R F[2]) {
    const R Z1[2] = {w.b1 * w.cL, w.b1};
    const R Z2[2] = {-w.b2 * w.cR, w.b2};
    am[0] = Z1[0]; am[1] = Z1[1];
    ap[0] = Z2[0]; ap[1] = Z2[1];
    F[0] = R(0); F[1] = R(0);
    if (order < 2 || w.wall) return;
    {   // wave 1, upwind edge to the right
        const R U[2] = {wp.b1 * wp.cL, wp.b1};
        const R zz = Z1[0] * Z1[0] + Z1[1] * Z1[1];
        R th = R(0);
        if (zz != R(0)) th = adj_div(U[0] * Z1[0] + U[1] * Z1[1], zz);
        const R coef = R(0.5) * R(-1) * (R(1) - nu * w.cL) * mc_phi(th);
        F[0] += coef * Z1[0];
        F[1] += coef * Z1[1];
    }
    {   // wave 2, upwind edge to the left
        const R U[2] = {-wm.b2 * wm.cR, wm.b2};
        const R zz = Z2[0] * Z2[0] + Z2[1] * Z2[1];
        R th = R(0);
        if (zz != R(0)) th = adj_div(U[0] * Z2[0] + U[1] * Z2[1], zz);
        const R coef = R(0.5) * (R(1) - nu * w.cR) * mc_phi(th);
        F[0] += coef * Z2[0];
        F[1] += coef * Z2[1];
    }
}

// One adjoint step of a TX x TY tile, dimensionally split in the reverse of
// the forward order: a y-sweep of every staged column, then an x-sweep of the
// y-swept state.  The tile and a 2-cell halo with corners are staged; the
// x-halo columns of the y-swept state come from y-sweeping index-mapped
// columns (the tangential component mu~ is passive in the y-sweep, so this is
// exactly the copy/mirror of the y-swept interior).  With walls the two
// sweeps are the transposes of the linear forward sweeps.
template <typename R, bool TWO_D, int TX, int TY>
__global__ void __launch_bounds__(TX *TY) adj_step_kernel(AdjParams<R> p) {
    constexpr int HX = 2, HY = TWO_D ? 2 : 0;
    constexpr int RX = TX + 2 * HX, RY = TY + 2 * HY;
    constexpr int NT = TX * TY;
    constexpr int NEX = RX - 1;
    constexpr int NEY = TWO_D ? RY - 1 : 1;
    __shared__ R s_e[RY][RX], s_m[RY][RX], s_g[RY][RX], s_c[RY][RX], s_gh[RY][RX];
    __shared__ union WaveBuf {
        AdjWave<R> y[NEY][RX];
        AdjWave<R> x[TY][NEX];
    } wb;

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = tx + ty * TX;
    const int nx = p.nx, ny = p.ny;
    const int i0 = blockIdx.x * TX - HX, j0 = blockIdx.y * TY - HY;

    for (int r = tid; r < RX * RY; r += NT) {
        const int ry = r / RX, rx = r - ry * RX;
        bool fx, fy = false;
        const int ci = ghost_index(i0 + rx, nx, p.bc.lo_x, p.bc.hi_x, &fx);
        int cj = 0;
        if (TWO_D) cj = ghost_index(j0 + ry, ny, p.bc.lo_y, p.bc.hi_y, &fy);
        const size_t o = (size_t)cj * nx + ci;
        R m = p.src[1][o], g = TWO_D ? p.src[2][o] : R(0);
        if (fx) m = -m;
        if (fy) g = -g;
        s_e[ry][rx] = p.src[0][o];
        s_m[ry][rx] = m;
        s_g[ry][rx] = g;
        // double: the coefficient array holds hbar (c and g hbar derived here,
        // rounding as in the reference); float: it holds c (g hbar = c c)
        const R a = p.c[o];
        R c, gh;
        if (sizeof(R) == 8) {
            if (a > p.dry_tol) { gh = p.g * a; c = sqrt(gh); }
            else { gh = R(0); c = R(0); }
        } else {
            c = a;
            gh = a * a;
        }
        s_c[ry][rx] = c;
        s_gh[ry][rx] = gh;
    }
    __syncthreads();

    if (TWO_D) {
        // y-edge waves of every staged column (edge k between rows k, k+1)
        for (int e = tid; e < NEY * RX; e += NT) {
            const int k = e / RX, rx = e - k * RX;
            wb.y[k][rx] = adj_riemann<R>(s_e[k][rx], s_g[k][rx], s_c[k][rx], s_gh[k][rx],
                                         s_e[k + 1][rx], s_g[k + 1][rx], s_c[k + 1][rx],
                                         s_gh[k + 1][rx]);
        }
        __syncthreads();
        // y-sweep of the tile rows in every staged column
        R ye[(TY * RX + NT - 1) / NT], yg[(TY * RX + NT - 1) / NT];
        int k = 0;
        for (int i = tid; i < TY * RX; i += NT, k++) {
            const int row = i / RX, rx = i - row * RX, ry = row + HY;
            ye[k] = s_e[ry][rx];
            yg[k] = s_g[ry][rx];
            if (s_c[ry][rx] > R(0)) {
                R bm0[2], bp0[2], G0[2], bm1[2], bp1[2], G1[2];
                adj_flux<R>(wb.y[ry - 2][rx], wb.y[ry - 1][rx], wb.y[ry][rx], p.nuy, p.order, bm0, bp0, G0);
                adj_flux<R>(wb.y[ry - 1][rx], wb.y[ry][rx], wb.y[ry + 1][rx], p.nuy, p.order, bm1, bp1, G1);
                const R de = -p.nuy * (bp0[0] + bm1[0]) - p.nuy * (G1[0] - G0[0]);
                const R dg = -p.nuy * (bp0[1] + bm1[1]) - p.nuy * (G1[1] - G0[1]);
                ye[k] = ye[k] + de;
                yg[k] = yg[k] + dg;
            }
        }
        __syncthreads();  // every y-wave read before the union is reused
        k = 0;
        for (int i = tid; i < TY * RX; i += NT, k++) {
            const int row = i / RX, rx = i - row * RX, ry = row + HY;
            s_e[ry][rx] = ye[k];
            s_g[ry][rx] = yg[k];
        }
        __syncthreads();
    }

    // x-edge waves of the (y-swept) tile rows
    for (int e = tid; e < TY * NEX; e += NT) {
        const int row = e / NEX, k = e - row * NEX, ry = row + HY;
        wb.x[row][k] = adj_riemann<R>(s_e[ry][k], s_m[ry][k], s_c[ry][k], s_gh[ry][k],
                                      s_e[ry][k + 1], s_m[ry][k + 1], s_c[ry][k + 1],
                                      s_gh[ry][k + 1]);
    }
    __syncthreads();

    const int gi = blockIdx.x * TX + tx, gj = blockIdx.y * TY + ty;
    if (gi >= nx || gj >= ny) return;
    const int cx = tx + HX, cy = ty + HY;
    R ne = s_e[cy][cx], nm = s_m[cy][cx], ng = s_g[cy][cx];
    if (s_c[cy][cx] > R(0)) {
        R am0[2], ap0[2], F0[2], am1[2], ap1[2], F1[2];
        adj_flux<R>(wb.x[ty][tx], wb.x[ty][tx + 1], wb.x[ty][tx + 2], p.nux, p.order, am0, ap0, F0);
        adj_flux<R>(wb.x[ty][tx + 1], wb.x[ty][tx + 2], wb.x[ty][tx + 3], p.nux, p.order, am1, ap1, F1);
        const R de = -p.nux * (ap0[0] + am1[0]) - p.nux * (F1[0] - F0[0]);
        const R dm = -p.nux * (ap0[1] + am1[1]) - p.nux * (F1[1] - F0[1]);
        ne = ne + de;
        nm = nm + dm;
    }
    const size_t o = (size_t)gj * nx + gi;
    p.dst[0][o] = ne;
    p.dst[1][o] = nm;
    if (TWO_D) p.dst[2][o] = ng;
    if (p.snap_f) {
        p.snap_f[o] = (float)ne;
        p.snap_f[p.snap_comp_stride + o] = (float)nm;
        if (TWO_D) p.snap_f[2 * p.snap_comp_stride + o] = (float)ng;
    } else if (p.snap_d) {
        p.snap_d[o] = (double)ne;
        p.snap_d[p.snap_comp_stride + o] = (double)nm;
        if (TWO_D) p.snap_d[2 * p.snap_comp_stride + o] = (double)ng;
    }
    if ((p.snap_f || p.snap_d) && o == 0) *p.tau_dev = p.tau_val;
}

}  // namespace swadj
