// fwd_kernels.cuh -- forward nonlinear shallow-water step (Eq. swe_1d / swe, Sec. 3, 5)
// with a Roe-type f-wave Riemann solve per edge (Sec. 6), fused ghost fill and
// fused CFL max-reduction (next time step computed on the device).
//
// Storage per precision:
//   double (SWA_FP64): q = (h, hu, hv), bath = B.  eta = h + B per cell.
//   float  (SWA_FP32): q = (eta, hu, hv), bath = hbar = -B (perturbation
//                      form: metre-scale eta is stored directly instead of as
//                      the small difference of ~4000 m depths).
#pragma once
#include "fwd.cuh"

namespace swadj {

// Roe f-wave decomposition at one edge in the edge's frame (normal, tangential).
// Inputs per side: depth h, normal/tangential momentum mn/mt, normal/tangential
// velocity un/ut, sqrt(h), surface eta.  The momentum jump carries the
// bathymetry source as g*hhat*(eta_R - eta_L): zero jump for the ocean at rest.
// Output: uhat, chat and the strengths b1 (speed uhat-chat, vector
// (1, s1, vhat)), b2 (speed uhat, (0,0,1)), b3 (speed uhat+chat, (1, s3, vhat)).
template <typename R>
__device__ __forceinline__ void fwave_roe(R g, R hL, R mnL, R mtL, R unL, R utL,
                                          R sqL, R etaL, R hR, R mnR, R mtR,
                                          R unR, R utR, R sqR, R etaR, R &uhat,
                                          R &chat, R &b1, R &b2, R &b3, R &vhat) {
    R hhat = R(0.5) * (hL + hR);
    R den = sqL + sqR;
    uhat = (sqL * unL + sqR * unR) / den;
    vhat = (sqL * utL + sqR * utR) / den;
    chat = sqrt(g * hhat);
    R s1 = uhat - chat, s3 = uhat + chat;
    R df1 = mnR - mnL;
    R df2 = (mnR * unR - mnL * unL) + g * hhat * (etaR - etaL);
    R df3 = mnR * utR - mnL * utL;
    R w = s3 - s1;
    b1 = (s3 * df1 - df2) / w;
    b3 = (df2 - s1 * df1) / w;
    b2 = df3 - vhat * df1;
}

// Shore solver (the wet/dry option; the reading of Sec. 6's solver, robust
// near shore and inundation and Roe away from it): at an edge with a dry
// cell (h <= dry_tol) or a transonic rarefaction (u - c or u + c rising
// through zero from the left cell to the right one) the fluctuations come
// from the hydrostatic reconstruction of Audusse et al. (2004) with an HLL
// flux, first order.  h*_L = max(0, eta_L - max(B_L, B_R)), h*_R likewise,
// cell velocities (zero in a dry cell), speeds s_L = min(u_L - c_L, u_R -
// c_R), s_R = max(u_L + c_L, u_R + c_R) over the reconstructed states;
//   amdq = F + (0, g/2 (h_L^2 - h*_L^2), 0) - f(Q_L),
//   apdq = f(Q_R) - F - (0, g/2 (h_R^2 - h*_R^2), 0),
// F the HLL flux of the reconstructed states, f the physical flux.  Every
// expression in the order of the FP64 reference solver.
template <typename R>
__device__ __forceinline__ bool shore_edge(R g, R tol, R hL, R mnL, R hR, R mnR) {
    if (!(hL > tol) || !(hR > tol)) return true;
    const R uL = mnL / hL, uR = mnR / hR;
    const R cL = sqrt(g * hL), cR = sqrt(g * hR);
    return (uL - cL < R(0) && uR - cR > R(0)) || (uL + cL < R(0) && uR + cR > R(0));
}

template <typename R>
__device__ __forceinline__ void shore_fluct(R g, R tol, R hL, R mnL, R mtL, R etaL, R BL,
                                            R hR, R mnR, R mtR, R etaR, R BR, R am[3],
                                            R ap[3]) {
    const R uL = hL > tol ? mnL / hL : R(0), vL = hL > tol ? mtL / hL : R(0);
    const R uR = hR > tol ? mnR / hR : R(0), vR = hR > tol ? mtR / hR : R(0);
    const R Bm = BL > BR ? BL : BR;
    R hLs = etaL - Bm, hRs = etaR - Bm;
    if (hLs < R(0)) hLs = R(0);
    if (hRs < R(0)) hRs = R(0);
    const R pL = R(0.5) * g * (hL * hL), pR = R(0.5) * g * (hR * hR);
    const R pLs = R(0.5) * g * (hLs * hLs), pRs = R(0.5) * g * (hRs * hRs);
    const R FL[3] = {hLs * uL, hLs * uL * uL + pLs, hLs * uL * vL};
    const R FR[3] = {hRs * uR, hRs * uR * uR + pRs, hRs * uR * vR};
    const R QL[3] = {hLs, hLs * uL, hLs * vL}, QR[3] = {hRs, hRs * uR, hRs * vR};
    R F[3] = {R(0), R(0), R(0)};
    if (hLs > R(0) || hRs > R(0)) {
        const R cL = sqrt(g * hLs), cR = sqrt(g * hRs);
        const R sL = uL - cL < uR - cR ? uL - cL : uR - cR;
        const R sR = uL + cL > uR + cR ? uL + cL : uR + cR;
        if (sL >= R(0)) {
#pragma unroll
            for (int m = 0; m < 3; m++) F[m] = FL[m];
        } else if (sR <= R(0)) {
#pragma unroll
            for (int m = 0; m < 3; m++) F[m] = FR[m];
        } else {
#pragma unroll
            for (int m = 0; m < 3; m++)
                F[m] = (sR * FL[m] - sL * FR[m] + sL * sR * (QR[m] - QL[m])) / (sR - sL);
        }
    }
    const R fL[3] = {mnL, mnL * uL + pL, mnL * vL}, fR[3] = {mnR, mnR * uR + pR, mnR * vR};
    const R SL[3] = {R(0), pL - pLs, R(0)}, SR[3] = {R(0), pR - pRs, R(0)};
#pragma unroll
    for (int m = 0; m < 3; m++) {
        am[m] = (F[m] + SL[m]) - fL[m];
        ap[m] = fR[m] - (F[m] + SR[m]);
    }
}

// Fluctuations amdq (to the left cell), apdq (to the right cell) and the
// second-order correction flux F at edge e, from the waves at e and at its
// left/right neighbour edges (indices into wave arrays W[6][stride]).
// CFL number of one FP32 cell, the same expression wherever the FP32 path
// reduces it: max((|hu|/h + c)/dx, (|hv|/h + c)/dy), c = sqrt(g h) (each
// sweep of the split step is limited by its own Courant number).
__device__ __forceinline__ float cfl_f32(float h, float hu, float hv, float g, float rdx,
                                         float rdy, int two_d) {
    // rounding fixed in the source (no compiler fusion), as in the step
    const float q = rsqrt_ftz(h), ih = __fmul_rn(q, q);
    const float gh = __fmul_rn(g, h), cc = __fmul_rn(gh, rsqrt_ftz(gh));
    float s = __fmul_rn(fmaf(fabsf(hu), ih, cc), rdx);
    if (two_d) s = fmaxf(s, __fmul_rn(fmaf(fabsf(hv), ih, cc), rdy));
    return s;
}

template <typename R>
struct Wave6 {
    R uh, ch, b1, b2, b3, vh;
};

template <typename R>
__device__ __forceinline__ void wave_vec(const Wave6<R> &w, int p, R Z[3], R &s) {
    if (p == 0) {
        s = w.uh - w.ch;
        Z[0] = w.b1; Z[1] = w.b1 * s; Z[2] = w.b1 * w.vh;
    } else if (p == 1) {
        s = w.uh;
        Z[0] = R(0); Z[1] = R(0); Z[2] = w.b2;
    } else {
        s = w.uh + w.ch;
        Z[0] = w.b3; Z[1] = w.b3 * s; Z[2] = w.b3 * w.vh;
    }
}

template <typename R>
__device__ __forceinline__ void edge_flux(const Wave6<R> &wm, const Wave6<R> &w,
                                          const Wave6<R> &wp, R nu, int order,
                                          R am[3], R ap[3], R F[3]) {
#pragma unroll
    for (int m = 0; m < 3; m++) { am[m] = R(0); ap[m] = R(0); F[m] = R(0); }
#pragma unroll
    for (int p = 0; p < 3; p++) {
        R Z[3], s;
        wave_vec(w, p, Z, s);
#pragma unroll
        for (int m = 0; m < 3; m++) {
            if (s < R(0)) am[m] += Z[m];
            else if (s > R(0)) ap[m] += Z[m];
            else { am[m] += R(0.5) * Z[m]; ap[m] += R(0.5) * Z[m]; }
        }
        if (order >= 2) {
            R Zu[3], su;
            wave_vec(s > R(0) ? wm : wp, p, Zu, su);
            R zz = Z[0] * Z[0] + Z[1] * Z[1] + Z[2] * Z[2];
            R theta = R(0);
            if (zz != R(0)) theta = (Zu[0] * Z[0] + Zu[1] * Z[1] + Zu[2] * Z[2]) / zz;
            R coef = R(0.5) * sgnr(s) * (R(1) - nu * fabs(s)) * mc_phi(theta);
#pragma unroll
            for (int m = 0; m < 3; m++) F[m] += coef * Z[m];
        }
    }
}

// One forward step of a TX x TY tile, dimensionally split (x-sweep of every
// row, then y-sweep of the x-swept state).  The tile and a 2-cell halo
// *including corners* are staged: the y-sweep of the tile needs the x-swept
// state in its two halo rows, and x-sweeping a halo row needs its corner
// cells.  Halo rows outside the grid come from index mapping, so their
// x-sweep equals the x-sweep of the mirrored/copied interior row, which is
// what ghost cells of the x-swept state hold.  Expressions follow the FP64
// reference in order, so with contraction disabled the rounding matches it.
// WD: the wet/dry option (shore solver at dry and transonic edges, a cell
// at or below dry_tol keeps no momentum and no negative depth after each
// sweep, dry cells carry no waves in the CFL number).
template <typename R, bool PERT, bool TWO_D, int TX, int TY, bool WD = false>
__global__ void __launch_bounds__(TX *TY)
fwd_step_kernel(FwdParams<R> p) {
    constexpr int HX = 2, HY = TWO_D ? 2 : 0;
    constexpr int RX = TX + 2 * HX, RY = TY + 2 * HY;
    constexpr int NT = TX * TY;
    constexpr int NEX = RX - 1;
    constexpr int NEY = TWO_D ? RY - 1 : 1;
    constexpr int WYC = TWO_D ? TX : 1;
    __shared__ R s_h[RY][RX], s_mu[RY][RX], s_mv[RY][RX], s_eta[RY][RX];
    __shared__ R s_u[RY][RX], s_v[RY][RX], s_sq[RY][RX], s_b[RY][RX];
    __shared__ union WaveBuf {
        Wave6<R> x[RY][NEX];
        Wave6<R> y[NEY][WYC];
    } wb;
    __shared__ double red[32];
    __shared__ int am_last;

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = tx + ty * TX;
    volatile DevClock *clk = p.clk;
    const double t = clk->t;
    double dt = clk->dt_cfl;
    if (p.t_end - t < dt) dt = p.t_end - t;
    if (!(dt > 0.0)) return;  // clock already at t_end: no-op step
    const int cur = clk->cur;
    if (p.gauges.n > 0 && blockIdx.x == 0 && blockIdx.y == 0)   // the state this step starts from
        record_gauges<R, NT>(p.gauges, p.q[cur][0], p.bath, p.nx, p.ny, p.two_d, t);

    const R *q0 = p.q[cur][0], *q1 = p.q[cur][1], *q2 = p.q[cur][2];
    R *o0 = p.q[cur ^ 1][0], *o1 = p.q[cur ^ 1][1], *o2 = p.q[cur ^ 1][2];
    const int nx = p.nx, ny = p.ny;
    const int i0 = blockIdx.x * TX - HX, j0 = blockIdx.y * TY - HY;
    const R tol = p.dry_tol;

    // 1) tile + halo with corners into shared memory, ghost cells by mapping
    for (int r = tid; r < RX * RY; r += NT) {
        const int ry = r / RX, rx = r - ry * RX;
        bool fx, fy = false;
        const int ci = ghost_index(i0 + rx, nx, p.bc.lo_x, p.bc.hi_x, &fx);
        int cj = 0;
        if (TWO_D) cj = ghost_index(j0 + ry, ny, p.bc.lo_y, p.bc.hi_y, &fy);
        const size_t o = (size_t)cj * nx + ci;
        R a = q0[o], mu = q1[o], mv = TWO_D ? q2[o] : R(0), b = p.bath[o];
        if (fx) mu = -mu;
        if (fy) mv = -mv;
        R h, eta;
        if (PERT) { eta = a; h = a + b; }
        else { h = a; eta = a + b; }
        s_h[ry][rx] = h;
        s_mu[ry][rx] = mu;
        s_mv[ry][rx] = mv;
        s_eta[ry][rx] = eta;
        const bool wet = !WD || h > tol;
        s_u[ry][rx] = wet ? mu / h : R(0);
        s_v[ry][rx] = wet ? mv / h : R(0);
        s_sq[ry][rx] = sqrt(h);
        s_b[ry][rx] = b;
    }
    __syncthreads();
    // bottom elevation of a staged cell (the shore solver's reconstruction)
    auto bot = [&](int ry, int rx) { return PERT ? -s_b[ry][rx] : s_b[ry][rx]; };

    // 2) x-edge waves of every staged row
    for (int e = tid; e < RY * NEX; e += NT) {
        const int ry = e / NEX, k = e - ry * NEX;
        Wave6<R> w;
        if (WD && shore_edge<R>(p.g, tol, s_h[ry][k], s_mu[ry][k], s_h[ry][k + 1],
                                s_mu[ry][k + 1])) {
            // a shore edge: no waves for the neighbours' limiters (ch < 0 marks it)
            w.uh = R(0); w.ch = R(-1); w.b1 = R(0); w.b2 = R(0); w.b3 = R(0); w.vh = R(0);
        } else {
            fwave_roe<R>(p.g, s_h[ry][k], s_mu[ry][k], s_mv[ry][k], s_u[ry][k],
                         s_v[ry][k], s_sq[ry][k], s_eta[ry][k], s_h[ry][k + 1],
                         s_mu[ry][k + 1], s_mv[ry][k + 1], s_u[ry][k + 1],
                         s_v[ry][k + 1], s_sq[ry][k + 1], s_eta[ry][k + 1], w.uh,
                         w.ch, w.b1, w.b2, w.b3, w.vh);
        }
        wb.x[ry][k] = w;
    }
    __syncthreads();

    // 3) x-sweep of the tile's columns in every staged row (in place)
    const R nux = R(dt) / p.dx;
    R xs[3][(RY + TY - 1) / TY];
    int nrow = 0;
    for (int ry = ty; ry < RY; ry += TY) {
        const int cx = tx + HX;
        R am0[3], ap0[3], F0[3], am1[3], ap1[3], F1[3];
        // edge k of a staged row joins cells k and k + 1
        auto xedge = [&](int k, R am[3], R ap[3], R F[3]) {
            if (WD && wb.x[ry][k].ch < R(0)) {
                shore_fluct<R>(p.g, tol, s_h[ry][k], s_mu[ry][k], s_mv[ry][k], s_eta[ry][k],
                               bot(ry, k), s_h[ry][k + 1], s_mu[ry][k + 1], s_mv[ry][k + 1],
                               s_eta[ry][k + 1], bot(ry, k + 1), am, ap);
#pragma unroll
                for (int m = 0; m < 3; m++) F[m] = R(0);
            } else {
                edge_flux<R>(wb.x[ry][k - 1], wb.x[ry][k], wb.x[ry][k + 1], nux, p.order, am,
                             ap, F);
            }
        };
        xedge(tx + 1, am0, ap0, F0);
        xedge(tx + 2, am1, ap1, F1);
        R dq[3];
#pragma unroll
        for (int m = 0; m < 3; m++) dq[m] = -nux * (ap0[m] + am1[m]) - nux * (F1[m] - F0[m]);
        const R a0 = PERT ? s_eta[ry][cx] : s_h[ry][cx];
        xs[0][nrow] = a0 + dq[0];
        xs[1][nrow] = s_mu[ry][cx] + dq[1];
        xs[2][nrow] = s_mv[ry][cx] + dq[2];
        nrow++;
    }
    __syncthreads();  // all x-waves read; the cell arrays now take the x-swept state
    {
        int k = 0;
        for (int ry = ty; ry < RY; ry += TY) {
            const int cx = tx + HX;
            R h, eta;
            if (PERT) {
                eta = xs[0][k];
                h = eta + s_b[ry][cx];
            } else {
                h = xs[0][k];
                eta = h + s_b[ry][cx];
            }
            R mu = xs[1][k], mv = xs[2][k];
            k++;
            if (WD && !(h > tol)) {   // a dry cell keeps no momentum, no negative depth
                if (h < R(0)) {
                    h = R(0);
                    eta = PERT ? -s_b[ry][cx] : s_b[ry][cx];
                }
                mu = R(0);
                mv = R(0);
            }
            if (!TWO_D) {  // 1D: the x-swept state is the new state
                s_h[ry][cx] = h; s_eta[ry][cx] = eta; s_mu[ry][cx] = mu; s_mv[ry][cx] = mv;
                continue;
            }
            s_h[ry][cx] = h;
            s_mu[ry][cx] = mu;
            s_mv[ry][cx] = mv;
            s_eta[ry][cx] = eta;
            const bool wet = !WD || h > tol;
            s_u[ry][cx] = wet ? mu / h : R(0);
            s_v[ry][cx] = wet ? mv / h : R(0);
            s_sq[ry][cx] = sqrt(h);
        }
    }
    __syncthreads();

    const int gi = blockIdx.x * TX + tx, gj = blockIdx.y * TY + ty;
    const bool valid = gi < nx && gj < ny;
    const int cx = tx + HX, cy = ty + HY;
    R n0, n1, n2;
    if (TWO_D) {
        // 4) y-edge waves of the x-swept state, tile columns
        for (int e = tid; e < NEY * TX; e += NT) {
            const int k = e / TX, col = e - k * TX, rx = col + HX;
            Wave6<R> w;
            if (WD && shore_edge<R>(p.g, tol, s_h[k][rx], s_mv[k][rx], s_h[k + 1][rx],
                                    s_mv[k + 1][rx])) {
                w.uh = R(0); w.ch = R(-1); w.b1 = R(0); w.b2 = R(0); w.b3 = R(0); w.vh = R(0);
            } else {
                fwave_roe<R>(p.g, s_h[k][rx], s_mv[k][rx], s_mu[k][rx], s_v[k][rx],
                             s_u[k][rx], s_sq[k][rx], s_eta[k][rx], s_h[k + 1][rx],
                             s_mv[k + 1][rx], s_mu[k + 1][rx], s_v[k + 1][rx],
                             s_u[k + 1][rx], s_sq[k + 1][rx], s_eta[k + 1][rx], w.uh,
                             w.ch, w.b1, w.b2, w.b3, w.vh);
            }
            wb.y[k][col] = w;
        }
        __syncthreads();
        // 5) y-sweep (edge frame (h, hv, hu))
        const R nuy = R(dt) / p.dy;
        R bm0[3], bp0[3], G0[3], bm1[3], bp1[3], G1[3];
        // y-edge k of the tile column joins staged rows k and k + 1
        auto yedge = [&](int k, R am[3], R ap[3], R F[3]) {
            if (WD && wb.y[k][tx].ch < R(0)) {
                shore_fluct<R>(p.g, tol, s_h[k][cx], s_mv[k][cx], s_mu[k][cx], s_eta[k][cx],
                               bot(k, cx), s_h[k + 1][cx], s_mv[k + 1][cx], s_mu[k + 1][cx],
                               s_eta[k + 1][cx], bot(k + 1, cx), am, ap);
#pragma unroll
                for (int m = 0; m < 3; m++) F[m] = R(0);
            } else {
                edge_flux<R>(wb.y[k - 1][tx], wb.y[k][tx], wb.y[k + 1][tx], nuy, p.order, am, ap,
                             F);
            }
        };
        yedge(ty + 1, bm0, bp0, G0);
        yedge(ty + 2, bm1, bp1, G1);
        R d[3];
#pragma unroll
        for (int m = 0; m < 3; m++) d[m] = -nuy * (bp0[m] + bm1[m]) - nuy * (G1[m] - G0[m]);
        const R a0 = PERT ? s_eta[cy][cx] : s_h[cy][cx];
        n0 = a0 + d[0];
        n2 = s_mv[cy][cx] + d[1];
        n1 = s_mu[cy][cx] + d[2];
    } else {
        n0 = PERT ? s_eta[cy][cx] : s_h[cy][cx];
        n1 = s_mu[cy][cx];
        n2 = R(0);
    }

    double s_cell = 0.0;
    if (valid) {
        const size_t o = (size_t)gj * nx + gi;
        R hn = PERT ? n0 + p.bath[o] : n0;
        if (WD && !(hn > tol)) {   // a dry cell keeps no momentum, no negative depth
            if (hn < R(0)) {
                hn = R(0);
                n0 = PERT ? -p.bath[o] : R(0);
            }
            n1 = R(0);
            n2 = R(0);
        }
        o0[o] = n0;
        o1[o] = n1;
        if (TWO_D) o2[o] = n2;
        if (!(WD ? hn >= R(0) : hn > R(0)) || !isfinite(n1) || !isfinite(n2))
            atomicOr(p.err, ERR_UNSTABLE);
        // CFL number of the new state: max over directions of (|u|+c)/d
        const R c = sqrt(p.g * hn);
        R s = (fabs(n1 / hn) + c) / p.dx;
        if (TWO_D) {
            const R sy = (fabs(n2 / hn) + c) / p.dy;
            if (sy > s) s = sy;
        }
        s_cell = (double)s;
        if (!(s_cell >= 0.0) || (WD && !(hn > tol))) s_cell = 0.0;
    }

    // 6) block max -> partial, last block reduces and advances the clock
    const double bm = block_max<NT>(s_cell, red);
    const int bid = blockIdx.x + blockIdx.y * gridDim.x;
    if (tid == 0) {
        p.partial[bid] = bm;
        __threadfence();
        const unsigned int tk = atomicAdd((unsigned int *)&p.clk->ticket, 1u);
        am_last = (tk == (unsigned int)(p.nblocks - 1));
    }
    __syncthreads();
    if (am_last) {
        __threadfence();
        double m = 0.0;
        for (int k = tid; k < p.nblocks; k += NT) {
            const double v = __ldcg(p.partial + k);
            m = v > m ? v : m;
        }
        m = block_max<NT>(m, red);
        if (tid == 0) {
            clk->t = t + dt;
            clk->smax = m;
            clk->dt_cfl = p.cfl / m;
            clk->cur = cur ^ 1;
            clk->nsteps = clk->nsteps + 1;
            clk->ticket = 0u;
            clk->work = 0u;
        }
    }
}

// Initial CFL reduction over the current state (set_state), same per-cell rule.
template <typename R, bool PERT>
__global__ void __launch_bounds__(256) clock_init_kernel(FwdParams<R> p, double t0) {
    __shared__ double red[32];
    __shared__ int am_last;
    const int tid = threadIdx.x;
    const size_t n = (size_t)p.nx * p.ny;
    const R *q0 = p.q[0][0], *q1 = p.q[0][1], *q2 = p.q[0][2];
    // a new state: no unit has had waves yet (the quiet-unit hint)
    for (int k = blockIdx.x * 256 + tid; k < p.umap_n; k += gridDim.x * 256) p.umap[k] = 0;
    double mx = 0.0;
    for (size_t k = (size_t)blockIdx.x * 256 + tid; k < n; k += (size_t)gridDim.x * 256) {
        const R h = PERT ? q0[k] + p.bath[k] : q0[k];
        double sd;
        if (p.wetdry && !(h > p.dry_tol)) {
            if (p.err && !(h >= R(0))) atomicOr(p.err, ERR_UNSTABLE);
            continue;   // a dry cell carries no waves
        }
        if (PERT) {
            // the float rule of the fused step reduction (cfl_f32)
            sd = (double)cfl_f32((float)h, (float)q1[k], p.two_d ? (float)q2[k] : 0.f,
                                 (float)p.g, 1.f / (float)p.dx, 1.f / (float)p.dy, p.two_d);
        } else {
            const R c = sqrt(p.g * h);
            R s = (fabs(q1[k] / h) + c) / p.dx;
            if (p.two_d) {
                const R sy = (fabs(q2[k] / h) + c) / p.dy;
                if (sy > s) s = sy;
            }
            sd = (double)s;
        }
        if (p.err && !(h > R(0))) atomicOr(p.err, ERR_UNSTABLE);
        mx = sd > mx ? sd : mx;
    }
    const double bm = block_max<256>(mx, red);
    if (tid == 0) {
        p.partial[blockIdx.x] = bm;
        __threadfence();
        const unsigned int tk = atomicAdd(&p.clk->ticket, 1u);
        am_last = (tk == gridDim.x - 1);
    }
    __syncthreads();
    if (am_last) {
        __threadfence();
        double m = 0.0;
        for (int k = tid; k < (int)gridDim.x; k += 256) {
            const double v = __ldcg(p.partial + k);
            m = v > m ? v : m;
        }
        m = block_max<256>(m, red);
        if (tid == 0) {
            volatile DevClock *clk = p.clk;
            clk->t = t0;
            clk->smax = m;
            clk->dt_cfl = p.cfl / m;
            clk->cur = 0;
            clk->nsteps = 0;
            clk->ticket = 0u;
            clk->work = 0u;
        }
    }
}

}  // namespace swadj
