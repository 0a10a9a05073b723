// ctu_kernels.cuh -- unsplit 2D forward step with transverse waves: the
// wave-propagation method of the textbook the paper defers to for its
// finite volume methods (LeVeque 2002, multidimensional chapters; Sec. 6),
// an alternative to the dimensionally split step of fwd_kernels.cuh.
//
// Every x- and y-edge Riemann problem is solved from Q^n (the same f-wave
// Roe solve as the split step).  With nu_x = dt/dx, nu_y = dt/dy:
//   Q_ij += -nu_x (A+dQ_{i-1/2,j} + A-dQ_{i+1/2,j}) - nu_x (F_{i+1/2,j} - F_{i-1/2,j})
//           -nu_y (B+dQ_{i,j-1/2} + B-dQ_{i,j+1/2}) - nu_y (G_{i,j+1/2} - G_{i,j-1/2})
// An edge flux is the edge's MC-limited correction minus (nu_other / 2)
// times the transverse parts of the four fluctuations of the other direction
// that enter the two cells beside the edge and move towards it, e.g.
//   G_{i,j-1/2} = C_{i,j-1/2} - (nu_x/2) [B+A+dQ_{i-1/2,j-1} + B+A-dQ_{i+1/2,j-1}
//                                        + B-A+dQ_{i-1/2,j} + B-A-dQ_{i+1/2,j}]
// A fluctuation's transverse parts come from the eigenstructure of the
// tangential flux Jacobian at its edge's Roe state.  Stable up to a Courant
// number of 1 in each direction (the CFL rule is the split step's).
//
// One TX x TY tile per block, in four phases through shared memory:
//   A  stage the tile and a 2-cell halo (corners included, ghosts by index
//      mapping);
//   B  solve each x-edge and y-edge Riemann problem the tile reads, once;
//   C  per cell of the tile and of the 1-cell ring that phase D reads: the
//      transverse parts of the fluctuations entering it, summed per direction
//      of travel (P: +, M: -), and the fluctuations and limited correction of
//      its low x- and y-edge, as four lists of items shared by all threads;
//   D  per tile cell: edge fluxes C - (nu_other/2) (P(cell below) + M(cell
//      above)) and the update.
// Each edge term is computed once per block instead of once per reading
// cell.  Expressions and the order of every sum follow the FP64 reference, so
// with contraction disabled (the FP64 instantiation) the rounding matches
// it.
#pragma once
#include "fwd_kernels.cuh"

namespace swadj {

// Division and square root where the operand is a positive normal number
// (depths, 2c, sums of square roots of depths): exact in FP64, the
// reference's rounding; one-instruction approximations in FP32.
__device__ __forceinline__ double ctu_div(double a, double b) { return a / b; }
__device__ __forceinline__ float ctu_div(float a, float b) { return a * rcp_ftz(b); }
__device__ __forceinline__ double ctu_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float ctu_sqrt(float x) { return x * rsqrt_ftz(x); }

// The f-wave Roe solve of fwave_roe (FP64: that very function; FP32: the same
// expressions with ctu_div / ctu_sqrt).
template <typename R>
__device__ __forceinline__ void ctu_roe(R g, R hL, R mnL, R mtL, R unL, R utL, R sqL, R etaL,
                                        R hR, R mnR, R mtR, R unR, R utR, R sqR, R etaR,
                                        R &uh, R &ch, R &b1, R &b2, R &b3, R &vh) {
    if constexpr (sizeof(R) == 8) {
        fwave_roe<R>(g, hL, mnL, mtL, unL, utL, sqL, etaL, hR, mnR, mtR, unR, utR, sqR, etaR,
                     uh, ch, b1, b2, b3, vh);
    } else {
        const R hhat = R(0.5) * (hL + hR);
        const R rden = rcp_ftz(sqL + sqR);
        uh = (sqL * unL + sqR * unR) * rden;
        vh = (sqL * utL + sqR * utR) * rden;
        ch = ctu_sqrt(g * hhat);
        const R s1 = uh - ch, s3 = uh + ch;
        const R df1 = mnR - mnL;
        const R df2 = (mnR * unR - mnL * unL) + g * hhat * (etaR - etaL);
        const R df3 = mnR * utR - mnL * utL;
        const R rw = rcp_ftz(s3 - s1);
        b1 = (s3 * df1 - df2) * rw;
        b3 = (df2 - s1 * df1) * rw;
        b2 = df3 - vh * df1;
    }
}

// Fluctuations of one edge (the first-order part of edge_flux, same sums).
template <typename R>
__device__ __forceinline__ void ctu_fluct(const Wave6<R> &w, R am[3], R ap[3]) {
#pragma unroll
    for (int m = 0; m < 3; m++) { am[m] = R(0); ap[m] = R(0); }
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
    }
}

// Transverse split of fluctuation a (edge frame h, normal, tangential
// momentum) by the tangential flux Jacobian at the Roe state (uh normal, vh
// tangential velocity, ch): speeds vh - ch, vh, vh + ch, vectors
// (1, uh, vh - ch), (0, 1, 0), (1, uh, vh + ch).  bm / bp: the parts moving
// in the negative / positive tangential direction, each summed in p order.
template <typename R>
__device__ __forceinline__ void ctu_tsplit(const Wave6<R> &w, const R a[3], R bm[3], R bp[3]) {
    const R uh = w.uh, vh = w.vh, ch = w.ch;
    const R mu[3] = {vh - ch, vh, vh + ch};
    const R two_c = R(2) * ch;
    R beta[3];
    beta[0] = ctu_div((vh + ch) * a[0] - a[2], two_c);
    beta[1] = a[1] - uh * a[0];
    beta[2] = ctu_div(a[2] - (vh - ch) * a[0], two_c);
    const R r[3][3] = {{R(1), uh, vh - ch}, {R(0), R(1), R(0)}, {R(1), uh, vh + ch}};
#pragma unroll
    for (int m = 0; m < 3; m++) { bm[m] = R(0); bp[m] = R(0); }
#pragma unroll
    for (int p = 0; p < 3; p++) {
        const R c = mu[p] * beta[p];
#pragma unroll
        for (int m = 0; m < 3; m++) {
            if (mu[p] < R(0)) bm[m] += c * r[p][m];
            else if (mu[p] > R(0)) bp[m] += c * r[p][m];
        }
    }
}

// Shared-memory layout of one block's tile (TX x TY cells, 2-cell halo).
// Phase A (staging) and phase C (per-cell edge terms) share one region.
template <typename R, int TX, int TY>
struct CtuSmem {
    static constexpr int RX = TX + 4, RY = TY + 4;     // staged cells
    static constexpr int QX = TX + 2, QY = TY + 2;     // cells with edge terms
    static constexpr int NCELL = RX * RY, NQ = QX * QY;
    static constexpr int NA = 7 * NCELL, NC = 30 * NQ;  // values in each phase
    static constexpr int NU = NA > NC ? NA : NC;
    static constexpr int NWX = RY * (RX - 1), NWY = (RY - 1) * RX;
    // waves as 6 arrays per direction (uh, ch, b1, b2, b3, vh)
    static constexpr size_t bytes = sizeof(R) * (NU + 6 * (NWX + NWY)) + 32 * sizeof(double) + 16;
};

// Transverse terms of one cell, from its two edges of the other direction
// (lo: entering through the low edge, its own wave; hi: through the high
// edge): P = parts moving in + along this direction, M = parts moving in -,
// both in this direction's frame (components 1 and 2 exchanged), each the
// low-edge part plus the high-edge part.
template <typename R>
__device__ __forceinline__ void ctu_cell_terms(const Wave6<R> &lo, const Wave6<R> &hi,
                                               R P[3], R M[3]) {
    R am[3], ap_lo[3], am_hi[3], ap[3];
    ctu_fluct(lo, am, ap_lo);
    ctu_fluct(hi, am_hi, ap);
    R pm0[3], pp0[3], pm1[3], pp1[3];
    ctu_tsplit(lo, ap_lo, pm0, pp0);
    ctu_tsplit(hi, am_hi, pm1, pp1);
    P[0] = pp0[0] + pp1[0]; P[1] = pp0[2] + pp1[2]; P[2] = pp0[1] + pp1[1];
    M[0] = pm0[0] + pm1[0]; M[1] = pm0[2] + pm1[2]; M[2] = pm0[1] + pm1[1];
}

template <typename R, bool PERT, int TX, int TY>
__global__ void __launch_bounds__(TX *TY)
fwd_ctu_kernel(FwdParams<R> p) {
    using L = CtuSmem<R, TX, TY>;
    constexpr int H = 2, RX = L::RX, RY = L::RY, QX = L::QX, QY = L::QY;
    constexpr int NT = TX * TY, NCELL = L::NCELL;
    extern __shared__ __align__(16) unsigned char ctu_smem[];
    R *U = reinterpret_cast<R *>(ctu_smem);
    R *wxa = U + L::NU;             // x-edge waves, field f at wxa[f * NWX + i]
    R *wya = wxa + 6 * L::NWX;      // y-edge waves, field f at wya[f * NWY + i]
    double *red = reinterpret_cast<double *>(wya + 6 * L::NWY);
    __shared__ int am_last;
    // phase A: staged cells, 7 fields of RY x RX
    R *s_h = U, *s_mu = U + NCELL, *s_mv = U + 2 * NCELL, *s_eta = U + 3 * NCELL;
    R *s_u = U + 4 * NCELL, *s_v = U + 5 * NCELL, *s_sq = U + 6 * NCELL;
    // phase C: per cell of the QY x QX region (staged cell (qx+1, qy+1)),
    // 30 fields: P/M along x and y (3 each), then (am, ap, C) of the cell's
    // low x-edge and low y-edge (3 each)
    auto Q = [&](int f, int m, int qx, int qy) -> R & { return U[((f * 3 + m) * QY + qy) * QX + qx]; };
    enum { PX = 0, MX, PY, MY, XAM, XAP, XC, YAM, YAP, YC };
    auto wave_at = [&](const R *a, int n, int i) {
        Wave6<R> w;
        w.uh = a[i]; w.ch = a[n + i]; w.b1 = a[2 * n + i];
        w.b2 = a[3 * n + i]; w.b3 = a[4 * n + i]; w.vh = a[5 * n + i];
        return w;
    };
    auto wave_put = [&](R *a, int n, int i, const Wave6<R> &w) {
        a[i] = w.uh; a[n + i] = w.ch; a[2 * n + i] = w.b1;
        a[3 * n + i] = w.b2; a[4 * n + i] = w.b3; a[5 * n + i] = w.vh;
    };
    constexpr int NWX = L::NWX, NWY = L::NWY;
    auto WX = [&](int ry, int k) { return wave_at(wxa, NWX, ry * (RX - 1) + k); };
    auto WY = [&](int k, int rx) { return wave_at(wya, NWY, k * RX + rx); };

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = tx + ty * TX;
    volatile DevClock *clk = p.clk;
    const double t = clk->t;
    double dt = clk->dt_cfl;
    if (p.t_end - t < dt) dt = p.t_end - t;
    if (!(dt > 0.0)) return;   // clock already at t_end: no-op step
    const int cur = clk->cur;
    if (p.gauges.n > 0 && blockIdx.x == 0 && blockIdx.y == 0)   // the state this step starts from
        record_gauges<R, NT>(p.gauges, p.q[cur][0], p.bath, p.nx, p.ny, 1, t);

    const R *q0 = p.q[cur][0], *q1 = p.q[cur][1], *q2 = p.q[cur][2];
    R *o0 = p.q[cur ^ 1][0], *o1 = p.q[cur ^ 1][1], *o2 = p.q[cur ^ 1][2];
    const int nx = p.nx, ny = p.ny;
    const int i0 = blockIdx.x * TX - H, j0 = blockIdx.y * TY - H;

    // A) tile + halo with corners, ghost cells by index mapping on both axes
    for (int r = tid; r < NCELL; r += NT) {
        const int ry = r / RX, rx = r - ry * RX;
        bool fx, fy;
        const int ci = ghost_index(i0 + rx, nx, p.bc.lo_x, p.bc.hi_x, &fx);
        const int cj = ghost_index(j0 + ry, ny, p.bc.lo_y, p.bc.hi_y, &fy);
        const size_t o = (size_t)cj * nx + ci;
        R a = q0[o], mu = q1[o], mv = q2[o];
        const R b = p.bath[o];
        if (fx) mu = -mu;
        if (fy) mv = -mv;
        R h, eta;
        if (PERT) { eta = a; h = a + b; }
        else { h = a; eta = a + b; }
        s_h[r] = h;
        s_mu[r] = mu;
        s_mv[r] = mv;
        s_eta[r] = eta;
        if constexpr (sizeof(R) == 8) {
            s_u[r] = mu / h;
            s_v[r] = mv / h;
        } else {
            const R rh = rcp_ftz(h);
            s_u[r] = mu * rh;
            s_v[r] = mv * rh;
        }
        s_sq[r] = ctu_sqrt(h);
    }
    __syncthreads();

    // B) x-edge waves of rows 1 .. RY-2, y-edge waves of columns 1 .. RX-2,
    //    edge frames (h, hu, hv) / (h, hv, hu); the cell's own state is kept
    //    in registers (phase C overwrites the staging area)
    const int cx = tx + H, cy = ty + H, cc = cy * RX + cx;
    const R a0 = PERT ? s_eta[cc] : s_h[cc], mu0 = s_mu[cc], mv0 = s_mv[cc];
    constexpr int NBX = (RY - 2) * (RX - 1), NBY = (RY - 1) * (RX - 2);
    for (int e = tid; e < NBX + NBY; e += NT) {
        Wave6<R> w;
        if (e < NBX) {
            const int ry = 1 + e / (RX - 1), k = e % (RX - 1);
            const int a = ry * RX + k, b = a + 1;
            ctu_roe<R>(p.g, s_h[a], s_mu[a], s_mv[a], s_u[a], s_v[a], s_sq[a], s_eta[a],
                       s_h[b], s_mu[b], s_mv[b], s_u[b], s_v[b], s_sq[b], s_eta[b], w.uh,
                       w.ch, w.b1, w.b2, w.b3, w.vh);
            wave_put(wxa, NWX, ry * (RX - 1) + k, w);
        } else {
            const int f = e - NBX;
            const int k = f / (RX - 2), rx = 1 + f % (RX - 2);
            const int a = k * RX + rx, b = a + RX;
            ctu_roe<R>(p.g, s_h[a], s_mv[a], s_mu[a], s_v[a], s_u[a], s_sq[a], s_eta[a],
                       s_h[b], s_mv[b], s_mu[b], s_v[b], s_u[b], s_sq[b], s_eta[b], w.uh,
                       w.ch, w.b1, w.b2, w.b3, w.vh);
            wave_put(wya, NWY, k * RX + rx, w);
        }
    }
    __syncthreads();

    // C) four item lists over the region cells (rx, ry) = (qx + 1, qy + 1),
    //    each covering only the cells phase D reads:
    //    1. P/M along x (from the cell's y-edges): qx 0 .. TX+1, qy 1 .. TY
    //    2. P/M along y (from its x-edges):        qx 1 .. TX,   qy 0 .. TY+1
    //    3. (am, ap, C) of its low x-edge:          qx 1 .. TX+1, qy 1 .. TY
    //    4. (am, ap, C) of its low y-edge:          qx 1 .. TX,   qy 1 .. TY+1
    const R nux = R(dt) / p.dx, nuy = R(dt) / p.dy;
    constexpr int N1 = QX * TY, N2 = TX * QY, N3 = (TX + 1) * TY, N4 = TX * (TY + 1);
    for (int e = tid; e < N1 + N2 + N3 + N4; e += NT) {
        if (e < N1) {
            const int qy = 1 + e / QX, qx = e % QX, rx = qx + 1, ry = qy + 1;
            R P[3], M[3];
            ctu_cell_terms(WY(ry - 1, rx), WY(ry, rx), P, M);
#pragma unroll
            for (int m = 0; m < 3; m++) { Q(PX, m, qx, qy) = P[m]; Q(MX, m, qx, qy) = M[m]; }
        } else if (e < N1 + N2) {
            const int f = e - N1;
            const int qy = f / TX, qx = 1 + f % TX, rx = qx + 1, ry = qy + 1;
            R P[3], M[3];
            ctu_cell_terms(WX(ry, rx - 1), WX(ry, rx), P, M);
#pragma unroll
            for (int m = 0; m < 3; m++) { Q(PY, m, qx, qy) = P[m]; Q(MY, m, qx, qy) = M[m]; }
        } else if (e < N1 + N2 + N3) {
            const int f = e - N1 - N2;
            const int qy = 1 + f / (TX + 1), qx = 1 + f % (TX + 1), rx = qx + 1, ry = qy + 1;
            R am[3], ap[3], C[3];
            edge_flux<R>(WX(ry, rx - 2), WX(ry, rx - 1), WX(ry, rx), nux, p.order, am, ap, C);
#pragma unroll
            for (int m = 0; m < 3; m++) {
                Q(XAM, m, qx, qy) = am[m]; Q(XAP, m, qx, qy) = ap[m]; Q(XC, m, qx, qy) = C[m];
            }
        } else {
            const int f = e - N1 - N2 - N3;
            const int qy = 1 + f / TX, qx = 1 + f % TX, rx = qx + 1, ry = qy + 1;
            R am[3], ap[3], C[3];
            edge_flux<R>(WY(ry - 2, rx), WY(ry - 1, rx), WY(ry, rx), nuy, p.order, am, ap, C);
#pragma unroll
            for (int m = 0; m < 3; m++) {
                Q(YAM, m, qx, qy) = am[m]; Q(YAP, m, qx, qy) = ap[m]; Q(YC, m, qx, qy) = C[m];
            }
        }
    }
    __syncthreads();

    // D) assemble the cell (region coordinates tx + 1, ty + 1)
    const R kx = R(0.5) * nuy, ky = R(0.5) * nux;
    const int qx = tx + 1, qy = ty + 1;
    R dxq[3], dyq[3];
#pragma unroll
    for (int m = 0; m < 3; m++) {
        const R FL = Q(XC, m, qx, qy) - kx * (Q(PX, m, qx - 1, qy) + Q(MX, m, qx, qy));
        const R FR = Q(XC, m, qx + 1, qy) - kx * (Q(PX, m, qx, qy) + Q(MX, m, qx + 1, qy));
        const R GB = Q(YC, m, qx, qy) - ky * (Q(PY, m, qx, qy - 1) + Q(MY, m, qx, qy));
        const R GT = Q(YC, m, qx, qy + 1) - ky * (Q(PY, m, qx, qy) + Q(MY, m, qx, qy + 1));
        dxq[m] = -nux * (Q(XAP, m, qx, qy) + Q(XAM, m, qx + 1, qy)) - nux * (FR - FL);
        dyq[m] = -nuy * (Q(YAP, m, qx, qy) + Q(YAM, m, qx, qy + 1)) - nuy * (GT - GB);
    }
    const R n0 = (a0 + dxq[0]) + dyq[0];
    const R n1 = (mu0 + dxq[1]) + dyq[2];
    const R n2 = (mv0 + dxq[2]) + dyq[1];

    const int gi = blockIdx.x * TX + tx, gj = blockIdx.y * TY + ty;
    double s_cell = 0.0;
    if (gi < nx && gj < ny) {
        const size_t o = (size_t)gj * nx + gi;
        const R hn = PERT ? n0 + p.bath[o] : n0;
        o0[o] = n0;
        o1[o] = n1;
        o2[o] = n2;
        if (!(hn > R(0)) || !isfinite(n1) || !isfinite(n2)) atomicOr(p.err, ERR_UNSTABLE);
        if (PERT) {
            s_cell = (double)cfl_f32((float)hn, (float)n1, (float)n2, (float)p.g,
                                     1.f / (float)p.dx, 1.f / (float)p.dy, 1);
        } else {
            const R c = sqrt(p.g * hn);
            R s = (fabs(n1 / hn) + c) / p.dx;
            const R sy = (fabs(n2 / hn) + c) / p.dy;
            if (sy > s) s = sy;
            s_cell = (double)s;
        }
        if (!(s_cell >= 0.0)) s_cell = 0.0;
    }

    // E) block max -> partial, the last block reduces and advances the clock
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

template <typename R, bool PERT, int TX, int TY>
int ctu_launch(FwdParams<R> p, cudaStream_t st, const char *name) {
    constexpr size_t smem = CtuSmem<R, TX, TY>::bytes;
    static_assert(smem <= 227 * 1024, "tile does not fit in shared memory");
    // set on every launch: the attribute belongs to the current device
    const int rc = swadj_host::cuda_check(
        cudaFuncSetAttribute(fwd_ctu_kernel<R, PERT, TX, TY>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
        name);
    if (rc) return rc;
    dim3 grid((p.nx + TX - 1) / TX, (p.ny + TY - 1) / TY);
    p.nblocks = (int)(grid.x * grid.y);
    fwd_ctu_kernel<R, PERT, TX, TY><<<grid, dim3(TX, TY), smem, st>>>(p);
    return swadj_host::cuda_check(cudaGetLastError(), name);
}

template <int TX, int TY>
inline int ctu_blocks(int nx, int ny) {
    return ((nx + TX - 1) / TX) * ((ny + TY - 1) / TY);
}

}  // namespace swadj
