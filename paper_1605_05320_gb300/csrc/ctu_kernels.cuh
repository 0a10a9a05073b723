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
// One TX x TY tile per block, staged with a 2-cell halo including corners;
// the x-edge waves of the rows and the y-edge waves of the columns a cell
// needs are solved once per block into shared memory, then each thread
// assembles its cell.  Expressions and the order of every sum follow the
// FP64 reference, so with contraction disabled (the FP64 instantiation) the
// rounding matches it.
#pragma once
#include "fwd_kernels.cuh"

namespace swadj {

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
// (1, uh, vh - ch), (0, 1, 0), (1, uh, vh + ch).  Adds the part moving in
// the negative tangential direction to bm and the positive one to bp, each
// a fresh sum in p order (then accumulated by the caller in the same order
// as the reference).
template <typename R>
__device__ __forceinline__ void ctu_tsplit(const Wave6<R> &w, const R a[3], R bm[3], R bp[3]) {
    const R uh = w.uh, vh = w.vh, ch = w.ch;
    const R mu[3] = {vh - ch, vh, vh + ch};
    const R two_c = R(2) * ch;
    R beta[3];
    beta[0] = ((vh + ch) * a[0] - a[2]) / two_c;
    beta[1] = a[1] - uh * a[0];
    beta[2] = (a[2] - (vh - ch) * a[0]) / two_c;
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

// Accumulate the transverse parts (in the frame of the other direction) into
// tr, components 1 and 2 exchanged (back to this direction's frame).
template <typename R>
__device__ __forceinline__ void ctu_acc(R tr[3], const R b[3]) {
    tr[0] += b[0];
    tr[1] += b[2];
    tr[2] += b[1];
}

// One direction of a cell's update, in that direction's edge frame.
// W(k): the waves of this direction's edge k (between cells k-1 and k along
// it, relative to the cell: k = 0 is the low edge); T(s, e): the waves of
// the other direction's edge e (0 low, 1 high) of the cell at offset s
// (-1, 0, 1) along this direction.  Returns the fluctuations entering the
// cell through its low/high edge and the low/high edge fluxes.
template <typename R, typename WF, typename TF>
__device__ __forceinline__ void ctu_dir(WF W, TF T, R nu, R k, int order, R ap_lo[3],
                                        R am_hi[3], R F_lo[3], R F_hi[3]) {
    R am_lo[3], ap_hi[3];
    edge_flux<R>(W(-1), W(0), W(1), nu, order, am_lo, ap_lo, F_lo);
    edge_flux<R>(W(0), W(1), W(2), nu, order, am_hi, ap_hi, F_hi);
    R tr_lo[3] = {R(0), R(0), R(0)}, tr_hi[3] = {R(0), R(0), R(0)};
#pragma unroll
    for (int s = -1; s <= 1; s++) {
        const Wave6<R> lo = T(s, 0), hi = T(s, 1);
        R am[3], apL[3], amH[3], ap[3];
        ctu_fluct(lo, am, apL);   // enters the cell at s through its low edge
        ctu_fluct(hi, amH, ap);   // ... through its high edge
        R pm0[3], pp0[3], pm1[3], pp1[3];
        ctu_tsplit(lo, apL, pm0, pp0);
        ctu_tsplit(hi, amH, pm1, pp1);
        if (s == -1) {
            ctu_acc(tr_lo, pp0); ctu_acc(tr_lo, pp1);
        } else if (s == 0) {
            ctu_acc(tr_lo, pm0); ctu_acc(tr_hi, pp0);
            ctu_acc(tr_lo, pm1); ctu_acc(tr_hi, pp1);
        } else {
            ctu_acc(tr_hi, pm0); ctu_acc(tr_hi, pm1);
        }
    }
#pragma unroll
    for (int m = 0; m < 3; m++) {
        F_lo[m] = F_lo[m] - k * tr_lo[m];
        F_hi[m] = F_hi[m] - k * tr_hi[m];
    }
}

template <typename R, bool PERT, int TX, int TY>
__global__ void __launch_bounds__(TX *TY)
fwd_ctu_kernel(FwdParams<R> p) {
    constexpr int H = 2;
    constexpr int RX = TX + 2 * H, RY = TY + 2 * H;
    constexpr int NT = TX * TY;
    __shared__ R s_h[RY][RX], s_mu[RY][RX], s_mv[RY][RX], s_eta[RY][RX];
    __shared__ R s_u[RY][RX], s_v[RY][RX], s_sq[RY][RX];
    __shared__ Wave6<R> wx[RY][RX - 1];   // x-edge (k|k+1) of staged row ry
    __shared__ Wave6<R> wy[RY - 1][RX];   // y-edge (k|k+1) of staged column rx
    __shared__ double red[32];
    __shared__ int am_last;

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

    // 1) tile + halo with corners, ghost cells by index mapping on both axes
    for (int r = tid; r < RX * RY; r += NT) {
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
        s_h[ry][rx] = h;
        s_mu[ry][rx] = mu;
        s_mv[ry][rx] = mv;
        s_eta[ry][rx] = eta;
        s_u[ry][rx] = mu / h;
        s_v[ry][rx] = mv / h;
        s_sq[ry][rx] = sqrt(h);
    }
    __syncthreads();

    // 2) x-edge waves of rows 1 .. RY-2 and y-edge waves of columns 1 .. RX-2
    //    (those the tile's cells read), edge frames (h, hu, hv) / (h, hv, hu)
    constexpr int NWX = (RY - 2) * (RX - 1), NWY = (RY - 1) * (RX - 2);
    for (int e = tid; e < NWX + NWY; e += NT) {
        Wave6<R> w;
        if (e < NWX) {
            const int ry = 1 + e / (RX - 1), k = e % (RX - 1);
            fwave_roe<R>(p.g, s_h[ry][k], s_mu[ry][k], s_mv[ry][k], s_u[ry][k], s_v[ry][k],
                         s_sq[ry][k], s_eta[ry][k], s_h[ry][k + 1], s_mu[ry][k + 1],
                         s_mv[ry][k + 1], s_u[ry][k + 1], s_v[ry][k + 1], s_sq[ry][k + 1],
                         s_eta[ry][k + 1], w.uh, w.ch, w.b1, w.b2, w.b3, w.vh);
            wx[ry][k] = w;
        } else {
            const int f = e - NWX;
            const int k = f / (RX - 2), rx = 1 + f % (RX - 2);
            fwave_roe<R>(p.g, s_h[k][rx], s_mv[k][rx], s_mu[k][rx], s_v[k][rx], s_u[k][rx],
                         s_sq[k][rx], s_eta[k][rx], s_h[k + 1][rx], s_mv[k + 1][rx],
                         s_mu[k + 1][rx], s_v[k + 1][rx], s_u[k + 1][rx], s_sq[k + 1][rx],
                         s_eta[k + 1][rx], w.uh, w.ch, w.b1, w.b2, w.b3, w.vh);
            wy[k][rx] = w;
        }
    }
    __syncthreads();

    // 3) assemble the cell
    const int cx = tx + H, cy = ty + H;
    const R nux = R(dt) / p.dx, nuy = R(dt) / p.dy;
    const R kx = R(0.5) * nuy, ky = R(0.5) * nux;
    R apL[3], amR[3], FL[3], FR[3], bpB[3], bmT[3], GB[3], GT[3];
    // x: edge k of the cell is x-edge (cx-1+k | cx+k); the other direction's
    // edges of the cell at offset s are y-edges (cy-1 | cy) and (cy | cy+1)
    ctu_dir<R>([&](int k) { return wx[cy][cx - 1 + k]; },
               [&](int s, int e) { return wy[cy - 1 + e][cx + s]; }, nux, kx, p.order, apL,
               amR, FL, FR);
    ctu_dir<R>([&](int k) { return wy[cy - 1 + k][cx]; },
               [&](int s, int e) { return wx[cy + s][cx - 1 + e]; }, nuy, ky, p.order, bpB,
               bmT, GB, GT);
    R dxq[3], dyq[3];
#pragma unroll
    for (int m = 0; m < 3; m++) {
        dxq[m] = -nux * (apL[m] + amR[m]) - nux * (FR[m] - FL[m]);
        dyq[m] = -nuy * (bpB[m] + bmT[m]) - nuy * (GT[m] - GB[m]);
    }
    const R a0 = PERT ? s_eta[cy][cx] : s_h[cy][cx];
    const R n0 = (a0 + dxq[0]) + dyq[0];
    const R n1 = (s_mu[cy][cx] + dxq[1]) + dyq[2];
    const R n2 = (s_mv[cy][cx] + dxq[2]) + dyq[1];

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

    // 4) block max -> partial, the last block reduces and advances the clock
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
        }
    }
}

template <typename R, bool PERT, int TX, int TY>
int ctu_launch(FwdParams<R> p, cudaStream_t st, const char *name) {
    dim3 grid((p.nx + TX - 1) / TX, (p.ny + TY - 1) / TY);
    p.nblocks = (int)(grid.x * grid.y);
    fwd_ctu_kernel<R, PERT, TX, TY><<<grid, dim3(TX, TY), 0, st>>>(p);
    return swadj_host::cuda_check(cudaGetLastError(), name);
}

template <int TX, int TY>
inline int ctu_blocks(int nx, int ny) {
    return ((nx + TX - 1) / TX) * ((ny + TY - 1) / TY);
}

}  // namespace swadj
