// fwd_tiles.cuh -- FP32 tile machinery of the forward step, shared by the
// single-grid step (fwd_f32.cu) and the batched patch step (patches.cu).
//
// A tile is TX x TY cells of one grid ("view").  Phases per tile: (0) stage
// the tile and a 2-cell halo (no corners) as derived cell data in shared
// memory, (1) solve every x- and y-edge the tile needs, (2) form every
// edge's net fluxes, limiter evaluated once per edge, (3) update the cells.
// Each phase is a flat loop of independent items over 256 threads.  A
// persistent block walks its share of a tile list; the raw values of the
// next tile are loaded into registers while the current one is computed.
//
// The MC-limited correction needs no division by the wave norm: for
// Z = b (1, s, vhat) and its upwind neighbour Zu = bu (1, su, vu),
// theta b = bu (1 + su s + vu vhat) / (1 + s^2 + vhat^2) and
// phi(theta) b = sign(b) max(0, min((|b| + sign(b) theta b)/2, 2|b|,
// 2 sign(b) theta b)), which is phi(theta) b for every b including b = 0.
#pragma once
#include "fwd_kernels.cuh"

namespace swadj {
namespace tile {

constexpr int NT = 256;  // threads per block

__device__ __forceinline__ float rcpf(float x) { return __fdividef(1.0f, x); }
// 1 if s > 0, 0 if s < 0, 1/2 if s == 0 (an f-wave of speed 0 is split)
__device__ __forceinline__ float pos1(float s) { return s > 0.f ? 1.f : (s < 0.f ? 0.f : 0.5f); }
// sign(s) / 2
__device__ __forceinline__ float hsg1(float s) { return s > 0.f ? 0.5f : (s < 0.f ? -0.5f : 0.f); }
// phi(theta) b for the MC limiter, r = theta b
__device__ __forceinline__ float mc1(float b, float r) {
    const float sg = b < 0.f ? -1.f : 1.f;
    const float B = fabsf(b), Rr = sg * r;
    float m = fminf(0.5f * (B + Rr), 2.f * B);
    m = fminf(m, 2.f * Rr);
    return sg * fmaxf(m, 0.f);
}

struct EdgeS {           // wave data of one edge
    float s1, s3, vh, b1, b2, b3;
};

// Roe f-wave decomposition at an edge in its (normal, tangential) frame.
__device__ __forceinline__ EdgeS solve1(float g, float hL, float mnL, float mtL, float unL,
                                        float utL, float sqL, float etaL, float hR, float mnR,
                                        float mtR, float unR, float utR, float sqR, float etaR) {
    EdgeS w;
    const float hh = 0.5f * (hL + hR);
    const float rd = rcpf(sqL + sqR);
    const float uh = (sqL * unL + sqR * unR) * rd;
    const float vh = (sqL * utL + sqR * utR) * rd;
    const float gh = g * hh;
    const float rc = rsqrtf(gh);
    const float ch = gh * rc;
    const float s1 = uh - ch, s3 = uh + ch;
    const float df1 = mnR - mnL;
    const float df2 = (mnR * unR - mnL * unL) + gh * (etaR - etaL);
    const float df3 = mnR * utR - mnL * utL;
    const float hr = 0.5f * rc;  // 1 / (s3 - s1)
    w.s1 = s1;
    w.s3 = s3;
    w.vh = vh;
    w.b1 = (s3 * df1 - df2) * hr;
    w.b3 = (df2 - s1 * df1) * hr;
    w.b2 = df3 - vh * df1;
    return w;
}

// Net fluxes of edge w (neighbours wl, wr): L into the left cell, R into the
// right cell (Q -= nu * net).  SUB: every edge of the warp is subsonic
// (s1 < 0 < s3), so the sign logic of waves 1 and 3 is fixed; same numbers.
template <bool SUB>
__device__ __forceinline__ void net1(const EdgeS &wl, const EdgeS &w, const EdgeS &wr, float nu,
                                     int order, float L[3], float R[3]) {
    const float s2 = 0.5f * (w.s1 + w.s3);
    const float p2 = pos1(s2);
    float ap0, ap1, ap2, am0, am1, am2;
    if (SUB) {
        ap0 = w.b3; ap1 = w.b3 * w.s3; ap2 = w.b3 * w.vh + p2 * w.b2;
        am0 = w.b1; am1 = w.b1 * w.s1; am2 = w.b1 * w.vh + (w.b2 - p2 * w.b2);
    } else {
        const float a1 = pos1(w.s1) * w.b1, a3 = pos1(w.s3) * w.b3;
        ap0 = a1 + a3; ap1 = a1 * w.s1 + a3 * w.s3; ap2 = (a1 + a3) * w.vh + p2 * w.b2;
        const float t0 = w.b1 + w.b3;
        am0 = t0 - ap0;
        am1 = (w.b1 * w.s1 + w.b3 * w.s3) - ap1;
        am2 = (t0 * w.vh + w.b2) - ap2;
    }
    float F0 = 0.f, F1 = 0.f, F2 = 0.f;
    if (order >= 2) {
        const EdgeS &u1 = (!SUB && w.s1 > 0.f) ? wl : wr;
        const EdgeS &u3 = (SUB || w.s3 > 0.f) ? wl : wr;
        const float m1 = fmaf(w.s1, w.s1, fmaf(w.vh, w.vh, 1.f));
        const float d1 = fmaf(u1.s1, w.s1, fmaf(u1.vh, w.vh, 1.f));
        const float l1 = mc1(w.b1, u1.b1 * d1 * rcpf(m1));
        const float m3 = fmaf(w.s3, w.s3, fmaf(w.vh, w.vh, 1.f));
        const float d3 = fmaf(u3.s3, w.s3, fmaf(u3.vh, w.vh, 1.f));
        const float l3 = mc1(w.b3, u3.b3 * d3 * rcpf(m3));
        const float l2 = mc1(w.b2, s2 > 0.f ? wl.b2 : wr.b2);
        float c1, c3;
        if (SUB) {
            c1 = -0.5f * fmaf(nu, w.s1, 1.f) * l1;
            c3 = 0.5f * fmaf(-nu, w.s3, 1.f) * l3;
        } else {
            c1 = hsg1(w.s1) * fmaf(-nu, fabsf(w.s1), 1.f) * l1;
            c3 = hsg1(w.s3) * fmaf(-nu, fabsf(w.s3), 1.f) * l3;
        }
        const float c2 = hsg1(s2) * fmaf(-nu, fabsf(s2), 1.f) * l2;
        F0 = c1 + c3;
        F1 = c1 * w.s1 + c3 * w.s3;
        F2 = F0 * w.vh + c2;
    }
    L[0] = am0 + F0; L[1] = am1 + F1; L[2] = am2 + F2;
    R[0] = ap0 - F0; R[1] = ap1 - F1; R[2] = ap2 - F2;
}

__device__ __forceinline__ bool sub1(const EdgeS &w) { return w.s1 < 0.f && w.s3 > 0.f; }

// One grid or patch as a tile sees it.
struct View {
    const float *q0, *q1, *q2, *hb;   // current state (eta, hu, hv) and hbar
    float *o0, *o1, *o2;              // new state
    int nx, ny;
    float dx, dy;
    BcSpec bc;
};

template <int TX, int TY>
struct Smem {
    static constexpr int RX = TX + 4, RY = TY + 4;
    static constexpr int NEX = TX + 3, NEY = TY + 3;
    union U {   // cell data of tile + halo; reused for the net fluxes
        struct C {
            float h[RY][RX], mu[RY][RX], mv[RY][RX], u[RY][RX], v[RY][RX], sq[RY][RX],
                eta[RY][RX];
        } c;
        struct N {
            float xl[3][TY][TX + 1], xr[3][TY][TX + 1];
            float yl[3][TY + 1][TX], yr[3][TY + 1][TX];
        } n;
    } u;
    float xw[6][TY][NEX];
    float yw[6][NEY][TX];
};

// Raw values of a thread's share of a tile's staged region (RPT items).
template <int TX, int TY>
struct Raw {
    static constexpr int RX = TX + 4, RY = TY + 4;
    static constexpr int RPT = (RX * RY + NT - 1) / NT;
    float eta[RPT], mu[RPT], mv[RPT], hb[RPT];
};

template <int TX, int TY>
__device__ __forceinline__ void load_raw(const View &V, int i0, int j0, Raw<TX, TY> &R) {
    constexpr int RX = TX + 4, RY = TY + 4;
    const bool interior = i0 - 2 >= 0 && i0 + TX + 2 <= V.nx && j0 - 2 >= 0 &&
                          j0 + TY + 2 <= V.ny;
#pragma unroll
    for (int k = 0; k < Raw<TX, TY>::RPT; k++) {
        const int r = threadIdx.x + k * NT;
        const int ry = r / RX, rx = r - ry * RX;
        const bool xin = rx >= 2 && rx < TX + 2, yin = ry >= 2 && ry < TY + 2;
        if (r >= RX * RY || (!xin && !yin)) continue;
        int ci = i0 + rx - 2, cj = j0 + ry - 2;
        bool fx = false, fy = false;
        if (!interior) {
            ci = ghost_index(ci, V.nx, V.bc.lo_x, V.bc.hi_x, &fx);
            cj = ghost_index(cj, V.ny, V.bc.lo_y, V.bc.hi_y, &fy);
        }
        const size_t o = (size_t)cj * V.nx + ci;
        R.eta[k] = __ldg(V.q0 + o);
        R.hb[k] = __ldg(V.hb + o);
        const float mu = __ldg(V.q1 + o), mv = __ldg(V.q2 + o);
        R.mu[k] = fx ? -mu : mu;
        R.mv[k] = fy ? -mv : mv;
    }
}

// Phases 0-3 for one tile whose raw values are in R.  Returns the tile's
// maximum CFL number over its new cells.
template <int TX, int TY>
__device__ __forceinline__ float tile_compute(Smem<TX, TY> &S, const View &V, int i0, int j0,
                                              const Raw<TX, TY> &R, float nux, float nuy,
                                              float g, int order, bool &bad) {
    constexpr int RX = TX + 4, RY = TY + 4, NEX = TX + 3, NEY = TY + 3;
    const int tid = threadIdx.x;
    // phase 0: derived cell data
#pragma unroll
    for (int k = 0; k < Raw<TX, TY>::RPT; k++) {
        const int r = tid + k * NT;
        const int ry = r / RX, rx = r - ry * RX;
        const bool xin = rx >= 2 && rx < TX + 2, yin = ry >= 2 && ry < TY + 2;
        if (r >= RX * RY || (!xin && !yin)) continue;
        const float h = R.eta[k] + R.hb[k];
        const float q = rsqrtf(h);
        const float ih = q * q;
        S.u.c.h[ry][rx] = h;
        S.u.c.mu[ry][rx] = R.mu[k];
        S.u.c.mv[ry][rx] = R.mv[k];
        S.u.c.u[ry][rx] = R.mu[k] * ih;
        S.u.c.v[ry][rx] = R.mv[k] * ih;
        S.u.c.sq[ry][rx] = h * q;
        S.u.c.eta[ry][rx] = R.eta[k];
    }
    __syncthreads();
    constexpr int CPT = TX * TY / NT;
    float own_eta[CPT], own_mu[CPT], own_mv[CPT], own_h[CPT];
#pragma unroll
    for (int k = 0; k < CPT; k++) {
        const int c = tid + k * NT, ry = c / TX + 2, rx = c % TX + 2;
        own_eta[k] = S.u.c.eta[ry][rx];
        own_mu[k] = S.u.c.mu[ry][rx];
        own_mv[k] = S.u.c.mv[ry][rx];
        own_h[k] = S.u.c.h[ry][rx];
    }
    // phase 1: edge waves
    for (int i = tid; i < TY * NEX + NEY * TX; i += NT) {
        if (i < TY * NEX) {
            const int row = i / NEX, e = i - row * NEX, ry = row + 2;
            const EdgeS w = solve1(g, S.u.c.h[ry][e], S.u.c.mu[ry][e], S.u.c.mv[ry][e],
                                   S.u.c.u[ry][e], S.u.c.v[ry][e], S.u.c.sq[ry][e],
                                   S.u.c.eta[ry][e], S.u.c.h[ry][e + 1], S.u.c.mu[ry][e + 1],
                                   S.u.c.mv[ry][e + 1], S.u.c.u[ry][e + 1], S.u.c.v[ry][e + 1],
                                   S.u.c.sq[ry][e + 1], S.u.c.eta[ry][e + 1]);
            S.xw[0][row][e] = w.s1; S.xw[1][row][e] = w.s3; S.xw[2][row][e] = w.vh;
            S.xw[3][row][e] = w.b1; S.xw[4][row][e] = w.b2; S.xw[5][row][e] = w.b3;
        } else {
            const int k = i - TY * NEX, e = k / TX, col = k - e * TX, rx = col + 2;
            const EdgeS w = solve1(g, S.u.c.h[e][rx], S.u.c.mv[e][rx], S.u.c.mu[e][rx],
                                   S.u.c.v[e][rx], S.u.c.u[e][rx], S.u.c.sq[e][rx],
                                   S.u.c.eta[e][rx], S.u.c.h[e + 1][rx], S.u.c.mv[e + 1][rx],
                                   S.u.c.mu[e + 1][rx], S.u.c.v[e + 1][rx], S.u.c.u[e + 1][rx],
                                   S.u.c.sq[e + 1][rx], S.u.c.eta[e + 1][rx]);
            S.yw[0][e][col] = w.s1; S.yw[1][e][col] = w.s3; S.yw[2][e][col] = w.vh;
            S.yw[3][e][col] = w.b1; S.yw[4][e][col] = w.b2; S.yw[5][e][col] = w.b3;
        }
    }
    __syncthreads();
    // phase 2: net fluxes (the cell data are dead; their space holds the nets)
    for (int i = tid; i < TY * (TX + 1) + (TY + 1) * TX; i += NT) {
        EdgeS a, b, c;
        float nu;
        const bool isx = i < TY * (TX + 1);
        int row = 0, e = 0, col = 0;
        if (isx) {
            row = i / (TX + 1);
            e = 1 + (i - row * (TX + 1));
#define SWADJ_LOADX(W, E)                                                         \
    W.s1 = S.xw[0][row][E]; W.s3 = S.xw[1][row][E]; W.vh = S.xw[2][row][E];     \
    W.b1 = S.xw[3][row][E]; W.b2 = S.xw[4][row][E]; W.b3 = S.xw[5][row][E];
            SWADJ_LOADX(a, e - 1) SWADJ_LOADX(b, e) SWADJ_LOADX(c, e + 1)
#undef SWADJ_LOADX
            nu = nux;
        } else {
            const int k = i - TY * (TX + 1);
            e = 1 + k / TX;
            col = k - (e - 1) * TX;
#define SWADJ_LOADY(W, E)                                                         \
    W.s1 = S.yw[0][E][col]; W.s3 = S.yw[1][E][col]; W.vh = S.yw[2][E][col];     \
    W.b1 = S.yw[3][E][col]; W.b2 = S.yw[4][E][col]; W.b3 = S.yw[5][E][col];
            SWADJ_LOADY(a, e - 1) SWADJ_LOADY(b, e) SWADJ_LOADY(c, e + 1)
#undef SWADJ_LOADY
            nu = nuy;
        }
        float L[3], Rr[3];
        if (__all_sync(__activemask(), sub1(b))) net1<true>(a, b, c, nu, order, L, Rr);
        else net1<false>(a, b, c, nu, order, L, Rr);
        if (isx) {
#pragma unroll
            for (int m = 0; m < 3; m++) { S.u.n.xl[m][row][e - 1] = L[m]; S.u.n.xr[m][row][e - 1] = Rr[m]; }
        } else {
#pragma unroll
            for (int m = 0; m < 3; m++) { S.u.n.yl[m][e - 1][col] = L[m]; S.u.n.yr[m][e - 1][col] = Rr[m]; }
        }
    }
    __syncthreads();
    // phase 3: update; x nets: left edge -> R at index col, right edge -> L at
    // col + 1; y nets are in (h, hv, hu) order
    float smax = 0.f;
    const float rdx = 1.f / V.dx, rdy = 1.f / V.dy;
#pragma unroll
    for (int k = 0; k < CPT; k++) {
        const int c = tid + k * NT, row = c / TX, col = c % TX;
        const int gi = i0 + col, gj = j0 + row;
        if (gi < V.nx && gj < V.ny) {
            const float d0 = -nux * (S.u.n.xr[0][row][col] + S.u.n.xl[0][row][col + 1])
                             - nuy * (S.u.n.yr[0][row][col] + S.u.n.yl[0][row + 1][col]);
            const float d1 = -nux * (S.u.n.xr[1][row][col] + S.u.n.xl[1][row][col + 1])
                             - nuy * (S.u.n.yr[2][row][col] + S.u.n.yl[2][row + 1][col]);
            const float d2 = -nux * (S.u.n.xr[2][row][col] + S.u.n.xl[2][row][col + 1])
                             - nuy * (S.u.n.yr[1][row][col] + S.u.n.yl[1][row + 1][col]);
            const float ne = own_eta[k] + d0, nmu = own_mu[k] + d1, nmv = own_mv[k] + d2;
            const size_t o = (size_t)gj * V.nx + gi;
            V.o0[o] = ne;
            V.o1[o] = nmu;
            V.o2[o] = nmv;
            const float h = own_h[k] + d0;
            bad |= !(h > 0.f) || !isfinite(nmu) || !isfinite(nmv);
            smax = fmaxf(smax, cfl_f32(h, nmu, nmv, g, rdx, rdy, 1));
        }
    }
    __syncthreads();  // the next tile overwrites the shared buffers
    return smax;
}

// Walk tiles blockIdx.x, blockIdx.x + gridDim.x, ... of `src`, prefetching
// the next tile's raw values while computing the current one.
template <int TX, int TY, typename Src>
__device__ __forceinline__ float run_tiles(Smem<TX, TY> &S, const Src &src, float nux, float nuy,
                                           float g, int order, bool &bad) {
    float smax = 0.f;
    const int n = src.count();
    int k = blockIdx.x;
    if (k >= n) return smax;
    View v;
    int i0, j0;
    src.get(k, v, i0, j0);
    Raw<TX, TY> cur;
    load_raw<TX, TY>(v, i0, j0, cur);
    while (true) {
        const int kn = k + gridDim.x;
        View vn = v;
        int in0 = 0, jn0 = 0;
        Raw<TX, TY> nxt;
        if (kn < n) {
            src.get(kn, vn, in0, jn0);
            load_raw<TX, TY>(vn, in0, jn0, nxt);
        }
        smax = fmaxf(smax, tile_compute<TX, TY>(S, v, i0, j0, cur, nux, nuy, g, order, bad));
        if (kn >= n) break;
        k = kn; v = vn; i0 = in0; j0 = jn0; cur = nxt;
    }
    return smax;
}

// Thread 0 reads the clock and broadcasts nu_x, nu_y and the buffer index;
// false when the clock has reached t_end (no-op step).
__device__ __forceinline__ bool begin_step(DevClock *clkp, double t_end, double dx, double dy,
                                           float *s_nu, int *s_cur, int *s_run, double &t_now,
                                           double &dt) {
    if (threadIdx.x == 0) {
        volatile DevClock *clk = clkp;
        t_now = clk->t;
        dt = clk->dt_cfl;
        if (t_end - t_now < dt) dt = t_end - t_now;
        *s_run = dt > 0.0;
        s_nu[0] = (float)(dt / dx);
        s_nu[1] = (float)(dt / dy);
        *s_cur = clk->cur;
    }
    __syncthreads();
    return *s_run != 0;
}

// Block max of the CFL number (float, exact) -> partial[block]; the last block
// to arrive reduces the partials and advances the clock (t, dt, buffer,
// steps).  Only that block's thread 0 does FP64 work.
template <int NTH>
__device__ __forceinline__ void finish_step(DevClock *clkp, double *partial, int nblocks,
                                            double cfl, float sm, float *red, int *am_last,
                                            double t_now, double dt, int cur) {
    const int t = threadIdx.x;
    for (int o = 16; o > 0; o >>= 1) sm = fmaxf(sm, __shfl_xor_sync(0xffffffffu, sm, o));
    if ((t & 31) == 0) red[t >> 5] = sm;
    __syncthreads();
    const int bid = blockIdx.x + blockIdx.y * gridDim.x;
    if (t == 0) {
        float m = red[0];
        for (int k = 1; k < NTH / 32; k++) m = fmaxf(m, red[k]);
        reinterpret_cast<float *>(partial)[bid] = m;
        __threadfence();
        const unsigned int tk = atomicAdd(&clkp->ticket, 1u);
        *am_last = (tk == (unsigned int)(nblocks - 1));
    }
    __syncthreads();
    if (*am_last) {
        __threadfence();
        float m = 0.0f;
        const float *pf = reinterpret_cast<const float *>(partial);
        for (int k = t; k < nblocks; k += NTH) m = fmaxf(m, __ldcg(pf + k));
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        __syncthreads();
        if ((t & 31) == 0) red[t >> 5] = m;
        __syncthreads();
        if (t == 0) {
            for (int k = 0; k < NTH / 32; k++) m = fmaxf(m, red[k]);
            volatile DevClock *clk = clkp;
            clk->t = t_now + dt;
            clk->smax = (double)m;
            clk->dt_cfl = cfl / (double)m;
            clk->cur = cur ^ 1;
            clk->nsteps = clk->nsteps + 1;
            clk->ticket = 0u;
        }
    }
}

}  // namespace tile
}  // namespace swadj
