// fwd_tiles.cuh -- FP32 tile machinery of the forward step, shared by the
// single-grid step (fwd_f32.cu) and the batched patch step (patches.cu).
//
// A tile is TX x TY cells of one grid ("view").  The step is dimensionally
// split (x-sweep, then y-sweep of the x-swept state).  Phases per tile:
// (0) stage the tile and a 2-cell halo including corners as derived cell
// data in shared memory; (1) x-edge waves of every staged row; (2) their net
// fluxes (limiter once per edge); (3) x-sweep of the tile's columns in every
// staged row, in place (the y-sweep needs the x-swept state in the two halo
// rows); (4) y-edge waves of the x-swept state; (5) their net fluxes;
// (6) y-sweep update of the tile's cells.  Each phase is a flat loop of
// independent items over 256 threads.  Cell data, edge waves and net fluxes
// are kept as 16- and 8-byte records so that each item moves them with a few
// vector shared-memory accesses.  A persistent block walks its share of a
// tile list; the raw values of the next tile are loaded into registers while
// the current one is computed.
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

__device__ __forceinline__ float rcpf(float x) { return rcp_ftz(x); }
// Rounded single operations that the compiler never fuses: with these and
// explicit fmaf the rounding of every expression below is fixed in the
// source, so an edge's numbers do not depend on the kernel that inlines it.
__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
// 1 if s > 0, 0 if s < 0, 1/2 if s == 0 (an f-wave of speed 0 is split)
__device__ __forceinline__ float pos1(float s) { return s > 0.f ? 1.f : (s < 0.f ? 0.f : 0.5f); }
// sign(s) / 2
__device__ __forceinline__ float hsg1(float s) { return s > 0.f ? 0.5f : (s < 0.f ? -0.5f : 0.f); }
// phi(theta) b for the MC limiter, r = theta b
__device__ __forceinline__ float mc1(float b, float r) {
    const float sg = b < 0.f ? -1.f : 1.f;
    const float B = fabsf(b), Rr = mul(sg, r);
    float m = fminf(mul(0.5f, add(B, Rr)), mul(2.f, B));
    m = fminf(m, mul(2.f, Rr));
    return mul(sg, fmaxf(m, 0.f));
}

struct EdgeS {           // wave data of one edge
    float s1, s3, vh, b1, b2, b3;
};

// Roe f-wave decomposition at an edge in its (normal, tangential) frame.
__device__ __forceinline__ EdgeS solve1(float g, float hL, float mnL, float mtL, float unL,
                                        float utL, float sqL, float etaL, float hR, float mnR,
                                        float mtR, float unR, float utR, float sqR, float etaR) {
    EdgeS w;
    const float hh = mul(0.5f, add(hL, hR));
    const float rd = rcpf(add(sqL, sqR));
    const float uh = mul(fmaf(sqL, unL, mul(sqR, unR)), rd);
    const float vh = mul(fmaf(sqL, utL, mul(sqR, utR)), rd);
    const float gh = mul(g, hh);
    const float rc = rsqrt_ftz(gh);
    const float ch = mul(gh, rc);
    const float s1 = sub(uh, ch), s3 = add(uh, ch);
    const float df1 = sub(mnR, mnL);
    const float df2 = fmaf(gh, sub(etaR, etaL), fmaf(mnR, unR, -mul(mnL, unL)));
    const float df3 = fmaf(mnR, utR, -mul(mnL, utL));
    const float hr = mul(0.5f, rc);  // 1 / (s3 - s1)
    w.s1 = s1;
    w.s3 = s3;
    w.vh = vh;
    w.b1 = mul(fmaf(s3, df1, -df2), hr);
    w.b3 = mul(fmaf(-s1, df1, df2), hr);
    w.b2 = fmaf(-vh, df1, df3);
    return w;
}

// Net fluxes of edge w (neighbours wl, wr): L into the left cell, R into the
// right cell (Q -= nu * net).  SUB: the edge is subsonic (s1 < 0 < s3), so
// the sign logic of waves 1 and 3 is fixed.  The two forms round
// differently, so callers pick SUB exactly when sub1(w) holds: the result of
// an edge then depends on that edge alone, not on its warp.
template <bool SUB>
__device__ __forceinline__ void net1(const EdgeS &wl, const EdgeS &w, const EdgeS &wr, float nu,
                                     int order, float L[3], float R[3]) {
    const float s2 = mul(0.5f, add(w.s1, w.s3));
    const float p2 = pos1(s2);
    float ap0, ap1, ap2, am0, am1, am2;
    if (SUB) {
        ap0 = w.b3; ap1 = mul(w.b3, w.s3); ap2 = fmaf(p2, w.b2, mul(w.b3, w.vh));
        am0 = w.b1; am1 = mul(w.b1, w.s1); am2 = add(mul(w.b1, w.vh), fmaf(-p2, w.b2, w.b2));
    } else {
        const float a1 = mul(pos1(w.s1), w.b1), a3 = mul(pos1(w.s3), w.b3);
        ap0 = add(a1, a3); ap1 = fmaf(a1, w.s1, mul(a3, w.s3)); ap2 = fmaf(p2, w.b2, mul(ap0, w.vh));
        const float t0 = add(w.b1, w.b3);
        am0 = sub(t0, ap0);
        am1 = sub(fmaf(w.b1, w.s1, mul(w.b3, w.s3)), ap1);
        am2 = sub(fmaf(t0, w.vh, w.b2), ap2);
    }
    float F0 = 0.f, F1 = 0.f, F2 = 0.f;
    if (order >= 2) {
        const EdgeS &u1 = (!SUB && w.s1 > 0.f) ? wl : wr;
        const EdgeS &u3 = (SUB || w.s3 > 0.f) ? wl : wr;
        const float m1 = fmaf(w.s1, w.s1, fmaf(w.vh, w.vh, 1.f));
        const float d1 = fmaf(u1.s1, w.s1, fmaf(u1.vh, w.vh, 1.f));
        const float l1 = mc1(w.b1, mul(mul(u1.b1, d1), rcpf(m1)));
        const float m3 = fmaf(w.s3, w.s3, fmaf(w.vh, w.vh, 1.f));
        const float d3 = fmaf(u3.s3, w.s3, fmaf(u3.vh, w.vh, 1.f));
        const float l3 = mc1(w.b3, mul(mul(u3.b3, d3), rcpf(m3)));
        const float l2 = mc1(w.b2, s2 > 0.f ? wl.b2 : wr.b2);
        float c1, c3;
        if (SUB) {
            c1 = mul(mul(-0.5f, fmaf(nu, w.s1, 1.f)), l1);
            c3 = mul(mul(0.5f, fmaf(-nu, w.s3, 1.f)), l3);
        } else {
            c1 = mul(mul(hsg1(w.s1), fmaf(-nu, fabsf(w.s1), 1.f)), l1);
            c3 = mul(mul(hsg1(w.s3), fmaf(-nu, fabsf(w.s3), 1.f)), l3);
        }
        const float c2 = mul(mul(hsg1(s2), fmaf(-nu, fabsf(s2), 1.f)), l2);
        F0 = add(c1, c3);
        F1 = fmaf(c1, w.s1, mul(c3, w.s3));
        F2 = fmaf(F0, w.vh, c2);
    }
    L[0] = add(am0, F0); L[1] = add(am1, F1); L[2] = add(am2, F2);
    R[0] = sub(ap0, F0); R[1] = sub(ap1, F1); R[2] = sub(ap2, F2);
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
    // cell data of the tile + halo (with corners), x-swept in place, as two
    // 16-byte records read with one vector load each:
    // a = (h, hu, hv, eta), b = (u, v, sqrt(h), unused)
    float4 a[RY][RX], b[RY][RX];
    union W {   // edge waves p = (s1, s3, vhat, b1), q = (b2, b3): x (phases 1-2), then y (4-5)
        struct X { float4 p[RY][NEX]; float2 q[RY][NEX]; } x;
        struct Y { float4 p[NEY][TX]; float2 q[NEY][TX]; } y;
    } w;
    union N {   // net fluxes lr = (L0, L1, L2, R0), r = (R1, R2): x (phases 2-3), then y (5-6)
        struct X { float4 lr[RY][TX + 1]; float2 r[RY][TX + 1]; } x;
        struct Y { float4 lr[TY + 1][TX]; float2 r[TY + 1][TX]; } y;
    } n;
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
        if (r >= RX * RY) continue;
        const int ry = r / RX, rx = r - ry * RX;
        int ci = i0 + rx - 2, cj = j0 + ry - 2;
        bool fx = false, fy = false;
        if (!interior) {
            ci = ghost_index(ci, V.nx, V.bc.lo_x, V.bc.hi_x, &fx);
            cj = ghost_index(cj, V.ny, V.bc.lo_y, V.bc.hi_y, &fy);
        }
        const size_t o = (size_t)cj * V.nx + ci;
        R.eta[k] = ld_early(V.q0 + o);
        R.hb[k] = ld_early(V.hb + o);
        const float mu = ld_early(V.q1 + o), mv = ld_early(V.q2 + o);
        R.mu[k] = fx ? -mu : mu;
        R.mv[k] = fy ? -mv : mv;
    }
}

template <typename SM>
__device__ __forceinline__ void put_cell(SM &S, int ry, int rx, float eta, float h, float mu,
                                         float mv) {
    const float q = rsqrt_ftz(h);
    const float ih = mul(q, q);
    S.a[ry][rx] = make_float4(h, mu, mv, eta);
    S.b[ry][rx] = make_float4(mul(mu, ih), mul(mv, ih), mul(h, q), 0.f);
}

__device__ __forceinline__ EdgeS edge_of(const float4 &p, const float2 &q) {
    EdgeS w;
    w.s1 = p.x; w.s3 = p.y; w.vh = p.z; w.b1 = p.w; w.b2 = q.x; w.b3 = q.y;
    return w;
}

// Net fluxes L (into the left / lower cell) and R (into the right / upper
// cell) of the middle edge b, neighbours a and c.
__device__ __forceinline__ void net_of(const EdgeS &a, const EdgeS &b, const EdgeS &c, float nu,
                                       int order, float4 &lr, float2 &r) {
    float L[3], Rr[3];
    if (sub1(b)) net1<true>(a, b, c, nu, order, L, Rr);
    else net1<false>(a, b, c, nu, order, L, Rr);
    lr = make_float4(L[0], L[1], L[2], Rr[0]);
    r = make_float2(Rr[1], Rr[2]);
}

// Phases 0-6 for one tile whose raw values are in R.  Returns the tile's
// maximum CFL number over its new cells.
template <int TX, int TY>
__device__ __forceinline__ float tile_compute(Smem<TX, TY> &S, const View &V, int i0, int j0,
                                              const Raw<TX, TY> &R, float nux, float nuy,
                                              float g, int order, bool &bad) {
    constexpr int RX = TX + 4, RY = TY + 4, NEX = TX + 3, NEY = TY + 3;
    const int tid = threadIdx.x;
    // phase 0: derived cell data of the whole staged region
#pragma unroll
    for (int k = 0; k < Raw<TX, TY>::RPT; k++) {
        const int r = tid + k * NT;
        if (r >= RX * RY) continue;
        const int ry = r / RX, rx = r - ry * RX;
        put_cell(S, ry, rx, R.eta[k], R.eta[k] + R.hb[k], R.mu[k], R.mv[k]);
    }
    __syncthreads();
    // phase 1: x-edge waves of every staged row (edge e between cols e, e+1)
    for (int i = tid; i < RY * NEX; i += NT) {
        const int ry = i / NEX, e = i - ry * NEX;
        const float4 aL = S.a[ry][e], bL = S.b[ry][e], aR = S.a[ry][e + 1], bR = S.b[ry][e + 1];
        const EdgeS w = solve1(g, aL.x, aL.y, aL.z, bL.x, bL.y, bL.z, aL.w, aR.x, aR.y, aR.z,
                               bR.x, bR.y, bR.z, aR.w);
        S.w.x.p[ry][e] = make_float4(w.s1, w.s3, w.vh, w.b1);
        S.w.x.q[ry][e] = make_float2(w.b2, w.b3);
    }
    __syncthreads();
    // phase 2: x net fluxes of edges 1 .. TX+1 in every staged row
    for (int i = tid; i < RY * (TX + 1); i += NT) {
        const int ry = i / (TX + 1), e = 1 + (i - ry * (TX + 1));
        const EdgeS wa = edge_of(S.w.x.p[ry][e - 1], S.w.x.q[ry][e - 1]);
        const EdgeS wb = edge_of(S.w.x.p[ry][e], S.w.x.q[ry][e]);
        const EdgeS wc = edge_of(S.w.x.p[ry][e + 1], S.w.x.q[ry][e + 1]);
        net_of(wa, wb, wc, nux, order, S.n.x.lr[ry][e - 1], S.n.x.r[ry][e - 1]);
    }
    __syncthreads();
    // phase 3: x-sweep of the tile's columns in every staged row, in place
    for (int i = tid; i < RY * TX; i += NT) {
        const int ry = i / TX, col = i - ry * TX, rx = col + 2;
        // left edge of column col -> R at index col, right edge -> L at col + 1
        const float4 le = S.n.x.lr[ry][col];
        const float2 lr = S.n.x.r[ry][col];
        const float4 re = S.n.x.lr[ry][col + 1];
        const float4 c = S.a[ry][rx];
        const float d0 = mul(-nux, add(le.w, re.x));
        const float d1 = mul(-nux, add(lr.x, re.y));
        const float d2 = mul(-nux, add(lr.y, re.z));
        put_cell(S, ry, rx, add(c.w, d0), add(c.x, d0), add(c.y, d1), add(c.z, d2));
    }
    __syncthreads();
    // phase 4: y-edge waves of the x-swept state, tile columns (frame (h, hv, hu))
    for (int i = tid; i < NEY * TX; i += NT) {
        const int e = i / TX, col = i - e * TX, rx = col + 2;
        const float4 aL = S.a[e][rx], bL = S.b[e][rx], aR = S.a[e + 1][rx], bR = S.b[e + 1][rx];
        const EdgeS w = solve1(g, aL.x, aL.z, aL.y, bL.y, bL.x, bL.z, aL.w, aR.x, aR.z, aR.y,
                               bR.y, bR.x, bR.z, aR.w);
        S.w.y.p[e][col] = make_float4(w.s1, w.s3, w.vh, w.b1);
        S.w.y.q[e][col] = make_float2(w.b2, w.b3);
    }
    __syncthreads();
    // phase 5: y net fluxes of edges 1 .. TY+1
    for (int i = tid; i < (TY + 1) * TX; i += NT) {
        const int e = 1 + i / TX, col = i - (e - 1) * TX;
        const EdgeS wa = edge_of(S.w.y.p[e - 1][col], S.w.y.q[e - 1][col]);
        const EdgeS wb = edge_of(S.w.y.p[e][col], S.w.y.q[e][col]);
        const EdgeS wc = edge_of(S.w.y.p[e + 1][col], S.w.y.q[e + 1][col]);
        net_of(wa, wb, wc, nuy, order, S.n.y.lr[e - 1][col], S.n.y.r[e - 1][col]);
    }
    __syncthreads();
    // phase 6: y-sweep update of the tile's cells; y nets are in (h, hv, hu)
    // order, lower edge of row -> R at index row, upper edge -> L at row + 1
    float smax = 0.f;
    const float rdx = 1.f / V.dx, rdy = 1.f / V.dy;
    constexpr int CPT = TX * TY / NT;
#pragma unroll
    for (int k = 0; k < CPT; k++) {
        const int c = tid + k * NT, row = c / TX, col = c % TX;
        const int gi = i0 + col, gj = j0 + row;
        const int ry = row + 2, rx = col + 2;
        if (gi < V.nx && gj < V.ny) {
            const float4 lo = S.n.y.lr[row][col];
            const float2 lr = S.n.y.r[row][col];
            const float4 up = S.n.y.lr[row + 1][col];
            const float4 cc = S.a[ry][rx];
            const float d0 = mul(-nuy, add(lo.w, up.x));
            const float d2 = mul(-nuy, add(lr.x, up.y));
            const float d1 = mul(-nuy, add(lr.y, up.z));
            const float ne = add(cc.w, d0), nmu = add(cc.y, d1), nmv = add(cc.z, d2);
            const size_t o = (size_t)gj * V.nx + gi;
            V.o0[o] = ne;
            V.o1[o] = nmu;
            V.o2[o] = nmv;
            const float h = add(cc.x, d0);
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
                                            double t_now, double dt, int cur,
                                            bool fence_all = false) {
    const int t = threadIdx.x;
    // with fused gauges the last block reads the new state of every block:
    // each thread makes its own writes visible before the block signals
    if (fence_all) __threadfence();
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
