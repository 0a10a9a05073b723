// fwd_edge.cuh -- FP32 edge arithmetic of the forward step (Roe f-wave
// solve, MC-limited net fluxes) and the step's clock handshake, shared by
// the single-grid step (fwd_f32.cu) and the batched patch step (patches.cu)
// through the warp-strip machinery of strips.cuh.
//
// The MC-limited correction needs no division by the wave norm: for
// Z = b (1, s, vhat) and its upwind neighbour Zu = bu (1, su, vu),
// theta b = bu (1 + su s + vu vhat) / (1 + s^2 + vhat^2) and
// phi(theta) b = sign(b) max(0, min((|b| + sign(b) theta b)/2, 2|b|,
// 2 sign(b) theta b)), which is phi(theta) b for every b including b = 0.
#pragma once
#include "fwd_kernels.cuh"

namespace swadj {
namespace fwave {

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

}  // namespace fwave
}  // namespace swadj
