// fwd_pair.cuh -- FP32 edge arithmetic of the forward step (Sec. 6: Roe-type
// f-wave solver for the shallow water equations with bathymetry; the
// wave-propagation update with MC-limited corrections), written once for a
// float and for a pair of floats holding two independent edges.
//
// Every operation rounds as written (__fadd_rn/__fmul_rn, which the
// compiler never fuses, and explicit fmaf), so an edge gets the same bits
// whichever kernel computes it and whichever edges share its warp: the
// single-grid strips, the patch strips and the 1D step agree bit for bit.
//
// The update is branch-free.  A wave of speed s goes right with weight
// (1 + sign s)/2 (1, 1/2 at s = 0, 0) and left with the rest, so the
// fluctuations are A+dQ = sum (1 + sign s^p)/2 Z^p and A-dQ the rest (an
// f-wave of speed 0 is split half and half).  The MC-limited correction
// needs no division by the wave norm: for Z = b (1, s, vhat) and its upwind
// neighbour Zu = bu (1, su, vu), theta b = bu (1 + su s + vu vhat) /
// (1 + s^2 + vhat^2), and phi(theta) b is formed from b and theta b alone
// (zero when b = 0).  A warp whose edges are all subsonic (s1 < 0 < s3)
// takes the SUB form, which drops the operations whose outcome that fixes
// (weights 0 and 1, upwind sides, signs); it gives the same numbers as the
// general form, up to the sign of an exact zero.
#pragma once
#include "swadj_internal.cuh"

namespace swadj {
namespace fp {

// A pair of independent floats (two edges or two columns), each operated on
// by the scalar operations.  Packed FP32x2 instructions were measured for
// this: no faster in these kernels, and they did not reproduce the scalar
// bits.
struct __align__(8) f2 {
    float x, y;
};
__device__ __forceinline__ f2 mk(float x, float y) { f2 r; r.x = x; r.y = y; return r; }

__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float fms(float a, float b, float c) { return fmaf(a, b, -c); }   // ab - c
__device__ __forceinline__ float fnma(float a, float b, float c) { return fmaf(-a, b, c); }  // c - ab

__device__ __forceinline__ float neg(float a) { return -a; }
__device__ __forceinline__ f2 neg(f2 a) { return mk(-a.x, -a.y); }
__device__ __forceinline__ f2 add(f2 a, f2 b) { return mk(add(a.x, b.x), add(a.y, b.y)); }
__device__ __forceinline__ f2 sub(f2 a, f2 b) { return mk(sub(a.x, b.x), sub(a.y, b.y)); }
__device__ __forceinline__ f2 mul(f2 a, f2 b) { return mk(mul(a.x, b.x), mul(a.y, b.y)); }
__device__ __forceinline__ f2 fma(f2 a, f2 b, f2 c) {
    return mk(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
}
__device__ __forceinline__ f2 fms(f2 a, f2 b, f2 c) { return mk(fms(a.x, b.x, c.x), fms(a.y, b.y, c.y)); }
__device__ __forceinline__ f2 fnma(f2 a, f2 b, f2 c) {
    return mk(fnma(a.x, b.x, c.x), fnma(a.y, b.y, c.y));
}

template <class V> __device__ __forceinline__ V splat(float c);
template <> __device__ __forceinline__ float splat<float>(float c) { return c; }
template <> __device__ __forceinline__ f2 splat<f2>(float c) { return mk(c, c); }

__device__ __forceinline__ float rcp(float x) { return rcp_ftz(x); }
__device__ __forceinline__ f2 rcp(f2 x) { return mk(rcp_ftz(x.x), rcp_ftz(x.y)); }
__device__ __forceinline__ float rsq(float x) { return rsqrt_ftz(x); }
__device__ __forceinline__ f2 rsq(f2 x) { return mk(rsqrt_ftz(x.x), rsqrt_ftz(x.y)); }

// sign(s) in {-1, 0, 1}
__device__ __forceinline__ float sgn(float s) { return s > 0.f ? 1.f : (s < 0.f ? -1.f : 0.f); }
__device__ __forceinline__ f2 sgn(f2 s) { return mk(sgn(s.x), sgn(s.y)); }
// s > 0 ? a : b, per element
__device__ __forceinline__ float pick(float s, float a, float b) { return s > 0.f ? a : b; }
__device__ __forceinline__ f2 pick(f2 s, f2 a, f2 b) {
    return mk(s.x > 0.f ? a.x : b.x, s.y > 0.f ? a.y : b.y);
}
__device__ __forceinline__ bool subsonic(float s1, float s3) { return s1 < 0.f && s3 > 0.f; }
__device__ __forceinline__ bool subsonic(f2 s1, f2 s3) {
    return subsonic(s1.x, s3.x) && subsonic(s1.y, s3.y);
}

// Half the MC-limited wave strength: phi(theta) b / 2 for the MC limiter
// phi = max(0, min((1 + theta)/2, 2, 2 theta)), given b and r = theta b:
// sg max(0, min((|b| + sg r)/4, |b|, sg r)) with sg = sign(b) (+-1; the
// result is 0 at b = 0).  The factor 1/2 is exact, so twice this is the
// limited strength to the last bit.
__device__ __forceinline__ float mch(float b, float r) {
    const float sg = copysignf(1.f, b);
    const float B = fabsf(b), R = mul(sg, r);
    const float m = fminf(fminf(mul(0.25f, add(B, R)), B), R);
    return mul(sg, fmaxf(m, 0.f));
}
__device__ __forceinline__ f2 mch(f2 b, f2 r) { return mk(mch(b.x, r.x), mch(b.y, r.y)); }

// ------------------------------------------------------------------ records
// A cell in the frame of a sweep (mn the momentum normal to the edges, mt
// the tangential one) with the data its edges need: sqrt(h), sqrt(h) times
// the normal and tangential velocity (mn / sqrt(h), mt / sqrt(h)), the
// normal momentum flux mn^2 / h and the cross flux mn mt / h.
template <class V>
struct Cell {
    V h, mn, mt, sq, su, sv, P, T, eta;
};

// Waves of one edge: speeds s1 = uh - ch, s3 = uh + ch (and uh of the shear
// wave), the tangential Roe velocity and the strengths of the waves
// b1 (1, s1, vh), b2 (0, 0, 1), b3 (1, s3, vh).
template <class V>
struct Edge {
    V s1, s3, vh, b1, b2, b3, uh;
};

// The upwind neighbour of wave 1 or 3 for the limiter: its speed, tangential
// Roe velocity and strength.
template <class V>
struct Up {
    V s, vh, b;
};

// Net fluxes of an edge: L into the left (lower) cell, R into the right
// (upper) cell, in the edge's frame (Q -= nu * net).
template <class V>
struct Net {
    V L0, L1, L2, R0, R1, R2;
};

// Cell data in the frame of a sweep from (eta, h, mn, mt).
template <class V>
__device__ __forceinline__ Cell<V> derive(V eta, V h, V mn, V mt) {
    const V q = rsq(h);
    Cell<V> c;
    c.h = h; c.mn = mn; c.mt = mt; c.eta = eta;
    c.sq = mul(h, q);
    c.su = mul(mn, q);
    c.sv = mul(mt, q);
    c.P = mul(c.su, c.su);
    c.T = mul(c.su, c.sv);
    return c;
}

// Roe f-wave decomposition (Sec. 6 solver): hhat = (hL + hR)/2, uhat and
// vhat sqrt(h)-weighted ((sqrt(hL) uL + sqrt(hR) uR) / (sqrt(hL) +
// sqrt(hR))), chat = sqrt(g hhat); the momentum jump carries the bathymetry
// source as g hhat (etaR - etaL), so the ocean at rest has no waves.
// 1 / (s3 - s1) = 1 / (2 chat) comes from the same rsqrt as chat.
template <class V>
__device__ __forceinline__ Edge<V> solve(V g_half, const Cell<V> &L, const Cell<V> &R) {
    Edge<V> w;
    const V gh = mul(g_half, add(L.h, R.h));   // g hhat
    const V rd = rcp(add(L.sq, R.sq));
    w.uh = mul(add(L.su, R.su), rd);
    w.vh = mul(add(L.sv, R.sv), rd);
    const V rc = rsq(gh);
    const V ch = mul(gh, rc);
    w.s1 = sub(w.uh, ch);
    w.s3 = add(w.uh, ch);
    const V df1 = sub(R.mn, L.mn);
    const V df2 = fma(gh, sub(R.eta, L.eta), sub(R.P, L.P));
    const V df3 = sub(R.T, L.T);
    const V hr = mul(splat<V>(0.5f), rc);
    w.b1 = mul(fms(w.s3, df1, df2), hr);
    w.b3 = mul(fnma(w.s1, df1, df2), hr);
    w.b2 = fnma(w.vh, df1, df3);
    return w;
}

// Fluctuations and MC-limited correction of edge w: L = A-dQ + F into the
// left cell, R = A+dQ - F into the right cell.  A wave of speed s goes right
// with weight (1 + sign s)/2 (half each way at s = 0); F = sum_p sign(s^p)/2
// (1 - nu |s^p|) phi(theta^p) Z^p, computed as (sign(s) - nu s) times half
// the limited strength (the same number).  u1, u3: the upwind neighbours of
// waves 1 and 3 (the left edge for s > 0, the right one otherwise); b2l,
// b2r: the shear-wave strengths of the left and right edges.  SUB: every
// edge of w is subsonic (s1 < 0 < s3), so wave 1 goes left and wave 3 right.
template <class V, bool SUB>
__device__ __forceinline__ Net<V> net(const Edge<V> &w, const Up<V> &u1, const Up<V> &u3, V b2l,
                                      V b2r, V nu, int order) {
    const V one = splat<V>(1.f), half = splat<V>(0.5f);
    const V g2 = sgn(w.uh);
    V ap0, ap1, am0, am1, k1, k3;
    if (SUB) {
        ap0 = w.b3;
        ap1 = mul(w.b3, w.s3);
        am0 = w.b1;
        am1 = mul(w.b1, w.s1);
        k1 = neg(fma(nu, w.s1, one));   // sign(s1) - nu s1
        k3 = fnma(nu, w.s3, one);
    } else {
        const V g1 = sgn(w.s1), g3 = sgn(w.s3);
        const V a1 = mul(fma(half, g1, half), w.b1), a3 = mul(fma(half, g3, half), w.b3);
        const V e1 = sub(w.b1, a1), e3 = sub(w.b3, a3);
        ap0 = add(a1, a3);
        am0 = add(e1, e3);
        ap1 = fma(a1, w.s1, mul(a3, w.s3));
        am1 = fma(e1, w.s1, mul(e3, w.s3));
        k1 = fnma(nu, w.s1, g1);
        k3 = fnma(nu, w.s3, g3);
    }
    const V a2 = mul(fma(half, g2, half), w.b2), e2 = sub(w.b2, a2);
    const V ap2 = fma(ap0, w.vh, a2), am2 = fma(am0, w.vh, e2);
    Net<V> n;
    if (order >= 2) {
        // theta^p b^p = b_up (1 + s_up s + v_up vhat) / (1 + s^2 + vhat^2)
        const V v2 = fma(w.vh, w.vh, one);
        const V m1 = fma(w.s1, w.s1, v2), m3 = fma(w.s3, w.s3, v2);
        const V d1 = fma(u1.s, w.s1, fma(u1.vh, w.vh, one));
        const V d3 = fma(u3.s, w.s3, fma(u3.vh, w.vh, one));
        const V l1 = mch(w.b1, mul(mul(u1.b, d1), rcp(m1)));
        const V l3 = mch(w.b3, mul(mul(u3.b, d3), rcp(m3)));
        const V l2 = mch(w.b2, pick(w.uh, b2l, b2r));
        const V c1 = mul(k1, l1), c3 = mul(k3, l3);
        const V c2 = mul(fnma(nu, w.uh, g2), l2);
        const V F0 = add(c1, c3);
        const V F1 = fma(c1, w.s1, mul(c3, w.s3));
        const V F2 = fma(F0, w.vh, c2);
        n.L0 = add(am0, F0); n.L1 = add(am1, F1); n.L2 = add(am2, F2);
        n.R0 = sub(ap0, F0); n.R1 = sub(ap1, F1); n.R2 = sub(ap2, F2);
    } else {
        n.L0 = am0; n.L1 = am1; n.L2 = am2;
        n.R0 = ap0; n.R1 = ap1; n.R2 = ap2;
    }
    return n;
}

// Upwind neighbours of an edge from its left (wl) and right (wr) edges.
template <class V>
__device__ __forceinline__ void upwind(const Edge<V> &w, const Edge<V> &wl, const Edge<V> &wr,
                                       Up<V> &u1, Up<V> &u3) {
    u1.s = pick(w.s1, wl.s1, wr.s1); u1.vh = pick(w.s1, wl.vh, wr.vh);
    u1.b = pick(w.s1, wl.b1, wr.b1);
    u3.s = pick(w.s3, wl.s3, wr.s3); u3.vh = pick(w.s3, wl.vh, wr.vh);
    u3.b = pick(w.s3, wl.b3, wr.b3);
}

// Net fluxes of the middle edge of three consecutive edges held by one
// thread (1D step, y-sweeps): the form is SUB when `all_sub`.
template <class V>
__device__ __forceinline__ Net<V> net3(const Edge<V> &wl, const Edge<V> &w, const Edge<V> &wr,
                                       V nu, int order, bool all_sub) {
    Up<V> u1, u3;
    if (all_sub) {
        u1.s = wr.s1; u1.vh = wr.vh; u1.b = wr.b1;
        u3.s = wl.s3; u3.vh = wl.vh; u3.b = wl.b3;
        return net<V, true>(w, u1, u3, wl.b2, wr.b2, nu, order);
    }
    upwind(w, wl, wr, u1, u3);
    return net<V, false>(w, u1, u3, wl.b2, wr.b2, nu, order);
}

}  // namespace fp
}  // namespace swadj
