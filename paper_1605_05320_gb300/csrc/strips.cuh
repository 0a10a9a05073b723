// strips.cuh -- warp-strip machinery of the FP32 2D forward step (Sec. 5,
// Sec. 6 solver; dimensionally split, x-sweep then y-sweep), shared by the
// single-grid step (fwd_f32.cu) and the batched patch step (patches.cu).
//
// A warp owns a strip of 32 columns (lanes) of one grid or patch, the
// middle 28 its output, and `rows` output rows, which it walks downwards.
// Each loaded row (the output rows and two halo rows above and below) is
// x-swept across the warp with shuffles, lane l solving and limiting edge
// (l|l+1) once; the y-sweep of the x-swept rows runs in registers over a
// sliding window of rows, each y-edge solved and limited once.  Rows are
// loaded one iteration ahead of their use.  Ghost cells outside the grid are
// index-mapped on load (copy, or mirror with the normal momentum negated);
// the x-sweep commutes with the y-mirror, so ghost rows may be x-swept like
// any other.  Per edge the arithmetic is fwd_edge.cuh's, so results depend
// neither on the strip height nor on how edges share a warp.
#pragma once
#include "fwd_edge.cuh"
#include "fwd_kernels.cuh"

namespace swadj {
namespace strip {

constexpr int kLanes = 32;
constexpr int kOut = kLanes - 4;        // output columns per strip
constexpr int kThreads = 128;           // 4 warps per block (~90 registers a thread)
constexpr unsigned kFull = 0xffffffffu;

// One grid or patch as a strip sees it.
struct View {
    const float *q0, *q1, *q2, *hb;   // current state (eta, hu, hv) and hbar = -B
    float *o0, *o1, *o2;              // new state
    int nx, ny;
    float rdx, rdy;                   // 1 / dx, 1 / dy (for the CFL term)
    BcSpec bc;
};

struct XCell {   // derived cell data
    float h, mu, mv, u, v, sq, eta;
};

__device__ __forceinline__ XCell derive(float eta, float h, float mu, float mv) {
    const float q = rsqrt_ftz(h);
    const float ih = fwave::mul(q, q);
    XCell c;
    c.h = h; c.mu = mu; c.mv = mv;
    c.u = fwave::mul(mu, ih); c.v = fwave::mul(mv, ih); c.sq = fwave::mul(h, q);
    c.eta = eta;
    return c;
}

__device__ __forceinline__ float dn(float x) { return __shfl_down_sync(kFull, x, 1); }
__device__ __forceinline__ float up(float x) { return __shfl_up_sync(kFull, x, 1); }

__device__ __forceinline__ fwave::EdgeS edge_dn(const fwave::EdgeS &w) {
    fwave::EdgeS r;
    r.s1 = dn(w.s1); r.s3 = dn(w.s3); r.vh = dn(w.vh);
    r.b1 = dn(w.b1); r.b2 = dn(w.b2); r.b3 = dn(w.b3);
    return r;
}
__device__ __forceinline__ fwave::EdgeS edge_up(const fwave::EdgeS &w) {
    fwave::EdgeS r;
    r.s1 = up(w.s1); r.s3 = up(w.s3); r.vh = up(w.vh);
    r.b1 = up(w.b1); r.b2 = up(w.b2); r.b3 = up(w.b3);
    return r;
}

// x-sweep of one row held across the warp; valid in lanes 2..29.
__device__ __forceinline__ XCell xsweep(const XCell &c, float g, float nux, int order) {
    const fwave::EdgeS w = fwave::solve1(g, c.h, c.mu, c.mv, c.u, c.v, c.sq, c.eta, dn(c.h),
                                         dn(c.mu), dn(c.mv), dn(c.u), dn(c.v), dn(c.sq),
                                         dn(c.eta));   // edge (l|l+1)
    float4 lr;
    float2 r;
    fwave::net_of(edge_up(w), w, edge_dn(w), nux, order, lr, r);
    // left edge of the cell -> R of edge (l-1|l), right edge -> L of edge (l|l+1)
    const float d0 = fwave::mul(-nux, fwave::add(up(lr.w), lr.x));
    const float d1 = fwave::mul(-nux, fwave::add(up(r.x), lr.y));
    const float d2 = fwave::mul(-nux, fwave::add(up(r.y), lr.z));
    return derive(fwave::add(c.eta, d0), fwave::add(c.h, d0), fwave::add(c.mu, d1),
                  fwave::add(c.mv, d2));
}

// y-edge waves between x-swept cells a (below) and b (above), frame (h, hv, hu)
__device__ __forceinline__ fwave::EdgeS ysolve(const XCell &a, const XCell &b, float g) {
    return fwave::solve1(g, a.h, a.mv, a.mu, a.v, a.u, a.sq, a.eta, b.h, b.mv, b.mu, b.v, b.u,
                         b.sq, b.eta);
}

struct Raw4 {
    float eta, mu, mv, hb;
};

__device__ __forceinline__ Raw4 load_raw(const View &v, int col, bool fx, int row, bool fy) {
    const size_t o = (size_t)row * v.nx + col;
    Raw4 r;
    r.eta = ld_early(v.q0 + o);
    r.hb = ld_early(v.hb + o);
    const float mu = ld_early(v.q1 + o), mv = ld_early(v.q2 + o);
    r.mu = fx ? -mu : mu;
    r.mv = fy ? -mv : mv;
    return r;
}

// One strip of view v: output columns x0 .. x0 + 27 and rows y0 .. y0 +
// rows - 1 (clipped to the view).  Called by all 32 lanes of a warp.
// Accumulates the CFL maximum of the new cells into smax and sets bad on a
// non-positive depth or non-finite momentum.
__device__ __forceinline__ void strip_unit(const View &v, int x0, int y0, int rows, float nux,
                                           float nuy, float g, int order, float &smax,
                                           bool &bad) {
    const int lane = threadIdx.x & 31;
    const int ylast = (y0 + rows < v.ny ? y0 + rows : v.ny) - 1;
    const int gi = x0 - 2 + lane;
    bool fx, fy;
    const int col = ghost_index(gi, v.nx, v.bc.lo_x, v.bc.hi_x, &fx);
    const bool out = lane >= 2 && lane < kLanes - 2 && gi < v.nx;
    XCell A = {}, B = {};            // x-swept rows j-2, j-1
    fwave::EdgeS W1 = {}, W2 = {};   // y-edges (j-3|j-2), (j-2|j-1)
    float4 nlr = make_float4(0.f, 0.f, 0.f, 0.f);   // y-net of edge (j-3|j-2)
    float2 nr = make_float2(0.f, 0.f);
    // strips away from the lower and upper boundary need no row mapping
    const bool yin = y0 - 2 >= 0 && ylast + 2 < v.ny;
    fy = false;
    int row = yin ? y0 - 2 : ghost_index(y0 - 2, v.ny, v.bc.lo_y, v.bc.hi_y, &fy);
    Raw4 Rn = load_raw(v, col, fx, row, fy);
#pragma unroll 3
    for (int j = y0 - 2; j <= ylast + 2; j++) {
        const Raw4 Rc = Rn;
        if (j < ylast + 2) {
            if (yin) row = j + 1;
            else row = ghost_index(j + 1, v.ny, v.bc.lo_y, v.bc.hi_y, &fy);
            Rn = load_raw(v, col, fx, row, fy);
        }
        const XCell C = xsweep(derive(Rc.eta, Rc.eta + Rc.hb, Rc.mu, Rc.mv), g, nux, order);
        fwave::EdgeS Wn = W2;
        if (j >= y0 - 1) Wn = ysolve(B, C, g);   // edge (j-1|j)
        float4 lr = make_float4(0.f, 0.f, 0.f, 0.f);
        float2 r = make_float2(0.f, 0.f);
        if (j >= y0 + 1) fwave::net_of(W1, W2, Wn, nuy, order, lr, r);   // edge (j-2|j-1)
        if (j >= y0 + 2 && out) {
            // y-sweep of row j-2: lower edge -> R of the previous net, upper
            // edge -> L of this one; nets are in (h, hv, hu) order
            const float d0 = fwave::mul(-nuy, fwave::add(nlr.w, lr.x));
            const float d2 = fwave::mul(-nuy, fwave::add(nr.x, lr.y));
            const float d1 = fwave::mul(-nuy, fwave::add(nr.y, lr.z));
            const float ne = fwave::add(A.eta, d0), nmu = fwave::add(A.mu, d1);
            const float nmv = fwave::add(A.mv, d2);
            const size_t o = (size_t)(j - 2) * v.nx + gi;
            v.o0[o] = ne;
            v.o1[o] = nmu;
            v.o2[o] = nmv;
            const float h = fwave::add(A.h, d0);
            bad |= !(h > 0.f) || !isfinite(nmu) || !isfinite(nmv);
            smax = fmaxf(smax, cfl_f32(h, nmu, nmv, g, v.rdx, v.rdy, 1));
        }
        A = B; B = C;
        W1 = W2; W2 = Wn;
        nlr = lr; nr = r;
    }
}

}  // namespace strip
}  // namespace swadj
