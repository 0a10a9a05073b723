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
// any other.  Per edge the arithmetic is fwd_pair.cuh's, so results depend
// neither on the strip height nor on how edges share a warp.
#pragma once
#include "fwd_edge.cuh"
#include "fwd_kernels.cuh"
#include "fwd_pair.cuh"

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

__device__ __forceinline__ float dn(float x) { return __shfl_down_sync(kFull, x, 1); }
__device__ __forceinline__ float up(float x) { return __shfl_up_sync(kFull, x, 1); }

// How a lane reaches the cells and edges beside its own along x: one
// column per lane, the neighbours are the lanes beside it (a policy, so the
// x-sweep below serves other lane layouts too).  ok(): whether
// the warp may take the SUB form, given this lane's edge (the nets of edges
// (1|2) .. (29|30) are used).
struct Nb1 {
    typedef float V;
    static __device__ __forceinline__ float l(float x) { return up(x); }
    static __device__ __forceinline__ float r(float x) { return dn(x); }
    static __device__ __forceinline__ bool ok(const fp::Edge<float> &w, int lane) {
        return lane < 1 || lane > kLanes - 3 || fp::subsonic(w.s1, w.s3);
    }
};

// Net fluxes of a lane's x-edge(s) w, fetching the neighbour edges the
// limiter needs from the lanes beside it: in the SUB form only the upwind
// values (wave 1 from the right edge, wave 3 from the left, both shear
// strengths), otherwise both neighbours in full.
template <class NB>
__device__ __forceinline__ fp::Net<typename NB::V> xnet(const fp::Edge<typename NB::V> &w,
                                                        typename NB::V nu, int order,
                                                        bool all_sub) {
    typedef typename NB::V V;
    fp::Up<V> u1, u3;
    if (all_sub) {
        V b2l = w.b2, b2r = w.b2;
        if (order >= 2) {
            u1.s = NB::r(w.s1); u1.vh = NB::r(w.vh); u1.b = NB::r(w.b1);
            u3.s = NB::l(w.s3); u3.vh = NB::l(w.vh); u3.b = NB::l(w.b3);
            b2l = NB::l(w.b2); b2r = NB::r(w.b2);
        }
        return fp::net<V, true>(w, u1, u3, b2l, b2r, nu, order);
    }
    fp::Edge<V> wl = w, wr = w;
    if (order >= 2) {
        wl.s1 = NB::l(w.s1); wl.s3 = NB::l(w.s3); wl.vh = NB::l(w.vh);
        wl.b1 = NB::l(w.b1); wl.b2 = NB::l(w.b2); wl.b3 = NB::l(w.b3);
        wr.s1 = NB::r(w.s1); wr.s3 = NB::r(w.s3); wr.vh = NB::r(w.vh);
        wr.b1 = NB::r(w.b1); wr.b2 = NB::r(w.b2); wr.b3 = NB::r(w.b3);
    }
    fp::upwind(w, wl, wr, u1, u3);
    return fp::net<V, false>(w, u1, u3, wl.b2, wr.b2, nu, order);
}

// x-sweep of one row held across the warp (x frame: mn = hu, mt = hv).
// Returns the x-swept cell(s) in the y frame (mn = hv).  Lanes see their
// right neighbour cells through NB::r; a cell takes R of the edge on its left
// and L of the edge on its right.
template <class NB>
__device__ __forceinline__ fp::Cell<typename NB::V> xsweep(const fp::Cell<typename NB::V> &c,
                                                           typename NB::V g_half, float nux,
                                                           int order, int lane) {
    typedef typename NB::V V;
    fp::Cell<V> r;
    r.h = NB::r(c.h); r.mn = NB::r(c.mn); r.mt = c.mt; r.sq = NB::r(c.sq);
    r.su = NB::r(c.su); r.sv = NB::r(c.sv); r.P = NB::r(c.P); r.T = NB::r(c.T);
    r.eta = NB::r(c.eta);
    const fp::Edge<V> w = fp::solve(g_half, c, r);
    const fp::Net<V> n =
        xnet<NB>(w, fp::splat<V>(nux), order, __all_sync(kFull, NB::ok(w, lane)));
    const V mnu = fp::splat<V>(-nux);
    const V d0 = fp::mul(mnu, fp::add(NB::l(n.R0), n.L0));
    const V d1 = fp::mul(mnu, fp::add(NB::l(n.R1), n.L1));
    const V d2 = fp::mul(mnu, fp::add(NB::l(n.R2), n.L2));
    return fp::derive(fp::add(c.eta, d0), fp::add(c.h, d0), fp::add(c.mt, d2),
                      fp::add(c.mn, d1));
}

struct Raw4 {
    float eta, mu, mv, hb;
};

// Rows are staged through a per-warp ring of shared memory by asynchronous
// copies (cp.async), kRing rows in flight, so that a warp walking its strip
// keeps enough loads outstanding to cover the memory latency.  Each lane
// copies and later reads only its own column of a row, so the ring needs no
// synchronisation beyond the lane's own wait for its copy groups.
constexpr int kRing = 8;                 // rows in flight per warp (a power of 2)
struct Ring {
    float v[kRing][4][kLanes];           // [slot][eta, hu, hv, hbar][lane]
};


__device__ __forceinline__ void fetch_row(Ring &R, int slot, const View &v, int col, int row,
                                          int lane) {
    const size_t o = (size_t)row * v.nx + col;
    cp_async4(&R.v[slot][0][lane], v.q0 + o);
    cp_async4(&R.v[slot][1][lane], v.q1 + o);
    cp_async4(&R.v[slot][2][lane], v.q2 + o);
    cp_async4(&R.v[slot][3][lane], v.hb + o);
}

// One strip of view v: output columns x0 .. x0 + 27 and rows y0 .. y0 +
// rows - 1 (clipped to the view).  Called by all 32 lanes of a warp, with
// the warp's own ring R.  Accumulates the CFL maximum of the new cells into
// smax and sets bad on a non-positive depth or non-finite momentum.  skip:
// take the exact shortcut of wave-free rows (false computes them in full,
// with the same result).
__device__ __forceinline__ void strip_unit(const View &v, int x0, int y0, int rows, float nux,
                                           float nuy, float g, int order, Ring &R, float &smax,
                                           bool &bad, bool skip = true) {
    const int lane = threadIdx.x & 31;
    const int ylast = (y0 + rows < v.ny ? y0 + rows : v.ny) - 1;
    const int gi = x0 - 2 + lane;
    bool fx, fy;
    const int col = ghost_index(gi, v.nx, v.bc.lo_x, v.bc.hi_x, &fx);
    const bool out = lane >= 2 && lane < kLanes - 2 && gi < v.nx;
    const float gh = 0.5f * g;
    fp::Cell<float> A = {}, B = {};   // x-swept rows j-2, j-1 (y frame)
    fp::Edge<float> W1 = {}, W2 = {};  // y-edges (j-3|j-2), (j-2|j-1)
    fp::Net<float> N1 = {};            // net of edge (j-3|j-2)
    // rest: bit k set when row j-k is exactly at rest (eta = hu = hv = 0) in
    // every lane of the warp.  There every wave is exactly zero, so the
    // x-sweep of such a row is the identity, an edge between two such rows
    // has no waves, and a net whose three edges lie in such rows is zero:
    // that work is skipped and its exact result used (the ocean ahead of a
    // tsunami is at rest).  The record of a wave-free edge has zero
    // strengths, so any limiter ratio formed with it is zero as well.
    unsigned rest = 0;
    fp::Edge<float> still = {};
    still.s1 = -1.f;
    still.s3 = 1.f;
    // strips away from the lower and upper boundary need no row mapping
    const bool yin = y0 - 2 >= 0 && ylast + 2 < v.ny;
    const int jend = ylast + 2;
    int jn = y0 - 2, sn = 0;   // next row to fetch and its ring slot
#pragma unroll
    for (int k = 0; k < kRing - 1; k++) {
        if (jn <= jend) {
            const int row = yin ? jn : ghost_index(jn, v.ny, v.bc.lo_y, v.bc.hi_y, &fy);
            fetch_row(R, sn, v, col, row, lane);
        }
        cp_commit();
        jn++;
        sn = (sn + 1) & (kRing - 1);
    }
    int sc = 0;   // ring slot of row j
#pragma unroll 3
    for (int j = y0 - 2; j <= jend; j++) {
        if (jn <= jend) {
            const int row = yin ? jn : ghost_index(jn, v.ny, v.bc.lo_y, v.bc.hi_y, &fy);
            fetch_row(R, sn, v, col, row, lane);
        }
        cp_commit();
        jn++;
        sn = (sn + 1) & (kRing - 1);
        cp_wait<kRing - 1>();   // row j has landed
        fy = false;
        if (!yin) ghost_index(j, v.ny, v.bc.lo_y, v.bc.hi_y, &fy);
        Raw4 Rc;
        Rc.eta = R.v[sc][0][lane];
        const float mu = R.v[sc][1][lane], mv = R.v[sc][2][lane];
        Rc.hb = R.v[sc][3][lane];
        Rc.mu = fx ? -mu : mu;
        Rc.mv = fy ? -mv : mv;
        sc = (sc + 1) & (kRing - 1);
        const bool at_rest =
            __all_sync(kFull, skip && Rc.eta == 0.f && Rc.mu == 0.f && Rc.mv == 0.f);
        rest = (rest << 1) | (at_rest ? 1u : 0u);
        const float h = fp::add(Rc.eta, Rc.hb);
        const fp::Cell<float> C = at_rest
                                      ? fp::derive(Rc.eta, h, Rc.mv, Rc.mu)
                                      : xsweep<Nb1>(fp::derive(Rc.eta, h, Rc.mu, Rc.mv), gh, nux,
                                                    order, lane);
        fp::Edge<float> Wn = W2;
        if (j >= y0 - 1) Wn = (rest & 3u) == 3u ? still : fp::solve(gh, B, C);   // edge (j-1|j)
        fp::Net<float> N = {};
        if (j >= y0 + 1 && (rest & 15u) != 15u) {   // net of edge (j-2|j-1)
            const bool all_sub = __all_sync(kFull, !out || fp::subsonic(W2.s1, W2.s3));
            N = fp::net3(W1, W2, Wn, nuy, order, all_sub);
        }
        if (j >= y0 + 2 && out) {
            // y-sweep of row j-2: lower edge -> R of the previous net, upper
            // edge -> L of this one (y frame: component 1 is hv, 2 is hu)
            const float d0 = fp::mul(-nuy, fp::add(N1.R0, N.L0));
            const float d1 = fp::mul(-nuy, fp::add(N1.R1, N.L1));
            const float d2 = fp::mul(-nuy, fp::add(N1.R2, N.L2));
            const float ne = fp::add(A.eta, d0), nmv = fp::add(A.mn, d1);
            const float nmu = fp::add(A.mt, d2);
            const size_t o = (size_t)(j - 2) * v.nx + gi;
            v.o0[o] = ne;
            v.o1[o] = nmu;
            v.o2[o] = nmv;
            const float h = fp::add(A.h, d0);
            bad |= !(h > 0.f) || !isfinite(nmu) || !isfinite(nmv);
            smax = fmaxf(smax, cfl_f32(h, nmu, nmv, g, v.rdx, v.rdy, 1));
        }
        A = B; B = C;
        W1 = W2; W2 = Wn;
        N1 = N;
    }
}

// ------------------------------------------------------------ quiet units
// A unit is quiet when every cell its step reads (its own cells and the two
// rows and columns around them, ghost cells index-mapped) is exactly at rest
// (eta = hu = hv = 0).  Every wave of such a window is zero, so the step
// leaves the unit's cells at rest, and the CFL term of each is that of the
// ocean at rest on its depth, cfl_f32(hbar, 0, 0), a function of the
// bathymetry alone.  quiet_unit() decides this from one streaming pass over
// the window (batches of three or six rows, two batches of loads in flight
// per lane, a warp vote per batch, leaving at the first batch with a wave),
// then writes the unit's cells at rest and takes their CFL maximum from
// rest_tab, the single grid's table of those rest terms (per strip sx and
// row j, the maximum over the strip's output columns, NaN where a column has
// hbar <= 0), or, for patches, forms them from hbar loaded with the window.
// A unit with a cell of hbar <= 0 takes the full path, which flags the
// depth.  The unit gets the state and the maximum the full path gives, up to
// the sign of an exact zero, at a fraction of the instructions: the ocean
// ahead of a tsunami is at rest.

// Loads of one batch of NB rows of a quiet scan: eta, hu, hv (and hbar when
// HB) of rows j0 .. j0 + NB - 1 (clipped to jend; a short last batch
// re-reads jend) in column col, rows index-mapped unless the window lies
// inside the grid.
template <bool HB, int NB>
struct QuietBatch {
    float e[NB], a[NB], b[NB], h[HB ? NB : 1];
    __device__ __forceinline__ void load(const View &v, int col, int j0, int jend, bool yin) {
#pragma unroll
        for (int k = 0; k < NB; k++) {
            const int j = j0 + k <= jend ? j0 + k : jend;
            bool fy;
            const int row = yin ? j : ghost_index(j, v.ny, v.bc.lo_y, v.bc.hi_y, &fy);
            const size_t o = (size_t)row * v.nx + col;
            e[k] = ld_early(v.q0 + o);
            a[k] = ld_early(v.q1 + o);
            b[k] = ld_early(v.q2 + o);
            if (HB) h[HB ? k : 0] = ld_early(v.hb + o);
        }
    }
    // Whether the batch is at rest in every lane of the warp.  With HB, also
    // the rest CFL terms of its output cells (rows y0 .. ylast, output lanes)
    // into t, and ok cleared where such a cell has hbar <= 0.
    __device__ __forceinline__ bool rest(const View &v, int j0, int y0, int ylast, bool outl,
                                         float g, float &t, bool &ok) const {
        bool r = true;
#pragma unroll
        for (int k = 0; k < NB; k++) {
            r = r && e[k] == 0.f && a[k] == 0.f && b[k] == 0.f;
            if (HB && outl && j0 + k >= y0 && j0 + k <= ylast) {
                const float hb = h[HB ? k : 0];
                ok = ok && hb > 0.f;
                t = fmaxf(t, cfl_f32(hb, 0.f, 0.f, g, v.rdx, v.rdy, 1));
            }
        }
        return __all_sync(kFull, r);
    }
};

// TAB: rest_tab is the single grid's table of rest CFL terms (per strip sx
// and row); otherwise the terms are formed from hbar, loaded with the window
// (patches).
template <bool TAB>
__device__ __forceinline__ bool quiet_unit(const View &v, const float *rest_tab, int sx, int x0,
                                           int y0, int rows, float g, float &smax) {
    constexpr int NB = TAB ? 6 : 3;   // rows per batch
    const int lane = threadIdx.x & 31;
    const int ylast = (y0 + rows < v.ny ? y0 + rows : v.ny) - 1;
    const int gi = x0 - 2 + lane;
    bool fx;
    const int col = ghost_index(gi, v.nx, v.bc.lo_x, v.bc.hi_x, &fx);
    const bool yin = y0 - 2 >= 0 && ylast + 2 < v.ny;
    const bool outl = lane >= 2 && lane < kLanes - 2 && gi < v.nx;
    const int jend = ylast + 2;
    float t = 0.f;
    bool ok = true;
    if (TAB) {   // the rest CFL terms of the unit's rows, loaded first
        for (int j = y0 + lane; j <= ylast; j += kLanes) {
            const float c = rest_tab[(size_t)sx * v.ny + j];
            ok = ok && c == c;
            t = fmaxf(t, c);
        }
    }
    // the window, two batches of rows in flight
    QuietBatch<!TAB, NB> P, Q;
    int j0 = y0 - 2;
    P.load(v, col, j0, jend, yin);
    for (;;) {
        bool more = j0 + NB <= jend;
        if (more) Q.load(v, col, j0 + NB, jend, yin);
        if (!P.rest(v, j0, y0, ylast, outl, g, t, ok)) return false;
        if (!more) break;
        j0 += NB;
        more = j0 + NB <= jend;
        if (more) P.load(v, col, j0 + NB, jend, yin);
        if (!Q.rest(v, j0, y0, ylast, outl, g, t, ok)) return false;
        if (!more) break;
        j0 += NB;
    }
    if (!__all_sync(kFull, ok)) return false;
    if (outl) {
        for (int j = y0; j <= ylast; j++) {
            const size_t o = (size_t)j * v.nx + gi;
            v.o0[o] = 0.f;
            v.o1[o] = 0.f;
            v.o2[o] = 0.f;
        }
    }
    smax = fmaxf(smax, t);
    return true;
}

}  // namespace strip
}  // namespace swadj
