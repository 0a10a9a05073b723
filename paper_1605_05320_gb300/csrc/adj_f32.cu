// adj_f32.cu -- FP32 adjoint step (Sec. 4; the time-reversed linear adjoint
// of adj_kernels.cuh, dimensionally split y then x).
//
// 2D grids run the warp-strip kernel below: per edge the same waves and
// limited net fluxes as the FP64 kernel, each edge solved once, the y-sweep
// in registers and the x-sweep across a warp by shuffles.  1D grids keep the
// one-tile-per-block kernel of adj_kernels.cuh.
//
// The limiter needs no division by the wave norm: for Z = b (c, 1) and its
// upwind neighbour Zu = bu (cu, 1), theta b = bu (cu c + 1) / (c^2 + 1), and
// phi(theta) b is formed from (b, theta b) directly (zero for b = 0, where
// the division form sets theta = 0).
#include "adj_kernels.cuh"

namespace swadj {
namespace adjt {

__device__ __forceinline__ float rcpf(float x) { return rcp_ftz(x); }
// Rounded single operations that the compiler never fuses (with explicit
// fmaf the rounding of every expression is fixed in the source).
__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }

// phi(theta) b for the MC limiter, r = theta b
__device__ __forceinline__ float mc1(float b, float r) {
    const float sg = b < 0.f ? -1.f : 1.f;
    const float B = fabsf(b), Rr = mul(sg, r);
    float m = fminf(mul(0.5f, add(B, Rr)), mul(2.f, B));
    m = fminf(m, mul(2.f, Rr));
    return mul(sg, fmaxf(m, 0.f));
}

struct EdgeA {   // waves of one edge: strengths and the (substituted) speeds
    float b1, b2, cl, cr;
    bool wall;     // a wet / dry edge: no second-order correction
};

// Waves at the edge between (eL, mL, cL) and (eR, mR, cR), m the normal
// component; c = 0 marks a dry cell, mirrored from its wet neighbour.  DRY =
// false: the grid has no dry cell (no wall edges), which gives the same
// numbers without the checks.
template <bool DRY = true>
__device__ __forceinline__ EdgeA solve_a(float eL, float mL, float cL, float eR, float mR,
                                         float cR) {
    EdgeA w;
    w.wall = false;
    if (DRY) {
        const bool dL = !(cL > 0.f), dR = !(cR > 0.f);
        w.wall = dL || dR;
        if (dL && dR) { w.b1 = 0.f; w.b2 = 0.f; w.cl = 0.f; w.cr = 0.f; return w; }
        if (dL) { eL = eR; mL = -mR; cL = cR; }
        if (dR) { eR = eL; mR = -mL; cR = cL; }
    }
    // flux jump of F = -(g hbar m, eta), g hbar = c^2
    const float d1 = fmaf(mul(cL, cL), mL, -mul(mul(cR, cR), mR));
    const float d2 = sub(eL, eR);
    const float rs = rcpf(add(cL, cR));
    w.b1 = mul(fmaf(cR, d2, d1), rs);
    w.b2 = mul(fmaf(cL, d2, -d1), rs);
    w.cl = cL;
    w.cr = cR;
    return w;
}

// Net fluxes of edge w (neighbour edges wl, wr) as (L0, L1, R0, R1): L into
// the left cell, R into the right cell (Q -= nu * net); components
// (eta~, normal).
template <bool DRY = true>
__device__ __forceinline__ float4 net_a(const EdgeA &wl, const EdgeA &w, const EdgeA &wr,
                                        float nu, int order) {
    float F0 = 0.f, F1 = 0.f;
    if (order >= 2 && (!DRY || !w.wall)) {
        // wave 1 (speed -cl) is upwinded from the right edge, wave 2 (+cr)
        // from the left edge
        const float r1 = mul(mul(wr.b1, fmaf(wr.cl, w.cl, 1.f)), rcpf(fmaf(w.cl, w.cl, 1.f)));
        const float r2 = mul(mul(wl.b2, fmaf(wl.cr, w.cr, 1.f)), rcpf(fmaf(w.cr, w.cr, 1.f)));
        const float k1 = mul(mul(-0.5f, fmaf(-nu, w.cl, 1.f)), mc1(w.b1, r1));
        const float k2 = mul(mul(0.5f, fmaf(-nu, w.cr, 1.f)), mc1(w.b2, r2));
        F0 = fmaf(k1, w.cl, -mul(k2, w.cr));
        F1 = add(k1, k2);
    }
    return make_float4(fmaf(w.b1, w.cl, F0), add(w.b1, F1), sub(-mul(w.b2, w.cr), F0),
                       sub(w.b2, F1));
}

// ---------------------------------------------------------------- strips
// A warp owns a strip of 32 columns (lanes) of which the middle 28 are its
// output, and SH output rows, which it walks downwards.  The y-sweep runs in
// registers with a sliding window over rows (each y-edge solved and limited
// once); every y-swept row is then x-swept across the warp with shuffles
// (each x-edge solved and limited once by the lane on its left).  Lanes 0-1
// and 30-31 are the x-halo: their y-swept values feed the output lanes' x
// edges.  Rows arrive through the warp's own ring of shared memory
// (cp.async, 8 rows in flight); there are no barriers.  The two-step kernel
// further down keeps one row of register prefetch.
constexpr int kLanes = 32;
constexpr int kOut = kLanes - 4;   // output columns per strip
constexpr int kRows = 32;          // output rows per strip
constexpr unsigned kFull = 0xffffffffu;

struct CellA {
    float e, m, g, c;   // eta~, mu~, gamma~, c = sqrt(g hbar) (0 if dry)
};

__device__ __forceinline__ CellA load_cell(const AdjParams<float> &p, int col, bool fx, int row,
                                           bool fy) {
    const size_t o = (size_t)row * p.nx + col;
    CellA q;
    q.e = ld_early(p.src[0] + o);
    const float mu = ld_early(p.src[1] + o), ga = ld_early(p.src[2] + o);
    q.m = fx ? -mu : mu;
    q.g = fy ? -ga : ga;
    q.c = ld_early(p.c + o);
    return q;
}

// Whether the strip unit with columns col (this lane's, index-mapped) and
// rows y0 .. ylast is quiet: every cell its step reads (its rows and two
// rows above and below, its columns and two either side) is exactly zero.
// Every wave of that window is then zero and the step leaves the unit zero.
// One streaming pass over the window in batches of six rows, two batches of
// loads in flight per lane, leaving at the first batch with a nonzero value.
// Far from the target the adjoint is still exactly zero for much of the
// solve.
constexpr int kQuietBatch = 6;
struct QuietBatchA {
    float e[kQuietBatch], m[kQuietBatch], g[kQuietBatch];
    __device__ __forceinline__ void load(const AdjParams<float> &p, int col, int j0, int jend,
                                         bool yin) {
#pragma unroll
        for (int k = 0; k < kQuietBatch; k++) {
            const int j = j0 + k <= jend ? j0 + k : jend;   // a short last batch re-reads
            bool fy;
            const int row = yin ? j : ghost_index(j, p.ny, p.bc.lo_y, p.bc.hi_y, &fy);
            const size_t o = (size_t)row * p.nx + col;
            e[k] = ld_early(p.src[0] + o);
            m[k] = ld_early(p.src[1] + o);
            g[k] = ld_early(p.src[2] + o);
        }
    }
    __device__ __forceinline__ bool zero() const {
        bool z = true;
#pragma unroll
        for (int k = 0; k < kQuietBatch; k++) z = z && e[k] == 0.f && m[k] == 0.f && g[k] == 0.f;
        return __all_sync(kFull, z);
    }
};
__device__ __forceinline__ bool quiet_a(const AdjParams<float> &p, int col, int y0, int ylast,
                                        bool yin) {
    const int jend = ylast + 2;
    QuietBatchA P, Q;
    int j0 = y0 - 2;
    P.load(p, col, j0, jend, yin);
    for (;;) {
        bool more = j0 + kQuietBatch <= jend;
        if (more) Q.load(p, col, j0 + kQuietBatch, jend, yin);
        if (!P.zero()) return false;
        if (!more) return true;
        j0 += kQuietBatch;
        more = j0 + kQuietBatch <= jend;
        if (more) P.load(p, col, j0 + kQuietBatch, jend, yin);
        if (!Q.zero()) return false;
        if (!more) return true;
        j0 += kQuietBatch;
    }
}

constexpr int kRingA = 8;   // rows in flight per warp (a power of 2)
struct RingA {
    float v[kRingA][4][kLanes];   // [slot][eta~, mu~, gamma~, c][lane]
};

// DRY: the grid has dry cells (wall checks on); ORD: the order of the
// scheme (1 or 2), fixed at compile time.
template <bool DRY, int ORD>
__global__ void __launch_bounds__(256, 4) adj_f32_strips(AdjParams<float> p) {
    __shared__ RingA ring[8];   // one per warp of the 256-thread block
    const int lane = threadIdx.x & 31;
    const int nsx = (p.nx + kOut - 1) / kOut, nsy = (p.ny + kRows - 1) / kRows;
    const int unit = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if ((p.snap_f || p.snap_d) && blockIdx.x == 0 && threadIdx.x == 0) *p.tau_dev = p.tau_val;
    if (unit >= nsx * nsy) return;   // warp-uniform
    const int sy = unit / nsx, sx = unit - sy * nsx;
    const int x0 = sx * kOut, y0 = sy * kRows;
    const int ylast = (y0 + kRows < p.ny ? y0 + kRows : p.ny) - 1;
    const int gi = x0 - 2 + lane;
    bool fx;
    const int col = ghost_index(gi, p.nx, p.bc.lo_x, p.bc.hi_x, &fx);
    const bool out = lane >= 2 && lane < kLanes - 2 && gi < p.nx;
    const float nux = p.nux, nuy = p.nuy;
    const int order = ORD;
    // row j of the strip, index-mapped (strips away from the lower and
    // upper boundary need no mapping; past the last row the load is clamped
    // and its values unused)
    const bool yin = y0 - 2 >= 0 && ylast + 2 < p.ny;
    // A unit that has had a nonzero value keeps having them: it skips the
    // quiet scan (the map is only a hint; the scan alone decides quiet).
    const bool scan = p.umap && (unit >= p.umap_n || p.umap[unit] == 0);
    if (scan && quiet_a(p, col, y0, ylast, yin)) {   // quiet: the unit stays zero
        if (out) {
            for (int j = y0; j <= ylast; j++) {
                const size_t o = (size_t)j * p.nx + gi;
                p.dst[0][o] = 0.f;
                p.dst[1][o] = 0.f;
                p.dst[2][o] = 0.f;
                if (p.snap_f) {
                    __stcs(p.snap_f + o, 0.f);
                    __stcs(p.snap_f + p.snap_comp_stride + o, 0.f);
                    __stcs(p.snap_f + 2 * p.snap_comp_stride + o, 0.f);
                } else if (p.snap_d) {
                    __stcs(p.snap_d + o, 0.0);
                    __stcs(p.snap_d + p.snap_comp_stride + o, 0.0);
                    __stcs(p.snap_d + 2 * p.snap_comp_stride + o, 0.0);
                }
            }
        }
        return;
    }
    if (scan && lane == 0 && unit < p.umap_n) p.umap[unit] = 1;
    // Rows stream through the warp's ring of shared memory by cp.async,
    // kRingA - 1 rows ahead of the one read, in the order they are used:
    // y0 - 2, y0 - 1, ..., ylast + 3 (past the last row the fetch is
    // clamped and its values unused).  Each lane copies and reads only its
    // own column, so the ring needs no synchronisation beyond the lane's own
    // wait for its copy groups.
    RingA &R = ring[threadIdx.x >> 5];
    int jf = y0 - 2, sf = 0;   // next row to fetch, its slot
    int jc = y0 - 2, sc = 0;   // next row to read, its slot
    const int jlast = ylast + 3;
    auto fetch = [&]() {
        if (jf <= jlast) {
            bool fy;
            int row;
            if (yin) row = jf < p.ny ? jf : p.ny - 1;
            else row = ghost_index(jf, p.ny, p.bc.lo_y, p.bc.hi_y, &fy);
            const size_t o = (size_t)row * p.nx + col;
            cp_async4(&R.v[sf][0][lane], p.src[0] + o);
            cp_async4(&R.v[sf][1][lane], p.src[1] + o);
            cp_async4(&R.v[sf][2][lane], p.src[2] + o);
            cp_async4(&R.v[sf][3][lane], p.c + o);
        }
        cp_commit();
        jf++;
        sf = (sf + 1) & (kRingA - 1);
    };
#pragma unroll
    for (int k = 0; k < kRingA - 1; k++) fetch();
    auto load = [&]() -> CellA {
        fetch();
        cp_wait<kRingA - 1>();   // row jc has landed
        bool fy = false;
        if (!yin) ghost_index(jc, p.ny, p.bc.lo_y, p.bc.hi_y, &fy);
        CellA q;
        q.e = R.v[sc][0][lane];
        const float mu = R.v[sc][1][lane], ga = R.v[sc][2][lane];
        q.m = fx ? -mu : mu;
        q.g = fy ? -ga : ga;
        q.c = R.v[sc][3][lane];
        jc++;
        sc = (sc + 1) & (kRingA - 1);
        return q;
    };
    // prologue, rows y0-2 .. y0+1 (rows are read one step ahead of use)
    CellA A = load();                                        // row y0-2
    CellA Cn = load();
    CellA B = Cn;                                            // row y0-1
    Cn = load();
    EdgeA W1 = solve_a<DRY>(A.e, A.g, A.c, B.e, B.g, B.c);        // edge (y0-2|y0-1)
    A = B;
    B = Cn;                                                  // row y0
    Cn = load();
    EdgeA W2 = solve_a<DRY>(A.e, A.g, A.c, B.e, B.g, B.c);        // edge (y0-1|y0)
    CellA C = Cn;                                            // row y0+1
    Cn = load();
    EdgeA Wn = solve_a<DRY>(B.e, B.g, B.c, C.e, C.g, C.c);        // edge (y0|y0+1)
    float4 nn = net_a<DRY>(W1, W2, Wn, nuy, order);               // edge (y0-1|y0)
    A = B; B = C;                                            // rows j-2, j-1
    W1 = W2; W2 = Wn;                                        // y-edges (j-3|j-2), (j-2|j-1)
    float rp0 = nn.z, rp1 = nn.w;   // R part of the y-net of edge (j-3|j-2)
    // main loop without branches on j
#pragma unroll 3
    for (int j = y0 + 2; j <= ylast + 2; j++) {
        C = Cn;
        Cn = load();                                          // row j+1
        Wn = solve_a<DRY>(B.e, B.g, B.c, C.e, C.g, C.c);          // edge (j-1|j)
        nn = net_a<DRY>(W1, W2, Wn, nuy, order);                  // edge (j-2|j-1)
        {
            // y-sweep of row r = j - 2: lower edge -> R of the previous net,
            // upper edge -> L of this one
            float e = A.e, g = A.g;
            const float m = A.m, c = A.c;
            if (!DRY || c > 0.f) {
                e = add(e, mul(-nuy, add(rp0, nn.x)));
                g = add(g, mul(-nuy, add(rp1, nn.y)));
            }
            // x-sweep of row r: lane l solves edge (l|l+1)
            const float eR = __shfl_down_sync(kFull, e, 1);
            const float mR = __shfl_down_sync(kFull, m, 1);
            const float cR = __shfl_down_sync(kFull, c, 1);
            const EdgeA X = solve_a<DRY>(e, m, c, eR, mR, cR);
            EdgeA XL = X, XR = X;   // only the fields net_a reads are exchanged
            XL.b2 = __shfl_up_sync(kFull, X.b2, 1);
            XL.cr = __shfl_up_sync(kFull, X.cr, 1);
            XR.b1 = __shfl_down_sync(kFull, X.b1, 1);
            XR.cl = __shfl_down_sync(kFull, X.cl, 1);
            const float4 xn = net_a<DRY>(XL, X, XR, nux, order);
            const float xr0 = __shfl_up_sync(kFull, xn.z, 1);   // R of edge (l-1|l)
            const float xr1 = __shfl_up_sync(kFull, xn.w, 1);
            float ne = e, nm = m;
            if (!DRY || c > 0.f) {
                ne = add(ne, mul(-nux, add(xr0, xn.x)));
                nm = add(nm, mul(-nux, add(xr1, xn.y)));
            }
            if (out) {
                const size_t o = (size_t)(j - 2) * p.nx + gi;
                p.dst[0][o] = ne;
                p.dst[1][o] = nm;
                p.dst[2][o] = g;
                if (p.snap_f) {
                    __stcs(p.snap_f + o, ne);
                    __stcs(p.snap_f + p.snap_comp_stride + o, nm);
                    __stcs(p.snap_f + 2 * p.snap_comp_stride + o, g);
                } else if (p.snap_d) {
                    __stcs(p.snap_d + o, (double)ne);
                    __stcs(p.snap_d + p.snap_comp_stride + o, (double)nm);
                    __stcs(p.snap_d + 2 * p.snap_comp_stride + o, (double)g);
                }
            }
        }
        A = B; B = C;
        W1 = W2; W2 = Wn;
        rp0 = nn.z; rp1 = nn.w;
    }
}

// ------------------------------------------- two steps per pass (temporal blocking)
// The adjoint's step is fixed, so two of its steps can be taken in one pass
// over the state: a warp loads its strip once and feeds every row through
// the y-then-x pipeline of the first step, whose finished rows feed the
// same pipeline of the second step, and only the second step's rows are
// written.  Each step needs two cells either side, so a strip of 32 lanes
// outputs 24 columns and reads 4 halo rows above and below.  Every edge is
// solved and limited by the same arithmetic as in the one-step kernel, and
// the intermediate state's ghost cells are the index-mapped interior cells
// the one-step path would load (a column mapped by a shuffle from the lane
// holding its source, a row from the interior rows kept for it), so two
// steps per pass give the one-step path's state bit for bit.
constexpr int kOut2 = kLanes - 8;   // output columns per two-step strip
constexpr int kRows2 = 32;          // output rows per two-step strip

// One step's pipeline over the rows of a strip.  Rows are fed in order; the
// feed of the fifth and every later row r completes row r - 2 (y-sweep, then
// x-sweep across the warp), valid in lanes 2..29.
struct Pipe {
    CellA A, B;       // rows r-2, r-1
    EdgeA W1, W2;     // y-edges (r-3|r-2), (r-2|r-1)
    float rp0, rp1;   // R part of the net of edge (r-3|r-2)
    int n;            // rows fed so far (warp-uniform)
};

__device__ __forceinline__ bool feed(Pipe &P, const CellA &C, float nux, float nuy, int order,
                                     CellA &out) {
    EdgeA Wn = P.W2;
    if (P.n >= 1) Wn = solve_a(P.B.e, P.B.g, P.B.c, C.e, C.g, C.c);   // edge (r-1|r)
    float4 nn = make_float4(0.f, 0.f, 0.f, 0.f);
    if (P.n >= 3) nn = net_a(P.W1, P.W2, Wn, nuy, order);             // edge (r-2|r-1)
    const bool done = P.n >= 4;
    if (done) {
        float e = P.A.e, g = P.A.g;
        const float m = P.A.m, c = P.A.c;
        if (c > 0.f) {
            e = add(e, mul(-nuy, add(P.rp0, nn.x)));
            g = add(g, mul(-nuy, add(P.rp1, nn.y)));
        }
        const float eR = __shfl_down_sync(kFull, e, 1);
        const float mR = __shfl_down_sync(kFull, m, 1);
        const float cR = __shfl_down_sync(kFull, c, 1);
        const EdgeA X = solve_a(e, m, c, eR, mR, cR);
        EdgeA XL = X, XR = X;
        XL.b2 = __shfl_up_sync(kFull, X.b2, 1);
        XL.cr = __shfl_up_sync(kFull, X.cr, 1);
        XR.b1 = __shfl_down_sync(kFull, X.b1, 1);
        XR.cl = __shfl_down_sync(kFull, X.cl, 1);
        const float4 xn = net_a(XL, X, XR, nux, order);
        const float xr0 = __shfl_up_sync(kFull, xn.z, 1);
        const float xr1 = __shfl_up_sync(kFull, xn.w, 1);
        float ne = e, nm = m;
        if (c > 0.f) {
            ne = add(ne, mul(-nux, add(xr0, xn.x)));
            nm = add(nm, mul(-nux, add(xr1, xn.y)));
        }
        out.e = ne; out.m = nm; out.g = g; out.c = c;
    }
    P.A = P.B; P.B = C;
    P.W1 = P.W2; P.W2 = Wn;
    P.rp0 = nn.z; P.rp1 = nn.w;
    P.n++;
    return done;
}

// the ghost row the one-step path would load for row r < 0 or r >= ny, from
// the interior rows lo0 = 0, lo1 = 1, hi0 = ny - 1, hi1 = ny - 2
__device__ __forceinline__ CellA ghost_row(int r, int ny, int bc_lo, int bc_hi, const CellA &lo0,
                                           const CellA &lo1, const CellA &hi0, const CellA &hi1) {
    CellA q;
    bool wall;
    if (r < 0) {
        wall = bc_lo == SWA_BC_WALL;
        q = (wall && r == -2) ? lo1 : lo0;
    } else {
        wall = bc_hi == SWA_BC_WALL;
        q = (wall && r == ny + 1) ? hi1 : hi0;
    }
    if (wall) q.g = -q.g;
    return q;
}

__global__ void __launch_bounds__(256, 3) adj_f32_strips2(AdjParams<float> p) {
    const int lane = threadIdx.x & 31;
    const int nsx = (p.nx + kOut2 - 1) / kOut2, nsy = (p.ny + kRows2 - 1) / kRows2;
    const int unit = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if ((p.snap_f || p.snap_d) && blockIdx.x == 0 && threadIdx.x == 0) *p.tau_dev = p.tau_val;
    if (unit >= nsx * nsy) return;   // warp-uniform
    const int sy = unit / nsx, sx = unit - sy * nsx;
    const int x0 = sx * kOut2, y0 = sy * kRows2;
    const int ny = p.ny;
    const int ylast = (y0 + kRows2 < ny ? y0 + kRows2 : ny) - 1;
    const int gi = x0 - 4 + lane;
    bool fx;
    const int col = ghost_index(gi, p.nx, p.bc.lo_x, p.bc.hi_x, &fx);
    // the lane holding this lane's column of the intermediate state
    const int src = (gi >= 0 && gi < p.nx) ? lane : col - (x0 - 4);
    const bool out = lane >= 4 && lane < kLanes - 4 && gi < p.nx;
    const float nux = p.nux, nuy = p.nuy;
    const int order = p.order;
    const bool yin = y0 - 4 >= 0 && ylast + 4 < ny;
    auto load = [&](int j) -> CellA {
        bool fy = false;
        int row;
        if (yin) row = j;
        else row = ghost_index(j, ny, p.bc.lo_y, p.bc.hi_y, &fy);
        return load_cell(p, col, fx, row, fy);
    };
    Pipe P1, P2;
    P1.n = 0; P2.n = 0;
    P1.rp0 = P1.rp1 = P2.rp0 = P2.rp1 = 0.f;
    CellA lo0 = {}, lo1 = {}, hi0 = {}, hi1 = {};
    CellA Cn = load(y0 - 4);
    for (int j = y0 - 4; j <= ylast + 4; j++) {   // input row j (warp-uniform)
        const CellA C = Cn;
        if (j < ylast + 4) Cn = load(j + 1);
        CellA S;
        if (!feed(P1, C, nux, nuy, order, S)) continue;
        const int r = j - 2;   // the finished row of the first step
        // its ghost columns: the mapped interior columns, as a load would give
        S.e = __shfl_sync(kFull, S.e, src);
        S.m = __shfl_sync(kFull, S.m, src);
        S.g = __shfl_sync(kFull, S.g, src);
        if (fx) S.m = -S.m;
        if (r == 0) lo0 = S;
        if (r == 1) lo1 = S;
        if (r == ny - 1) hi0 = S;
        if (r == ny - 2) hi1 = S;
        // rows below the grid are fed once rows 0 and 1 are known
        if (r < 0 || (y0 - 2 < 0 && r == 0)) continue;
        int nfeed = 1, rf = r;
        if (y0 - 2 < 0 && r == 1) { nfeed = 4; rf = -2; }   // rows -2, -1, 0, 1
        for (int k = 0; k < nfeed; k++, rf++) {
            CellA F = S;
            if (rf < 0 || rf >= ny) F = ghost_row(rf, ny, p.bc.lo_y, p.bc.hi_y, lo0, lo1, hi0, hi1);
            else if (rf != r) F = rf == 0 ? lo0 : lo1;
            CellA Q;
            if (!feed(P2, F, nux, nuy, order, Q)) continue;
            const int ro = rf - 2;   // the finished row of the second step
            if (out && ro >= y0 && ro <= ylast) {
                const size_t o = (size_t)ro * p.nx + gi;
                p.dst[0][o] = Q.e;
                p.dst[1][o] = Q.m;
                p.dst[2][o] = Q.g;
                if (p.snap_f) {
                    __stcs(p.snap_f + o, Q.e);
                    __stcs(p.snap_f + p.snap_comp_stride + o, Q.m);
                    __stcs(p.snap_f + 2 * p.snap_comp_stride + o, Q.g);
                } else if (p.snap_d) {
                    __stcs(p.snap_d + o, (double)Q.e);
                    __stcs(p.snap_d + p.snap_comp_stride + o, (double)Q.m);
                    __stcs(p.snap_d + 2 * p.snap_comp_stride + o, (double)Q.g);
                }
            }
        }
    }
}

}  // namespace adjt

int adj_f32_unit_map_bytes(int nx, int ny) {
    return ((nx + adjt::kOut - 1) / adjt::kOut) * ((ny + adjt::kRows - 1) / adjt::kRows);
}

template <>
int adj_launch_step<float>(const AdjParams<float> &p, cudaStream_t st) {
    if (p.two_d && p.two_steps) {
        const long long units = (long long)((p.nx + adjt::kOut2 - 1) / adjt::kOut2) *
                                ((p.ny + adjt::kRows2 - 1) / adjt::kRows2);
        const unsigned blocks = (unsigned)((units + 7) / 8);
        adjt::adj_f32_strips2<<<blocks, 256, 0, st>>>(p);
        return swadj_host::cuda_check(cudaGetLastError(), "adj_f32_strips2");
    }
    if (p.two_d) {
        const long long units = (long long)((p.nx + adjt::kOut - 1) / adjt::kOut) *
                                ((p.ny + adjt::kRows - 1) / adjt::kRows);
        const unsigned blocks = (unsigned)((units + 7) / 8);
        if (p.all_wet && p.order == 2)
            adjt::adj_f32_strips<false, 2><<<blocks, 256, 0, st>>>(p);
        else if (p.all_wet)
            adjt::adj_f32_strips<false, 1><<<blocks, 256, 0, st>>>(p);
        else if (p.order == 2)
            adjt::adj_f32_strips<true, 2><<<blocks, 256, 0, st>>>(p);
        else
            adjt::adj_f32_strips<true, 1><<<blocks, 256, 0, st>>>(p);
        return swadj_host::cuda_check(cudaGetLastError(), "adj_f32_strips");
    }
    dim3 grid((p.nx + 127) / 128, 1);
    adj_step_kernel<float, false, 128, 1><<<grid, dim3(128, 1), 0, st>>>(p);
    return swadj_host::cuda_check(cudaGetLastError(), "adj_step_kernel<float>");
}

}  // namespace swadj
