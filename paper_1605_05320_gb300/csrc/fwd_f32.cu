// fwd_f32.cu -- FP32 perturbation-form forward step (Eq. swe, Sec. 5; Roe-type
// f-wave solver per edge, Sec. 6) for GB300.
//
// Storage: eta = h + B, hu, hv and hbar = -B in float.  Depth h = eta + hbar
// enters only wave speeds and Roe averages; the surface jump that drives the
// bathymetry-balanced momentum flux is taken from eta directly, so decimetre
// waves on 4000 m are resolved to float precision of eta, not of h.
//
// 2D grids run the warp-strip kernel below (per edge the arithmetic of
// fwd_tiles.cuh); 1D grids run a one-thread-per-cell kernel.  The CFL maximum is
// reduced in float (max is exact); the last block to finish turns it into the
// next time step in double.
#include "fwd_tiles.cuh"

namespace swadj {
namespace f32 {

// ------------------------------------------------------------ warp strips
// 2D grids.  A warp owns a strip of 32 columns (lanes), the middle 28 its
// output, and `rows` output rows, and walks them downwards.  Each loaded row
// (the output rows and two halo rows above and below) is x-swept across the
// warp with shuffles, lane l solving and limiting edge (l|l+1) once; the
// y-sweep of the x-swept rows runs in registers over a sliding window of
// rows, each y-edge solved and limited once.  Per edge the arithmetic is the
// tile machinery's (solve1, net1), so results do not depend on the launch
// shape.  No shared memory and no barriers except the CFL reduction.
namespace strip {

constexpr int kLanes = 32;
constexpr int kOut = kLanes - 4;   // output columns per strip
constexpr unsigned kFull = 0xffffffffu;

struct XCell {   // derived cell data, as put_cell forms it
    float h, mu, mv, u, v, sq, eta;
};

__device__ __forceinline__ XCell derive(float eta, float h, float mu, float mv) {
    const float q = rsqrt_ftz(h);
    const float ih = tile::mul(q, q);
    XCell c;
    c.h = h; c.mu = mu; c.mv = mv;
    c.u = tile::mul(mu, ih); c.v = tile::mul(mv, ih); c.sq = tile::mul(h, q);
    c.eta = eta;
    return c;
}

__device__ __forceinline__ float dn(float x) { return __shfl_down_sync(kFull, x, 1); }
__device__ __forceinline__ float up(float x) { return __shfl_up_sync(kFull, x, 1); }

__device__ __forceinline__ tile::EdgeS edge_dn(const tile::EdgeS &w) {
    tile::EdgeS r;
    r.s1 = dn(w.s1); r.s3 = dn(w.s3); r.vh = dn(w.vh);
    r.b1 = dn(w.b1); r.b2 = dn(w.b2); r.b3 = dn(w.b3);
    return r;
}
__device__ __forceinline__ tile::EdgeS edge_up(const tile::EdgeS &w) {
    tile::EdgeS r;
    r.s1 = up(w.s1); r.s3 = up(w.s3); r.vh = up(w.vh);
    r.b1 = up(w.b1); r.b2 = up(w.b2); r.b3 = up(w.b3);
    return r;
}

// x-sweep of one row held across the warp; valid in lanes 2..29.
__device__ __forceinline__ XCell xsweep(const XCell &c, float g, float nux, int order) {
    const tile::EdgeS w = tile::solve1(g, c.h, c.mu, c.mv, c.u, c.v, c.sq, c.eta, dn(c.h),
                                       dn(c.mu), dn(c.mv), dn(c.u), dn(c.v), dn(c.sq),
                                       dn(c.eta));   // edge (l|l+1)
    float4 lr;
    float2 r;
    tile::net_of(edge_up(w), w, edge_dn(w), nux, order, lr, r);
    // left edge of the cell -> R of edge (l-1|l), right edge -> L of edge (l|l+1)
    const float d0 = tile::mul(-nux, tile::add(up(lr.w), lr.x));
    const float d1 = tile::mul(-nux, tile::add(up(r.x), lr.y));
    const float d2 = tile::mul(-nux, tile::add(up(r.y), lr.z));
    return derive(tile::add(c.eta, d0), tile::add(c.h, d0), tile::add(c.mu, d1),
                  tile::add(c.mv, d2));
}

// y-edge waves between x-swept cells a (below) and b (above), frame (h, hv, hu)
__device__ __forceinline__ tile::EdgeS ysolve(const XCell &a, const XCell &b, float g) {
    return tile::solve1(g, a.h, a.mv, a.mu, a.v, a.u, a.sq, a.eta, b.h, b.mv, b.mu, b.v, b.u,
                        b.sq, b.eta);
}

struct Raw4 {
    float eta, mu, mv, hb;
};

__device__ __forceinline__ Raw4 load_raw(const FwdParams<float> &p, int cur, int col, bool fx,
                                         int row, bool fy) {
    const size_t o = (size_t)row * p.nx + col;
    Raw4 r;
    r.eta = ld_early(p.q[cur][0] + o);
    r.hb = ld_early(p.bath + o);
    const float mu = ld_early(p.q[cur][1] + o), mv = ld_early(p.q[cur][2] + o);
    r.mu = fx ? -mu : mu;
    r.mv = fy ? -mv : mv;
    return r;
}

constexpr int kStripThreads = 128;   // 4 warps: at ~90 registers, 5 blocks per SM

__global__ void __launch_bounds__(kStripThreads) fwd_f32_strips(FwdParams<float> p, int rows) {
    __shared__ float s_nu[2];
    __shared__ int s_cur, s_run;
    __shared__ float red[kStripThreads / 32];
    __shared__ int am_last;
    double t_now = 0.0, dt = 0.0;
    if (!tile::begin_step(p.clk, p.t_end, (double)p.dx, (double)p.dy, s_nu, &s_cur, &s_run,
                          t_now, dt))
        return;
    const int cur = s_cur;
    const float nux = s_nu[0], nuy = s_nu[1], g = p.g;
    const float rdx = 1.f / p.dx, rdy = 1.f / p.dy;
    const int lane = threadIdx.x & 31;
    const int nsx = (p.nx + kOut - 1) / kOut, nsy = (p.ny + rows - 1) / rows;
    const int unit = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    float smax = 0.f;
    bool bad = false;
    if (unit < nsx * nsy) {   // warp-uniform
        const int sy = unit / nsx, sx = unit - sy * nsx;
        const int x0 = sx * kOut, y0 = sy * rows;
        const int ylast = (y0 + rows < p.ny ? y0 + rows : p.ny) - 1;
        const int gi = x0 - 2 + lane;
        bool fx, fy;
        const int col = ghost_index(gi, p.nx, p.bc.lo_x, p.bc.hi_x, &fx);
        const bool out = lane >= 2 && lane < kLanes - 2 && gi < p.nx;
        float *const o0 = p.q[cur ^ 1][0], *const o1 = p.q[cur ^ 1][1], *const o2 = p.q[cur ^ 1][2];
        XCell A = {}, B = {};           // x-swept rows j-2, j-1
        tile::EdgeS W1 = {}, W2 = {};   // y-edges (j-3|j-2), (j-2|j-1)
        float4 nlr = make_float4(0.f, 0.f, 0.f, 0.f);   // y-net of edge (j-3|j-2)
        float2 nr = make_float2(0.f, 0.f);
        // rows are loaded one iteration ahead of their use
        int row = ghost_index(y0 - 2, p.ny, p.bc.lo_y, p.bc.hi_y, &fy);
        Raw4 Rn = load_raw(p, cur, col, fx, row, fy);
#pragma unroll 3
        for (int j = y0 - 2; j <= ylast + 2; j++) {
            const Raw4 Rc = Rn;
            if (j < ylast + 2) {
                row = ghost_index(j + 1, p.ny, p.bc.lo_y, p.bc.hi_y, &fy);
                Rn = load_raw(p, cur, col, fx, row, fy);
            }
            const XCell C = xsweep(derive(Rc.eta, Rc.eta + Rc.hb, Rc.mu, Rc.mv), g, nux,
                                   p.order);
            tile::EdgeS Wn = W2;
            if (j >= y0 - 1) Wn = ysolve(B, C, g);   // edge (j-1|j)
            float4 lr = make_float4(0.f, 0.f, 0.f, 0.f);
            float2 r = make_float2(0.f, 0.f);
            if (j >= y0 + 1) tile::net_of(W1, W2, Wn, nuy, p.order, lr, r);   // edge (j-2|j-1)
            if (j >= y0 + 2 && out) {
                // y-sweep of row j-2: lower edge -> R of the previous net,
                // upper edge -> L of this one; nets are in (h, hv, hu) order
                const float d0 = tile::mul(-nuy, tile::add(nlr.w, lr.x));
                const float d2 = tile::mul(-nuy, tile::add(nr.x, lr.y));
                const float d1 = tile::mul(-nuy, tile::add(nr.y, lr.z));
                const float ne = tile::add(A.eta, d0), nmu = tile::add(A.mu, d1);
                const float nmv = tile::add(A.mv, d2);
                const size_t o = (size_t)(j - 2) * p.nx + gi;
                o0[o] = ne;
                o1[o] = nmu;
                o2[o] = nmv;
                const float h = tile::add(A.h, d0);
                bad |= !(h > 0.f) || !isfinite(nmu) || !isfinite(nmv);
                smax = fmaxf(smax, cfl_f32(h, nmu, nmv, g, rdx, rdy, 1));
            }
            A = B; B = C;
            W1 = W2; W2 = Wn;
            nlr = lr; nr = r;
        }
    }
    if (bad) atomicOr(p.err, ERR_UNSTABLE);
    tile::finish_step<kStripThreads>(p.clk, p.partial, p.nblocks, p.cfl, smax, red, &am_last,
                                     t_now, dt, cur, p.gauges.n > 0);
    if (p.gauges.n > 0 && am_last)
        record_gauges<float, kStripThreads>(p.gauges, p.q[cur ^ 1][0], p.bath, p.nx, p.ny, 1,
                                            t_now + dt);
}

}  // namespace strip

// 1D grids: one thread per cell, solving the four edges it needs itself
// (1D grids are small; the redundancy costs nothing that matters).
__global__ void __launch_bounds__(256) fwd_f32_1d(FwdParams<float> p) {
    __shared__ float s_nu[2];
    __shared__ int s_cur, s_run;
    __shared__ float red[8];
    __shared__ int am_last;
    double t_now = 0.0, dt = 0.0;
    if (!tile::begin_step(p.clk, p.t_end, (double)p.dx, (double)p.dy, s_nu, &s_cur, &s_run,
                          t_now, dt))
        return;
    const int cur = s_cur;
    const float nux = s_nu[0], g = p.g;
    const float *q0 = p.q[cur][0], *q1 = p.q[cur][1];
    const int i = blockIdx.x * 256 + threadIdx.x;
    float sm = 0.f;
    bool bad = false;
    if (i < p.nx) {
        float h[5], mu[5], u[5], sq[5], eta[5];
#pragma unroll
        for (int k = 0; k < 5; k++) {
            bool fx;
            const int c = ghost_index(i - 2 + k, p.nx, p.bc.lo_x, p.bc.hi_x, &fx);
            eta[k] = q0[c];
            mu[k] = fx ? -q1[c] : q1[c];
            h[k] = eta[k] + p.bath[c];
            const float q = rsqrt_ftz(h[k]);
            sq[k] = tile::mul(h[k], q);
            u[k] = tile::mul(mu[k], tile::mul(q, q));
        }
        tile::EdgeS w[4];
#pragma unroll
        for (int k = 0; k < 4; k++)
            w[k] = tile::solve1(g, h[k], mu[k], 0.f, u[k], 0.f, sq[k], eta[k], h[k + 1],
                                mu[k + 1], 0.f, u[k + 1], 0.f, sq[k + 1], eta[k + 1]);
        float L0[3], R0[3], L1[3], R1[3];
        if (tile::sub1(w[1])) tile::net1<true>(w[0], w[1], w[2], nux, p.order, L0, R0);
        else tile::net1<false>(w[0], w[1], w[2], nux, p.order, L0, R0);
        if (tile::sub1(w[2])) tile::net1<true>(w[1], w[2], w[3], nux, p.order, L1, R1);
        else tile::net1<false>(w[1], w[2], w[3], nux, p.order, L1, R1);
        const float d0 = tile::mul(-nux, tile::add(R0[0], L1[0]));
        const float ne = tile::add(eta[2], d0);
        const float nmu = tile::add(mu[2], tile::mul(-nux, tile::add(R0[1], L1[1])));
        p.q[cur ^ 1][0][i] = ne;
        p.q[cur ^ 1][1][i] = nmu;
        const float hn = tile::add(h[2], d0);
        bad = !(hn > 0.f) || !isfinite(nmu);
        sm = cfl_f32(hn, nmu, 0.f, g, 1.f / p.dx, 1.f / p.dy, 0);
    }
    if (bad) atomicOr(p.err, ERR_UNSTABLE);
    tile::finish_step<256>(p.clk, p.partial, p.nblocks, p.cfl, sm, red, &am_last, t_now, dt,
                           cur, p.gauges.n > 0);
    if (p.gauges.n > 0 && am_last)
        record_gauges<float, 256>(p.gauges, p.q[cur ^ 1][0], p.bath, p.nx, p.ny, 0,
                                  t_now + dt);
}

}  // namespace f32

static int strip_blocks(int nx, int ny, int rows) {
    const long long units = (long long)((nx + f32::strip::kOut - 1) / f32::strip::kOut) *
                            ((ny + rows - 1) / rows);
    constexpr int wpb = f32::strip::kStripThreads / 32;
    return (int)((units + wpb - 1) / wpb);
}

// Strip height requested for the FP32 2D step (16, 32 or 64), else 0.
static int requested_rows(const FwdParams<float> &p) {
    return (p.fwd_rows == 16 || p.fwd_rows == 32 || p.fwd_rows == 64) ? p.fwd_rows : 0;
}

// Default strip height: the one minimising (waves of strips) x (rows + 4),
// the rows a strip x-sweeps, with a wave = the warps resident on all SMs.
// All heights give the same results.
static int default_rows(int nx, int ny) {
    static long long slots = 0;
    if (slots == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f32::strip::fwd_f32_strips,
                                                      f32::strip::kStripThreads, 0);
        slots = (long long)(sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1) *
                (f32::strip::kStripThreads / 32);
    }
    int best = 32;
    long long best_cost = -1;
    for (int rows : {64, 32, 16}) {
        const long long units = (long long)((nx + f32::strip::kOut - 1) / f32::strip::kOut) *
                                ((ny + rows - 1) / rows);
        const long long cost = ((units + slots - 1) / slots) * (rows + 4);
        if (best_cost < 0 || cost < best_cost) { best = rows; best_cost = cost; }
    }
    return best;
}

template <>
int fwd_launch_step<float>(const FwdParams<float> &p0, cudaStream_t st) {
    FwdParams<float> p = p0;
    if (p.two_d) {
        const int req = requested_rows(p);
        const int rows = req ? req : default_rows(p.nx, p.ny);
        p.nblocks = strip_blocks(p.nx, p.ny, rows);
        f32::strip::fwd_f32_strips<<<p.nblocks, f32::strip::kStripThreads, 0, st>>>(p, rows);
        return swadj_host::cuda_check(cudaGetLastError(), "fwd_f32_strips");
    }
    dim3 grid((p.nx + 255) / 256, 1);
    p.nblocks = (int)grid.x;
    f32::fwd_f32_1d<<<grid, 256, 0, st>>>(p);
    return swadj_host::cuda_check(cudaGetLastError(), "fwd_f32_1d");
}

template <>
int fwd_step_blocks<float>(const FwdParams<float> &p) {
    // one reduction slot per block: of the requested strip height, else of
    // the lowest one (an upper bound for the default)
    if (p.two_d) {
        const int req = requested_rows(p);
        return strip_blocks(p.nx, p.ny, req ? req : 16);
    }
    return (p.nx + 255) / 256;
}

template <>
int fwd_launch_clock_init<float>(const FwdParams<float> &p, double t0, cudaStream_t st) {
    const size_t n = (size_t)p.nx * p.ny;
    int blocks = (int)((n + 255) / 256);
    if (blocks > kInitBlocks) blocks = kInitBlocks;
    clock_init_kernel<float, true><<<blocks, 256, 0, st>>>(p, t0);
    return swadj_host::cuda_check(cudaGetLastError(), "clock_init_kernel<float>");
}

}  // namespace swadj
