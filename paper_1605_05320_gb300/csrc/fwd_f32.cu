// fwd_f32.cu -- FP32 perturbation-form forward step (Eq. swe, Sec. 5; Roe-type
// f-wave solver per edge, Sec. 6) for GB300.
//
// Storage: eta = h + B, hu, hv and hbar = -B in float.  Depth h = eta + hbar
// enters only wave speeds and Roe averages; the surface jump that drives the
// bathymetry-balanced momentum flux is taken from eta directly, so decimetre
// waves on 4000 m are resolved to float precision of eta, not of h.
//
// 2D grids run the warp strips of strips.cuh (per edge the arithmetic of
// fwd_pair.cuh); 1D grids run a one-thread-per-cell kernel with the same
// arithmetic.  The CFL maximum
// is reduced in float (max is exact); the last block to finish turns it into
// the next time step in double.
#include "ctu_kernels.cuh"
#include "strips.cuh"

namespace swadj {
namespace f32 {


// 2D grids: persistent warps take work units from the clock's counter, one
// unit a strip of 28 output columns by `rows` rows, in row-major order.
// Where the ocean is at rest a unit costs little (strips.cuh), so units are
// short and taken as warps free up: the active part of the domain spreads
// over every SM instead of over the few warps whose strips it crosses.
// ORD: the order of the scheme (1 or 2), fixed at compile time.
template <int ORD>
__global__ void __launch_bounds__(strip::kThreads, 4)
    fwd_f32_strips(FwdParams<float> p, int rows, int nunits) {
    __shared__ float s_nu[2];
    __shared__ int s_cur, s_run;
    __shared__ float red[strip::kThreads / 32];
    __shared__ int am_last;
    __shared__ strip::Ring ring[strip::kThreads / 32];
    double t_now = 0.0, dt = 0.0;
    if (!fwave::begin_step(p.clk, p.t_end, (double)p.dx, (double)p.dy, s_nu, &s_cur, &s_run,
                           t_now, dt))
        return;
    const int cur = s_cur;
    // with gauge recording, the last block first samples the state the step
    // starts from (the others write the other buffer)
    if (p.gauges.n > 0 && blockIdx.x == gridDim.x - 1)
        record_gauges<float, strip::kThreads>(p.gauges, p.q[cur][0], p.bath, p.nx, p.ny, 1,
                                              t_now);
    const int nsx = (p.nx + strip::kOut - 1) / strip::kOut;
    strip::View v;
    v.q0 = p.q[cur][0]; v.q1 = p.q[cur][1]; v.q2 = p.q[cur][2]; v.hb = p.bath;
    v.o0 = p.q[cur ^ 1][0]; v.o1 = p.q[cur ^ 1][1]; v.o2 = p.q[cur ^ 1][2];
    v.nx = p.nx; v.ny = p.ny;
    v.rdx = 1.f / p.dx; v.rdy = 1.f / p.dy;
    v.bc = p.bc;
    float smax = 0.f;
    bool bad = false;
    const int lane = threadIdx.x & 31;
    const bool quiet = p.rest_tab && p.umap && !p.keep_rest;
    for (;;) {   // warp-uniform
        int u = 0;
        if (lane == 0) u = (int)atomicAdd(&p.clk->work, 1u);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (u >= nunits) break;
        const int sy = u / nsx, sx = u - sy * nsx;
        // A unit that had waves at an earlier step keeps them (the ocean does
        // not return exactly to rest behind a wave): it skips the quiet scan.
        // The map is only a hint; the scan alone decides that a unit is quiet.
        if (quiet && (u >= p.umap_n || p.umap[u] == 0)) {
            if (strip::quiet_unit<true>(v, p.rest_tab, sx, sx * strip::kOut, sy * rows, rows, p.g,
                                        smax))
                continue;
            if (lane == 0 && u < p.umap_n) p.umap[u] = 1;
        }
        // Units with waves take the full path: quiet units cover the ocean
        // at rest, and the strip loop without its row skipping is leaner.
        strip::strip_unit(v, sx * strip::kOut, sy * rows, rows, s_nu[0], s_nu[1], p.g, ORD,
                          ring[threadIdx.x >> 5], smax, bad, false);
    }
    if (bad) atomicOr(p.err, ERR_UNSTABLE);
    fwave::finish_step<strip::kThreads>(p.clk, p.partial, p.nblocks, p.cfl, smax, red, &am_last,
                                        t_now, dt, cur);
}

// 1D grids: one thread per cell, solving the four edges it needs itself
// (1D grids are small; the redundancy costs nothing that matters).
__global__ void __launch_bounds__(256) fwd_f32_1d(FwdParams<float> p) {
    __shared__ float s_nu[2];
    __shared__ int s_cur, s_run;
    __shared__ float red[8];
    __shared__ int am_last;
    double t_now = 0.0, dt = 0.0;
    if (!fwave::begin_step(p.clk, p.t_end, (double)p.dx, (double)p.dy, s_nu, &s_cur, &s_run,
                          t_now, dt))
        return;
    const int cur = s_cur;
    if (p.gauges.n > 0 && blockIdx.x == 0)   // the state this step starts from
        record_gauges<float, 256>(p.gauges, p.q[cur][0], p.bath, p.nx, p.ny, 0, t_now);
    const float nux = s_nu[0], g = p.g;
    const float *q0 = p.q[cur][0], *q1 = p.q[cur][1];
    const int i = blockIdx.x * 256 + threadIdx.x;
    float sm = 0.f;
    bool bad = false;
    if (i < p.nx) {
        fp::Cell<float> c[5];
#pragma unroll
        for (int k = 0; k < 5; k++) {
            bool fx;
            const int ci = ghost_index(i - 2 + k, p.nx, p.bc.lo_x, p.bc.hi_x, &fx);
            const float eta = q0[ci], mu = fx ? -q1[ci] : q1[ci];
            c[k] = fp::derive(eta, fp::add(eta, p.bath[ci]), mu, 0.f);
        }
        const float gh = 0.5f * g;
        fp::Edge<float> w[4];
#pragma unroll
        for (int k = 0; k < 4; k++) w[k] = fp::solve(gh, c[k], c[k + 1]);
        const fp::Net<float> n0 =
            fp::net3(w[0], w[1], w[2], nux, p.order, fp::subsonic(w[1].s1, w[1].s3));
        const fp::Net<float> n1 =
            fp::net3(w[1], w[2], w[3], nux, p.order, fp::subsonic(w[2].s1, w[2].s3));
        const float d0 = fp::mul(-nux, fp::add(n0.R0, n1.L0));
        const float ne = fp::add(c[2].eta, d0);
        const float nmu = fp::add(c[2].mn, fp::mul(-nux, fp::add(n0.R1, n1.L1)));
        p.q[cur ^ 1][0][i] = ne;
        p.q[cur ^ 1][1][i] = nmu;
        const float hn = fp::add(c[2].h, d0);
        bad = !(hn > 0.f) || !isfinite(nmu);
        sm = cfl_f32(hn, nmu, 0.f, g, 1.f / p.dx, 1.f / p.dy, 0);
    }
    if (bad) atomicOr(p.err, ERR_UNSTABLE);
    fwave::finish_step<256>(p.clk, p.partial, p.nblocks, p.cfl, sm, red, &am_last, t_now, dt,
                            cur);
}

// The rest CFL table of quiet units (strips.cuh): per strip sx and row j,
// the maximum over the strip's output columns of cfl_f32(hbar, 0, 0), the
// step's CFL term of a cell at rest, with the step's own 1/dx and 1/dy; NaN
// where a column has hbar <= 0.
__global__ void rest_cfl_table(FwdParams<float> p, float *tab) {
    const int nsx = (p.nx + strip::kOut - 1) / strip::kOut;
    const float rdx = 1.f / p.dx, rdy = 1.f / p.dy;
    const size_t n = (size_t)nsx * p.ny;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x) {
        const int sx = (int)(k / p.ny), j = (int)(k - (size_t)sx * p.ny);
        const int x1 = (sx + 1) * strip::kOut < p.nx ? (sx + 1) * strip::kOut : p.nx;
        float t = 0.f;
        bool ok = true;
        for (int i = sx * strip::kOut; i < x1; i++) {
            const float hb = p.bath[(size_t)j * p.nx + i];
            ok = ok && hb > 0.f;
            t = fmaxf(t, cfl_f32(hb, 0.f, 0.f, p.g, rdx, rdy, 1));
        }
        tab[k] = ok ? t : __int_as_float(0x7fc00000);
    }
}

}  // namespace f32

// Entries of the unit map: units of the lowest strip height (16 rows).
int fwd_f32_unit_map_bytes(int nx, int ny) {
    return ((nx + strip::kOut - 1) / strip::kOut) * ((ny + 15) / 16);
}

size_t fwd_f32_rest_table_floats(int nx, int ny) {
    return (size_t)((nx + strip::kOut - 1) / strip::kOut) * ny;
}

int fwd_f32_rest_table(const FwdParams<float> &p, float *tab, cudaStream_t st) {
    const size_t n = fwd_f32_rest_table_floats(p.nx, p.ny);
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    f32::rest_cfl_table<<<blocks, 256, 0, st>>>(p, tab);
    return swadj_host::cuda_check(cudaGetLastError(), "rest_cfl_table");
}

// Rows of a work unit of the FP32 2D step: the requested strip height (16,
// 32 or 64), else kUnitRows.  All heights give the same results.
constexpr int kUnitRows = 32;
// Persistent blocks at most (reduction slots of the grid workspace).
constexpr int kMaxStepBlocks = 4096;

static int unit_rows(const FwdParams<float> &p) {
    return (p.fwd_rows == 16 || p.fwd_rows == 32 || p.fwd_rows == 64) ? p.fwd_rows : kUnitRows;
}

static int strip_units(int nx, int ny, int rows) {
    return ((nx + strip::kOut - 1) / strip::kOut) * ((ny + rows - 1) / rows);
}

// Blocks of one resident wave of the strip kernel on the current device.
static int resident_blocks() {
    static int blocks = 0;
    if (blocks == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f32::fwd_f32_strips<2>,
                                                      strip::kThreads, 0);
        blocks = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
        if (blocks > kMaxStepBlocks) blocks = kMaxStepBlocks;
    }
    return blocks;
}

template <>
int fwd_launch_step<float>(const FwdParams<float> &p0, cudaStream_t st) {
    FwdParams<float> p = p0;
    if (p.two_d) {
        const int rows = unit_rows(p);
        const int units = strip_units(p.nx, p.ny, rows);
        constexpr int wpb = strip::kThreads / 32;
        int blocks = (units + wpb - 1) / wpb;
        const int wave = resident_blocks();
        if (blocks > wave) blocks = wave;
        p.nblocks = blocks + (p.gauges.n > 0 ? 1 : 0);
        if (p.order == 2)
            f32::fwd_f32_strips<2><<<p.nblocks, strip::kThreads, 0, st>>>(p, rows, units);
        else
            f32::fwd_f32_strips<1><<<p.nblocks, strip::kThreads, 0, st>>>(p, rows, units);
        return swadj_host::cuda_check(cudaGetLastError(), "fwd_f32_strips");
    }
    dim3 grid((p.nx + 255) / 256, 1);
    p.nblocks = (int)grid.x;
    f32::fwd_f32_1d<<<grid, 256, 0, st>>>(p);
    return swadj_host::cuda_check(cudaGetLastError(), "fwd_f32_1d");
}

template <>
int fwd_step_blocks<float>(const FwdParams<float> &p) {
    // one reduction slot per block: at most one block per 4 units (of the
    // lowest height), at most kMaxStepBlocks, and the gauge block
    if (p.two_d) {
        const int b = (strip_units(p.nx, p.ny, 16) + 3) / 4;
        return (b < kMaxStepBlocks ? b : kMaxStepBlocks) + 1;
    }
    return (p.nx + 255) / 256;
}

// The wet/dry option runs the tiled split step (fwd_kernels.cuh) with the
// shore solver, in the perturbation form.
template <>
int fwd_launch_wd<float>(const FwdParams<float> &p0, cudaStream_t st) {
    FwdParams<float> p = p0;
    if (p.two_d) {
        dim3 grid((p.nx + 31) / 32, (p.ny + 3) / 4);
        p.nblocks = (int)(grid.x * grid.y);
        fwd_step_kernel<float, true, true, 32, 4, true><<<grid, dim3(32, 4), 0, st>>>(p);
    } else {
        dim3 grid((p.nx + 127) / 128, 1);
        p.nblocks = (int)grid.x;
        fwd_step_kernel<float, true, false, 128, 1, true><<<grid, dim3(128, 1), 0, st>>>(p);
    }
    return swadj_host::cuda_check(cudaGetLastError(), "fwd_step_kernel<float, wet/dry>");
}

template <>
int fwd_wd_blocks<float>(const FwdParams<float> &p) {
    if (p.two_d) return ((p.nx + 31) / 32) * ((p.ny + 3) / 4);
    return (p.nx + 127) / 128;
}

template <>
int fwd_launch_ctu<float>(const FwdParams<float> &p, cudaStream_t st) {
    return ctu_launch<float, true, 32, 16>(p, st, "fwd_ctu_kernel<float>");
}

template <>
int fwd_ctu_blocks<float>(const FwdParams<float> &p) {
    return ctu_blocks<32, 16>(p.nx, p.ny);
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
