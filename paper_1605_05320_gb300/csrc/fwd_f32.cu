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


// 2D grids: warp strips, one strip per warp.
__global__ void __launch_bounds__(strip::kThreads, 5) fwd_f32_strips(FwdParams<float> p, int rows) {
    __shared__ float s_nu[2];
    __shared__ int s_cur, s_run;
    __shared__ float red[strip::kThreads / 32];
    __shared__ int am_last;
    double t_now = 0.0, dt = 0.0;
    if (!fwave::begin_step(p.clk, p.t_end, (double)p.dx, (double)p.dy, s_nu, &s_cur, &s_run,
                           t_now, dt))
        return;
    const int cur = s_cur;
    // with gauge recording, one extra block (the last) samples the state the
    // step starts from while the others step it
    if (p.gauges.n > 0 && blockIdx.x == gridDim.x - 1)
        record_gauges<float, strip::kThreads>(p.gauges, p.q[cur][0], p.bath, p.nx, p.ny, 1,
                                           t_now);
    const int nsx = (p.nx + strip::kOut - 1) / strip::kOut, nsy = (p.ny + rows - 1) / rows;
    const int unit = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    float smax = 0.f;
    bool bad = false;
    if (unit < nsx * nsy) {   // warp-uniform
        const int sy = unit / nsx, sx = unit - sy * nsx;
        strip::View v;
        v.q0 = p.q[cur][0]; v.q1 = p.q[cur][1]; v.q2 = p.q[cur][2]; v.hb = p.bath;
        v.o0 = p.q[cur ^ 1][0]; v.o1 = p.q[cur ^ 1][1]; v.o2 = p.q[cur ^ 1][2];
        v.nx = p.nx; v.ny = p.ny;
        v.rdx = 1.f / p.dx; v.rdy = 1.f / p.dy;
        v.bc = p.bc;
        strip::strip_unit(v, sx * strip::kOut, sy * rows, rows, s_nu[0], s_nu[1], p.g, p.order, smax,
                       bad);
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

}  // namespace f32

static int strip_blocks(int nx, int ny, int rows) {
    const long long units = (long long)((nx + strip::kOut - 1) / strip::kOut) *
                            ((ny + rows - 1) / rows);
    constexpr int wpb = strip::kThreads / 32;
    return (int)((units + wpb - 1) / wpb);
}

// Strip height requested for the FP32 2D step (16, 32 or 64), else 0.
static int requested_rows(const FwdParams<float> &p) {
    return (p.fwd_rows == 16 || p.fwd_rows == 32 || p.fwd_rows == 64) ? p.fwd_rows : 0;
}

// Default strip height.  Warps of one resident wave (all SMs full) hide
// each other's latency best, so the default is the lowest height (at least
// 16 rows) whose strips all fit in one wave, one block kept for the gauge
// block; when none does (very large grids), the one of 16 .. 256 rows
// minimising (waves of strips) x (rows + 4), the rows a strip x-sweeps.
// All heights give the same results.
static int default_rows(int nx, int ny) {
    static long long slots = 0;
    if (slots == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f32::fwd_f32_strips,
                                                      strip::kThreads, 0);
        slots = (long long)(sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1) *
                (strip::kThreads / 32);
    }
    const long long nsx = (nx + strip::kOut - 1) / strip::kOut;
    const long long per_col = (slots - strip::kThreads / 32) / nsx;   // strips down a column
    if (per_col >= 1) {
        long long rows = (ny + per_col - 1) / per_col;
        if (rows < 16) rows = 16;
        if (rows <= 256) return (int)rows;
    }
    int best = 32;
    long long best_cost = -1;
    for (int rows : {256, 128, 64, 32, 16}) {
        const long long units = nsx * ((ny + rows - 1) / rows);
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
        p.nblocks = strip_blocks(p.nx, p.ny, rows) + (p.gauges.n > 0 ? 1 : 0);
        f32::fwd_f32_strips<<<p.nblocks, strip::kThreads, 0, st>>>(p, rows);
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
    // the lowest one (an upper bound for the default), and the gauge block
    if (p.two_d) {
        const int req = requested_rows(p);
        return strip_blocks(p.nx, p.ny, req ? req : 16) + 1;   // + the gauge block
    }
    return (p.nx + 255) / 256;
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
