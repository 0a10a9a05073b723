// gauge.cuh -- gauge sampling (Sec. 6 gauges): surface elevation at a point
// by bilinear interpolation of cell-centre values, clamped to the outermost
// centres.  Used by the stand-alone gauge kernel and by the step kernels'
// fused gauge recording.
#pragma once

#include "swadj_internal.cuh"

namespace swadj {

// Fused recording into a device series; n == 0 turns it off.
struct GaugeRec {
    int n;                // gauges
    const double *xy;     // [n][2] coordinates
    double *series;       // [cap][n] surface elevation at the start of each step
    double *times;        // [cap] time at the start of each step, or null
    long long cap;        // rows of the series
    long long *row;       // device row counter (rows recorded so far)
    double x_lo, y_lo, dx, dy;   // geometry of the grid
};

// eta at (x, y) from the state array q0 (eta for float grids, h for double
// grids, eta = h + B) and the bathymetry array of the grid.
template <typename R>
__device__ __forceinline__ double gauge_eta(const R *q0, const R *bath, int nx, int ny,
                                            int two_d, double x_lo, double y_lo, double dx,
                                            double dy, double x, double y) {
    double fx = (x - x_lo) / dx - 0.5;
    fx = fx < 0.0 ? 0.0 : (fx > (double)(nx - 1) ? (double)(nx - 1) : fx);
    int i0 = (int)floor(fx);
    if (i0 > nx - 2) i0 = nx - 2;
    if (i0 < 0) i0 = 0;
    double ax = fx - (double)i0;
    const int i1 = nx > 1 ? i0 + 1 : i0;
    if (nx == 1) ax = 0.0;
    size_t st[4];
    double wt[4];
    if (!two_d) {
        st[0] = i0; st[1] = i1; st[2] = 0; st[3] = 0;
        wt[0] = 1.0 - ax; wt[1] = ax; wt[2] = 0.0; wt[3] = 0.0;
    } else {
        double fy = (y - y_lo) / dy - 0.5;
        fy = fy < 0.0 ? 0.0 : (fy > (double)(ny - 1) ? (double)(ny - 1) : fy);
        int j0 = (int)floor(fy);
        if (j0 > ny - 2) j0 = ny - 2;
        if (j0 < 0) j0 = 0;
        double ay = fy - (double)j0;
        const int j1 = ny > 1 ? j0 + 1 : j0;
        if (ny == 1) ay = 0.0;
        st[0] = (size_t)j0 * nx + i0; wt[0] = (1.0 - ax) * (1.0 - ay);
        st[1] = (size_t)j0 * nx + i1; wt[1] = ax * (1.0 - ay);
        st[2] = (size_t)j1 * nx + i0; wt[2] = (1.0 - ax) * ay;
        st[3] = (size_t)j1 * nx + i1; wt[3] = ax * ay;
    }
    // rounded operations (never fused), so every translation unit gives the
    // same number, and the one an unfused FP64 evaluation gives
    double v = 0.0;
#pragma unroll
    for (int c = 0; c < 4; c++) {
        double eta;
        if (sizeof(R) == 4) eta = (double)__ldcg(q0 + st[c]);
        else eta = __dadd_rn((double)__ldcg(q0 + st[c]), (double)bath[st[c]]);
        v = __dadd_rn(v, __dmul_rn(wt[c], eta));
    }
    return v;
}

// Called by every thread of one block of a step kernel (block-uniform call)
// with the state the step starts from (q0, complete since the previous
// launch) and its time t.  Writes the next row of the series; rows past cap
// are not written.
template <typename R, int NTH>
__device__ __forceinline__ void record_gauges(const GaugeRec &g, const R *q0, const R *bath,
                                              int nx, int ny, int two_d, double t) {
    __shared__ long long s_row;
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        s_row = *g.row;
        *g.row = s_row + 1;
    }
    __syncthreads();
    const long long r = s_row;
    if (r >= g.cap) return;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    for (int k = tid; k < g.n; k += NTH)
        g.series[r * g.n + k] = gauge_eta<R>(q0, bath, nx, ny, two_d, g.x_lo, g.y_lo, g.dx,
                                             g.dy, g.xy[2 * k], g.xy[2 * k + 1]);
    if (tid == 0 && g.times) g.times[r] = t;
}

}  // namespace swadj
