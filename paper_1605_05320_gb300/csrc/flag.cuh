// flag.cuh -- flag-pass and gauge kernel parameters.
#pragma once

#include "swadj_internal.cuh"

namespace swadj {

template <typename R, typename S>
struct FlagParams {
    // forward grid (state read from the buffer the device clock points at)
    int nx, ny, two_d;
    double x_lo, y_lo, dx, dy;
    R dry_tol;
    const R *q[2][3];
    const R *bath;           // B (double) or hbar (float)
    const DevClock *clk;
    // adjoint grid and snapshots
    int anx, any, same_grid;
    double ax_lo, ay_lo, adx, ady;
    // the same map in float for the FP32 pass: the adjoint-grid coordinate
    // of forward cell i (in cell widths, from the first centre) is
    // (i + 1/2) * frx + fcx; exact in float when the grids align
    float frx, fcx, fry, fcy;
    const uint8_t *awet;     // 1 where the adjoint cell is wet
    const S *snaps;          // [K][ncomp][na]
    size_t snap_stride;      // ncomp * na
    size_t na;
    int ncomp;
    const double *tau;       // [K], strictly decreasing
    int K;
    double t_s, t_f, tol;
    int mode;
    uint8_t *flags;
    float *maxip;
    unsigned long long *count;
    // snapshot envelope (FP32 2D stores, or null): per group of kEnvGroup
    // consecutive snapshots and per quad of 4 consecutive cells, the maximum
    // |component| of each component, [group][ncomp][na / 4]
    const float *env;
};

// Snapshots per envelope group.
constexpr int kEnvGroup = 8;

template <typename R, typename S>
int flag_launch(const FlagParams<R, S> &p, cudaStream_t st);

// Fold snapshot slot `slot` ([3][na] floats, na % 4 == 0) into its envelope
// group `env_group` ([3][na / 4]): overwrite when `first`, else max.
int env_launch_update(const float *slot, size_t na, float *env_group, int first,
                      cudaStream_t st);

template <typename R>
struct SurfParams {
    size_t n;
    const R *q[2][3];
    const R *bath;
    const DevClock *clk;
    R tol, dry_tol;
    uint8_t *flags;
    unsigned long long *count;
};

template <typename R>
int surface_launch(const SurfParams<R> &p, cudaStream_t st);

template <typename R>
struct GaugeParams {
    int nx, ny, two_d;
    double x_lo, y_lo, dx, dy;
    const R *q[2][3];
    const R *bath;
    const DevClock *clk;
    int n;
    const double *xy;
    double *out;
};

template <typename R>
int gauge_launch(const GaugeParams<R> &p, cudaStream_t st);

}  // namespace swadj
