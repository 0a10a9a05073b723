// fwd.cuh -- forward-step kernel parameters and host launchers.
#pragma once

#include "gauge.cuh"
#include "swadj_internal.cuh"

namespace swadj {

constexpr int kInitBlocks = 1024;  // blocks of the initial CFL reduction

template <typename R>
struct FwdParams {
    int nx, ny, two_d, order;
    BcSpec bc;
    R dx, dy, g;
    double cfl, t_end;
    R *q[2][3];        // ping-pong state buffers
    const R *bath;     // B (double) or hbar = -B (float, perturbation form)
    DevClock *clk;
    double *partial;   // one double per block
    int nblocks;
    int *err;          // device error word (ERR_* bits)
    int fwd_rows;      // FP32 strip height (rows per block), 0 = default
    int keep_rest;     // FP32 2D: 1 computes wave-free rows in full (no skipping)
    const float *rest_tab;   // FP32 2D grid: rest CFL table of quiet units (null: none)
    unsigned char *umap;     // FP32 2D grid: 1 = unit had waves at an earlier step
    int umap_n;              // entries of umap
    GaugeRec gauges;   // fused gauge recording (n = 0: off)
    int wetdry;        // 1: the shore solver at dry and transonic edges
    R dry_tol;         // a cell with h <= dry_tol is dry
};

template <typename R>
int fwd_launch_step(const FwdParams<R> &p, cudaStream_t st);
// rest CFL table of the FP32 2D grid step (floats, and the kernel filling it)
size_t fwd_f32_rest_table_floats(int nx, int ny);
int fwd_f32_unit_map_bytes(int nx, int ny);
int fwd_f32_rest_table(const FwdParams<float> &p, float *tab, cudaStream_t st);
template <typename R>
int fwd_step_blocks(const FwdParams<R> &p);
template <typename R>
int fwd_launch_clock_init(const FwdParams<R> &p, double t0, cudaStream_t st);
template <> int fwd_launch_step<double>(const FwdParams<double> &, cudaStream_t);
template <> int fwd_launch_step<float>(const FwdParams<float> &, cudaStream_t);
template <> int fwd_step_blocks<double>(const FwdParams<double> &);
template <> int fwd_step_blocks<float>(const FwdParams<float> &);
// unsplit 2D step with transverse waves (ctu_kernels.cuh)
template <typename R>
int fwd_launch_ctu(const FwdParams<R> &p, cudaStream_t st);
template <typename R>
int fwd_ctu_blocks(const FwdParams<R> &p);
template <> int fwd_launch_ctu<double>(const FwdParams<double> &, cudaStream_t);
template <> int fwd_launch_ctu<float>(const FwdParams<float> &, cudaStream_t);
template <> int fwd_ctu_blocks<double>(const FwdParams<double> &);
template <> int fwd_ctu_blocks<float>(const FwdParams<float> &);
// split step with the shore solver (fwd_kernels.cuh, WD)
template <typename R>
int fwd_launch_wd(const FwdParams<R> &p, cudaStream_t st);
template <typename R>
int fwd_wd_blocks(const FwdParams<R> &p);
template <> int fwd_launch_wd<double>(const FwdParams<double> &, cudaStream_t);
template <> int fwd_launch_wd<float>(const FwdParams<float> &, cudaStream_t);
template <> int fwd_wd_blocks<double>(const FwdParams<double> &);
template <> int fwd_wd_blocks<float>(const FwdParams<float> &);
template <> int fwd_launch_clock_init<double>(const FwdParams<double> &, double, cudaStream_t);
template <> int fwd_launch_clock_init<float>(const FwdParams<float> &, double, cudaStream_t);

}  // namespace swadj
