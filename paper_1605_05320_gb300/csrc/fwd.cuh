// fwd.cuh -- forward-step kernel parameters and host launchers.
#pragma once

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
};

template <typename R>
int fwd_launch_step(const FwdParams<R> &p, cudaStream_t st);
template <typename R>
int fwd_step_blocks(const FwdParams<R> &p);
template <typename R>
int fwd_launch_clock_init(const FwdParams<R> &p, double t0, cudaStream_t st);
int fwd_read_clear_err(cudaStream_t st, int *out);

}  // namespace swadj
