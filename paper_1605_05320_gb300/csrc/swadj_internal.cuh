// swadj_internal.cuh -- device-side definitions shared by the libswadj kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "swadj.h"

namespace swadj {

// Device-resident clock of a forward grid.  Written only by the last block of
// each step kernel (after every block has read it), read at the start of the
// next one: time, step and buffer parity never leave the device, so step
// sequences can be captured in a CUDA graph.
struct DevClock {
    double t;           // current time t_n
    double dt_cfl;      // cfl / s_max(Q^n)
    long long nsteps;   // steps taken
    int cur;            // buffer index holding Q^n
    unsigned int ticket;  // last-block-done counter, 0 between launches
    unsigned int work;    // next work unit of a persistent step kernel, 0 between launches
    double smax;        // s_max(Q^n)
};

// Bits set in the device error word.
enum : int {
    ERR_UNSTABLE = 1,   // non-finite state or depth <= 0
    ERR_LAG = 2         // an AMR step's levels did not reach its end time
};

struct BcSpec {
    int lo_x, hi_x, lo_y, hi_y;
};

// Map a possibly out-of-range index onto the grid for ghost cells: copy the
// nearest cell (extrapolation) or mirror it (wall, with *flip set so the
// normal momentum is negated).  The result is clamped into [0, n).
__device__ __forceinline__ int ghost_index(int g, int n, int bc_lo, int bc_hi,
                                           bool *flip) {
    *flip = false;
    if (g < 0) {
        if (bc_lo == SWA_BC_WALL) { g = -g - 1; *flip = true; }
        else g = 0;
    } else if (g >= n) {
        if (bc_hi == SWA_BC_WALL) { g = 2 * n - 1 - g; *flip = true; }
        else g = n - 1;
    }
    g = g < 0 ? 0 : (g >= n ? n - 1 : g);
    return g;
}

// Read-only global load as volatile inline PTX: it stays ahead of the
// barriers that follow it in program order, so a register prefetch of the
// next tile is issued before the current tile's work instead of being moved
// next to its first use.
__device__ __forceinline__ float ld_early(const float *p) {
    float v;
    asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

// Asynchronous 4-byte copy global -> shared (cp.async), its commit and the
// wait until at most N of this thread's newest copy groups are pending.
__device__ __forceinline__ void cp_async4(float *dst, const float *src) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(a), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// One-instruction approximate reciprocal and reciprocal square root
// (hand-written PTX) with subnormals flushed to zero.  Their inputs in the
// FP32 kernels are positive normal numbers: depths, sums of square roots of
// depths, 1 + s^2 terms.
__device__ __forceinline__ float rcp_ftz(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// MC limiter: max(0, min((1+theta)/2, 2, 2 theta)).
template <typename R>
__device__ __forceinline__ R mc_phi(R theta) {
    R a = R(0.5) * (R(1) + theta);
    R m = a < R(2) ? a : R(2);
    R c = R(2) * theta;
    m = c < m ? c : m;
    return m > R(0) ? m : R(0);
}

template <typename R>
__device__ __forceinline__ R sgnr(R s) {
    return s > R(0) ? R(1) : (s < R(0) ? R(-1) : R(0));
}

// Block-wide max of a non-negative double, result valid in thread 0.
template <int NT>
__device__ __forceinline__ double block_max(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) {
        double w = __shfl_xor_sync(0xffffffffu, v, o);
        v = v > w ? v : w;
    }
    const int lane = threadIdx.x & 31;
    const int wid = (threadIdx.x + threadIdx.y * blockDim.x) >> 5;
    if (NT > 32) {
        if (lane == 0) red[wid] = v;
        __syncthreads();
        if (wid == 0) {
            v = (lane < NT / 32) ? red[lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) {
                double w = __shfl_xor_sync(0xffffffffu, v, o);
                v = v > w ? v : w;
            }
        }
    }
    return v;
}

}  // namespace swadj

// Host-side helpers shared by the translation units (defined in api.cu).
namespace swadj {
// Internal view of a forward grid (api.cu), for the AMR glue (patches.cu).
struct GridRefs {
    swa_grid_desc d;
    void *q[2][3];      // ping-pong state buffers
    const void *bath;   // B (FP64) or hbar = -B (FP32)
    DevClock *clk;
    int state_set;
    int scheme;         // SWA_SCHEME_SPLIT or SWA_SCHEME_CTU
};
int grid_refs(const swa_grid *g, GridRefs *out);
// FP64 mass audit (audit.cu)
int mass_launch(const void *const q0[2], const void *bath, int fp32, const DevClock *clk,
                size_t n, double area, double *partial, int max_blocks, double *out,
                cudaStream_t st);
}  // namespace swadj

namespace swadj_host {
int set_error(int code, const char *fmt, ...);
int cuda_check(cudaError_t e, const char *what);
int *error_word();  // device address of the error word of the current device
}  // namespace swadj_host
