// fwd_edge.cuh -- the clock handshake of the FP32 step kernels (read the
// device clock at the start; reduce the CFL number and advance the clock at
// the end), shared by the single-grid step (fwd_f32.cu) and the batched
// patch step (patches.cu).  The edge arithmetic is in fwd_pair.cuh.
#pragma once
#include "fwd_kernels.cuh"

namespace swadj {
namespace fwave {

// Thread 0 reads the clock and broadcasts nu_x, nu_y and the buffer index;
// false when the clock has reached t_end (no-op step).
__device__ __forceinline__ bool begin_step(DevClock *clkp, double t_end, double dx, double dy,
                                           float *s_nu, int *s_cur, int *s_run, double &t_now,
                                           double &dt) {
    if (threadIdx.x == 0) {
        volatile DevClock *clk = clkp;
        t_now = clk->t;
        dt = clk->dt_cfl;
        if (t_end - t_now < dt) dt = t_end - t_now;
        *s_run = dt > 0.0;
        s_nu[0] = (float)(dt / dx);
        s_nu[1] = (float)(dt / dy);
        *s_cur = clk->cur;
    }
    __syncthreads();
    return *s_run != 0;
}

// Block max of the CFL number (float, exact) -> partial[block]; the last block
// to arrive reduces the partials and advances the clock (t, dt, buffer,
// steps).  Only that block's thread 0 does FP64 work.
template <int NTH>
__device__ __forceinline__ void finish_step(DevClock *clkp, double *partial, int nblocks,
                                            double cfl, float sm, float *red, int *am_last,
                                            double t_now, double dt, int cur) {
    const int t = threadIdx.x;
    for (int o = 16; o > 0; o >>= 1) sm = fmaxf(sm, __shfl_xor_sync(0xffffffffu, sm, o));
    if ((t & 31) == 0) red[t >> 5] = sm;
    __syncthreads();
    const int bid = blockIdx.x + blockIdx.y * gridDim.x;
    if (t == 0) {
        float m = red[0];
        for (int k = 1; k < NTH / 32; k++) m = fmaxf(m, red[k]);
        reinterpret_cast<float *>(partial)[bid] = m;
        __threadfence();
        const unsigned int tk = atomicAdd(&clkp->ticket, 1u);
        *am_last = (tk == (unsigned int)(nblocks - 1));
    }
    __syncthreads();
    if (*am_last) {
        __threadfence();
        float m = 0.0f;
        const float *pf = reinterpret_cast<const float *>(partial);
        for (int k = t; k < nblocks; k += NTH) m = fmaxf(m, __ldcg(pf + k));
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        __syncthreads();
        if ((t & 31) == 0) red[t >> 5] = m;
        __syncthreads();
        if (t == 0) {
            for (int k = 0; k < NTH / 32; k++) m = fmaxf(m, red[k]);
            volatile DevClock *clk = clkp;
            clk->t = t_now + dt;
            clk->smax = (double)m;
            clk->dt_cfl = cfl / (double)m;
            clk->cur = cur ^ 1;
            clk->nsteps = clk->nsteps + 1;
            clk->ticket = 0u;
            clk->work = 0u;
        }
    }
}

}  // namespace fwave
}  // namespace swadj
