// audit.cu -- FP64 audit of the conserved mass of a grid: M = sum_i h_i dx dy
// over the interior cells, the quantity the conservative update of Eq. (swe)
// keeps constant between closed boundaries.
//
// The sum is formed in double whatever the storage precision: for the FP32
// perturbation form h = (double) eta + (double) hbar, so the audit sees the
// mass to FP64 rounding while the state itself is held in float.  The order
// of summation is fixed (a grid-stride sum per thread, a tree in each block,
// then one block over the block sums), so repeated audits of the same state
// give the same bits.
#include "swadj_internal.cuh"

namespace swadj {
namespace {

constexpr int kAuditThreads = 256;

template <typename R, bool PERT>
__global__ void __launch_bounds__(kAuditThreads)
    mass_partial_kernel(const R *q0a, const R *q0b, const R *bath, const DevClock *clk,
                        size_t n, double *partial) {
    __shared__ double red[kAuditThreads];
    const R *q0 = clk->cur ? q0b : q0a;   // the buffer holding the current state
    double s = 0.0;
    for (size_t k = (size_t)blockIdx.x * kAuditThreads + threadIdx.x; k < n;
         k += (size_t)gridDim.x * kAuditThreads)
        s += PERT ? (double)q0[k] + (double)bath[k] : (double)q0[k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = kAuditThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(kAuditThreads)
    mass_final_kernel(const double *partial, int nb, double area, double *out) {
    __shared__ double red[kAuditThreads];
    double s = 0.0;
    for (int k = threadIdx.x; k < nb; k += kAuditThreads) s += partial[k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = kAuditThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0] * area;
}

}  // namespace

// q0[2]: the depth (FP64) or surface (FP32) array of both state buffers;
// partial: at least `max_blocks` doubles of scratch.
int mass_launch(const void *const q0[2], const void *bath, int fp32, const DevClock *clk,
                size_t n, double area, double *partial, int max_blocks, double *out,
                cudaStream_t st) {
    int blocks = (int)((n + kAuditThreads - 1) / kAuditThreads);
    if (blocks > max_blocks) blocks = max_blocks;
    if (blocks < 1) blocks = 1;
    if (fp32)
        mass_partial_kernel<float, true><<<blocks, kAuditThreads, 0, st>>>(
            (const float *)q0[0], (const float *)q0[1], (const float *)bath, clk, n, partial);
    else
        mass_partial_kernel<double, false><<<blocks, kAuditThreads, 0, st>>>(
            (const double *)q0[0], (const double *)q0[1], nullptr, clk, n, partial);
    const int rc = swadj_host::cuda_check(cudaGetLastError(), "mass_partial_kernel");
    if (rc != SWA_OK) return rc;
    mass_final_kernel<<<1, kAuditThreads, 0, st>>>(partial, blocks, area, out);
    return swadj_host::cuda_check(cudaGetLastError(), "mass_final_kernel");
}

}  // namespace swadj
