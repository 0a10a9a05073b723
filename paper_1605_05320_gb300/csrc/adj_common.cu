// adj_common.cu -- adjoint set-up and snapshot-copy kernels.
#include "adj.cuh"

namespace swadj {

__device__ __forceinline__ void atomic_max_nonneg(double *a, double v) {
    // non-negative doubles order like their bit patterns as unsigned integers
    atomicMax((unsigned long long *)a, (unsigned long long)__double_as_longlong(v));
}

// Coefficient array: hbar = max(-B, 0) for double adjoints, c = sqrt(g hbar)
// (0 where dry) for float ones.  smax = max over wet cells of c/dx [+ c/dy].
template <typename R>
__global__ void adj_init_kernel(const double *B, R *c, size_t n, int two_d,
                                double g, double dx, double dy, double dry_tol,
                                double *smax) {
    double mx = 0.0;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x) {
        const double hb = -B[k] > 0.0 ? -B[k] : 0.0;
        double cc = 0.0, s = 0.0;
        if (hb > dry_tol) {
            cc = sqrt(g * hb);
            s = cc / dx;
            if (two_d && cc / dy > s) s = cc / dy;
        }
        c[k] = sizeof(R) == 8 ? (R)hb : (R)cc;
        mx = s > mx ? s : mx;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double w = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = w > mx ? w : mx;
    }
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(smax, mx);
}

template <typename R>
int adj_launch_init(const double *B, R *c, size_t n, int two_d, double g,
                    double dx, double dy, double dry_tol, double *smax,
                    cudaStream_t st) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 2048) blocks = 2048;
    adj_init_kernel<R><<<blocks, 256, 0, st>>>(B, c, n, two_d, g, dx, dy, dry_tol, smax);
    return swadj_host::cuda_check(cudaGetLastError(), "adj_init_kernel");
}

template <typename R>
__global__ void adj_store_kernel(const R *s0, const R *s1, const R *s2, int ncomp,
                                 size_t n, float *sf, double *sd, size_t cs,
                                 double *tau_dev, double tau_val) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x) {
        if (sf) {
            sf[k] = (float)s0[k];
            sf[cs + k] = (float)s1[k];
            if (ncomp == 3) sf[2 * cs + k] = (float)s2[k];
        } else {
            sd[k] = (double)s0[k];
            sd[cs + k] = (double)s1[k];
            if (ncomp == 3) sd[2 * cs + k] = (double)s2[k];
        }
        if (k == 0) *tau_dev = tau_val;
    }
}

template <typename R>
int adj_launch_store(const R *const src[3], int ncomp, size_t n, float *snap_f,
                     double *snap_d, size_t comp_stride, double *tau_dev,
                     double tau_val, cudaStream_t st) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    adj_store_kernel<R><<<blocks, 256, 0, st>>>(src[0], src[1], src[2], ncomp, n,
                                                snap_f, snap_d, comp_stride,
                                                tau_dev, tau_val);
    return swadj_host::cuda_check(cudaGetLastError(), "adj_store_kernel");
}

template int adj_launch_init<double>(const double *, double *, size_t, int, double,
                                     double, double, double, double *, cudaStream_t);
template int adj_launch_init<float>(const double *, float *, size_t, int, double,
                                    double, double, double, double *, cudaStream_t);
template int adj_launch_store<double>(const double *const[3], int, size_t, float *,
                                      double *, size_t, double *, double, cudaStream_t);
template int adj_launch_store<float>(const float *const[3], int, size_t, float *,
                                     double *, size_t, double *, double, cudaStream_t);

}  // namespace swadj
