// fwd_f64.cu -- FP64 forward-step instantiations.  This translation unit is
// compiled without floating-point contraction (-fmad=false) and the kernels
// evaluate every expression in the same order as the FP64 reference solver,
// so the FP64 path rounds exactly like it.  In (h, hu) form one ulp of a
// 4000 m depth (4.5e-13 m) already moves the momentum by ~1e-11 per step
// through g*hhat*(eta_R - eta_L); matching rounding is what keeps the FP64
// path within 1e-12 of the reference after thousands of steps.
#include "ctu_kernels.cuh"

namespace swadj {

template <typename R, bool PERT, bool TWO_D, int TX, int TY, bool WD = false>
static int launch_step(FwdParams<R> p, cudaStream_t st) {
    dim3 grid((p.nx + TX - 1) / TX, TWO_D ? (p.ny + TY - 1) / TY : 1);
    p.nblocks = (int)(grid.x * grid.y);
    fwd_step_kernel<R, PERT, TWO_D, TX, TY, WD><<<grid, dim3(TX, TY), 0, st>>>(p);
    return swadj_host::cuda_check(cudaGetLastError(), "fwd_step_kernel<double>");
}

template <>
int fwd_launch_step<double>(const FwdParams<double> &p, cudaStream_t st) {
    if (p.two_d) return launch_step<double, false, true, 32, 4>(p, st);
    return launch_step<double, false, false, 128, 1>(p, st);
}

template <>
int fwd_step_blocks<double>(const FwdParams<double> &p) {
    if (p.two_d) return ((p.nx + 31) / 32) * ((p.ny + 3) / 4);
    return (p.nx + 127) / 128;
}

template <>
int fwd_launch_wd<double>(const FwdParams<double> &p, cudaStream_t st) {
    if (p.two_d) return launch_step<double, false, true, 32, 4, true>(p, st);
    return launch_step<double, false, false, 128, 1, true>(p, st);
}

template <>
int fwd_wd_blocks<double>(const FwdParams<double> &p) {
    return fwd_step_blocks<double>(p);
}

template <>
int fwd_launch_ctu<double>(const FwdParams<double> &p, cudaStream_t st) {
    return ctu_launch<double, false, 16, 8>(p, st, "fwd_ctu_kernel<double>");
}

template <>
int fwd_ctu_blocks<double>(const FwdParams<double> &p) {
    return ctu_blocks<16, 8>(p.nx, p.ny);
}

template <>
int fwd_launch_clock_init<double>(const FwdParams<double> &p, double t0, cudaStream_t st) {
    const size_t n = (size_t)p.nx * p.ny;
    int blocks = (int)((n + 255) / 256);
    if (blocks > kInitBlocks) blocks = kInitBlocks;
    clock_init_kernel<double, false><<<blocks, 256, 0, st>>>(p, t0);
    return swadj_host::cuda_check(cudaGetLastError(), "clock_init_kernel<double>");
}

}  // namespace swadj
