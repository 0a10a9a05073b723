// adj_f64.cu -- FP64 adjoint-step instantiations, compiled without
// floating-point contraction (-fmad=false); expressions are evaluated in
// the same order as the FP64 reference solver, so the rounding matches it.
#include "adj_kernels.cuh"

namespace swadj {

template <typename R, bool TWO_D, int TX, int TY>
static int launch_adj(const AdjParams<R> &p, cudaStream_t st) {
    dim3 grid((p.nx + TX - 1) / TX, TWO_D ? (p.ny + TY - 1) / TY : 1);
    adj_step_kernel<R, TWO_D, TX, TY><<<grid, dim3(TX, TY), 0, st>>>(p);
    return swadj_host::cuda_check(cudaGetLastError(), "adj_step_kernel<double>");
}

template <>
int adj_launch_step<double>(const AdjParams<double> &p, cudaStream_t st) {
    if (p.two_d) return launch_adj<double, true, 32, 4>(p, st);
    return launch_adj<double, false, 128, 1>(p, st);
}

}  // namespace swadj
