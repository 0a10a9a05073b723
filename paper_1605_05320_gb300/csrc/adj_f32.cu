// adj_f32.cu -- FP32 adjoint-step instantiations.
#include "adj_kernels.cuh"

namespace swadj {

template <typename R, bool TWO_D, int TX, int TY>
static int launch_adj(const AdjParams<R> &p, cudaStream_t st) {
    dim3 grid((p.nx + TX - 1) / TX, TWO_D ? (p.ny + TY - 1) / TY : 1);
    adj_step_kernel<R, TWO_D, TX, TY><<<grid, dim3(TX, TY), 0, st>>>(p);
    return swadj_host::cuda_check(cudaGetLastError(), "adj_step_kernel<float>");
}

template <>
int adj_launch_step<float>(const AdjParams<float> &p, cudaStream_t st) {
    if (p.two_d) return launch_adj<float, true, 32, 8>(p, st);
    return launch_adj<float, false, 128, 1>(p, st);
}

}  // namespace swadj
