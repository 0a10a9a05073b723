// alu_peak.cu -- swa_alu_probe: throughput probes of the arithmetic units the
// step kernels are bound by, so that rooflines can be stated against peaks
// measured on the device at hand rather than against data-sheet figures.
//
// Each thread runs kChains independent dependency chains of one operation
// for `iters` rounds (independent chains hide the pipeline latency), then
// folds them into one store so nothing is optimised away.  Operations:
//   SWA_PROBE_FFMA64   fma.rn.f64           (2 flops each)
//   SWA_PROBE_FFMA32   fma.rn.f32           (2 flops each)
//   SWA_PROBE_FFMA32X2 fma.rn.f32x2         (4 flops each, two lanes' worth)
//   SWA_PROBE_RSQRT32  rsqrt.approx.ftz.f32 (1 op each; the special-function unit)
// The caller times the launch (CUDA events on `stream`) and divides
// swa_alu_probe_ops() by the time.
#include "swadj_internal.cuh"

namespace swadj {
namespace {

constexpr int kChains = 8;

template <int KIND>
__global__ void __launch_bounds__(256) alu_probe_kernel(float *sink, int iters, float seed) {
    const float s = seed + 1e-7f * (float)threadIdx.x;
    if (KIND == SWA_PROBE_FFMA64) {
        double a[kChains];
        const double b = 0.999999, c = 1e-7 * (double)s;
#pragma unroll
        for (int k = 0; k < kChains; k++) a[k] = (double)s + k;
        for (int i = 0; i < iters; i++)
#pragma unroll
            for (int k = 0; k < kChains; k++) a[k] = fma(a[k], b, c);
        double t = 0.0;
#pragma unroll
        for (int k = 0; k < kChains; k++) t += a[k];
        if (t == 1234.5) sink[blockIdx.x] = (float)t;
    } else if (KIND == SWA_PROBE_FFMA32) {
        float a[kChains];
        const float b = 0.999999f, c = 1e-7f * s;
#pragma unroll
        for (int k = 0; k < kChains; k++) a[k] = s + k;
        for (int i = 0; i < iters; i++)
#pragma unroll
            for (int k = 0; k < kChains; k++) a[k] = fmaf(a[k], b, c);
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < kChains; k++) t += a[k];
        if (t == 1234.5f) sink[blockIdx.x] = t;
    } else if (KIND == SWA_PROBE_FFMA32X2) {
        float2 a[kChains];
        const float2 b = make_float2(0.999999f, 0.999998f), c = make_float2(1e-7f * s, 2e-7f * s);
#pragma unroll
        for (int k = 0; k < kChains; k++) a[k] = make_float2(s + k, s - k);
        for (int i = 0; i < iters; i++)
#pragma unroll
            for (int k = 0; k < kChains; k++) a[k] = __ffma2_rn(a[k], b, c);
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < kChains; k++) t += a[k].x + a[k].y;
        if (t == 1234.5f) sink[blockIdx.x] = t;
    } else {
        float a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; k++) a[k] = s + 0.25f * k;
        for (int i = 0; i < iters; i++)
#pragma unroll
            for (int k = 0; k < kChains; k++) a[k] = rsqrt_ftz(a[k]);
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < kChains; k++) t += a[k];
        if (t == 1234.5f) sink[blockIdx.x] = t;
    }
}

}  // namespace
}  // namespace swadj

extern "C" {

double swa_alu_probe_ops(int kind, int blocks, int threads, int iters) {
    const double per = kind == SWA_PROBE_FFMA32X2 ? 4.0 : (kind == SWA_PROBE_RSQRT32 ? 1.0 : 2.0);
    return per * swadj::kChains * (double)blocks * (double)threads * (double)iters;
}

int swa_alu_probe(int kind, int blocks, int threads, int iters, float *sink_dev, void *stream) {
    using namespace swadj;
    if (blocks < 1 || threads < 32 || threads > 256 || (threads & 31) || iters < 1 || !sink_dev)
        return swadj_host::set_error(SWA_EINVAL, "alu probe: bad launch shape or null sink");
    cudaStream_t st = (cudaStream_t)stream;
    switch (kind) {
        case SWA_PROBE_FFMA64:
            alu_probe_kernel<SWA_PROBE_FFMA64><<<blocks, threads, 0, st>>>(sink_dev, iters, 1.f);
            break;
        case SWA_PROBE_FFMA32:
            alu_probe_kernel<SWA_PROBE_FFMA32><<<blocks, threads, 0, st>>>(sink_dev, iters, 1.f);
            break;
        case SWA_PROBE_FFMA32X2:
            alu_probe_kernel<SWA_PROBE_FFMA32X2><<<blocks, threads, 0, st>>>(sink_dev, iters, 1.f);
            break;
        case SWA_PROBE_RSQRT32:
            alu_probe_kernel<SWA_PROBE_RSQRT32><<<blocks, threads, 0, st>>>(sink_dev, iters, 1.f);
            break;
        default:
            return swadj_host::set_error(SWA_EINVAL, "alu probe: unknown kind %d", kind);
    }
    return swadj_host::cuda_check(cudaGetLastError(), "alu_probe_kernel");
}

}  // extern "C"
