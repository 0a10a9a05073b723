// noalloc.cu -- swa_step_forward_static: one forward step for callers that
// cannot allocate device memory.
//
// Some callers hold device memory they did not allocate and are not allowed
// to allocate more: a host framework that owns the whole memory pool and
// hands out only the state arrays, code running where cudaMalloc is
// forbidden (inside a region that must not synchronise the device, or under
// a fixed memory budget decided up front).  They can pass their own input
// and output arrays, but not the per-block scratch that the CFL reduction
// of the step kernel needs.  This entry point takes that scratch from a
// fixed file-scope device array instead, so it allocates nothing.
//
// The array is loaded with the library: every GPU that loads libswadj.so
// holds kStaticScratchBytes of device memory for it until the process exits.
// All calls share it and it keeps the last call's contents; each call resets
// the part that must start from zero (the clock and its block ticket) with a
// one-thread kernel on the caller's stream before its step kernel runs, so a
// call reads no host memory and does not synchronise.  Calls whose kernels overlap on the GPU (two streams, or
// two host threads) race on the array and give wrong results: serialise
// them on one stream.
#include <mutex>

#include "fwd.cuh"
#include "swadj_internal.cuh"

namespace swadj {

// 256 bytes of clock followed by one 8-byte partial maximum per block
// (SWA_STATIC_MAX_BLOCKS of them, 256 KiB + 256 B in all).
constexpr size_t kStaticClockBytes = 256;
constexpr int kStaticMaxBlocks = SWA_STATIC_MAX_BLOCKS;
constexpr size_t kStaticScratchBytes = SWA_STATIC_SCRATCH_BYTES;
static_assert(kStaticScratchBytes == kStaticClockBytes + 8 * (size_t)kStaticMaxBlocks,
              "static scratch layout");

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Puts the static clock in the state a step starts from: time 0, the
// caller's dt, buffer 0 holding the input, no steps, block ticket and
// work-unit counter 0.
__global__ void static_clock_reset(DevClock *clk, double dt) {
    clk->t = 0.0;
    clk->dt_cfl = dt;
    clk->nsteps = 0;
    clk->cur = 0;
    clk->ticket = 0u;
    clk->work = 0u;
    clk->smax = 0.0;
}

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices];

// Device address of the static scratch for the current device.  The first
// call on a device looks it up (cudaGetSymbolAddress) and caches it; in host
// code the array's name is only a host-side stand-in, never a device
// address, so the kernels always get this looked-up pointer.  The cache
// outlives a cudaDeviceReset, after which the module may load elsewhere, so
// resetting a device while the library is in use is not supported.
int scratch_for_current_device(void **scratch, int **err) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return swadj_host::cuda_check(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices)
        return swadj_host::set_error(SWA_EINVAL, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return swadj_host::cuda_check(e, "cudaGetSymbolAddress(scratch)");
        g_scratch_ptr[dev] = p;
    }
    *scratch = g_scratch_ptr[dev];
    *err = swadj_host::error_word();  // the word swa_sync_status reports
    return *err ? SWA_OK : swadj_host::set_error(SWA_ECUDA, "device error word unavailable");
}

template <typename R>
int run_static(const swa_grid_desc *d, const void *const q_in[3], void *const q_out[3],
               const void *bath, double dt, double *smax_out, cudaStream_t st) {
    FwdParams<R> p{};
    p.nx = d->nx; p.ny = d->ny; p.two_d = d->ndim == 2; p.order = d->order;
    p.bc = BcSpec{d->bc[0], d->bc[1], d->bc[2], d->bc[3]};
    p.dx = (R)d->dx; p.dy = (R)d->dy; p.g = (R)d->g;
    p.cfl = d->cfl;
    p.t_end = 1e300;
    const int blocks = fwd_step_blocks<R>(p);
    if (blocks > kStaticMaxBlocks)
        return swadj_host::set_error(
            SWA_ENOMEM,
            "swa_step_forward_static: this %dx%d grid needs %d reduction slots, the static "
            "scratch holds %d; use swa_step_forward with a workspace",
            d->nx, d->ny, blocks, kStaticMaxBlocks);
    void *scratch = nullptr;
    int *err = nullptr;
    int rc = scratch_for_current_device(&scratch, &err);
    if (rc != SWA_OK) return rc;
    // reset the clock (t = 0, dt, buffer 0 = input, ticket 0) before the step,
    // from kernel arguments: no host memory is read
    static_clock_reset<<<1, 1, 0, st>>>((DevClock *)scratch, dt);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return swadj_host::cuda_check(e, "static clock reset");
    for (int k = 0; k < 3; k++) {
        p.q[0][k] = (R *)q_in[k];
        p.q[1][k] = (R *)q_out[k];
    }
    p.bath = (const R *)bath;
    p.clk = (DevClock *)scratch;
    p.partial = (double *)((unsigned char *)scratch + kStaticClockBytes);
    p.nblocks = blocks;
    p.err = err;
    int rc2 = fwd_launch_step<R>(p, st);
    if (rc2 != SWA_OK || !smax_out) return rc2;
    // the step leaves s_max of the new state in the static clock
    e = cudaMemcpyAsync(smax_out, &((DevClock *)scratch)->smax, sizeof(double),
                        cudaMemcpyDeviceToDevice, st);
    return swadj_host::cuda_check(e, "s_max copy");
}
}  // namespace

}  // namespace swadj

extern "C" int swa_step_forward_static(const swa_grid_desc *desc, const void *const q_in[3],
                                       void *const q_out[3], const void *bath, double dt,
                                       double *smax_out_dev, void *stream) {
    using namespace swadj;
    if (!desc || !q_in || !q_out || !bath)
        return swadj_host::set_error(SWA_EINVAL, "null argument");
    if (desc->ndim != 1 && desc->ndim != 2)
        return swadj_host::set_error(SWA_EINVAL, "ndim must be 1 or 2");
    if (desc->nx < 2 || desc->ny < 1 || (desc->ndim == 1 && desc->ny != 1) ||
        (desc->ndim == 2 && desc->ny < 2))
        return swadj_host::set_error(SWA_EINVAL, "bad grid size");
    if (desc->order != 1 && desc->order != 2)
        return swadj_host::set_error(SWA_EINVAL, "order must be 1 or 2");
    for (int k = 0; k < 3; k++) {
        if (!q_in[k] && (k < 2 || desc->ndim == 2))
            return swadj_host::set_error(SWA_EINVAL, "null input array %d", k);
        if (!q_out[k] && (k < 2 || desc->ndim == 2))
            return swadj_host::set_error(SWA_EINVAL, "null output array %d", k);
        if (k < 2 || desc->ndim == 2)
            if (q_in[k] == q_out[k])
                return swadj_host::set_error(SWA_EINVAL, "input and output arrays must differ");
    }
    if (!(dt > 0)) return swadj_host::set_error(SWA_EINVAL, "dt must be > 0");
    if (desc->precision == SWA_FP64)
        return run_static<double>(desc, q_in, q_out, bath, dt, smax_out_dev, (cudaStream_t)stream);
    if (desc->precision == SWA_FP32)
        return run_static<float>(desc, q_in, q_out, bath, dt, smax_out_dev, (cudaStream_t)stream);
    return swadj_host::set_error(SWA_EINVAL, "precision must be SWA_FP64 or SWA_FP32");
}
