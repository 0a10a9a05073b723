// fwd_f32.cu -- FP32 perturbation-form forward step (Eq. swe, Sec. 5; Roe-type
// f-wave solver per edge, Sec. 6) for GB300.
//
// Storage: eta = h + B, hu, hv and hbar = -B in float.  Depth h = eta + hbar
// enters only wave speeds and Roe averages; the surface jump that drives the
// bathymetry-balanced momentum flux is taken from eta directly, so decimetre
// waves on 4000 m are resolved to float precision of eta, not of h.
//
// 2D grids run the persistent tile kernel of fwd_tiles.cuh over the grid's
// tiles; 1D grids run a one-thread-per-cell kernel.  The CFL maximum is
// reduced in float (max is exact); the last block to finish turns it into the
// next time step in double.
#include "fwd_tiles.cuh"

namespace swadj {
namespace f32 {

// Tiles of one grid, row-major.
struct GridTiles {
    tile::View v;
    int ntx, nty, TX, TY;
    __device__ __forceinline__ int count() const { return ntx * nty; }
    __device__ __forceinline__ void get(int k, tile::View &out, int &i0, int &j0) const {
        out = v;
        const int ty = k / ntx;
        i0 = (k - ty * ntx) * TX;
        j0 = ty * TY;
    }
};

template <int TX, int TY>
__global__ void __launch_bounds__(256) fwd_f32_tiles(FwdParams<float> p) {
    extern __shared__ __align__(16) unsigned char dsm[];
    tile::Smem<TX, TY> &S = *reinterpret_cast<tile::Smem<TX, TY> *>(dsm);
    __shared__ float s_nu[2];
    __shared__ int s_cur, s_run;
    __shared__ float red[8];
    __shared__ int am_last;
    double t_now = 0.0, dt = 0.0;
    if (!tile::begin_step(p.clk, p.t_end, (double)p.dx, (double)p.dy, s_nu, &s_cur, &s_run,
                          t_now, dt))
        return;
    const int cur = s_cur;
    GridTiles src;
    src.v.q0 = p.q[cur][0]; src.v.q1 = p.q[cur][1]; src.v.q2 = p.q[cur][2]; src.v.hb = p.bath;
    src.v.o0 = p.q[cur ^ 1][0]; src.v.o1 = p.q[cur ^ 1][1]; src.v.o2 = p.q[cur ^ 1][2];
    src.v.nx = p.nx; src.v.ny = p.ny; src.v.dx = p.dx; src.v.dy = p.dy; src.v.bc = p.bc;
    src.ntx = (p.nx + TX - 1) / TX;
    src.nty = (p.ny + TY - 1) / TY;
    src.TX = TX;
    src.TY = TY;
    bool bad = false;
    const float sm = tile::run_tiles<TX, TY>(S, src, s_nu[0], s_nu[1], p.g, p.order, bad);
    if (bad) atomicOr(p.err, ERR_UNSTABLE);
    tile::finish_step<256>(p.clk, p.partial, p.nblocks, p.cfl, sm, red, &am_last, t_now, dt,
                           cur);
}

// 1D grids: one thread per cell, solving the four edges it needs itself
// (1D grids are small; the redundancy costs nothing that matters).
__global__ void __launch_bounds__(256) fwd_f32_1d(FwdParams<float> p) {
    __shared__ float s_nu[2];
    __shared__ int s_cur, s_run;
    __shared__ float red[8];
    __shared__ int am_last;
    double t_now = 0.0, dt = 0.0;
    if (!tile::begin_step(p.clk, p.t_end, (double)p.dx, (double)p.dy, s_nu, &s_cur, &s_run,
                          t_now, dt))
        return;
    const int cur = s_cur;
    const float nux = s_nu[0], g = p.g;
    const float *q0 = p.q[cur][0], *q1 = p.q[cur][1];
    const int i = blockIdx.x * 256 + threadIdx.x;
    float sm = 0.f;
    bool bad = false;
    if (i < p.nx) {
        float h[5], mu[5], u[5], sq[5], eta[5];
#pragma unroll
        for (int k = 0; k < 5; k++) {
            bool fx;
            const int c = ghost_index(i - 2 + k, p.nx, p.bc.lo_x, p.bc.hi_x, &fx);
            eta[k] = q0[c];
            mu[k] = fx ? -q1[c] : q1[c];
            h[k] = eta[k] + p.bath[c];
            const float q = rsqrtf(h[k]);
            sq[k] = h[k] * q;
            u[k] = mu[k] * q * q;
        }
        tile::EdgeS w[4];
#pragma unroll
        for (int k = 0; k < 4; k++)
            w[k] = tile::solve1(g, h[k], mu[k], 0.f, u[k], 0.f, sq[k], eta[k], h[k + 1],
                                mu[k + 1], 0.f, u[k + 1], 0.f, sq[k + 1], eta[k + 1]);
        float L0[3], R0[3], L1[3], R1[3];
        tile::net1<false>(w[0], w[1], w[2], nux, p.order, L0, R0);
        tile::net1<false>(w[1], w[2], w[3], nux, p.order, L1, R1);
        const float d0 = -nux * (R0[0] + L1[0]);
        const float ne = eta[2] + d0;
        const float nmu = mu[2] - nux * (R0[1] + L1[1]);
        p.q[cur ^ 1][0][i] = ne;
        p.q[cur ^ 1][1][i] = nmu;
        const float hn = h[2] + d0;
        bad = !(hn > 0.f) || !isfinite(nmu);
        sm = cfl_f32(hn, nmu, 0.f, g, 1.f / p.dx, 1.f / p.dy, 0);
    }
    if (bad) atomicOr(p.err, ERR_UNSTABLE);
    tile::finish_step<256>(p.clk, p.partial, p.nblocks, p.cfl, sm, red, &am_last, t_now, dt,
                           cur);
}

}  // namespace f32

constexpr int kTX = 32;

// Tile height of the FP32 step: 16 rows by default, 8 on request (the
// autotuner's choice); both give the same results.
static int tile_rows(const FwdParams<float> &p) { return p.fwd_rows == 8 ? 8 : 16; }

// Blocks of the persistent launch: every SM filled with as many blocks as
// fit, never more than there are tiles.
template <int TY>
static int persistent_blocks(int ntiles) {
    static int per_sm = 0, sms = 0;
    if (per_sm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(f32::fwd_f32_tiles<kTX, TY>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(tile::Smem<kTX, TY>));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, f32::fwd_f32_tiles<kTX, TY>, 256, sizeof(tile::Smem<kTX, TY>));
        if (per_sm < 1) per_sm = 1;
        if (sms < 1) sms = 1;
    }
    const int b = per_sm * sms;
    return ntiles < b ? ntiles : b;
}

template <int TY>
static int launch_tiles(FwdParams<float> p, cudaStream_t st) {
    const int ntiles = ((p.nx + kTX - 1) / kTX) * ((p.ny + TY - 1) / TY);
    p.nblocks = persistent_blocks<TY>(ntiles);
    f32::fwd_f32_tiles<kTX, TY><<<p.nblocks, 256, sizeof(tile::Smem<kTX, TY>), st>>>(p);
    return swadj_host::cuda_check(cudaGetLastError(), "fwd_f32_tiles");
}

template <>
int fwd_launch_step<float>(const FwdParams<float> &p0, cudaStream_t st) {
    FwdParams<float> p = p0;
    if (p.two_d) return tile_rows(p) == 8 ? launch_tiles<8>(p, st) : launch_tiles<16>(p, st);
    dim3 grid((p.nx + 255) / 256, 1);
    p.nblocks = (int)grid.x;
    f32::fwd_f32_1d<<<grid, 256, 0, st>>>(p);
    return swadj_host::cuda_check(cudaGetLastError(), "fwd_f32_1d");
}

template <>
int fwd_step_blocks<float>(const FwdParams<float> &p) {
    if (p.two_d) {
        // at most one reduction slot per tile (the persistent grid is smaller)
        const int TY = tile_rows(p);
        return ((p.nx + kTX - 1) / kTX) * ((p.ny + TY - 1) / TY);
    }
    return (p.nx + 255) / 256;
}

template <>
int fwd_launch_clock_init<float>(const FwdParams<float> &p, double t0, cudaStream_t st) {
    const size_t n = (size_t)p.nx * p.ny;
    int blocks = (int)((n + 255) / 256);
    if (blocks > kInitBlocks) blocks = kInitBlocks;
    clock_init_kernel<float, true><<<blocks, 256, 0, st>>>(p, t0);
    return swadj_host::cuda_check(cudaGetLastError(), "clock_init_kernel<float>");
}

}  // namespace swadj
