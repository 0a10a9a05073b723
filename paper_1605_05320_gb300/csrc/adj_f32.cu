// adj_f32.cu -- FP32 adjoint step (Sec. 4; the time-reversed linear adjoint
// of adj_kernels.cuh, dimensionally split y then x).
//
// 2D grids run a persistent tile kernel in the style of the forward step:
// a TX x TY tile and a 2-cell halo with corners are staged in shared memory;
// phases (1) y-edge waves of every staged column, (2) their net fluxes (the
// limiter once per edge), (3) y-sweep of the tile rows in every staged
// column, in place (the x-sweep needs the y-swept state in the halo
// columns), (4) x-edge waves of the tile rows, (5) their net fluxes, (6)
// x-sweep update, written to the new state and, every snapshot step, to the
// snapshot slot.  The raw values of the next tile are loaded into registers
// while the current one is computed.  1D grids keep the one-tile-per-block
// kernel of adj_kernels.cuh.
//
// The limiter needs no division by the wave norm: for Z = b (c, 1) and its
// upwind neighbour Zu = bu (cu, 1), theta b = bu (cu c + 1) / (c^2 + 1), and
// phi(theta) b is formed from (b, theta b) directly (zero for b = 0, where
// the division form sets theta = 0).
#include "adj_kernels.cuh"

namespace swadj {
namespace adjt {

constexpr int NT = 256;

__device__ __forceinline__ float rcpf(float x) { return __fdividef(1.0f, x); }

// phi(theta) b for the MC limiter, r = theta b
__device__ __forceinline__ float mc1(float b, float r) {
    const float sg = b < 0.f ? -1.f : 1.f;
    const float B = fabsf(b), Rr = sg * r;
    float m = fminf(0.5f * (B + Rr), 2.f * B);
    m = fminf(m, 2.f * Rr);
    return sg * fmaxf(m, 0.f);
}

struct EdgeA {   // waves of one edge: strengths and the (substituted) speeds
    float b1, b2, cl, cr;
    bool wall;     // a wet / dry edge: no second-order correction
};

// Waves at the edge between (eL, mL, cL) and (eR, mR, cR), m the normal
// component; c = 0 marks a dry cell, mirrored from its wet neighbour.
__device__ __forceinline__ EdgeA solve_a(float eL, float mL, float cL, float eR, float mR,
                                         float cR) {
    EdgeA w;
    const bool dL = !(cL > 0.f), dR = !(cR > 0.f);
    w.wall = dL || dR;
    if (dL && dR) { w.b1 = 0.f; w.b2 = 0.f; w.cl = 0.f; w.cr = 0.f; return w; }
    if (dL) { eL = eR; mL = -mR; cL = cR; }
    if (dR) { eR = eL; mR = -mL; cR = cL; }
    // flux jump of F = -(g hbar m, eta), g hbar = c^2
    const float d1 = cL * cL * mL - cR * cR * mR;
    const float d2 = eL - eR;
    const float rs = rcpf(cL + cR);
    w.b1 = (d1 + cR * d2) * rs;
    w.b2 = (cL * d2 - d1) * rs;
    w.cl = cL;
    w.cr = cR;
    return w;
}

// Shared-memory record of an edge, (b1, b2, cl, cr) with the wall flag in
// the sign bit of cl (cl >= 0, so |cl| restores it exactly).
__device__ __forceinline__ float4 pack_edge(const EdgeA &w) {
    return make_float4(w.b1, w.b2, w.wall ? -w.cl : w.cl, w.cr);
}
__device__ __forceinline__ EdgeA unpack_edge(const float4 &r) {
    EdgeA w;
    w.b1 = r.x; w.b2 = r.y; w.cl = fabsf(r.z); w.cr = r.w;
    w.wall = signbit(r.z);
    return w;
}

// Net fluxes of edge w (neighbour edges wl, wr) as (L0, L1, R0, R1): L into
// the left cell, R into the right cell (Q -= nu * net); components
// (eta~, normal).
__device__ __forceinline__ float4 net_a(const EdgeA &wl, const EdgeA &w, const EdgeA &wr,
                                        float nu, int order) {
    float F0 = 0.f, F1 = 0.f;
    if (order >= 2 && !w.wall) {
        // wave 1 (speed -cl) is upwinded from the right edge, wave 2 (+cr)
        // from the left edge
        const float r1 = wr.b1 * fmaf(wr.cl, w.cl, 1.f) * rcpf(fmaf(w.cl, w.cl, 1.f));
        const float r2 = wl.b2 * fmaf(wl.cr, w.cr, 1.f) * rcpf(fmaf(w.cr, w.cr, 1.f));
        const float k1 = -0.5f * fmaf(-nu, w.cl, 1.f) * mc1(w.b1, r1);
        const float k2 = 0.5f * fmaf(-nu, w.cr, 1.f) * mc1(w.b2, r2);
        F0 = k1 * w.cl - k2 * w.cr;
        F1 = k1 + k2;
    }
    return make_float4(w.b1 * w.cl + F0, w.b1 + F1, -(w.b2 * w.cr) - F0, w.b2 - F1);
}

template <int TX, int TY>
struct Smem {
    static constexpr int RX = TX + 4, RY = TY + 4, NEX = TX + 3, NEY = TY + 3;
    float4 q[RY][RX];   // cell records (eta~, mu~, gamma~, c)
    union W {           // edge records: y (phases 1-2), then x (4-5)
        float4 y[NEY][RX];
        float4 x[TY][NEX];
    } w;
    union N {           // net fluxes (L0, L1, R0, R1): y (phases 2-3), then x (5-6)
        float4 y[TY + 1][RX];
        float4 x[TY][TX + 1];
    } n;
};

template <int TX, int TY>
struct Raw {
    static constexpr int RX = TX + 4, RY = TY + 4;
    static constexpr int RPT = (RX * RY + NT - 1) / NT;
    float e[RPT], m[RPT], g[RPT], c[RPT];
};

template <int TX, int TY>
__device__ __forceinline__ void load_raw(const AdjParams<float> &p, int i0, int j0,
                                         Raw<TX, TY> &R) {
    constexpr int RX = TX + 4, RY = TY + 4;
    const bool interior = i0 - 2 >= 0 && i0 + TX + 2 <= p.nx && j0 - 2 >= 0 &&
                          j0 + TY + 2 <= p.ny;
#pragma unroll
    for (int k = 0; k < Raw<TX, TY>::RPT; k++) {
        const int r = threadIdx.x + k * NT;
        if (r >= RX * RY) continue;
        const int ry = r / RX, rx = r - ry * RX;
        int ci = i0 + rx - 2, cj = j0 + ry - 2;
        bool fx = false, fy = false;
        if (!interior) {
            ci = ghost_index(ci, p.nx, p.bc.lo_x, p.bc.hi_x, &fx);
            cj = ghost_index(cj, p.ny, p.bc.lo_y, p.bc.hi_y, &fy);
        }
        const size_t o = (size_t)cj * p.nx + ci;
        R.e[k] = ld_early(p.src[0] + o);
        R.c[k] = ld_early(p.c + o);
        const float mu = ld_early(p.src[1] + o), ga = ld_early(p.src[2] + o);
        R.m[k] = fx ? -mu : mu;
        R.g[k] = fy ? -ga : ga;
    }
}

template <int TX, int TY>
__device__ __forceinline__ void tile_compute(Smem<TX, TY> &S, const AdjParams<float> &p,
                                             int i0, int j0, const Raw<TX, TY> &R) {
    constexpr int RX = TX + 4, RY = TY + 4, NEX = TX + 3, NEY = TY + 3;
    const int tid = threadIdx.x;
    const float nux = p.nux, nuy = p.nuy;
    const int order = p.order;
    // phase 0: stage
#pragma unroll
    for (int k = 0; k < Raw<TX, TY>::RPT; k++) {
        const int r = tid + k * NT;
        if (r >= RX * RY) continue;
        const int ry = r / RX, rx = r - ry * RX;
        S.q[ry][rx] = make_float4(R.e[k], R.m[k], R.g[k], R.c[k]);
    }
    __syncthreads();
    // phase 1: y-edge waves of every staged column (edge k between rows k, k+1)
    for (int i = tid; i < NEY * RX; i += NT) {
        const int k = i / RX, rx = i - k * RX;
        const float4 a = S.q[k][rx], b = S.q[k + 1][rx];
        S.w.y[k][rx] = pack_edge(solve_a(a.x, a.z, a.w, b.x, b.z, b.w));
    }
    __syncthreads();
    // phase 2: y net fluxes of edges 1 .. TY+1 in every staged column
    for (int i = tid; i < (TY + 1) * RX; i += NT) {
        const int e = 1 + i / RX, rx = i - (e - 1) * RX;
        S.n.y[e - 1][rx] = net_a(unpack_edge(S.w.y[e - 1][rx]), unpack_edge(S.w.y[e][rx]),
                                 unpack_edge(S.w.y[e + 1][rx]), nuy, order);
    }
    __syncthreads();
    // phase 3: y-sweep of the tile rows in every staged column, in place;
    // lower edge of row -> R at index row, upper edge -> L at row + 1
    for (int i = tid; i < TY * RX; i += NT) {
        const int row = i / RX, rx = i - row * RX, ry = row + 2;
        float4 c = S.q[ry][rx];
        if (c.w > 0.f) {
            const float4 lo = S.n.y[row][rx], up = S.n.y[row + 1][rx];
            c.x += -nuy * (lo.z + up.x);
            c.z += -nuy * (lo.w + up.y);
            S.q[ry][rx] = c;
        }
    }
    __syncthreads();
    // phase 4: x-edge waves of the y-swept tile rows (edge k between cols k, k+1)
    for (int i = tid; i < TY * NEX; i += NT) {
        const int row = i / NEX, k = i - row * NEX, ry = row + 2;
        const float4 a = S.q[ry][k], b = S.q[ry][k + 1];
        S.w.x[row][k] = pack_edge(solve_a(a.x, a.y, a.w, b.x, b.y, b.w));
    }
    __syncthreads();
    // phase 5: x net fluxes of edges 1 .. TX+1 of the tile rows
    for (int i = tid; i < TY * (TX + 1); i += NT) {
        const int row = i / (TX + 1), e = 1 + (i - row * (TX + 1));
        S.n.x[row][e - 1] = net_a(unpack_edge(S.w.x[row][e - 1]), unpack_edge(S.w.x[row][e]),
                                  unpack_edge(S.w.x[row][e + 1]), nux, order);
    }
    __syncthreads();
    // phase 6: x-sweep of the tile cells -> new state (+ snapshot)
    constexpr int CPT = TX * TY / NT;
#pragma unroll
    for (int k = 0; k < CPT; k++) {
        const int cidx = tid + k * NT, row = cidx / TX, col = cidx % TX;
        const int gi = i0 + col, gj = j0 + row;
        const int ry = row + 2, rx = col + 2;
        if (gi < p.nx && gj < p.ny) {
            const float4 c = S.q[ry][rx];
            float ne = c.x, nm = c.y;
            const float ng = c.z;
            if (c.w > 0.f) {
                const float4 le = S.n.x[row][col], re = S.n.x[row][col + 1];
                ne += -nux * (le.z + re.x);
                nm += -nux * (le.w + re.y);
            }
            const size_t o = (size_t)gj * p.nx + gi;
            p.dst[0][o] = ne;
            p.dst[1][o] = nm;
            p.dst[2][o] = ng;
            if (p.snap_f) {
                __stcs(p.snap_f + o, ne);
                __stcs(p.snap_f + p.snap_comp_stride + o, nm);
                __stcs(p.snap_f + 2 * p.snap_comp_stride + o, ng);
            } else if (p.snap_d) {
                __stcs(p.snap_d + o, (double)ne);
                __stcs(p.snap_d + p.snap_comp_stride + o, (double)nm);
                __stcs(p.snap_d + 2 * p.snap_comp_stride + o, (double)ng);
            }
        }
    }
    __syncthreads();  // the next tile overwrites the shared buffers
}

template <int TX, int TY>
__global__ void __launch_bounds__(NT) adj_f32_tiles(AdjParams<float> p) {
    extern __shared__ __align__(16) unsigned char dsm[];
    Smem<TX, TY> &S = *reinterpret_cast<Smem<TX, TY> *>(dsm);
    const int ntx = (p.nx + TX - 1) / TX;
    const int n = ntx * ((p.ny + TY - 1) / TY);
    if ((p.snap_f || p.snap_d) && blockIdx.x == 0 && threadIdx.x == 0) *p.tau_dev = p.tau_val;
    int k = blockIdx.x;
    if (k >= n) return;
    int ty = k / ntx;
    int i0 = (k - ty * ntx) * TX, j0 = ty * TY;
    Raw<TX, TY> cur;
    load_raw<TX, TY>(p, i0, j0, cur);
    while (true) {
        const int kn = k + gridDim.x;
        int in0 = 0, jn0 = 0;
        Raw<TX, TY> nxt;
        if (kn < n) {
            const int tyn = kn / ntx;
            in0 = (kn - tyn * ntx) * TX;
            jn0 = tyn * TY;
            load_raw<TX, TY>(p, in0, jn0, nxt);
        }
        tile_compute<TX, TY>(S, p, i0, j0, cur);
        if (kn >= n) break;
        k = kn; i0 = in0; j0 = jn0; cur = nxt;
    }
}

}  // namespace adjt

constexpr int kATX = 32, kATY = 16;

// Blocks of the persistent launch: every SM filled with as many blocks as
// fit, never more than there are tiles.
static int adj_persistent_blocks(int ntiles) {
    static int per_sm = 0, sms = 0;
    if (per_sm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(adjt::adj_f32_tiles<kATX, kATY>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(adjt::Smem<kATX, kATY>));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, adjt::adj_f32_tiles<kATX, kATY>, adjt::NT,
            sizeof(adjt::Smem<kATX, kATY>));
        if (per_sm < 1) per_sm = 1;
        if (sms < 1) sms = 1;
    }
    const int b = per_sm * sms;
    return ntiles < b ? ntiles : b;
}

template <>
int adj_launch_step<float>(const AdjParams<float> &p, cudaStream_t st) {
    if (p.two_d) {
        const int ntiles = ((p.nx + kATX - 1) / kATX) * ((p.ny + kATY - 1) / kATY);
        const int blocks = adj_persistent_blocks(ntiles);
        adjt::adj_f32_tiles<kATX, kATY>
            <<<blocks, adjt::NT, sizeof(adjt::Smem<kATX, kATY>), st>>>(p);
        return swadj_host::cuda_check(cudaGetLastError(), "adj_f32_tiles");
    }
    dim3 grid((p.nx + 127) / 128, 1);
    adj_step_kernel<float, false, 128, 1><<<grid, dim3(128, 1), 0, st>>>(p);
    return swadj_host::cuda_check(cudaGetLastError(), "adj_step_kernel<float>");
}

}  // namespace swadj
