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
};

// Waves at the edge between (eL, mL, cL) and (eR, mR, cR), m the normal
// component; c = 0 marks a dry cell, mirrored from its wet neighbour.
__device__ __forceinline__ EdgeA solve_a(float eL, float mL, float cL, float eR, float mR,
                                         float cR) {
    EdgeA w;
    const bool dL = !(cL > 0.f), dR = !(cR > 0.f);
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

// Net fluxes of edge w (neighbour edges wl, wr): L into the left cell, R into
// the right cell (Q -= nu * net); components (eta~, normal).  `wall`: a wet /
// dry edge, which carries no second-order correction.
__device__ __forceinline__ void net_a(const EdgeA &wl, const EdgeA &w, const EdgeA &wr,
                                      float nu, int order, bool wall, float L[2], float R[2]) {
    float F0 = 0.f, F1 = 0.f;
    if (order >= 2 && !wall) {
        // wave 1 (speed -cl) is upwinded from the right edge, wave 2 (+cr)
        // from the left edge
        const float r1 = wr.b1 * fmaf(wr.cl, w.cl, 1.f) * rcpf(fmaf(w.cl, w.cl, 1.f));
        const float r2 = wl.b2 * fmaf(wl.cr, w.cr, 1.f) * rcpf(fmaf(w.cr, w.cr, 1.f));
        const float k1 = -0.5f * fmaf(-nu, w.cl, 1.f) * mc1(w.b1, r1);
        const float k2 = 0.5f * fmaf(-nu, w.cr, 1.f) * mc1(w.b2, r2);
        F0 = k1 * w.cl - k2 * w.cr;
        F1 = k1 + k2;
    }
    L[0] = w.b1 * w.cl + F0;
    L[1] = w.b1 + F1;
    R[0] = -(w.b2 * w.cr) - F0;
    R[1] = w.b2 - F1;
}

template <int TX, int TY>
struct Smem {
    static constexpr int RX = TX + 4, RY = TY + 4, NEX = TX + 3, NEY = TY + 3;
    float e[RY][RX], m[RY][RX], g[RY][RX], c[RY][RX];
    union W {   // edge waves (b1, b2, cl, cr): y (phases 1-2), then x (4-5)
        float y[4][NEY][RX];
        float x[4][TY][NEX];
    } w;
    union N {   // net fluxes: y (phases 2-3), then x (5-6)
        struct Y { float l[2][TY + 1][RX], r[2][TY + 1][RX]; } y;
        struct X { float l[2][TY][TX + 1], r[2][TY][TX + 1]; } x;
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
        R.e[k] = __ldg(p.src[0] + o);
        R.c[k] = __ldg(p.c + o);
        const float mu = __ldg(p.src[1] + o), ga = __ldg(p.src[2] + o);
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
        S.e[ry][rx] = R.e[k];
        S.m[ry][rx] = R.m[k];
        S.g[ry][rx] = R.g[k];
        S.c[ry][rx] = R.c[k];
    }
    __syncthreads();
    // phase 1: y-edge waves of every staged column (edge k between rows k, k+1)
    for (int i = tid; i < NEY * RX; i += NT) {
        const int k = i / RX, rx = i - k * RX;
        const EdgeA w = solve_a(S.e[k][rx], S.g[k][rx], S.c[k][rx], S.e[k + 1][rx],
                                S.g[k + 1][rx], S.c[k + 1][rx]);
        S.w.y[0][k][rx] = w.b1; S.w.y[1][k][rx] = w.b2;
        S.w.y[2][k][rx] = w.cl; S.w.y[3][k][rx] = w.cr;
    }
    __syncthreads();
    // phase 2: y net fluxes of edges 1 .. TY+1 in every staged column
    for (int i = tid; i < (TY + 1) * RX; i += NT) {
        const int e = 1 + i / RX, rx = i - (e - 1) * RX;
        EdgeA a, b, c;
        a.b1 = S.w.y[0][e - 1][rx]; a.b2 = S.w.y[1][e - 1][rx];
        a.cl = S.w.y[2][e - 1][rx]; a.cr = S.w.y[3][e - 1][rx];
        b.b1 = S.w.y[0][e][rx]; b.b2 = S.w.y[1][e][rx];
        b.cl = S.w.y[2][e][rx]; b.cr = S.w.y[3][e][rx];
        c.b1 = S.w.y[0][e + 1][rx]; c.b2 = S.w.y[1][e + 1][rx];
        c.cl = S.w.y[2][e + 1][rx]; c.cr = S.w.y[3][e + 1][rx];
        const bool wall = !(S.c[e][rx] > 0.f) || !(S.c[e + 1][rx] > 0.f);
        float L[2], Rr[2];
        net_a(a, b, c, nuy, order, wall, L, Rr);
        S.n.y.l[0][e - 1][rx] = L[0]; S.n.y.l[1][e - 1][rx] = L[1];
        S.n.y.r[0][e - 1][rx] = Rr[0]; S.n.y.r[1][e - 1][rx] = Rr[1];
    }
    __syncthreads();
    // phase 3: y-sweep of the tile rows in every staged column, in place;
    // lower edge of row -> R at index row, upper edge -> L at row + 1
    for (int i = tid; i < TY * RX; i += NT) {
        const int row = i / RX, rx = i - row * RX, ry = row + 2;
        if (S.c[ry][rx] > 0.f) {
            S.e[ry][rx] += -nuy * (S.n.y.r[0][row][rx] + S.n.y.l[0][row + 1][rx]);
            S.g[ry][rx] += -nuy * (S.n.y.r[1][row][rx] + S.n.y.l[1][row + 1][rx]);
        }
    }
    __syncthreads();
    // phase 4: x-edge waves of the y-swept tile rows (edge k between cols k, k+1)
    for (int i = tid; i < TY * NEX; i += NT) {
        const int row = i / NEX, k = i - row * NEX, ry = row + 2;
        const EdgeA w = solve_a(S.e[ry][k], S.m[ry][k], S.c[ry][k], S.e[ry][k + 1],
                                S.m[ry][k + 1], S.c[ry][k + 1]);
        S.w.x[0][row][k] = w.b1; S.w.x[1][row][k] = w.b2;
        S.w.x[2][row][k] = w.cl; S.w.x[3][row][k] = w.cr;
    }
    __syncthreads();
    // phase 5: x net fluxes of edges 1 .. TX+1 of the tile rows
    for (int i = tid; i < TY * (TX + 1); i += NT) {
        const int row = i / (TX + 1), e = 1 + (i - row * (TX + 1)), ry = row + 2;
        EdgeA a, b, c;
        a.b1 = S.w.x[0][row][e - 1]; a.b2 = S.w.x[1][row][e - 1];
        a.cl = S.w.x[2][row][e - 1]; a.cr = S.w.x[3][row][e - 1];
        b.b1 = S.w.x[0][row][e]; b.b2 = S.w.x[1][row][e];
        b.cl = S.w.x[2][row][e]; b.cr = S.w.x[3][row][e];
        c.b1 = S.w.x[0][row][e + 1]; c.b2 = S.w.x[1][row][e + 1];
        c.cl = S.w.x[2][row][e + 1]; c.cr = S.w.x[3][row][e + 1];
        const bool wall = !(S.c[ry][e] > 0.f) || !(S.c[ry][e + 1] > 0.f);
        float L[2], Rr[2];
        net_a(a, b, c, nux, order, wall, L, Rr);
        S.n.x.l[0][row][e - 1] = L[0]; S.n.x.l[1][row][e - 1] = L[1];
        S.n.x.r[0][row][e - 1] = Rr[0]; S.n.x.r[1][row][e - 1] = Rr[1];
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
            float ne = S.e[ry][rx], nm = S.m[ry][rx];
            const float ng = S.g[ry][rx];
            if (S.c[ry][rx] > 0.f) {
                ne += -nux * (S.n.x.r[0][row][col] + S.n.x.l[0][row][col + 1]);
                nm += -nux * (S.n.x.r[1][row][col] + S.n.x.l[1][row][col + 1]);
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
