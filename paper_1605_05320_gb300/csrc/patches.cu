// patches.cu -- batched uneven patches: one launch per level step.
//
// Every patch of a level is cut into warp strips (28 output columns x `rows`
// rows, strips.cuh); the level's strip list (patch, x0, y0) is built on the
// host at creation and kept on the device.  A level step is one launch of
// resident warps that walk that list, so small and large patches share the
// launch and the tail of small patches does not leave SMs idle.  The
// level's clock (time, step, buffer parity, next dt from the fused CFL
// reduction) lives on the device, as for a single grid.
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "strips.cuh"

namespace swadj {
namespace patches {

constexpr int kMaxBlocks = 4096;  // reduction slots per level

struct PatchDevice {
    float *q[2][3];
    const float *hb;
    int nx, ny;
    float dx, dy, rdx, rdy;
    BcSpec bc;
};

// ------------------------------------------------------------ ring fills
// The AMR glue's ring fill of one cell (see the AMR section below for the
// maps): a sibling copy, or the parent linear in time between its buffers
// before and after its step (alpha in [0, 1]) then limited linear in space
// within the parent cell (minmod slopes from the parent's array, zero where
// a neighbour lies outside it).  Entry m = (patch, cell, src, idx): src >= 0
// a sibling patch and idx its cell; src < 0 the parent cell idx (in patch
// par, or the coarse grid for par < 0) with the ring cell at -src - 1 = sx +
// r sy inside it.  Used by the fill kernel and by level launches that fill
// their own rings.
struct RingFill {
    const int4 *fill;           // the level's entries, patch by patch, ring cells row-major
    const int *par;             // parent patch per entry (-1: the coarse grid)
    const int *base;            // per patch-set patch: its first entry (-1: not on the level)
    const PatchDevice *coarse;  // the coarse grid's buffers, as a patch without ring
    const DevClock *pclk;       // the parent's clock (its current buffer)
    int r;
    double t_p, dt_p;           // the parent's step
};

// index of ring cell (i, j) among its patch's ring cells in row-major order
__host__ __device__ __forceinline__ int ring_index(int i, int j, int nx, int ny) {
    if (j < 2) return j * nx + i;
    if (j >= ny - 2) return 2 * nx + (ny - 4) * 4 + (j - (ny - 2)) * nx + i;
    return 2 * nx + (j - 2) * 4 + (i < 2 ? i : i - (nx - 4));
}

__host__ __device__ __forceinline__ bool ring_cell(int i, int j, int nx, int ny) {
    return i < 2 || i >= nx - 2 || j < 2 || j >= ny - 2;
}

__device__ __forceinline__ float minmod(float a, float b) {
    if (a * b <= 0.f) return 0.f;
    return fabsf(a) < fabsf(b) ? a : b;
}

// component k of ring entry m at alpha af; fcur, pcur: the level's and the
// parent's current buffers
__device__ __forceinline__ float ring_value(const PatchDevice *table, const PatchDevice *coarse,
                                            int4 m, int par, int k, int r, float af, int fcur,
                                            int pcur) {
    if (m.z >= 0) return table[m.z].q[fcur][k][m.w];
    const int sub = -m.z - 1, sx = sub % r, sy = sub / r;
    const PatchDevice &Q = par < 0 ? *coarse : table[par];
    const int nx = Q.nx, ny = Q.ny;
    const int c = m.w, ic = c % nx, jc = c / nx;
    const float xi = (float)(2 * sx + 1 - r) / (float)(2 * r);
    const float zeta = (float)(2 * sy + 1 - r) / (float)(2 * r);
    const float *o = Q.q[pcur ^ 1][k], *nw = Q.q[pcur][k];
    auto at = [&](int i) { return fmaf(af, nw[i] - o[i], o[i]); };
    const float qc = at(c);
    float s_x = 0.f, s_y = 0.f;
    if (ic > 0 && ic < nx - 1) s_x = minmod(qc - at(c - 1), at(c + 1) - qc);
    if (jc > 0 && jc < ny - 1) s_y = minmod(qc - at(c - nx), at(c + nx) - qc);
    return fmaf(s_y, zeta, fmaf(s_x, xi, qc));
}

// What a reader of a patch's current buffer needs to form its ring cells
// itself, before the level launch's own fill of them is known to be done.
struct RingCtx {
    const PatchDevice *table;
    const RingFill *rf;
    int pid, fcur, pcur;
    float af;
};

// ------------------------------------------------------------ refluxing
// Mass flux through an edge of cell (i, j), low (side < 0) or high (side >
// 0), along `axis`, as the FP32 split step forms it: x-edges from the state
// (x-sweep), y-edges from the x-swept state (y-sweep).  The edge's flux is
// F = mn_L + L0, the normal momentum of the cell below it plus the net the
// update gives that cell (in exact arithmetic also mn_R - R0, the cell
// above it), so a cell's update is dh = -nu (F_high - F_low) per sweep and
// both sides of an edge see the same number.  The edge arithmetic is the
// strip kernel's (fwd_pair.cuh), each net in the form its own edge picks
// (the warp-uniform choice of the kernel gives the same numbers).
namespace reflux {

struct CellRaw {
    float eta, mu, mv, hb;
};

// cell (i, j) of view v, ghost-mapped; with a ring context its ring cells
// are formed from the fill map instead of read
__device__ __forceinline__ CellRaw raw_at(const strip::View &v, int i, int j,
                                          const RingCtx *rc = nullptr) {
    bool fx, fy;
    const int ii = ghost_index(i, v.nx, v.bc.lo_x, v.bc.hi_x, &fx);
    const int jj = ghost_index(j, v.ny, v.bc.lo_y, v.bc.hi_y, &fy);
    const size_t o = (size_t)jj * v.nx + ii;
    CellRaw c;
    c.hb = v.hb[o];
    float mu, mv;
    if (rc && ring_cell(ii, jj, v.nx, v.ny)) {
        const RingFill &F = *rc->rf;
        const int e = F.base[rc->pid] + ring_index(ii, jj, v.nx, v.ny);
        const int4 m = F.fill[e];
        const int par = F.par[e];
        c.eta = ring_value(rc->table, F.coarse, m, par, 0, F.r, rc->af, rc->fcur, rc->pcur);
        mu = ring_value(rc->table, F.coarse, m, par, 1, F.r, rc->af, rc->fcur, rc->pcur);
        mv = ring_value(rc->table, F.coarse, m, par, 2, F.r, rc->af, rc->fcur, rc->pcur);
    } else {
        c.eta = v.q0[o];
        mu = v.q1[o];
        mv = v.q2[o];
    }
    c.mu = fx ? -mu : mu;
    c.mv = fy ? -mv : mv;
    return c;
}

// x-frame cell data of cell (i, j)
__device__ __forceinline__ fp::Cell<float> xcell(const strip::View &v, int i, int j,
                                                 const RingCtx *rc = nullptr) {
    const CellRaw c = raw_at(v, i, j, rc);
    return fp::derive(c.eta, fp::add(c.eta, c.hb), c.mu, c.mv);
}

// the x-swept cell (i, j) in the y frame, as the strip kernel's x-sweep
// leaves it
__device__ __forceinline__ fp::Cell<float> xswept(const strip::View &v, int i, int j, float gh,
                                                  float nux, int order,
                                                  const RingCtx *rc = nullptr) {
    fp::Cell<float> c[5];
#pragma unroll
    for (int k = 0; k < 5; k++) c[k] = xcell(v, i - 2 + k, j, rc);
    fp::Edge<float> w[4];
#pragma unroll
    for (int k = 0; k < 4; k++) w[k] = fp::solve(gh, c[k], c[k + 1]);
    const fp::Net<float> nl = fp::net3(w[0], w[1], w[2], nux, order, fp::subsonic(w[1].s1, w[1].s3));
    const fp::Net<float> nr = fp::net3(w[1], w[2], w[3], nux, order, fp::subsonic(w[2].s1, w[2].s3));
    const float d0 = fp::mul(-nux, fp::add(nl.R0, nr.L0));
    const float d1 = fp::mul(-nux, fp::add(nl.R1, nr.L1));
    const float d2 = fp::mul(-nux, fp::add(nl.R2, nr.L2));
    const fp::Cell<float> &a = c[2];
    return fp::derive(fp::add(a.eta, d0), fp::add(a.h, d0), fp::add(a.mt, d2), fp::add(a.mn, d1));
}

// Flux of the edge between stencil cells 1 and 2 of the 4 cells at offsets
// k0 .. k0 + 3 from (i, j) along `axis`, formed by a group of 4 lanes: lane
// q = lane & 3 forms stencil cell q (x-sweeping its row first for a y-edge),
// its edge to cell q + 1 and the neighbour edges come by shuffles, and the
// result is valid on the lane with q == 1.  All 32 lanes must call it.
__device__ __forceinline__ float group_flux(const strip::View &v, int i, int j, int axis, int k0,
                                            float gh, float nux, float nuy, int order,
                                            const RingCtx *rc = nullptr) {
    using strip::dn;
    using strip::up;
    const int q = threadIdx.x & 3;
    const fp::Cell<float> c =
        axis == 0 ? xcell(v, i + k0 + q, j, rc) : xswept(v, i, j + k0 + q, gh, nux, order, rc);
    fp::Cell<float> n = c;
    n.h = dn(c.h); n.mn = dn(c.mn); n.sq = dn(c.sq); n.su = dn(c.su); n.sv = dn(c.sv);
    n.P = dn(c.P); n.T = dn(c.T); n.eta = dn(c.eta);
    const fp::Edge<float> w = fp::solve(gh, c, n);   // edge (q | q + 1)
    fp::Edge<float> wl = w, wr = w;
    wl.s1 = up(w.s1); wl.s3 = up(w.s3); wl.vh = up(w.vh);
    wl.b1 = up(w.b1); wl.b2 = up(w.b2); wl.b3 = up(w.b3);
    wr.s1 = dn(w.s1); wr.s3 = dn(w.s3); wr.vh = dn(w.vh);
    wr.b1 = dn(w.b1); wr.b2 = dn(w.b2); wr.b3 = dn(w.b3);
    const fp::Net<float> N =
        fp::net3(wl, w, wr, axis == 0 ? nux : nuy, order, fp::subsonic(w.s1, w.s3));
    return fp::add(c.mn, N.L0);
}

// the step the coming launch takes on this clock (as begin_step forms it)
__device__ __forceinline__ double coming_dt(const DevClock *clk, double t_end) {
    volatile const DevClock *c = clk;
    double dt = c->dt_cfl;
    if (t_end - c->t < dt) dt = t_end - c->t;
    return dt > 0.0 ? dt : 0.0;
}

}  // namespace reflux

// Refluxing work of a level launch inside the AMR glue.  An edge e of
// level l joins a copy of an uncovered level-(l - 1) cell U to a cell V
// under a level-l patch interior: cf[e] = (U's patch or -1 for the coarse
// grid, U's cell, V's owner patch, its first cell along the edge), cfw[e] =
// axis | hi << 1 | stride << 2 (hi: V on U's high side; stride: from one of
// the r cells along the edge to the next), and 1 + r FP64 slots: the coarse
// part (level l - 1's own fluxes) then one fine part per cell along it.
//   fine parts (this level as the child, its own edges): slot[e (1 + r) + 1
//     + k] -= (dt / d) (1 / r) F_k, d the parent's cell width;
//   coarse parts (this level as the parent, the next level's edges):
//     slot2[e (1 + r2)] += (dt / d) F_U, d this level's cell width;
// with F signed into V.  nfine = ncoarse = 0: none.
struct LevelReflux {
    const int4 *cf;
    const int *cfw;
    double *slot;
    int nfine, r;           // items: edges x r
    double dpx, dpy;        // parent cell size
    const int4 *cf2;
    const int *cfw2;
    double *slot2;
    int ncoarse, r2;        // items: the next level's edges
    double dtx, dty;        // this level's cell size
};

struct LevelParams {
    const PatchDevice *table;
    int4 *units;         // (patch, x0, y0, hint): hint 1 = the strip has had waves
    int nunits, rows;
    DevClock *clk;
    double *partial;
    int nblocks;
    double t_end, cfl, dx, dy;
    float g;
    int order;
    int *err;
    LevelReflux rf;
    RingFill lf;       // the level fills its own rings (AMR glue) when fill_on
    int fill_on;
};

// Fill the ring cells of patch pid inside the stencil window of the strip at
// (x0, y0) (columns x0 - 2 .. x0 + 29, rows y0 - 2 .. the strip's last row +
// 2, clipped to the array) in the current buffer, the warp's lanes taking
// the window's cells in turn.  Strips of a patch share ring cells; each
// writes the same value, so the writes of two strips agree, and a strip
// reads only cells it has written itself.
__device__ __noinline__ void fill_window(const LevelParams &p, int pid, int x0, int y0, int cur,
                                         float af, int pcur) {
    const PatchDevice &P = p.table[pid];
    const int nx = P.nx, ny = P.ny;
    const int ylast = (y0 + p.rows < ny ? y0 + p.rows : ny) - 1;
    const int cx0 = x0 - 2 > 0 ? x0 - 2 : 0, cx1 = x0 + 29 < nx - 1 ? x0 + 29 : nx - 1;
    const int ry0 = y0 - 2 > 0 ? y0 - 2 : 0, ry1 = ylast + 2 < ny - 1 ? ylast + 2 : ny - 1;
    if (cx0 >= 2 && cx1 < nx - 2 && ry0 >= 2 && ry1 < ny - 2) return;   // no ring cell
    const int W = cx1 - cx0 + 1, H = ry1 - ry0 + 1;
    const int b = p.lf.base[pid];
    for (int q = threadIdx.x & 31; q < W * H; q += 32) {
        const int j = ry0 + q / W, i = cx0 + q % W;
        if (!ring_cell(i, j, nx, ny)) continue;
        const int e = b + ring_index(i, j, nx, ny);
        const int4 m = __ldg(p.lf.fill + e);
        const int par = __ldg(p.lf.par + e);
        const size_t o = (size_t)j * nx + i;
#pragma unroll
        for (int k = 0; k < 3; k++)
            P.q[cur][k][o] = ring_value(p.table, p.lf.coarse, m, par, k, p.lf.r, af, cur, pcur);
    }
}

// One task of a level launch's refluxing work: 8 items, 4 lanes each;
// tasks below ceil(nfine / 8) are fine parts, the rest coarse parts.
__device__ __noinline__ void level_reflux_task(const LevelParams &p, int task, int cur,
                                               float nux, float nuy, double dt, float af,
                                               int pcur) {
    const LevelReflux &R = p.rf;
    const int lane = threadIdx.x & 31;
    const int tf = (R.nfine + 7) / 8;
    const bool fine = task < tf;
    const int n = fine ? R.nfine : R.ncoarse;
    int item = (fine ? task : task - tf) * 8 + (lane >> 2);
    const bool live = item < n;
    if (!live) item = n - 1;   // idle lanes redo the last item for the shuffles
    const int e = fine ? item / R.r : item;
    const int4 m = fine ? R.cf[e] : R.cf2[e];
    const int w = fine ? R.cfw[e] : R.cfw2[e];
    const int axis = w & 1, side = (w & 2) ? 1 : -1, stride = w >> 2;
    // fine: a cell of V's patch along the edge, its low edge when V is on
    // U's high side (stencil from two cells below it), else its high edge;
    // coarse: U in its patch, its high edge when V is on its high side
    const int pid = fine ? m.z : m.x;
    const int c = fine ? m.w + (item - e * R.r) * stride : m.y;
    const int k0 = fine ? (side > 0 ? -2 : -1) : (side > 0 ? -1 : -2);
    const PatchDevice &P = p.table[pid];
    strip::View v;
    v.q0 = P.q[cur][0]; v.q1 = P.q[cur][1]; v.q2 = P.q[cur][2]; v.hb = P.hb;
    v.nx = P.nx; v.ny = P.ny; v.bc = P.bc;
    // with the level filling its own rings, ring cells are formed here (the
    // strip that writes them may not have run yet)
    RingCtx rc{p.table, &p.lf, pid, cur, pcur, af};
    const float f = reflux::group_flux(v, c % P.nx, c / P.nx, axis, k0, 0.5f * p.g, nux, nuy,
                                       p.order, p.fill_on ? &rc : nullptr);
    if (!live || (lane & 3) != 1) return;
    const double fs = (double)(side > 0 ? f : -f);
    if (fine)
        R.slot[(size_t)e * (1 + R.r) + 1 + (item - e * R.r)] -=
            dt / (axis == 0 ? R.dpx : R.dpy) / (double)R.r * fs;
    else
        R.slot2[(size_t)e * (1 + R.r2)] += dt / (axis == 0 ? R.dtx : R.dty) * fs;
}

// ORD: the order of the scheme (1 or 2), fixed at compile time.
template <int ORD>
__global__ void __launch_bounds__(strip::kThreads, 4) level_strip_kernel(LevelParams p) {
    __shared__ float s_nu[2];
    __shared__ int s_cur, s_run;
    __shared__ float red[strip::kThreads / 32];
    __shared__ int am_last;
    __shared__ strip::Ring ring[strip::kThreads / 32];
    __shared__ float s_af;
    __shared__ int s_pcur;
    double t_now = 0.0, dt = 0.0;
    if (!fwave::begin_step(p.clk, p.t_end, p.dx, p.dy, s_nu, &s_cur, &s_run, t_now, dt)) return;
    if (p.fill_on) {   // block-uniform
        if (threadIdx.x == 0) {
            double a = (t_now - p.lf.t_p) / p.lf.dt_p;
            a = a < 0.0 ? 0.0 : (a > 1.0 ? 1.0 : a);
            s_af = (float)a;
            s_pcur = ((volatile const DevClock *)p.lf.pclk)->cur;
        }
        __syncthreads();
    }
    const int cur = s_cur;
    const int wpb = blockDim.x >> 5;
    float smax = 0.f;
    bool bad = false;
    // warp-uniform walk of the level's strip list
    for (int u = blockIdx.x * wpb + (threadIdx.x >> 5); u < p.nunits; u += gridDim.x * wpb) {
        const int4 t = p.units[u];
        const PatchDevice &P = p.table[t.x];
        strip::View v;
        v.q0 = P.q[cur][0]; v.q1 = P.q[cur][1]; v.q2 = P.q[cur][2]; v.hb = P.hb;
        v.o0 = P.q[cur ^ 1][0]; v.o1 = P.q[cur ^ 1][1]; v.o2 = P.q[cur ^ 1][2];
        v.nx = P.nx; v.ny = P.ny; v.rdx = P.rdx; v.rdy = P.rdy; v.bc = P.bc;
        if (p.fill_on) {
            fill_window(p, t.x, t.y, t.z, cur, s_af, s_pcur);
            __threadfence_block();
            __syncwarp();   // the window's writes before the strip's loads
        }
        // A strip that has had waves keeps them: it skips the quiet scan (the
        // hint only; the scan alone decides that a strip is quiet).
        if (t.w == 0) {
            if (strip::quiet_unit<false>(v, nullptr, 0, t.y, t.z, p.rows, p.g, smax)) continue;
            if ((threadIdx.x & 31) == 0) p.units[u].w = 1;
        }
        strip::strip_unit(v, t.y, t.z, p.rows, s_nu[0], s_nu[1], p.g, ORD,
                          ring[threadIdx.x >> 5], smax, bad);
    }
    if (p.rf.nfine + p.rf.ncoarse > 0) {
        // the warps with one strip fewer start on the refluxing tasks; the
        // clock is not advanced before every block has finished them
        const int total = gridDim.x * wpb, gw = blockIdx.x * wpb + (threadIdx.x >> 5);
        const int ntasks = (p.rf.nfine + 7) / 8 + (p.rf.ncoarse + 7) / 8;
        const int rem = p.nunits % total;
        const double dt_now = reflux::coming_dt(p.clk, p.t_end);
        for (int t = (gw + total - rem) % total; t < ntasks; t += total)
            level_reflux_task(p, t, cur, s_nu[0], s_nu[1], dt_now, p.fill_on ? s_af : 0.f,
                              p.fill_on ? s_pcur : 0);
    }
    if (bad) atomicOr(p.err, ERR_UNSTABLE);
    fwave::finish_step<strip::kThreads>(p.clk, p.partial, p.nblocks, p.cfl, smax, red,
                                        &am_last, t_now, dt, s_cur);
}

__device__ __forceinline__ void atomic_max_nonneg(double *a, double v) {
    atomicMax((unsigned long long *)a, (unsigned long long)__double_as_longlong(v));
}

// CFL maximum of buffer 0 of every patch of the level (same per-cell rule as
// the step's fused reduction), into *smax.
__global__ void level_smax_kernel(LevelParams p, double *smax) {
    float m = 0.f;
    for (int k = blockIdx.x; k < p.nunits; k += gridDim.x) {
        const int4 t = p.units[k];
        const PatchDevice &P = p.table[t.x];
        for (int c = threadIdx.x; c < strip::kOut * p.rows; c += blockDim.x) {
            const int i = t.y + c % strip::kOut, j = t.z + c / strip::kOut;
            if (i >= P.nx || j >= P.ny) continue;
            const size_t o = (size_t)j * P.nx + i;
            const float h = P.q[0][0][o] + P.hb[o];
            const float s = cfl_f32(h, P.q[0][1][o], P.q[0][2][o], p.g, P.rdx, P.rdy, 1);
            if (!(h > 0.f)) atomicOr(p.err, ERR_UNSTABLE);
            m = fmaxf(m, s);
        }
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(smax, (double)m);
}

__global__ void level_clock_kernel(DevClock *clk, const double *smax, double t0, double cfl) {
    clk->t = t0;
    clk->smax = *smax;
    clk->dt_cfl = cfl / *smax;
    clk->cur = 0;
    clk->nsteps = 0;
    clk->ticket = 0u;
    clk->work = 0u;
}

__global__ void to_float_kernel(const double *src, float *dst, const double *sub, int negate,
                                size_t n) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x) {
        double v = src[k];
        if (sub) v = v - sub[k];
        if (negate) v = -v;
        dst[k] = (float)v;
    }
}

__global__ void to_double_kernel(const float *src, const float *add, double *dst, size_t n) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x) {
        double v = (double)src[k];
        if (add) v = v + (double)add[k];
        dst[k] = v;
    }
}

unsigned ew_blocks(size_t n) {
    size_t b = (n + 255) / 256;
    return (unsigned)(b > 4096 ? 4096 : (b < 1 ? 1 : b));
}

struct Level {
    int npatches = 0, nunits16 = 0, nunits32 = 0;
    long long ncells = 0;
    double dx = 0, dy = 0;
    int4 *units16 = nullptr, *units32 = nullptr;
    DevClock *clk = nullptr;
    double *partial = nullptr;
    double *smax = nullptr;
    int rows = 0;   // requested strip height (16 or 32), 0 = default 32
    bool started = false;
};

int occupancy_blocks() {
    static int per_sm = 0, sms = 0;
    if (per_sm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, level_strip_kernel<2>,
                                                      strip::kThreads, 0);
        if (per_sm < 1) per_sm = 1;
        if (sms < 1) sms = 1;
    }
    const int b = per_sm * sms;
    return b < kMaxBlocks ? b : kMaxBlocks;
}

}  // namespace patches
}  // namespace swadj

using namespace swadj;
using namespace swadj::patches;
using swadj_host::cuda_check;
using swadj_host::set_error;

struct swa_patchset {
    int n = 0;
    swa_grid_desc common;
    std::vector<swa_patch_desc> pd;
    std::vector<PatchDevice> host_table;
    PatchDevice *table = nullptr;
    double *staging = nullptr;
    size_t staging_n = 0;
    Level lev[SWA_MAX_LEVELS + 1];
};

#define TRY(x)                          \
    do {                                \
        int _rc = (x);                  \
        if (_rc != SWA_OK) return _rc;  \
    } while (0)

namespace {

struct Carve {
    char *base;
    size_t off = 0;
    explicit Carve(void *b) : base((char *)b) {}
    void *take(size_t bytes) {
        off = (off + 255) & ~(size_t)255;
        void *p = base ? base + off : nullptr;
        off += bytes;
        return p;
    }
};

int check_patches(int n, const swa_patch_desc *p, const swa_grid_desc *c) {
    if (n < 1 || !p || !c) return set_error(SWA_EINVAL, "need n >= 1 patches and a common descriptor");
    double ldx[SWA_MAX_LEVELS + 1] = {0}, ldy[SWA_MAX_LEVELS + 1] = {0};
    for (int k = 0; k < n; k++) {
        if (p[k].level < 1 || p[k].level > SWA_MAX_LEVELS)
            return set_error(SWA_EINVAL, "patch %d: level must be in [1, %d]", k, SWA_MAX_LEVELS);
        if (p[k].nx < 2 || p[k].ny < 2) return set_error(SWA_EINVAL, "patch %d: nx, ny must be >= 2", k);
        if (!(p[k].dx > 0) || !(p[k].dy > 0)) return set_error(SWA_EINVAL, "patch %d: dx, dy must be > 0", k);
        const int l = p[k].level;
        if (ldx[l] == 0) { ldx[l] = p[k].dx; ldy[l] = p[k].dy; }
        else if (ldx[l] != p[k].dx || ldy[l] != p[k].dy)
            return set_error(SWA_EINVAL, "patch %d: cell size differs from level %d's", k, l);
    }
    if (c->order != 1 && c->order != 2) return set_error(SWA_EINVAL, "order must be 1 or 2");
    for (int k = 0; k < 4; k++)
        if (c->bc[k] != SWA_BC_EXTRAP && c->bc[k] != SWA_BC_WALL)
            return set_error(SWA_EINVAL, "bad boundary condition");
    if (!(c->g > 0) || !(c->cfl > 0) || !(c->cfl <= 1.0)) return set_error(SWA_EINVAL, "need g > 0, 0 < cfl <= 1");
    return SWA_OK;
}

void strips_of(const swa_patch_desc &p, int k, int rows, std::vector<int4> &out) {
    for (int j0 = 0; j0 < p.ny; j0 += rows)
        for (int i0 = 0; i0 < p.nx; i0 += strip::kOut) out.push_back(make_int4(k, i0, j0, 0));
}

void layout(int n, const swa_patch_desc *p, Carve &c, swa_patchset *ps) {
    size_t maxn = 0;
    std::vector<int4> t16[SWA_MAX_LEVELS + 1], t32[SWA_MAX_LEVELS + 1];
    for (int k = 0; k < n; k++) {
        const size_t nn = (size_t)p[k].nx * p[k].ny;
        if (nn > maxn) maxn = nn;
        strips_of(p[k], k, 16, t16[p[k].level]);
        strips_of(p[k], k, 32, t32[p[k].level]);
    }
    PatchDevice *table = (PatchDevice *)c.take(sizeof(PatchDevice) * n);
    double *staging = (double *)c.take(maxn * 8);
    if (ps) {
        ps->table = table;
        ps->staging = staging;
        ps->staging_n = maxn;
        ps->host_table.resize(n);
    }
    for (int k = 0; k < n; k++) {
        const size_t nn = (size_t)p[k].nx * p[k].ny;
        PatchDevice d{};
        for (int b = 0; b < 2; b++)
            for (int m = 0; m < 3; m++) d.q[b][m] = (float *)c.take(nn * 4);
        d.hb = (const float *)c.take(nn * 4);
        if (ps) {
            d.nx = p[k].nx; d.ny = p[k].ny;
            d.dx = (float)p[k].dx; d.dy = (float)p[k].dy;
            d.rdx = 1.f / d.dx; d.rdy = 1.f / d.dy;
            d.bc = BcSpec{ps->common.bc[0], ps->common.bc[1], ps->common.bc[2], ps->common.bc[3]};
            ps->host_table[k] = d;
        }
    }
    for (int l = 1; l <= SWA_MAX_LEVELS; l++) {
        int4 *a = (int4 *)c.take(sizeof(int4) * (t16[l].size() + 1));
        int4 *b = (int4 *)c.take(sizeof(int4) * (t32[l].size() + 1));
        DevClock *clk = (DevClock *)c.take(sizeof(DevClock));
        double *part = (double *)c.take(8 * kMaxBlocks);
        double *smax = (double *)c.take(8);
        if (ps) {
            Level &L = ps->lev[l];
            L.units16 = a; L.units32 = b; L.clk = clk; L.partial = part; L.smax = smax;
            L.nunits16 = (int)t16[l].size();
            L.nunits32 = (int)t32[l].size();
        }
    }
}

}  // namespace

static LevelParams level_params(const swa_patchset *ps, int l, double t_end) {
    const Level &L = ps->lev[l];
    LevelParams p{};
    p.table = ps->table;
    // default: 16-row strips when a level has few enough of them for every
    // resident warp to take at most one (a latency-bound level, where
    // shorter strips shorten the critical path), 32 otherwise
    const int auto_rows = L.nunits16 <= occupancy_blocks() * (strip::kThreads / 32) ? 16 : 32;
    p.rows = L.rows == 16 ? 16 : (L.rows == 32 ? 32 : auto_rows);
    p.units = p.rows == 16 ? L.units16 : L.units32;
    p.nunits = p.rows == 16 ? L.nunits16 : L.nunits32;
    p.clk = L.clk;
    p.partial = L.partial;
    p.t_end = t_end;
    p.cfl = ps->common.cfl;
    p.dx = L.dx;
    p.dy = L.dy;
    p.g = (float)ps->common.g;
    p.order = ps->common.order;
    p.err = swadj_host::error_word();
    return p;
}

// nsteps launches of the level step, with the refluxing work rf in each.
static int level_launch(swa_patchset *ps, int level, int nsteps, double t_end,
                        const LevelReflux &rf, cudaStream_t st, const RingFill *lf = nullptr) {
    if (!ps || level < 1 || level > SWA_MAX_LEVELS) return set_error(SWA_EINVAL, "bad level");
    Level &L = ps->lev[level];
    if (L.npatches == 0) return set_error(SWA_EINVAL, "level %d has no patches", level);
    if (!L.started) return set_error(SWA_ESTATE, "level %d not started", level);
    if (nsteps < 0) return set_error(SWA_EINVAL, "nsteps < 0");
    LevelParams p = level_params(ps, level, t_end);
    p.rf = rf;
    if (lf) {
        p.lf = *lf;
        p.fill_on = 1;
    }
    constexpr int wpb = strip::kThreads / 32;
    const int need = (p.nunits + wpb - 1) / wpb;
    p.nblocks = occupancy_blocks();
    if (p.nblocks > need) p.nblocks = need;
    for (int s = 0; s < nsteps; s++)
        if (p.order == 2)
            level_strip_kernel<2><<<p.nblocks, strip::kThreads, 0, st>>>(p);
        else
            level_strip_kernel<1><<<p.nblocks, strip::kThreads, 0, st>>>(p);
    return cuda_check(cudaGetLastError(), "level_strip_kernel");
}

extern "C" {

size_t swa_patches_workspace_bytes(int n, const swa_patch_desc *patches,
                                   const swa_grid_desc *common) {
    if (check_patches(n, patches, common) != SWA_OK) return 0;
    Carve c(nullptr);
    layout(n, patches, c, nullptr);
    return c.off + 256;
}

int swa_create_patches(int n, const swa_patch_desc *patches, const double *const *bathy_host,
                       const swa_grid_desc *common, void *ws, size_t ws_bytes, void *stream,
                       swa_patchset **out) {
    TRY(check_patches(n, patches, common));
    if (!bathy_host || !ws || !out) return set_error(SWA_EINVAL, "null argument");
    if (((uintptr_t)ws & 255) != 0) return set_error(SWA_EINVAL, "workspace must be 256-byte aligned");
    const size_t need = swa_patches_workspace_bytes(n, patches, common);
    if (ws_bytes < need)
        return set_error(SWA_ENOMEM, "patch workspace %zu bytes < %zu needed", ws_bytes, need);
    swa_patchset *ps = new (std::nothrow) swa_patchset();
    if (!ps) return set_error(SWA_ENOMEM, "host allocation failed");
    ps->n = n;
    ps->common = *common;
    ps->pd.assign(patches, patches + n);
    Carve c(ws);
    layout(n, patches, c, ps);
    cudaStream_t st = (cudaStream_t)stream;
    int rc = cuda_check(cudaMemsetAsync(ws, 0, need - 256, st), "workspace clear");
    // per-level bookkeeping and strip lists
    std::vector<int4> t16[SWA_MAX_LEVELS + 1], t32[SWA_MAX_LEVELS + 1];
    for (int k = 0; k < n; k++) {
        Level &L = ps->lev[patches[k].level];
        L.npatches++;
        L.ncells += (long long)patches[k].nx * patches[k].ny;
        L.dx = patches[k].dx;
        L.dy = patches[k].dy;
        strips_of(patches[k], k, 16, t16[patches[k].level]);
        strips_of(patches[k], k, 32, t32[patches[k].level]);
    }
    for (int l = 1; l <= SWA_MAX_LEVELS && rc == SWA_OK; l++) {
        Level &L = ps->lev[l];
        if (L.npatches == 0) continue;
        rc = cuda_check(cudaMemcpyAsync(L.units16, t16[l].data(), sizeof(int4) * t16[l].size(),
                                        cudaMemcpyHostToDevice, st), "strip list upload");
        if (rc == SWA_OK)
            rc = cuda_check(cudaMemcpyAsync(L.units32, t32[l].data(), sizeof(int4) * t32[l].size(),
                                            cudaMemcpyHostToDevice, st), "strip list upload");
    }
    if (rc == SWA_OK)
        rc = cuda_check(cudaMemcpyAsync(ps->table, ps->host_table.data(),
                                        sizeof(PatchDevice) * n, cudaMemcpyHostToDevice, st),
                        "patch table upload");
    // bathymetry -> hbar, state -> ocean at rest (eta = 0, zero momenta from the clear)
    for (int k = 0; k < n && rc == SWA_OK; k++) {
        const size_t nn = (size_t)patches[k].nx * patches[k].ny;
        if (!bathy_host[k]) { rc = set_error(SWA_EINVAL, "null bathymetry for patch %d", k); break; }
        rc = cuda_check(cudaMemcpyAsync(ps->staging, bathy_host[k], nn * 8,
                                        cudaMemcpyHostToDevice, st), "bathymetry upload");
        if (rc != SWA_OK) break;
        to_float_kernel<<<ew_blocks(nn), 256, 0, st>>>(ps->staging, (float *)ps->host_table[k].hb,
                                                        nullptr, 1, nn);
        rc = cuda_check(cudaGetLastError(), "bathymetry convert");
    }
    if (rc == SWA_OK) rc = cuda_check(cudaStreamSynchronize(st), "create_patches");
    if (rc != SWA_OK) { delete ps; return rc; }
    *out = ps;
    return SWA_OK;
}

int swa_destroy_patches(swa_patchset *ps) {
    delete ps;
    return SWA_OK;
}

int swa_patches_set_state(swa_patchset *ps, int k, const double *eta, const double *hu,
                          const double *hv, int where, void *stream) {
    if (!ps || k < 0 || k >= ps->n || !eta || !hu || !hv) return set_error(SWA_EINVAL, "bad argument");
    if (where != SWA_HOST && where != SWA_DEVICE) return set_error(SWA_EINVAL, "bad where");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nn = (size_t)ps->pd[k].nx * ps->pd[k].ny;
    const double *src[3] = {eta, hu, hv};
    for (int m = 0; m < 3; m++) {
        const double *s = src[m];
        if (where == SWA_HOST) {
            TRY(cuda_check(cudaMemcpyAsync(ps->staging, s, nn * 8, cudaMemcpyHostToDevice, st),
                           "state upload"));
            s = ps->staging;
        }
        to_float_kernel<<<ew_blocks(nn), 256, 0, st>>>(s, ps->host_table[k].q[0][m], nullptr, 0, nn);
        TRY(cuda_check(cudaGetLastError(), "state convert"));
    }
    ps->lev[ps->pd[k].level].started = false;
    return SWA_OK;
}

// A level's new state: no strip has had waves yet (the quiet-strip hint).
__global__ void clear_hint_kernel(int4 *u, int n) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        u[k].w = 0;
}

int swa_patches_start_level(swa_patchset *ps, int level, double t, void *stream) {
    if (!ps || level < 1 || level > SWA_MAX_LEVELS) return set_error(SWA_EINVAL, "bad level");
    Level &L = ps->lev[level];
    if (L.npatches == 0) return set_error(SWA_EINVAL, "level %d has no patches", level);
    cudaStream_t st = (cudaStream_t)stream;
    LevelParams p = level_params(ps, level, 0.0);
    TRY(cuda_check(cudaMemsetAsync(L.smax, 0, 8, st), "smax clear"));
    if (L.nunits16 > 0)
        clear_hint_kernel<<<(L.nunits16 + 255) / 256, 256, 0, st>>>(L.units16, L.nunits16);
    if (L.nunits32 > 0)
        clear_hint_kernel<<<(L.nunits32 + 255) / 256, 256, 0, st>>>(L.units32, L.nunits32);
    TRY(cuda_check(cudaGetLastError(), "clear_hint_kernel"));
    int blocks = p.nunits < 2048 ? p.nunits : 2048;
    level_smax_kernel<<<blocks, 256, 0, st>>>(p, L.smax);
    TRY(cuda_check(cudaGetLastError(), "level_smax_kernel"));
    level_clock_kernel<<<1, 1, 0, st>>>(L.clk, L.smax, t, ps->common.cfl);
    TRY(cuda_check(cudaGetLastError(), "level_clock_kernel"));
    L.started = true;
    return SWA_OK;
}

int swa_patches_get_state(swa_patchset *ps, int k, double *h, double *hu, double *hv,
                          double *eta, int where, void *stream) {
    if (!ps || k < 0 || k >= ps->n) return set_error(SWA_EINVAL, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    DevClock clk;
    TRY(cuda_check(cudaMemcpyAsync(&clk, ps->lev[ps->pd[k].level].clk, sizeof(clk),
                                   cudaMemcpyDeviceToHost, st), "clock read"));
    TRY(cuda_check(cudaStreamSynchronize(st), "clock read"));
    const int cur = clk.cur;
    const size_t nn = (size_t)ps->pd[k].nx * ps->pd[k].ny;
    double *dst[4] = {h, hu, hv, eta};
    const PatchDevice &P = ps->host_table[k];
    for (int m = 0; m < 4; m++) {
        if (!dst[m]) continue;
        double *d = where == SWA_HOST ? ps->staging : dst[m];
        const float *src = P.q[cur][m == 3 ? 0 : m];
        to_double_kernel<<<ew_blocks(nn), 256, 0, st>>>(src, m == 0 ? P.hb : nullptr, d, nn);
        TRY(cuda_check(cudaGetLastError(), "state convert"));
        if (where == SWA_HOST) {
            TRY(cuda_check(cudaMemcpyAsync(dst[m], ps->staging, nn * 8, cudaMemcpyDeviceToHost, st),
                           "state download"));
            TRY(cuda_check(cudaStreamSynchronize(st), "state download"));
        }
    }
    return SWA_OK;
}

int swa_step_level(swa_patchset *ps, int level, int nsteps, double t_end, void *stream) {
    return level_launch(ps, level, nsteps, t_end, LevelReflux{}, (cudaStream_t)stream);
}

int swa_patches_get_time(swa_patchset *ps, int level, double *t, double *dt_next,
                         long long *nsteps, void *stream) {
    if (!ps || level < 1 || level > SWA_MAX_LEVELS) return set_error(SWA_EINVAL, "bad level");
    DevClock clk;
    TRY(cuda_check(cudaMemcpyAsync(&clk, ps->lev[level].clk, sizeof(clk), cudaMemcpyDeviceToHost,
                                   (cudaStream_t)stream), "clock read"));
    TRY(cuda_check(cudaStreamSynchronize((cudaStream_t)stream), "clock read"));
    if (t) *t = clk.t;
    if (dt_next) *dt_next = clk.dt_cfl;
    if (nsteps) *nsteps = clk.nsteps;
    return SWA_OK;
}

int swa_patches_level_info(const swa_patchset *ps, int level, int *npatches, int *ntiles,
                           long long *ncells) {
    if (!ps || level < 1 || level > SWA_MAX_LEVELS) return set_error(SWA_EINVAL, "bad level");
    const Level &L = ps->lev[level];
    if (npatches) *npatches = L.npatches;
    if (ntiles) *ntiles = L.npatches > 0 ? level_params(ps, level, 0.0).nunits : 0;
    if (ncells) *ncells = L.ncells;
    return SWA_OK;
}

int swa_patches_set_tile_rows(swa_patchset *ps, int level, int rows) {
    if (!ps || level < 1 || level > SWA_MAX_LEVELS) return set_error(SWA_EINVAL, "bad level");
    if (rows != 0 && rows != 16 && rows != 32)
        return set_error(SWA_EINVAL, "strip rows must be 0, 16 or 32");
    ps->lev[level].rows = rows;
    return SWA_OK;
}

}  // extern "C"

// ================================================================ AMR glue
//
// A coarse grid (FP32, 2D) and L nested levels of ringed patches of one
// patch set, level l refined from level l - 1 by an integer ratio r_l in
// space and in time (the hierarchy of Sec. 1 and Sec. 6).  Level l's cells
// are numbered on a virtual uniform grid over the domain ("global" level-l
// cells, P_l = r_1 ... r_l per coarse cell).  Each patch carries a 2-cell
// ring as ordinary cells; the level step updates the ring like any cell (it
// enters only the level's CFL maximum) and the fill before the next launch
// overwrites it.  Maps built on the host at creation, per level l:
//   fill:  per ring cell of a level-l patch (patch, cell, src, idx): src >=
//          0 the lowest-index other level-l patch whose interior holds the
//          cell and idx its cell there; else idx the parent cell holding it
//          (in the coarse grid at l = 1, else in the lowest-index level-(l -
//          1) patch whose interior holds it: fill_par) and -src - 1 = sx + r
//          sy the ring cell's position inside it.
//   avg:   per copy of a level-(l - 1) cell under a level-l interior (the
//          coarse cell, or the cell in each level-(l - 1) patch whose
//          interior holds it): (parent patch or -1, its cell, the
//          lowest-index level-l patch over it, that patch's first cell).
//   edges: the refluxing edges of level l (LevelReflux) and, per copy of an
//          uncovered level-(l - 1) cell with edges, the group (U's patch or
//          -1, U's cell, first edge, edges).
namespace swadj {
namespace amr {

constexpr int kRing = 2;

using patches::PatchDevice;
using patches::ew_blocks;

struct FillParams {
    const PatchDevice *table;
    RingFill rf;
    const DevClock *lclk;   // this level
    int nfill;
};

// Ring fill of a level at its current time as a kernel of its own (the
// level launch can also fill its rings itself): one thread per ring cell,
// the three components in turn (independent loads); the clocks and alpha
// (FP64) are read and formed once per block.
__global__ void __launch_bounds__(128) amr_fill_kernel(FillParams p) {
    __shared__ float s_a;
    __shared__ int s_fcur, s_pcur;
    if (threadIdx.x == 0) {
        volatile const DevClock *lc = p.lclk, *pc = p.rf.pclk;
        double a = (lc->t - p.rf.t_p) / p.rf.dt_p;
        a = a < 0.0 ? 0.0 : (a > 1.0 ? 1.0 : a);
        s_a = (float)a;
        s_fcur = lc->cur;
        s_pcur = pc->cur;
    }
    __syncthreads();
    const float af = s_a;
    const int fcur = s_fcur, pcur = s_pcur;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < p.nfill; e += gridDim.x * blockDim.x) {
        const int4 m = __ldg(p.rf.fill + e);
        const int par = __ldg(p.rf.par + e);
        const PatchDevice &D = p.table[m.x];
#pragma unroll
        for (int k = 0; k < 3; k++)
            D.q[fcur][k][m.y] =
                patches::ring_value(p.table, p.rf.coarse, m, par, k, p.rf.r, af, fcur, pcur);
    }
}

// Sum of an r x r block of fine cells, row by row (R > 0: r known at
// compile time).
template <int R>
__device__ __forceinline__ float block_sum(const float *f, int nx, int r) {
    float s = 0.f;
    if (R > 0) {
#pragma unroll
        for (int jj = 0; jj < R; jj++)
#pragma unroll
            for (int ii = 0; ii < R; ii++) s += f[jj * nx + ii];
    } else {
        for (int jj = 0; jj < r; jj++)
            for (int ii = 0; ii < r; ii++) s += f[jj * nx + ii];
    }
    return s;
}

struct AvgParams {
    const PatchDevice *table;
    const PatchDevice *coarse;     // the coarse grid's buffers
    const DevClock *lclk, *pclk;   // this level, its parent
    int r;
    const int4 *avg;
    int navg;
    const int4 *cfu;               // refluxing groups (ncfu = 0: none)
    int ncfu;
    double *slot;                  // 1 + r per edge
    double t_end;                  // the parent's step end
    int *err;
};

// Every copy of a parent cell under the level := mean of its r x r cells
// (eta, hu, hv); one thread per (entry, component).  Then, one thread per
// group (refluxing of the parent level): eta_U += the FP64 sum of its
// edges' slots (coarse part, then the fine parts, edge by edge), and the
// slots return to zero.  U is never under the level, so the two parts write
// different cells.  Also checks that both levels reached the step's end.
template <int R>
__global__ void amr_avg_kernel(AvgParams p) {
    volatile const DevClock *lc = p.lclk, *pc = p.pclk;
    __shared__ int s_fcur, s_pcur;
    if (threadIdx.x == 0) {
        s_fcur = lc->cur;
        s_pcur = pc->cur;
    }
    __syncthreads();
    const int fcur = s_fcur, pcur = s_pcur;
    const int r = R > 0 ? R : p.r;
    const float inv = 1.f / (float)(r * r);
    const int n3 = 3 * p.navg, n = n3 + p.ncfu;
    for (int e3 = blockIdx.x * blockDim.x + threadIdx.x; e3 < n; e3 += gridDim.x * blockDim.x) {
        if (e3 >= n3) {
            const int4 g = __ldg(p.cfu + (e3 - n3));
            double s = 0.0;
            for (int e = g.z; e < g.z + g.w; e++) {
                double *sl = p.slot + (size_t)e * (1 + r);
                double f = sl[0];
                for (int k = 1; k <= r; k++) f += sl[k];
                for (int k = 0; k <= r; k++) sl[k] = 0.0;
                s += f;
            }
            float *eta = (g.x < 0 ? *p.coarse : p.table[g.x]).q[pcur][0];
            eta[g.y] = fp::add(eta[g.y], (float)s);
            continue;
        }
        const int e = e3 / 3, k = e3 - 3 * e;
        const int4 m = __ldg(p.avg + e);
        const PatchDevice &S = p.table[m.z];
        float *dst = (m.x < 0 ? *p.coarse : p.table[m.x]).q[pcur][k];
        dst[m.y] = block_sum<R>(S.q[fcur][k] + m.w, S.nx, r) * inv;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double tol = 1e-12 * (fabs(p.t_end) > 1.0 ? fabs(p.t_end) : 1.0);
        if (!(fabs(lc->t - p.t_end) <= tol) || !(fabs(pc->t - p.t_end) <= tol))
            atomicOr(p.err, ERR_LAG);
    }
}

// Before the coarse step: checks that every level starts at t_n, then per
// level-1 edge the coarse part, slot[e (1 + r)] += (dt_c / d) F_U, the
// coarse flux through the edge as U's update will use it (signed into V).
// A group of 4 lanes per edge, 8 edges per warp.
struct CoarseReflux {
    const DevClock *cclk;
    const float *cq[2][3];
    const float *chb;
    int nxc, nyc;
    BcSpec cbc;
    double dxc, dyc;      // coarse cell size (the correction's scale)
    double nxc_d, nyc_d;  // the coarse step's nu divisors (its FP32 cell size)
    float g;
    int order;
    const int4 *cf;
    const int *cfw;
    double *slot;
    int ncf, r;
    double t_n, t_end;
    const DevClock *lclk[SWA_MAX_LEVELS];
    int nlev;
    int *err;
};

__global__ void reflux_coarse_kernel(CoarseReflux p) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double tol = 1e-12 * (fabs(p.t_n) > 1.0 ? fabs(p.t_n) : 1.0);
        bool ok = fabs(((volatile const DevClock *)p.cclk)->t - p.t_n) <= tol;
        for (int l = 0; l < p.nlev; l++)
            ok = ok && fabs(((volatile const DevClock *)p.lclk[l])->t - p.t_n) <= tol;
        if (!ok) atomicOr(p.err, ERR_LAG);
    }
    if (p.ncf == 0) return;
    const int lane = threadIdx.x & 31;
    const int warp = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    int e = warp * 8 + (lane >> 2);
    const bool live = e < p.ncf;
    if (!live) e = p.ncf - 1;   // idle lanes redo the last edge for the shuffles
    const double dt = reflux::coming_dt(p.cclk, p.t_end);
    const int cur = p.cclk->cur;
    strip::View v;
    v.q0 = p.cq[cur][0]; v.q1 = p.cq[cur][1]; v.q2 = p.cq[cur][2]; v.hb = p.chb;
    v.nx = p.nxc; v.ny = p.nyc; v.bc = p.cbc;
    const int4 m = p.cf[e];
    const int w = p.cfw[e];
    const int axis = w & 1, side = (w & 2) ? 1 : -1;
    // U's high edge: stencil from one cell below U; its low edge: from two
    const float f = reflux::group_flux(v, m.y % p.nxc, m.y / p.nxc, axis, side > 0 ? -1 : -2,
                                       0.5f * p.g, (float)(dt / p.nxc_d), (float)(dt / p.nyc_d),
                                       p.order);
    if (live && (lane & 3) == 1)
        p.slot[(size_t)e * (1 + p.r)] += (dt > 0.0 ? dt : 0.0) / (axis == 0 ? p.dxc : p.dyc) *
                                         (double)(side > 0 ? f : -f);
}

// ------------------------------------------------------------- host maps
// One patch in its level's global cells: array column 0 at (I0, J0);
// interior [I0 + 2, I0 + nx - 2) x [J0 + 2, J0 + ny - 2).
struct FineBox {
    long long I0, J0;
    int nx, ny;
    bool interior(long long I, long long J) const {
        return I >= I0 + kRing && I < I0 + nx - kRing && J >= J0 + kRing && J < J0 + ny - kRing;
    }
    int local(long long I, long long J) const { return (int)((J - J0) * nx + (I - I0)); }
};

// A hierarchy level's patches (patch-set indices ascending) and a bucket
// index over the coarse cells: the patches whose interior meets each.
struct LevelGeom {
    std::vector<int> ids;
    std::vector<FineBox> box;
    long long per = 1;        // level cells per coarse cell, per axis
    long long gnx = 0, gny = 0;
    int r = 1;
    double dx = 0, dy = 0;
    std::vector<int> head, list;

    // lowest-index patch (other than skip) whose interior holds global cell
    // (I, J); -1 if none
    int owner(long long I, long long J, int skip, int nxc) const {
        if (I < 0 || J < 0 || I >= gnx || J >= gny) return -1;
        const size_t c = (size_t)(J / per) * nxc + (size_t)(I / per);
        for (int k = head[c]; k < head[c + 1]; k++) {
            const int a = list[k];
            if (a != skip && box[a].interior(I, J)) return a;
        }
        return -1;
    }
};

struct HostMaps {
    std::vector<int4> fill, avg, cf, cfu;
    std::vector<int> par, cfw;
    std::vector<int> base;   // per patch-set patch: its first fill entry (-1: not on the level)
};

// Check the hierarchy and build every level's maps (host).  levels[l - 1]:
// the patch-set level of hierarchy level l; ratios[l - 1]: r_l.
int build_maps(const GridRefs &c, const swa_patchset *ps, int L, const int *levels,
               const int *ratios, std::vector<HostMaps> &out) {
    const swa_grid_desc &d = c.d;
    if (d.ndim != 2 || d.precision != SWA_FP32)
        return set_error(SWA_EINVAL, "the coarse grid must be 2D FP32");
    if (L < 1 || L > SWA_MAX_LEVELS) return set_error(SWA_EINVAL, "levels must be in [1, %d]",
                                                      SWA_MAX_LEVELS);
    // the fills overwrite every ring cell before each launch, so the patches
    // must extrapolate beyond their rings (a wall would change the ring's
    // edge waves and the level's CFL step)
    for (int k = 0; k < 4; k++)
        if (ps->common.bc[k] != SWA_BC_EXTRAP)
            return set_error(SWA_EINVAL,
                             "the fine patch set must use SWA_BC_EXTRAP on all four sides");
    std::vector<LevelGeom> G(L + 1);
    G[0].per = 1; G[0].gnx = d.nx; G[0].gny = d.ny; G[0].dx = d.dx; G[0].dy = d.dy;
    long long per = 1;
    for (int l = 1; l <= L; l++) {
        const int lev = levels[l - 1], r = ratios[l - 1];
        if (lev < 1 || lev > SWA_MAX_LEVELS || ps->lev[lev].npatches == 0)
            return set_error(SWA_EINVAL, "level %d has no patches", lev);
        for (int k = 1; k < l; k++)
            if (levels[k - 1] == lev)
                return set_error(SWA_EINVAL, "patch-set level %d used twice", lev);
        if (r < 1 || r > 64) return set_error(SWA_EINVAL, "ratio must be in [1, 64]");
        per *= r;
        if (per > (1LL << 20)) return set_error(SWA_EINVAL, "refinement too deep");
        LevelGeom &g = G[l];
        g.r = r; g.per = per; g.gnx = d.nx * per; g.gny = d.ny * per;
        g.dx = G[l - 1].dx / r; g.dy = G[l - 1].dy / r;
        for (int k = 0; k < ps->n; k++) {
            const swa_patch_desc &q = ps->pd[k];
            if (q.level != lev) continue;
            if (fabs(q.dx - g.dx) > 1e-9 * g.dx || fabs(q.dy - g.dy) > 1e-9 * g.dy)
                return set_error(SWA_EINVAL, "patch %d: cell size is not the parent's / %d", k, r);
            // interior lower-left on a parent cell corner
            const double fi = (q.x_lo + kRing * q.dx - d.x_lo) / G[l - 1].dx;
            const double fj = (q.y_lo + kRing * q.dy - d.y_lo) / G[l - 1].dy;
            const long long i0 = llround(fi), j0 = llround(fj);
            if (fabs(fi - (double)i0) > 1e-6 || fabs(fj - (double)j0) > 1e-6)
                return set_error(SWA_EINVAL, "patch %d: interior not on parent cell corners", k);
            if (q.nx <= 2 * kRing || q.ny <= 2 * kRing || (q.nx - 2 * kRing) % r != 0 ||
                (q.ny - 2 * kRing) % r != 0)
                return set_error(SWA_EINVAL, "patch %d: interior not whole parent cells", k);
            FineBox b{i0 * r - kRing, j0 * r - kRing, q.nx, q.ny};
            if (b.I0 < 0 || b.J0 < 0 || b.I0 + b.nx > g.gnx || b.J0 + b.ny > g.gny)
                return set_error(SWA_EINVAL, "patch %d: its ring leaves the domain", k);
            g.ids.push_back(k);
            g.box.push_back(b);
        }
        // bucket index (CSR over coarse cells, patch order kept)
        const size_t nc = (size_t)d.nx * d.ny;
        g.head.assign(nc + 1, 0);
        for (int pass = 0; pass < 2; pass++) {
            std::vector<int> fillp;
            if (pass == 1) {
                for (size_t i = 0; i < nc; i++) g.head[i + 1] += g.head[i];
                g.list.assign(g.head[nc], 0);
                fillp.assign(g.head.begin(), g.head.end() - 1);
            }
            for (int a = 0; a < (int)g.box.size(); a++) {
                const FineBox &b = g.box[a];
                const long long x0 = (b.I0 + kRing) / per, x1 = (b.I0 + b.nx - kRing - 1) / per;
                const long long y0 = (b.J0 + kRing) / per, y1 = (b.J0 + b.ny - kRing - 1) / per;
                for (long long y = y0; y <= y1; y++)
                    for (long long x = x0; x <= x1; x++) {
                        const size_t cc = (size_t)y * d.nx + (size_t)x;
                        if (pass == 0) g.head[cc + 1]++;
                        else g.list[fillp[cc]++] = a;
                    }
            }
        }
    }
    out.assign(L + 1, HostMaps());
    static const int dirs[4][2] = {{0, 1}, {0, -1}, {1, 1}, {1, -1}};
    for (int l = 1; l <= L; l++) {
        const LevelGeom &g = G[l], &gp = G[l - 1];
        const int r = g.r;
        HostMaps &M = out[l];
        M.base.assign(ps->n, -1);
        // fills (and the nesting check of every array cell)
        for (int a = 0; a < (int)g.box.size(); a++) {
            const FineBox &b = g.box[a];
            M.base[g.ids[a]] = (int)M.fill.size();
            for (int j = 0; j < b.ny; j++)
                for (int i = 0; i < b.nx; i++) {
                    const bool ring =
                        !(i >= kRing && i < b.nx - kRing && j >= kRing && j < b.ny - kRing);
                    const long long I = b.I0 + i, J = b.J0 + j;
                    const long long Ip = I / r, Jp = J / r;
                    int pb = -1;
                    if (l > 1) {
                        pb = gp.owner(Ip, Jp, -1, d.nx);
                        if (pb < 0)
                            return set_error(SWA_EINVAL, "patch %d: not nested in level %d",
                                             g.ids[a], levels[l - 2]);
                    }
                    if (!ring) continue;
                    const int src = g.owner(I, J, a, d.nx);
                    int4 m = make_int4(g.ids[a], j * b.nx + i, 0, 0);
                    int par = -1;
                    if (src >= 0) {
                        m.z = g.ids[src];
                        m.w = g.box[src].local(I, J);
                    } else {
                        m.z = -1 - (int)((I - Ip * r) + r * (J - Jp * r));
                        if (l == 1) {
                            m.w = (int)(Jp * d.nx + Ip);
                        } else {
                            m.w = gp.box[pb].local(Ip, Jp);
                            par = gp.ids[pb];
                        }
                    }
                    M.fill.push_back(m);
                    M.par.push_back(par);
                }
        }
        // copies of the parent level's interior cells, in order
        auto each_copy = [&](auto fn) {
            if (l == 1) {
                for (int jc = 0; jc < d.ny; jc++)
                    for (int ic = 0; ic < d.nx; ic++) fn(-1, jc * d.nx + ic, (long long)ic, (long long)jc);
                return;
            }
            for (int b = 0; b < (int)gp.box.size(); b++) {
                const FineBox &B = gp.box[b];
                for (int j = kRing; j < B.ny - kRing; j++)
                    for (int i = kRing; i < B.nx - kRing; i++)
                        fn(gp.ids[b], j * B.nx + i, B.I0 + i, B.J0 + j);
            }
        };
        each_copy([&](int pu, int u, long long I, long long J) {
            const int a = g.owner(I * r, J * r, -1, d.nx);
            if (a >= 0) {
                M.avg.push_back(make_int4(pu, u, g.ids[a], g.box[a].local(I * r, J * r)));
                return;
            }
            const int first = (int)M.cf.size();
            for (int k = 0; k < 4; k++) {
                const int axis = dirs[k][0], side = dirs[k][1];
                const long long Iv = axis == 0 ? I + side : I, Jv = axis == 0 ? J : J + side;
                if (Iv < 0 || Iv >= gp.gnx || Jv < 0 || Jv >= gp.gny) continue;
                const int q = g.owner(Iv * r, Jv * r, -1, d.nx);
                if (q < 0) continue;
                const FineBox &b = g.box[q];
                long long If = Iv * r, Jf = Jv * r;
                if (axis == 0) If += side > 0 ? 0 : r - 1;
                else Jf += side > 0 ? 0 : r - 1;
                const int stride = axis == 0 ? b.nx : 1;
                M.cf.push_back(make_int4(pu, u, g.ids[q], b.local(If, Jf)));
                M.cfw.push_back(axis | (side > 0 ? 2 : 0) | (stride << 2));
            }
            if ((int)M.cf.size() > first)
                M.cfu.push_back(make_int4(pu, u, first, (int)M.cf.size() - first));
        });
        if ((long long)M.cf.size() * (1 + r) > 0x7fffffffLL)
            return set_error(SWA_EINVAL, "too many coarse-fine edges at level %d", levels[l - 1]);
    }
    return SWA_OK;
}

// Workspace layout of one level's maps and slots, each on a 256-byte
// boundary.
struct Layout {
    size_t fill, par, base, avg, cf, cfw, cfu, slot, end;
};

inline size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

inline Layout layout_of(const HostMaps &M, int r, size_t at) {
    Layout Lo;
    Lo.fill = at;
    Lo.par = Lo.fill + round256(sizeof(int4) * M.fill.size());
    Lo.base = Lo.par + round256(sizeof(int) * M.par.size());
    Lo.avg = Lo.base + round256(sizeof(int) * M.base.size());
    Lo.cf = Lo.avg + round256(sizeof(int4) * M.avg.size());
    Lo.cfw = Lo.cf + round256(sizeof(int4) * M.cf.size());
    Lo.cfu = Lo.cfw + round256(sizeof(int) * M.cfw.size());
    Lo.slot = Lo.cfu + round256(sizeof(int4) * M.cfu.size());
    Lo.end = Lo.slot + round256(sizeof(double) * M.cf.size() * (size_t)(1 + r));
    return Lo;
}

// the coarse grid's descriptor heads the workspace
constexpr size_t kCoarseDesc = (sizeof(PatchDevice) + 255) & ~(size_t)255;

inline size_t total_bytes(const std::vector<HostMaps> &M, const int *ratios, int L) {
    size_t at = kCoarseDesc;
    for (int l = 1; l <= L; l++) at = layout_of(M[l], ratios[l - 1], at).end;
    return at + 256;
}

}  // namespace amr
}  // namespace swadj

struct AmrLevel {
    int lev = 0, r = 1;
    int4 *fill = nullptr, *avg = nullptr, *cf = nullptr, *cfu = nullptr;
    int *par = nullptr, *cfw = nullptr, *base = nullptr;
    double *slot = nullptr;
    int nfill = 0, navg = 0, ncf = 0, ncfu = 0;
    double dx = 0, dy = 0;
};

struct swa_amr {
    swa_grid *coarse = nullptr;
    swa_patchset *fine = nullptr;
    swadj::patches::PatchDevice *coarse_pd = nullptr;   // device
    int L = 0;
    AmrLevel lv[SWA_MAX_LEVELS + 1];   // 1 .. L
    int reflux = 1;
    int fill_mode = SWA_AMR_FILL_KERNEL;
};

namespace {

// Averaging of level l into its parent (and the refluxing of the parent
// from level l's edges), after the parent's step ending at t_end.
int amr_average(swa_amr *A, const GridRefs &c, int l, double t_end, bool reflux,
                cudaStream_t st) {
    using namespace swadj;
    AmrLevel &V = A->lv[l];
    amr::AvgParams p{};
    p.table = A->fine->table;
    p.coarse = A->coarse_pd;
    p.lclk = A->fine->lev[V.lev].clk;
    p.pclk = l == 1 ? c.clk : A->fine->lev[A->lv[l - 1].lev].clk;
    p.r = V.r;
    p.avg = V.avg; p.navg = V.navg;
    if (reflux) { p.cfu = V.cfu; p.ncfu = V.ncfu; }
    p.slot = V.slot;
    p.t_end = t_end;
    p.err = swadj_host::error_word();
    const size_t n = (size_t)3 * V.navg + (size_t)p.ncfu;
    const unsigned ab = patches::ew_blocks(n > 0 ? n : 1);
    switch (V.r) {
        case 1: amr::amr_avg_kernel<1><<<ab, 256, 0, st>>>(p); break;
        case 2: amr::amr_avg_kernel<2><<<ab, 256, 0, st>>>(p); break;
        case 4: amr::amr_avg_kernel<4><<<ab, 256, 0, st>>>(p); break;
        case 8: amr::amr_avg_kernel<8><<<ab, 256, 0, st>>>(p); break;
        default: amr::amr_avg_kernel<0><<<ab, 256, 0, st>>>(p); break;
    }
    return cuda_check(cudaGetLastError(), "amr_avg_kernel");
}

// Level l of the hierarchy over the parent step [t_p, t_p + dt_p]
// (Berger-Oliger): r_l substeps, each with its ring fills and launches
// (one launch for a level with children, m for the finest), then the
// children over the substep and their averaging (with the refluxing of
// this level).
int amr_run(swa_amr *A, const GridRefs &c, int l, double t_p, double dt_p, int m, bool reflux,
            cudaStream_t st) {
    using namespace swadj;
    AmrLevel &V = A->lv[l];
    const int r = V.r;
    patches::RingFill lf{};
    lf.fill = V.fill; lf.par = V.par; lf.base = V.base; lf.coarse = A->coarse_pd;
    lf.pclk = l == 1 ? c.clk : A->fine->lev[A->lv[l - 1].lev].clk;
    lf.r = r; lf.t_p = t_p; lf.dt_p = dt_p;
    const bool fused = A->fill_mode == SWA_AMR_FILL_FUSED;
    amr::FillParams f{};
    f.table = A->fine->table;
    f.rf = lf;
    f.lclk = A->fine->lev[V.lev].clk;
    f.nfill = V.nfill;
    size_t fbn = ((size_t)(V.nfill > 0 ? V.nfill : 1) + 127) / 128;
    const unsigned fb = (unsigned)(fbn < 65535 ? fbn : 65535);
    patches::LevelReflux rf{};
    const double dpx = l == 1 ? c.d.dx : A->lv[l - 1].dx, dpy = l == 1 ? c.d.dy : A->lv[l - 1].dy;
    if (reflux) {
        rf.cf = V.cf; rf.cfw = V.cfw; rf.slot = V.slot; rf.nfine = V.ncf * r; rf.r = r;
        rf.dpx = dpx; rf.dpy = dpy;
        if (l < A->L) {
            const AmrLevel &W = A->lv[l + 1];
            rf.cf2 = W.cf; rf.cfw2 = W.cfw; rf.slot2 = W.slot; rf.ncoarse = W.ncf; rf.r2 = W.r;
            rf.dtx = V.dx; rf.dty = V.dy;
        }
    }
    const int launches = l == A->L ? m : 1;
    for (int k = 1; k <= r; k++) {
        const double t_k = k == r ? t_p + dt_p : t_p + dt_p * (double)k / (double)r;
        const double t_km1 = k == 1 ? t_p : t_p + dt_p * (double)(k - 1) / (double)r;
        for (int j = 0; j < launches; j++) {
            if (!fused) {
                amr::amr_fill_kernel<<<fb, 128, 0, st>>>(f);
                TRY(cuda_check(cudaGetLastError(), "amr_fill_kernel"));
            }
            TRY(level_launch(A->fine, V.lev, 1, t_k, rf, st, fused ? &lf : nullptr));
        }
        if (l < A->L) {
            TRY(amr_run(A, c, l + 1, t_km1, t_k - t_km1, m, reflux, st));
            TRY(amr_average(A, c, l + 1, t_k, reflux, st));
        }
    }
    return SWA_OK;
}

}  // namespace

extern "C" {

size_t swa_amr_levels_workspace_bytes(const swa_grid *coarse, const swa_patchset *fine,
                                      int nlevels, const int *levels, const int *ratios) {
    GridRefs c;
    if (!fine || !levels || !ratios || grid_refs(coarse, &c) != SWA_OK) return 0;
    std::vector<amr::HostMaps> M;
    if (amr::build_maps(c, fine, nlevels, levels, ratios, M) != SWA_OK) return 0;
    return amr::total_bytes(M, ratios, nlevels);
}

int swa_create_amr_levels(swa_grid *coarse, swa_patchset *fine, int nlevels, const int *levels,
                          const int *ratios, void *ws, size_t ws_bytes, void *stream,
                          swa_amr **out) {
    GridRefs c;
    if (!fine || !ws || !out || !levels || !ratios) return set_error(SWA_EINVAL, "null argument");
    TRY(grid_refs(coarse, &c));
    if (((uintptr_t)ws & 255) != 0) return set_error(SWA_EINVAL, "workspace must be 256-byte aligned");
    std::vector<amr::HostMaps> M;
    TRY(amr::build_maps(c, fine, nlevels, levels, ratios, M));
    const size_t need = amr::total_bytes(M, ratios, nlevels);
    if (ws_bytes < need)
        return set_error(SWA_ENOMEM, "AMR workspace %zu bytes < %zu needed", ws_bytes, need);
    swa_amr *A = new (std::nothrow) swa_amr();
    if (!A) return set_error(SWA_ENOMEM, "host allocation failed");
    A->coarse = coarse; A->fine = fine; A->L = nlevels;
    cudaStream_t st = (cudaStream_t)stream;
    char *base = (char *)ws;
    size_t at = amr::kCoarseDesc;
    int rc = SWA_OK;
    // the coarse grid as a ringless patch: its ping-pong buffers and size
    patches::PatchDevice cpd{};
    for (int b = 0; b < 2; b++)
        for (int k = 0; k < 3; k++) cpd.q[b][k] = (float *)c.q[b][k];
    cpd.hb = (const float *)c.bath;
    cpd.nx = c.d.nx; cpd.ny = c.d.ny;
    A->coarse_pd = (patches::PatchDevice *)base;
    rc = cuda_check(cudaMemcpyAsync(A->coarse_pd, &cpd, sizeof(cpd), cudaMemcpyHostToDevice, st),
                    "AMR coarse descriptor upload");
    double dx = c.d.dx, dy = c.d.dy;
    for (int l = 1; l <= nlevels && rc == SWA_OK; l++) {
        const amr::HostMaps &H = M[l];
        const amr::Layout Lo = amr::layout_of(H, ratios[l - 1], at);
        at = Lo.end;
        AmrLevel &V = A->lv[l];
        V.lev = levels[l - 1]; V.r = ratios[l - 1];
        dx /= V.r; dy /= V.r;
        V.dx = dx; V.dy = dy;
        V.fill = (int4 *)(base + Lo.fill); V.par = (int *)(base + Lo.par);
        V.base = (int *)(base + Lo.base);
        V.avg = (int4 *)(base + Lo.avg); V.cf = (int4 *)(base + Lo.cf);
        V.cfw = (int *)(base + Lo.cfw); V.cfu = (int4 *)(base + Lo.cfu);
        V.slot = (double *)(base + Lo.slot);
        V.nfill = (int)H.fill.size(); V.navg = (int)H.avg.size();
        V.ncf = (int)H.cf.size(); V.ncfu = (int)H.cfu.size();
        struct Up { void *dst; const void *src; size_t bytes; const char *what; } up[] = {
            {V.fill, H.fill.data(), sizeof(int4) * H.fill.size(), "AMR fill map upload"},
            {V.par, H.par.data(), sizeof(int) * H.par.size(), "AMR fill parents upload"},
            {V.base, H.base.data(), sizeof(int) * H.base.size(), "AMR fill bases upload"},
            {V.avg, H.avg.data(), sizeof(int4) * H.avg.size(), "AMR average map upload"},
            {V.cf, H.cf.data(), sizeof(int4) * H.cf.size(), "AMR edge map upload"},
            {V.cfw, H.cfw.data(), sizeof(int) * H.cfw.size(), "AMR edge flags upload"},
            {V.cfu, H.cfu.data(), sizeof(int4) * H.cfu.size(), "AMR edge group upload"},
        };
        for (const Up &u : up)
            if (rc == SWA_OK && u.bytes > 0)
                rc = cuda_check(cudaMemcpyAsync(u.dst, u.src, u.bytes, cudaMemcpyHostToDevice, st),
                                u.what);
        const size_t sb = sizeof(double) * (size_t)V.ncf * (size_t)(1 + V.r);
        if (rc == SWA_OK && sb > 0)
            rc = cuda_check(cudaMemsetAsync(V.slot, 0, sb, st), "AMR slot clear");
    }
    if (rc == SWA_OK) rc = cuda_check(cudaStreamSynchronize(st), "create_amr");
    if (rc != SWA_OK) { delete A; return rc; }
    *out = A;
    return SWA_OK;
}

size_t swa_amr_workspace_bytes(const swa_grid *coarse, const swa_patchset *fine, int level,
                               int ratio) {
    return swa_amr_levels_workspace_bytes(coarse, fine, 1, &level, &ratio);
}

int swa_create_amr(swa_grid *coarse, swa_patchset *fine, int level, int ratio, void *ws,
                   size_t ws_bytes, void *stream, swa_amr **out) {
    return swa_create_amr_levels(coarse, fine, 1, &level, &ratio, ws, ws_bytes, stream, out);
}

int swa_destroy_amr(swa_amr *A) {
    delete A;
    return SWA_OK;
}

int swa_amr_set_reflux(swa_amr *A, int on) {
    if (!A) return set_error(SWA_EINVAL, "null AMR hierarchy");
    A->reflux = on != 0;
    return SWA_OK;
}

int swa_amr_set_fill_mode(swa_amr *A, int mode) {
    if (!A) return set_error(SWA_EINVAL, "null AMR hierarchy");
    if (mode != SWA_AMR_FILL_FUSED && mode != SWA_AMR_FILL_KERNEL)
        return set_error(SWA_EINVAL, "fill mode must be SWA_AMR_FILL_FUSED or SWA_AMR_FILL_KERNEL");
    A->fill_mode = mode;
    return SWA_OK;
}

int swa_amr_info(const swa_amr *A, int level, int *nfill, int *navg, int *nedges) {
    if (!A) return set_error(SWA_EINVAL, "null AMR hierarchy");
    if (level < 1 || level > A->L) return set_error(SWA_EINVAL, "level must be in [1, %d]", A->L);
    const AmrLevel &V = A->lv[level];
    if (nfill) *nfill = V.nfill;
    if (navg) *navg = V.navg;
    if (nedges) *nedges = V.ncf;
    return SWA_OK;
}

int swa_amr_step(swa_amr *A, double t_n, double dt_c, int max_launches, void *stream) {
    if (!A) return set_error(SWA_EINVAL, "null AMR hierarchy");
    if (!(dt_c > 0.0)) return set_error(SWA_EINVAL, "dt_c must be > 0");
    if (max_launches < 1) return set_error(SWA_EINVAL, "max_launches must be >= 1");
    GridRefs c;
    TRY(grid_refs(A->coarse, &c));
    if (!c.state_set) return set_error(SWA_ESTATE, "coarse state not set");
    bool edges = false;
    for (int l = 1; l <= A->L; l++) {
        if (!A->fine->lev[A->lv[l].lev].started)
            return set_error(SWA_ESTATE, "level %d not started", A->lv[l].lev);
        edges = edges || A->lv[l].ncf > 0;
    }
    const bool reflux = A->reflux != 0;
    if (reflux && edges && c.scheme != SWA_SCHEME_SPLIT)
        return set_error(SWA_EINVAL, "refluxing needs the split scheme on the coarse grid");
    cudaStream_t st = (cudaStream_t)stream;
    const double t_end = t_n + dt_c;
    amr::CoarseReflux q{};
    q.cclk = c.clk;
    for (int b = 0; b < 2; b++)
        for (int k = 0; k < 3; k++) q.cq[b][k] = (const float *)c.q[b][k];
    q.chb = (const float *)c.bath;
    q.nxc = c.d.nx; q.nyc = c.d.ny;
    q.cbc = BcSpec{c.d.bc[0], c.d.bc[1], c.d.bc[2], c.d.bc[3]};
    q.dxc = c.d.dx; q.dyc = c.d.dy;
    q.nxc_d = (double)(float)c.d.dx; q.nyc_d = (double)(float)c.d.dy;
    q.g = (float)c.d.g; q.order = c.d.order;
    q.cf = A->lv[1].cf; q.cfw = A->lv[1].cfw; q.slot = A->lv[1].slot;
    q.ncf = reflux ? A->lv[1].ncf : 0; q.r = A->lv[1].r;
    q.t_n = t_n; q.t_end = t_end;
    for (int l = 1; l <= A->L; l++) q.lclk[l - 1] = A->fine->lev[A->lv[l].lev].clk;
    q.nlev = A->L;
    q.err = swadj_host::error_word();
    const unsigned eb = (unsigned)(q.ncf > 0 ? (q.ncf + 31) / 32 : 1);   // 8 edges per warp
    amr::reflux_coarse_kernel<<<eb, 128, 0, st>>>(q);
    TRY(cuda_check(cudaGetLastError(), "reflux_coarse_kernel"));
    TRY(swa_step_forward(A->coarse, 1, t_end, stream));
    TRY(amr_run(A, c, 1, t_n, dt_c, max_launches, reflux, st));
    return amr_average(A, c, 1, t_end, reflux, st);
}

}  // extern "C"
