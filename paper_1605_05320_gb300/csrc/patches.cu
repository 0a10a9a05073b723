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

__device__ __forceinline__ CellRaw raw_at(const strip::View &v, int i, int j) {
    bool fx, fy;
    const int ii = ghost_index(i, v.nx, v.bc.lo_x, v.bc.hi_x, &fx);
    const int jj = ghost_index(j, v.ny, v.bc.lo_y, v.bc.hi_y, &fy);
    const size_t o = (size_t)jj * v.nx + ii;
    CellRaw c;
    c.eta = v.q0[o];
    c.hb = v.hb[o];
    const float mu = v.q1[o], mv = v.q2[o];
    c.mu = fx ? -mu : mu;
    c.mv = fy ? -mv : mv;
    return c;
}

// x-frame cell data of cell (i, j)
__device__ __forceinline__ fp::Cell<float> xcell(const strip::View &v, int i, int j) {
    const CellRaw c = raw_at(v, i, j);
    return fp::derive(c.eta, fp::add(c.eta, c.hb), c.mu, c.mv);
}

// the x-swept cell (i, j) in the y frame, as the strip kernel's x-sweep
// leaves it
__device__ __forceinline__ fp::Cell<float> xswept(const strip::View &v, int i, int j, float gh,
                                                  float nux, int order) {
    fp::Cell<float> c[5];
#pragma unroll
    for (int k = 0; k < 5; k++) c[k] = xcell(v, i - 2 + k, j);
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
                                            float gh, float nux, float nuy, int order) {
    using strip::dn;
    using strip::up;
    const int q = threadIdx.x & 3;
    const fp::Cell<float> c =
        axis == 0 ? xcell(v, i + k0 + q, j) : xswept(v, i, j + k0 + q, gh, nux, order);
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

// Refluxing work of a level launch inside the AMR glue: per coarse-fine
// edge e and fine cell k along it (item e r + k), dhf[item] -= (dt_f / d)
// (1 / r) F_f, the flux into the fine region across the edge over this
// launch.  nitems = 0: none.
struct LevelReflux {
    const int4 *cf;   // edges (U, patch, first fine cell, axis | hi << 1 | stride << 2)
    double *dhf;
    int nitems, r;
    double dxc, dyc;  // coarse cell size
};

struct LevelParams {
    const PatchDevice *table;
    const int4 *units;   // (patch, x0, y0, 0)
    int nunits, rows;
    DevClock *clk;
    double *partial;
    int nblocks;
    double t_end, cfl, dx, dy;
    float g;
    int order;
    int *err;
    LevelReflux rf;
};

// One task of a level launch's refluxing work: 8 items, 4 lanes each.
__device__ __noinline__ void level_reflux_task(const LevelParams &p, int task, int cur,
                                               float nux, float nuy, double dt) {
    const int lane = threadIdx.x & 31;
    int item = task * 8 + (lane >> 2);
    const bool live = item < p.rf.nitems;
    if (!live) item = p.rf.nitems - 1;   // idle lanes redo the last item for the shuffles
    const int e = item / p.rf.r, k = item - e * p.rf.r;
    const int4 m = p.rf.cf[e];
    const PatchDevice &P = p.table[m.y];
    strip::View v;
    v.q0 = P.q[cur][0]; v.q1 = P.q[cur][1]; v.q2 = P.q[cur][2]; v.hb = P.hb;
    v.nx = P.nx; v.ny = P.ny; v.bc = P.bc;
    const int axis = m.w & 1, side = (m.w & 2) ? 1 : -1, stride = m.w >> 2;
    const int c = m.z + k * stride;
    // V on U's high side: the fine cell's low edge (stencil from two cells
    // below it); else its high edge (from one below)
    const float f = reflux::group_flux(v, c % P.nx, c / P.nx, axis, side > 0 ? -2 : -1,
                                       0.5f * p.g, nux, nuy, p.order);
    if (live && (lane & 3) == 1)
        p.rf.dhf[item] -= dt / (axis == 0 ? p.rf.dxc : p.rf.dyc) / (double)p.rf.r *
                          (double)(side > 0 ? f : -f);
}

__global__ void __launch_bounds__(strip::kThreads, 5) level_strip_kernel(LevelParams p) {
    __shared__ float s_nu[2];
    __shared__ int s_cur, s_run;
    __shared__ float red[strip::kThreads / 32];
    __shared__ int am_last;
    __shared__ strip::Ring ring[strip::kThreads / 32];
    double t_now = 0.0, dt = 0.0;
    if (!fwave::begin_step(p.clk, p.t_end, p.dx, p.dy, s_nu, &s_cur, &s_run, t_now, dt)) return;
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
        strip::strip_unit(v, t.y, t.z, p.rows, s_nu[0], s_nu[1], p.g, p.order,
                          ring[threadIdx.x >> 5], smax, bad);
    }
    if (p.rf.nitems > 0) {
        // the warps with one strip fewer start on the refluxing tasks; the
        // clock is not advanced before every block has finished them
        const int total = gridDim.x * wpb, gw = blockIdx.x * wpb + (threadIdx.x >> 5);
        const int ntasks = (p.rf.nitems + 7) / 8, rem = p.nunits % total;
        const double dt_now = reflux::coming_dt(p.clk, p.t_end);
        for (int t = (gw + total - rem) % total; t < ntasks; t += total)
            level_reflux_task(p, t, cur, s_nu[0], s_nu[1], dt_now);
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
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, level_strip_kernel,
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
    p.rows = L.rows == 16 ? 16 : 32;
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
                        const LevelReflux &rf, cudaStream_t st) {
    if (!ps || level < 1 || level > SWA_MAX_LEVELS) return set_error(SWA_EINVAL, "bad level");
    Level &L = ps->lev[level];
    if (L.npatches == 0) return set_error(SWA_EINVAL, "level %d has no patches", level);
    if (!L.started) return set_error(SWA_ESTATE, "level %d not started", level);
    if (nsteps < 0) return set_error(SWA_EINVAL, "nsteps < 0");
    LevelParams p = level_params(ps, level, t_end);
    p.rf = rf;
    constexpr int wpb = strip::kThreads / 32;
    const int need = (p.nunits + wpb - 1) / wpb;
    p.nblocks = occupancy_blocks();
    if (p.nblocks > need) p.nblocks = need;
    for (int s = 0; s < nsteps; s++)
        level_strip_kernel<<<p.nblocks, strip::kThreads, 0, st>>>(p);
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

int swa_patches_start_level(swa_patchset *ps, int level, double t, void *stream) {
    if (!ps || level < 1 || level > SWA_MAX_LEVELS) return set_error(SWA_EINVAL, "bad level");
    Level &L = ps->lev[level];
    if (L.npatches == 0) return set_error(SWA_EINVAL, "level %d has no patches", level);
    cudaStream_t st = (cudaStream_t)stream;
    LevelParams p = level_params(ps, level, 0.0);
    TRY(cuda_check(cudaMemsetAsync(L.smax, 0, 8, st), "smax clear"));
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
    if (ntiles) *ntiles = L.rows == 16 ? L.nunits16 : L.nunits32;
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

// ======================================================= two-level AMR glue
//
// One coarse grid (FP32, 2D) and one level of fine patches refined by an
// integer ratio r in space and time (the AMR hierarchy of Sec. 1, Sec. 6).
// Each fine patch carries a 2-cell ring as ordinary cells; the level step
// updates the ring like any cell (it enters only the level's CFL maximum)
// and the fill before the next launch overwrites it.  The maps below are
// built on the host at creation from the patch geometry:
//   fill: per ring cell (patch, cell, source).  Source: the lowest-index
//         other patch whose interior holds the cell (patch, cell), else the
//         coarse cell containing it and the fine cell's position inside it.
//   avg:  per coarse cell under a patch interior (lowest patch index): the
//         patch and the index of its first fine cell.
namespace swadj {
namespace amr {

constexpr int kRing = 2;

using patches::PatchDevice;
using patches::ew_blocks;

struct AmrParams {
    const PatchDevice *table;
    const DevClock *lclk, *cclk;   // fine level, coarse grid
    float *cq[2][3];               // coarse state buffers (eta, hu, hv)
    int nxc, nyc, r;
    const int4 *fill;
    int nfill;
    const int4 *avg;
    int navg;
    const int4 *cfu;   // refluxing: (U, first edge, edges, 0); ncfu = 0: none
    int ncfu;
    const double *dh, *dhf;
    double t_n, dt_c, t_end;
    int *err;
};

__device__ __forceinline__ float minmod(float a, float b) {
    if (a * b <= 0.f) return 0.f;
    return fabsf(a) < fabsf(b) ? a : b;
}

// Ring fill at the fine level's current time: sibling copy, or the coarse
// level linear in time (alpha = (t - t_n) / dt_c in [0, 1]) then limited
// linear in space within the coarse cell (minmod slopes, zero at the domain
// edge).  Map entry (patch, cell, src, idx): src >= 0 is a sibling patch
// and idx its cell; src < 0 is the coarse cell idx, with the fine cell at
// (-src - 1) = sx + r sy inside it.  One thread per (entry, component);
// the clocks and alpha (FP64) are read and formed once per block.
__global__ void amr_fill_kernel(AmrParams p) {
    __shared__ float s_a;
    __shared__ int s_fcur, s_ccur;
    if (threadIdx.x == 0) {
        volatile const DevClock *lc = p.lclk, *cc = p.cclk;
        double a = (lc->t - p.t_n) / p.dt_c;
        a = a < 0.0 ? 0.0 : (a > 1.0 ? 1.0 : a);
        s_a = (float)a;
        s_fcur = lc->cur;
        s_ccur = cc->cur;
    }
    __syncthreads();
    const float af = s_a;
    const int fcur = s_fcur, ccur = s_ccur;
    const int r = p.r, nxc = p.nxc, nyc = p.nyc;
    const int n = 3 * p.nfill;
    for (int e3 = blockIdx.x * blockDim.x + threadIdx.x; e3 < n; e3 += gridDim.x * blockDim.x) {
        const int e = e3 / 3, k = e3 - 3 * e;
        const int4 m = __ldg(p.fill + e);
        float *dst = p.table[m.x].q[fcur][k];
        if (m.z >= 0) {
            dst[m.y] = p.table[m.z].q[fcur][k][m.w];
            continue;
        }
        const int sub = -m.z - 1, sx = sub % r, sy = sub / r;
        const int c = m.w, ic = c % nxc, jc = c / nxc;
        const float xi = (float)(2 * sx + 1 - r) / (float)(2 * r);
        const float zeta = (float)(2 * sy + 1 - r) / (float)(2 * r);
        const float *o = p.cq[ccur ^ 1][k], *nw = p.cq[ccur][k];
        auto at = [&](int i) { return fmaf(af, nw[i] - o[i], o[i]); };
        const float qc = at(c);
        float s_x = 0.f, s_y = 0.f;
        if (ic > 0 && ic < nxc - 1) s_x = minmod(qc - at(c - 1), at(c + 1) - qc);
        if (jc > 0 && jc < nyc - 1) s_y = minmod(qc - at(c - nxc), at(c + nxc) - qc);
        dst[m.y] = fmaf(s_y, zeta, fmaf(s_x, xi, qc));
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

// Coarse cells under a patch := mean of their r x r fine cells (eta, hu, hv).
// Entry (coarse cell, patch, first fine cell, 0); one thread per (entry,
// component).  Then, one thread per uncovered coarse cell U beside the fine
// level (refluxing): eta_U += the FP64 sum of its edges' corrections, coarse
// part plus fine parts, in a fixed order (U is never a covered cell, so the
// two parts write different cells).  Also checks that both levels reached
// the step's end time.
template <int R>
__global__ void amr_avg_kernel(AmrParams p) {
    volatile const DevClock *lc = p.lclk, *cc = p.cclk;
    __shared__ int s_fcur, s_ccur;
    if (threadIdx.x == 0) {
        s_fcur = lc->cur;
        s_ccur = cc->cur;
    }
    __syncthreads();
    const int fcur = s_fcur, ccur = s_ccur;
    const int r = R > 0 ? R : p.r;
    const float inv = 1.f / (float)(r * r);
    const int n3 = 3 * p.navg, n = n3 + p.ncfu;
    for (int e3 = blockIdx.x * blockDim.x + threadIdx.x; e3 < n; e3 += gridDim.x * blockDim.x) {
        if (e3 >= n3) {
            const int4 g = __ldg(p.cfu + (e3 - n3));
            double s = 0.0;
            for (int e = g.y; e < g.y + g.z; e++) {
                double f = p.dh[e];
                for (int k = 0; k < r; k++) f += p.dhf[(size_t)e * r + k];
                s += f;
            }
            float *eta = p.cq[ccur][0];
            eta[g.x] = fp::add(eta[g.x], (float)s);
            continue;
        }
        const int e = e3 / 3, k = e3 - 3 * e;
        const int4 m = __ldg(p.avg + e);
        const PatchDevice &S = p.table[m.y];
        p.cq[ccur][k][m.x] = block_sum<R>(S.q[fcur][k] + m.z, S.nx, r) * inv;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double tol = 1e-12 * (fabs(p.t_end) > 1.0 ? fabs(p.t_end) : 1.0);
        if (!(fabs(lc->t - p.t_end) <= tol) || !(fabs(cc->t - p.t_end) <= tol))
            atomicOr(p.err, ERR_LAG);
    }
}

// Before the coarse step, per edge: dh[e] = (dt_c / d) F_c, the coarse
// flux through the edge as U's update will use it (sign: + for V on U's
// high side), and the edge's fine parts start at zero.  A group of 4 lanes
// per edge, 8 edges per warp.
struct RefluxParams {
    const DevClock *cclk;
    const float *cq[2][3];
    const float *chb;
    int nxc, nyc, r;
    BcSpec cbc;
    double dxc, dyc;      // coarse cell size (the correction's scale)
    double nxc_d, nyc_d;  // the coarse step's nu divisors (its FP32 cell size)
    float g;
    int order;
    const int4 *cf;
    int ncf;
    double *dh, *dhf;
    double t_end;
};

__global__ void reflux_coarse_kernel(RefluxParams p) {
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
    const int axis = m.w & 1, side = (m.w & 2) ? 1 : -1;
    // U's high edge: stencil from one cell below U; its low edge: from two
    const float f = reflux::group_flux(v, m.x % p.nxc, m.x / p.nxc, axis, side > 0 ? -1 : -2,
                                       0.5f * p.g, (float)(dt / p.nxc_d), (float)(dt / p.nyc_d),
                                       p.order);
    if (live && (lane & 3) == 0)
        for (int k = 0; k < p.r; k++) p.dhf[(size_t)e * p.r + k] = 0.0;
    if (live && (lane & 3) == 1)
        p.dh[e] = (dt > 0.0 ? dt : 0.0) / (axis == 0 ? p.dxc : p.dyc) * (double)(side > 0 ? f : -f);
}

// Geometry of one fine patch in global fine cells: array column 0 at
// (I0, J0); interior [I0 + 2, I0 + nx - 2) x [J0 + 2, J0 + ny - 2).
// Building the maps costs O(coarse cells + ring cells + covered cells).
struct FineBox {
    long long I0, J0;
    int nx, ny;
};

// Check the hierarchy and build the maps (host).
int build_maps(const GridRefs &c, const swa_patchset *ps, int level, int r,
               std::vector<int4> &fill, std::vector<int4> &avg, std::vector<int4> &cf,
               std::vector<int4> &cfu) {
    const swa_grid_desc &d = c.d;
    if (d.ndim != 2 || d.precision != SWA_FP32)
        return set_error(SWA_EINVAL, "the coarse grid must be 2D FP32");
    if (r < 1 || r > 64) return set_error(SWA_EINVAL, "ratio must be in [1, 64]");
    if (level < 1 || level > SWA_MAX_LEVELS || ps->lev[level].npatches == 0)
        return set_error(SWA_EINVAL, "level %d has no patches", level);
    // the fills overwrite every ring cell before each launch, so the fine
    // patches must extrapolate beyond their rings (a wall would change the
    // ring's edge waves and the level's CFL step)
    for (int k = 0; k < 4; k++)
        if (ps->common.bc[k] != SWA_BC_EXTRAP)
            return set_error(SWA_EINVAL,
                             "the fine patch set must use SWA_BC_EXTRAP on all four sides");
    std::vector<int> ids;
    std::vector<FineBox> box;
    const double dxf = d.dx / r, dyf = d.dy / r;
    for (int k = 0; k < ps->n; k++) {
        const swa_patch_desc &q = ps->pd[k];
        if (q.level != level) continue;
        if (fabs(q.dx - dxf) > 1e-9 * dxf || fabs(q.dy - dyf) > 1e-9 * dyf)
            return set_error(SWA_EINVAL, "patch %d: cell size is not the coarse size / %d", k, r);
        // interior lower-left on a coarse cell corner
        const double fi = (q.x_lo + kRing * q.dx - d.x_lo) / d.dx;
        const double fj = (q.y_lo + kRing * q.dy - d.y_lo) / d.dy;
        const long long i0 = llround(fi), j0 = llround(fj);
        if (fabs(fi - (double)i0) > 1e-6 || fabs(fj - (double)j0) > 1e-6)
            return set_error(SWA_EINVAL, "patch %d: interior not on coarse cell corners", k);
        if (q.nx <= 2 * kRing || q.ny <= 2 * kRing || (q.nx - 2 * kRing) % r != 0 ||
            (q.ny - 2 * kRing) % r != 0)
            return set_error(SWA_EINVAL, "patch %d: interior not whole coarse cells", k);
        FineBox b{i0 * r - kRing, j0 * r - kRing, q.nx, q.ny};
        if (b.I0 < 0 || b.J0 < 0 || b.I0 + b.nx > (long long)d.nx * r ||
            b.J0 + b.ny > (long long)d.ny * r)
            return set_error(SWA_EINVAL, "patch %d: its ring leaves the coarse domain", k);
        ids.push_back(k);
        box.push_back(b);
    }
    const int np = (int)ids.size();
    // Interiors are whole coarse cells, so a fine cell's owners are its
    // coarse cell's: per coarse cell the two lowest-index patches (in the
    // order above) whose interiors cover it, -1 if none.
    std::vector<int2> own((size_t)d.nx * d.ny, make_int2(-1, -1));
    for (int a = 0; a < np; a++) {
        const FineBox &b = box[a];
        const long long i0 = (b.I0 + kRing) / r, j0 = (b.J0 + kRing) / r;
        const int mx = (b.nx - 2 * kRing) / r, my = (b.ny - 2 * kRing) / r;
        for (int jc = 0; jc < my; jc++)
            for (int ic = 0; ic < mx; ic++) {
                int2 &o = own[(size_t)(j0 + jc) * d.nx + (size_t)(i0 + ic)];
                if (o.x < 0) o.x = a;
                else if (o.y < 0) o.y = a;
            }
    }
    fill.clear();
    avg.clear();
    for (int a = 0; a < np; a++) {
        const FineBox &b = box[a];
        for (int j = 0; j < b.ny; j++)
            for (int i = 0; i < b.nx; i++) {
                if (i >= kRing && i < b.nx - kRing && j >= kRing && j < b.ny - kRing) continue;
                const long long I = b.I0 + i, J = b.J0 + j;
                const long long ic = I / r, jc = J / r;
                const int2 o = own[(size_t)jc * d.nx + (size_t)ic];
                const int src = o.x != a ? o.x : o.y;   // lowest-index other owner
                int4 m = make_int4(ids[a], j * b.nx + i, 0, 0);
                if (src >= 0) {
                    const FineBox &s = box[src];
                    m.z = ids[src];
                    m.w = (int)((J - s.J0) * s.nx + (I - s.I0));
                } else {
                    m.z = -1 - (int)((I - ic * r) + r * (J - jc * r));
                    m.w = (int)(jc * d.nx + ic);
                }
                fill.push_back(m);
            }
    }
    for (int jc = 0; jc < d.ny; jc++)
        for (int ic = 0; ic < d.nx; ic++) {
            const int a = own[(size_t)jc * d.nx + ic].x;
            if (a < 0) continue;
            const FineBox &b = box[a];
            const long long li = (long long)ic * r - b.I0, lj = (long long)jc * r - b.J0;
            avg.push_back(make_int4(jc * d.nx + ic, ids[a], (int)(lj * b.nx + li), 0));
        }
    // coarse-fine edges: per uncovered coarse cell U, its covered neighbours
    // V in the order (+x, -x, +y, -y); the r fine cells of V's owner along
    // the edge, from the corner nearest the lower left
    cf.clear();
    cfu.clear();
    static const int dirs[4][2] = {{0, 1}, {0, -1}, {1, 1}, {1, -1}};
    for (int jc = 0; jc < d.ny; jc++)
        for (int ic = 0; ic < d.nx; ic++) {
            if (own[(size_t)jc * d.nx + ic].x >= 0) continue;
            const int first = (int)cf.size();
            for (int k = 0; k < 4; k++) {
                const int axis = dirs[k][0], side = dirs[k][1];
                const int iv = axis == 0 ? ic + side : ic, jv = axis == 0 ? jc : jc + side;
                if (iv < 0 || iv >= d.nx || jv < 0 || jv >= d.ny) continue;
                const int a = own[(size_t)jv * d.nx + iv].x;
                if (a < 0) continue;
                const FineBox &b = box[a];
                long long I = (long long)iv * r, J = (long long)jv * r;
                if (axis == 0) I += side > 0 ? 0 : r - 1;
                else J += side > 0 ? 0 : r - 1;
                const int stride = axis == 0 ? b.nx : 1;
                cf.push_back(make_int4(jc * d.nx + ic, ids[a], (int)((J - b.J0) * b.nx + (I - b.I0)),
                                       axis | (side > 0 ? 2 : 0) | (stride << 2)));
            }
            if ((int)cf.size() > first)
                cfu.push_back(make_int4(jc * d.nx + ic, first, (int)cf.size() - first, 0));
        }
    return SWA_OK;
}

// Workspace layout: fill, avg, edge and edge-group maps (int4), then the
// per-edge corrections (double), each on a 256-byte boundary.
struct Layout {
    size_t fill, avg, cf, cfu, dh, dhf, total;
};

inline size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

inline Layout layout_of(size_t nfill, size_t navg, size_t ncf, size_t ncfu, int r) {
    Layout L;
    L.fill = 0;
    L.avg = L.fill + round256(sizeof(int4) * nfill);
    L.cf = L.avg + round256(sizeof(int4) * navg);
    L.cfu = L.cf + round256(sizeof(int4) * ncf);
    L.dh = L.cfu + round256(sizeof(int4) * ncfu);
    L.dhf = L.dh + round256(sizeof(double) * ncf);
    L.total = L.dhf + round256(sizeof(double) * ncf * (size_t)r) + 256;
    return L;
}

}  // namespace amr
}  // namespace swadj

struct swa_amr {
    swa_grid *coarse = nullptr;
    swa_patchset *fine = nullptr;
    int level = 0, r = 1;
    int4 *fill = nullptr, *avg = nullptr, *cf = nullptr, *cfu = nullptr;
    double *dh = nullptr, *dhf = nullptr;
    int nfill = 0, navg = 0, ncf = 0, ncfu = 0;
    int reflux = 1;
};

extern "C" {

size_t swa_amr_workspace_bytes(const swa_grid *coarse, const swa_patchset *fine, int level,
                               int ratio) {
    GridRefs c;
    if (!fine || grid_refs(coarse, &c) != SWA_OK) return 0;
    std::vector<int4> f, a, e, u;
    if (amr::build_maps(c, fine, level, ratio, f, a, e, u) != SWA_OK) return 0;
    return amr::layout_of(f.size(), a.size(), e.size(), u.size(), ratio).total;
}

int swa_create_amr(swa_grid *coarse, swa_patchset *fine, int level, int ratio, void *ws,
                   size_t ws_bytes, void *stream, swa_amr **out) {
    GridRefs c;
    if (!fine || !ws || !out) return set_error(SWA_EINVAL, "null argument");
    TRY(grid_refs(coarse, &c));
    if (((uintptr_t)ws & 255) != 0) return set_error(SWA_EINVAL, "workspace must be 256-byte aligned");
    std::vector<int4> f, a, e, u;
    TRY(amr::build_maps(c, fine, level, ratio, f, a, e, u));
    if ((long long)e.size() * ratio > 0x7fffffffLL)
        return set_error(SWA_EINVAL, "too many coarse-fine edges for ratio %d", ratio);
    const amr::Layout L = amr::layout_of(f.size(), a.size(), e.size(), u.size(), ratio);
    if (ws_bytes < L.total)
        return set_error(SWA_ENOMEM, "AMR workspace %zu bytes < %zu needed", ws_bytes, L.total);
    swa_amr *A = new (std::nothrow) swa_amr();
    if (!A) return set_error(SWA_ENOMEM, "host allocation failed");
    A->coarse = coarse; A->fine = fine; A->level = level; A->r = ratio;
    char *base = (char *)ws;
    A->fill = (int4 *)(base + L.fill);
    A->avg = (int4 *)(base + L.avg);
    A->cf = (int4 *)(base + L.cf);
    A->cfu = (int4 *)(base + L.cfu);
    A->dh = (double *)(base + L.dh);
    A->dhf = (double *)(base + L.dhf);
    A->nfill = (int)f.size();
    A->navg = (int)a.size();
    A->ncf = (int)e.size();
    A->ncfu = (int)u.size();
    cudaStream_t st = (cudaStream_t)stream;
    int rc = SWA_OK;
    const std::vector<int4> *src[4] = {&f, &a, &e, &u};
    int4 *dst[4] = {A->fill, A->avg, A->cf, A->cfu};
    const char *what[4] = {"AMR fill map upload", "AMR average map upload",
                           "AMR edge map upload", "AMR edge group upload"};
    for (int k = 0; k < 4 && rc == SWA_OK; k++)
        if (!src[k]->empty())
            rc = cuda_check(cudaMemcpyAsync(dst[k], src[k]->data(), sizeof(int4) * src[k]->size(),
                                            cudaMemcpyHostToDevice, st), what[k]);
    if (rc == SWA_OK) rc = cuda_check(cudaStreamSynchronize(st), "create_amr");
    if (rc != SWA_OK) { delete A; return rc; }
    *out = A;
    return SWA_OK;
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

int swa_amr_info(const swa_amr *A, int *nfill, int *navg, int *nedges) {
    if (!A) return set_error(SWA_EINVAL, "null AMR hierarchy");
    if (nfill) *nfill = A->nfill;
    if (navg) *navg = A->navg;
    if (nedges) *nedges = A->ncf;
    return SWA_OK;
}

int swa_amr_step(swa_amr *A, double t_n, double dt_c, int max_launches, void *stream) {
    if (!A) return set_error(SWA_EINVAL, "null AMR hierarchy");
    if (!(dt_c > 0.0)) return set_error(SWA_EINVAL, "dt_c must be > 0");
    if (max_launches < 1) return set_error(SWA_EINVAL, "max_launches must be >= 1");
    GridRefs c;
    TRY(grid_refs(A->coarse, &c));
    if (!c.state_set) return set_error(SWA_ESTATE, "coarse state not set");
    if (!A->fine->lev[A->level].started) return set_error(SWA_ESTATE, "fine level not started");
    const bool reflux = A->reflux && A->ncf > 0;
    if (reflux && c.scheme != SWA_SCHEME_SPLIT)
        return set_error(SWA_EINVAL, "refluxing needs the split scheme on the coarse grid");
    cudaStream_t st = (cudaStream_t)stream;
    amr::AmrParams p{};
    p.table = A->fine->table;
    p.lclk = A->fine->lev[A->level].clk;
    p.cclk = c.clk;
    for (int b = 0; b < 2; b++)
        for (int k = 0; k < 3; k++) p.cq[b][k] = (float *)c.q[b][k];
    p.nxc = c.d.nx; p.nyc = c.d.ny; p.r = A->r;
    p.fill = A->fill; p.nfill = A->nfill;
    p.avg = A->avg; p.navg = A->navg;
    p.t_n = t_n; p.dt_c = dt_c; p.t_end = t_n + dt_c;
    p.err = swadj_host::error_word();
    amr::RefluxParams q{};
    q.cclk = c.clk;
    for (int b = 0; b < 2; b++)
        for (int k = 0; k < 3; k++) q.cq[b][k] = p.cq[b][k];
    q.chb = (const float *)c.bath;
    q.nxc = c.d.nx; q.nyc = c.d.ny; q.r = A->r;
    q.cbc = BcSpec{c.d.bc[0], c.d.bc[1], c.d.bc[2], c.d.bc[3]};
    q.dxc = c.d.dx; q.dyc = c.d.dy;
    q.nxc_d = (double)(float)c.d.dx; q.nyc_d = (double)(float)c.d.dy;
    q.g = (float)c.d.g; q.order = c.d.order;
    q.cf = A->cf; q.ncf = A->ncf; q.dh = A->dh; q.dhf = A->dhf;
    q.t_end = p.t_end;
    patches::LevelReflux rf{};
    if (reflux) {
        rf.cf = A->cf; rf.dhf = A->dhf; rf.nitems = A->ncf * A->r; rf.r = A->r;
        rf.dxc = c.d.dx; rf.dyc = c.d.dy;
        p.cfu = A->cfu; p.ncfu = A->ncfu; p.dh = A->dh; p.dhf = A->dhf;
    }
    const unsigned fb = ew_blocks((size_t)3 * (A->nfill > 0 ? A->nfill : 1));
    const size_t navg_items = (size_t)3 * A->navg + (size_t)p.ncfu;
    const unsigned ab = ew_blocks(navg_items > 0 ? navg_items : 1);
    if (reflux) {
        const unsigned eb = (unsigned)((A->ncf + 31) / 32);   // 8 edges per warp, 4 warps
        amr::reflux_coarse_kernel<<<eb, 128, 0, st>>>(q);
        TRY(cuda_check(cudaGetLastError(), "reflux_coarse_kernel"));
    }
    TRY(swa_step_forward(A->coarse, 1, p.t_end, stream));
    for (int k = 1; k <= A->r; k++) {
        const double t_k = k == A->r ? p.t_end : t_n + dt_c * (double)k / (double)A->r;
        for (int j = 0; j < max_launches; j++) {
            amr::amr_fill_kernel<<<fb, 256, 0, st>>>(p);
            TRY(cuda_check(cudaGetLastError(), "amr_fill_kernel"));
            TRY(level_launch(A->fine, A->level, 1, t_k, rf, st));
        }
    }
    switch (A->r) {
        case 1: amr::amr_avg_kernel<1><<<ab, 256, 0, st>>>(p); break;
        case 2: amr::amr_avg_kernel<2><<<ab, 256, 0, st>>>(p); break;
        case 4: amr::amr_avg_kernel<4><<<ab, 256, 0, st>>>(p); break;
        case 8: amr::amr_avg_kernel<8><<<ab, 256, 0, st>>>(p); break;
        default: amr::amr_avg_kernel<0><<<ab, 256, 0, st>>>(p); break;
    }
    TRY(cuda_check(cudaGetLastError(), "amr_avg_kernel"));
    return SWA_OK;
}

}  // extern "C"
