// api.cu -- the extern "C" boundary of libswadj.so (declared in swadj.h).
//
// Host-side bookkeeping only: argument checks, workspace carving, stream-
// ordered copies and kernel launches.  Every arithmetic step of the method
// runs in the kernels of fwd.cu, adj.cu and flag.cu (plus the elementwise
// conversion kernels below).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "adj.cuh"
#include "flag.cuh"
#include "fwd.cuh"
#include "swadj_internal.cuh"

using namespace swadj;

// ------------------------------------------------------------------ errors
namespace swadj_host {
static thread_local char g_msg[512];

int set_error(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_check(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return SWA_OK;
    return set_error(SWA_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}
}  // namespace swadj_host

using swadj_host::cuda_check;
using swadj_host::set_error;

// Device error word shared by every object on a device (ERR_* bits).  Kernels
// in other translation units receive its address through their parameters.
__device__ int g_swa_err;

static int *err_word() {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_swa_err) != cudaSuccess) return nullptr;
    return (int *)p;
}

int *swadj_host::error_word() { return err_word(); }

#define TRY(x)                      \
    do {                            \
        int _rc = (x);              \
        if (_rc != SWA_OK) return _rc; \
    } while (0)

static cudaStream_t S(void *s) { return (cudaStream_t)s; }

// Bump allocator over a caller-provided workspace (or a size query if base is
// NULL).  Every array starts on a 256-byte boundary.
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

static int check_desc(const swa_grid_desc *d) {
    if (!d) return set_error(SWA_EINVAL, "null grid descriptor");
    if (d->ndim != 1 && d->ndim != 2) return set_error(SWA_EINVAL, "ndim must be 1 or 2");
    if (d->nx < 1 || d->ny < 1) return set_error(SWA_EINVAL, "nx, ny must be >= 1");
    if (d->ndim == 1 && d->ny != 1) return set_error(SWA_EINVAL, "ndim = 1 needs ny = 1");
    if (d->ndim == 2 && (d->nx < 2 || d->ny < 2))
        return set_error(SWA_EINVAL, "2D grids need nx, ny >= 2");
    if (d->ndim == 1 && d->nx < 2) return set_error(SWA_EINVAL, "1D grids need nx >= 2");
    if (!(d->dx > 0) || !(d->dy > 0)) return set_error(SWA_EINVAL, "dx, dy must be > 0");
    if (d->precision != SWA_FP64 && d->precision != SWA_FP32)
        return set_error(SWA_EINVAL, "precision must be SWA_FP64 or SWA_FP32");
    if (d->order != 1 && d->order != 2) return set_error(SWA_EINVAL, "order must be 1 or 2");
    for (int k = 0; k < 4; k++)
        if (d->bc[k] != SWA_BC_EXTRAP && d->bc[k] != SWA_BC_WALL)
            return set_error(SWA_EINVAL, "bc[%d] must be SWA_BC_EXTRAP or SWA_BC_WALL", k);
    if (!(d->g > 0) || !(d->cfl > 0) || !(d->cfl <= 1.0) || !(d->dry_tol >= 0))
        return set_error(SWA_EINVAL, "need g > 0, 0 < cfl <= 1, dry_tol >= 0");
    if ((double)d->nx * d->ny > 2.0e9) return set_error(SWA_EINVAL, "grid too large");
    return SWA_OK;
}

// -------------------------------------------------------- conversion kernels
// mode for conv_in: 0 dst = src; 1 dst = src - Bd (h from eta, double);
//                   2 dst = -src (hbar from B)
template <typename R>
__global__ void conv_in_kernel(const double *src, R *dst, const double *Bd, int mode,
                               size_t n) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x) {
        double v = src[k];
        if (mode == 1) v = v - Bd[k];
        else if (mode == 2) v = -v;
        dst[k] = (R)v;
    }
}

// mode for conv_out: 0 dst = src; 1 dst = src + bath (double B or float hbar)
template <typename R>
__global__ void conv_out_kernel(const R *src, const R *bath, double *dst, int mode,
                                size_t n) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x) {
        double v = (double)src[k];
        if (mode == 1) v = v + (double)bath[k];
        dst[k] = v;
    }
}

__global__ void fill_zero_f64(double *p, size_t n) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x)
        p[k] = 0.0;
}

// wet = coefficient above `thr` (double adjoints store hbar, thr = dry_tol;
// float adjoints store c, 0 where dry, thr = 0)
template <typename R>
__global__ void wet_mask_kernel(const R *c, R thr, uint8_t *wet, size_t n) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x)
        wet[k] = c[k] > thr ? 1 : 0;
}

static unsigned ew_blocks(size_t n) {
    size_t b = (n + 255) / 256;
    return (unsigned)(b > 4096 ? 4096 : (b < 1 ? 1 : b));
}

template <typename R>
static int conv_in(const double *src, R *dst, const double *Bd, int mode, size_t n,
                   cudaStream_t st) {
    conv_in_kernel<R><<<ew_blocks(n), 256, 0, st>>>(src, dst, Bd, mode, n);
    return cuda_check(cudaGetLastError(), "conv_in_kernel");
}

template <typename R>
static int conv_out(const R *src, const R *bath, double *dst, int mode, size_t n,
                    cudaStream_t st) {
    conv_out_kernel<R><<<ew_blocks(n), 256, 0, st>>>(src, bath, dst, mode, n);
    return cuda_check(cudaGetLastError(), "conv_out_kernel");
}

// ------------------------------------------------------------------- grid
struct swa_grid {
    swa_grid_desc d;
    size_t n;
    size_t esz;            // 8 (FP64) or 4 (FP32)
    void *q[2][3];
    void *bath;            // B (FP64) or hbar (FP32)
    double *Bd;            // FP64 B (FP64 grids only; equals bath)
    double *staging;       // n doubles
    DevClock *clk;
    double *partial;
    int step_blocks;
    int state_set;
    int strip_rows;        // FP32 launch shape (0 = default)
    int keep_rest;         // FP32 2D: compute wave-free rows in full
    int scheme;            // 2D update: SWA_SCHEME_SPLIT or SWA_SCHEME_CTU
    int wetdry;            // split step with the shore solver (dry cells allowed)
    long long *gauge_row;  // device row counter of the fused gauge recording
    GaugeRec gauges;       // fused gauge recording (n = 0: off)
    float *rest_tab;       // FP32 2D: rest CFL table of the step's quiet units
    unsigned char *umap;   // FP32 2D: units that have had waves (quiet-unit hint)
    int umap_n;
};

static int grid_step_blocks(const swa_grid_desc *d) {
    if (d->precision == SWA_FP64) {
        FwdParams<double> p{};
        p.nx = d->nx; p.ny = d->ny; p.two_d = d->ndim == 2;
        return fwd_step_blocks<double>(p);
    }
    FwdParams<float> p{};
    p.nx = d->nx; p.ny = d->ny; p.two_d = d->ndim == 2;
    return fwd_step_blocks<float>(p);
}

// Reduction slots for the smallest strip height the FP32 kernel accepts, or
// for the unsplit step's tiles if there are more of those.
static int grid_max_blocks(const swa_grid_desc *d) {
    int b = grid_step_blocks(d);
    int w;
    if (d->precision == SWA_FP32) {
        FwdParams<float> p{};
        p.nx = d->nx; p.ny = d->ny; p.two_d = d->ndim == 2;
        w = fwd_wd_blocks<float>(p);
    } else {
        FwdParams<double> p{};
        p.nx = d->nx; p.ny = d->ny; p.two_d = d->ndim == 2;
        w = fwd_wd_blocks<double>(p);
    }
    if (w > b) b = w;
    if (d->ndim != 2) return b;
    int c;
    if (d->precision == SWA_FP32) {
        FwdParams<float> p{};
        p.nx = d->nx; p.ny = d->ny; p.two_d = 1; p.fwd_rows = SWA_MIN_STRIP_ROWS;
        if (fwd_step_blocks<float>(p) > b) b = fwd_step_blocks<float>(p);
        c = fwd_ctu_blocks<float>(p);
    } else {
        FwdParams<double> p{};
        p.nx = d->nx; p.ny = d->ny; p.two_d = 1;
        c = fwd_ctu_blocks<double>(p);
    }
    return b > c ? b : c;
}

static void grid_layout(const swa_grid_desc *d, Carve &c, swa_grid *g) {
    const size_t n = (size_t)d->nx * d->ny;
    const size_t esz = d->precision == SWA_FP64 ? 8 : 4;
    void *q[2][3];
    for (int b = 0; b < 2; b++)
        for (int k = 0; k < 3; k++) q[b][k] = c.take(n * esz);
    void *bath = c.take(n * esz);
    double *staging = (double *)c.take(n * 8);
    DevClock *clk = (DevClock *)c.take(sizeof(DevClock));
    long long *grow = (long long *)c.take(sizeof(long long));
    int blocks = grid_max_blocks(d);
    if (blocks < kInitBlocks) blocks = kInitBlocks;
    double *partial = (double *)c.take((size_t)blocks * 8);
    float *rest_tab = nullptr;
    unsigned char *umap = nullptr;
    int umap_n = 0;
    if (d->precision == SWA_FP32 && d->ndim == 2) {
        rest_tab = (float *)c.take(fwd_f32_rest_table_floats(d->nx, d->ny) * sizeof(float));
        umap_n = fwd_f32_unit_map_bytes(d->nx, d->ny);
        umap = (unsigned char *)c.take((size_t)umap_n);
    }
    if (g) {
        g->rest_tab = rest_tab;
        g->umap = umap;
        g->umap_n = umap_n;
        for (int b = 0; b < 2; b++)
            for (int k = 0; k < 3; k++) g->q[b][k] = q[b][k];
        g->bath = bath;
        g->staging = staging;
        g->clk = clk;
        g->partial = partial;
        g->step_blocks = grid_step_blocks(d);
        g->gauge_row = grow;
    }
}

int swadj::grid_refs(const swa_grid *g, GridRefs *out) {
    if (!g || !out) return set_error(SWA_EINVAL, "null grid");
    out->d = g->d;
    for (int b = 0; b < 2; b++)
        for (int k = 0; k < 3; k++) out->q[b][k] = g->q[b][k];
    out->bath = g->bath;
    out->clk = g->clk;
    out->state_set = g->state_set;
    out->scheme = g->scheme;
    return SWA_OK;
}

template <typename R>
static FwdParams<R> fwd_params(const swa_grid *g, double t_end) {
    FwdParams<R> p{};
    p.nx = g->d.nx; p.ny = g->d.ny; p.two_d = g->d.ndim == 2; p.order = g->d.order;
    p.bc = BcSpec{g->d.bc[0], g->d.bc[1], g->d.bc[2], g->d.bc[3]};
    p.dx = (R)g->d.dx; p.dy = (R)g->d.dy; p.g = (R)g->d.g;
    p.cfl = g->d.cfl; p.t_end = t_end;
    for (int b = 0; b < 2; b++)
        for (int k = 0; k < 3; k++) p.q[b][k] = (R *)g->q[b][k];
    p.bath = (const R *)g->bath;
    p.clk = g->clk;
    p.partial = g->partial;
    p.nblocks = g->step_blocks;
    p.err = err_word();
    p.fwd_rows = g->strip_rows;
    p.keep_rest = g->keep_rest;
    p.rest_tab = g->rest_tab;
    p.umap = g->umap;
    p.umap_n = g->umap_n;
    p.gauges = g->gauges;
    p.wetdry = g->wetdry;
    p.dry_tol = (R)g->d.dry_tol;
    return p;
}

extern "C" {

const char *swa_version(void) { return "swadj 0.1 (sm_103a)"; }

const char *swa_last_error(void) { return swadj_host::g_msg; }

int swa_sync_status(void *stream) {
    cudaStream_t st = S(stream);
    TRY(cuda_check(cudaStreamSynchronize(st), "stream synchronize"));
    int err = 0, zero = 0;
    TRY(cuda_check(cudaMemcpyFromSymbolAsync(&err, g_swa_err, sizeof(int), 0,
                                             cudaMemcpyDeviceToHost, st), "error word read"));
    TRY(cuda_check(cudaMemcpyToSymbolAsync(g_swa_err, &zero, sizeof(int), 0,
                                           cudaMemcpyHostToDevice, st), "error word clear"));
    TRY(cuda_check(cudaStreamSynchronize(st), "error word"));
    if (err & ERR_UNSTABLE)
        return set_error(SWA_EUNSTABLE, "device saw a non-finite state or depth <= 0");
    if (err & ERR_LAG)
        return set_error(SWA_ESTATE, "an AMR step ended before its levels reached its end time");
    return SWA_OK;
}

size_t swa_grid_workspace_bytes(const swa_grid_desc *desc) {
    if (check_desc(desc) != SWA_OK) return 0;
    Carve c(nullptr);
    grid_layout(desc, c, nullptr);
    return c.off + 256;
}

static int set_state_impl(swa_grid *g, const double *eta, const double *hu, const double *hv,
                          double t, int where, void *stream, bool check);

int swa_create_grid(const swa_grid_desc *desc, const double *bathy_host, void *ws,
                    size_t ws_bytes, void *stream, swa_grid **out) {
    TRY(check_desc(desc));
    if (!bathy_host || !ws || !out) return set_error(SWA_EINVAL, "null argument");
    if (((uintptr_t)ws & 255) != 0) return set_error(SWA_EINVAL, "workspace must be 256-byte aligned");
    const size_t need = swa_grid_workspace_bytes(desc);
    if (ws_bytes < need)
        return set_error(SWA_ENOMEM, "grid workspace %zu bytes < %zu needed", ws_bytes, need);
    swa_grid *g = new (std::nothrow) swa_grid();
    if (!g) return set_error(SWA_ENOMEM, "host allocation failed");
    g->d = *desc;
    g->n = (size_t)desc->nx * desc->ny;
    g->esz = desc->precision == SWA_FP64 ? 8 : 4;
    Carve c(ws);
    grid_layout(desc, c, g);
    cudaStream_t st = S(stream);
    int rc = cuda_check(cudaMemsetAsync(ws, 0, need - 256, st), "workspace clear");
    if (rc == SWA_OK)
        rc = cuda_check(cudaMemcpyAsync(g->staging, bathy_host, g->n * 8,
                                        cudaMemcpyHostToDevice, st), "bathymetry upload");
    if (rc == SWA_OK) {
        if (desc->precision == SWA_FP64) {
            rc = cuda_check(cudaMemcpyAsync(g->bath, g->staging, g->n * 8,
                                            cudaMemcpyDeviceToDevice, st), "bathymetry copy");
            g->Bd = (double *)g->bath;
        } else {
            rc = conv_in<float>(g->staging, (float *)g->bath, nullptr, 2, g->n, st);
            g->Bd = nullptr;
            if (rc == SWA_OK && g->rest_tab)
                rc = fwd_f32_rest_table(fwd_params<float>(g, 0.0), g->rest_tab, st);
        }
    }
    // ocean at rest until swa_set_state: surface 0, no momentum
    if (rc == SWA_OK) {
        fill_zero_f64<<<ew_blocks(g->n), 256, 0, st>>>(g->staging, g->n);
        rc = cuda_check(cudaGetLastError(), "fill_zero");
    }
    if (rc == SWA_OK) rc = cuda_check(cudaStreamSynchronize(st), "create_grid");
    if (rc != SWA_OK) { delete g; return rc; }
    *out = g;
    rc = set_state_impl(g, g->staging, g->staging, g->staging, 0.0, SWA_DEVICE, stream, false);
    if (rc != SWA_OK) { delete g; *out = nullptr; return rc; }
    return SWA_OK;
}

int swa_destroy_grid(swa_grid *grid) {
    delete grid;
    return SWA_OK;
}

// check = false: the ocean at rest a new grid starts from, whose land cells
// (if any) have no valid depth yet, reports nothing to the error word.
static int set_state_impl(swa_grid *g, const double *eta, const double *hu, const double *hv,
                          double t, int where, void *stream, bool check) {
    if (!g || !eta || !hu) return set_error(SWA_EINVAL, "null argument");
    if (g->d.ndim == 2 && !hv) return set_error(SWA_EINVAL, "hv required for 2D grids");
    if (where != SWA_HOST && where != SWA_DEVICE) return set_error(SWA_EINVAL, "bad where");
    cudaStream_t st = S(stream);
    const double *src[3] = {eta, hu, hv};
    const int nf = g->d.ndim == 2 ? 3 : 2;
    for (int k = 0; k < nf; k++) {
        const double *s = src[k];
        if (where == SWA_HOST) {
            TRY(cuda_check(cudaMemcpyAsync(g->staging, s, g->n * 8, cudaMemcpyHostToDevice, st),
                           "state upload"));
            s = g->staging;
        }
        if (g->d.precision == SWA_FP64)
            TRY(conv_in<double>(s, (double *)g->q[0][k], g->Bd, k == 0 ? 1 : 0, g->n, st));
        else
            TRY(conv_in<float>(s, (float *)g->q[0][k], nullptr, 0, g->n, st));
    }
    if (nf == 2) {
        TRY(cuda_check(cudaMemsetAsync(g->q[0][2], 0, g->n * g->esz, st), "hv clear"));
    }
    TRY(cuda_check(cudaMemsetAsync(g->q[1][2], 0, g->n * g->esz, st), "hv clear"));
    if (g->d.precision == SWA_FP64) {
        FwdParams<double> p = fwd_params<double>(g, 0.0);
        if (!check) p.err = nullptr;
        TRY(fwd_launch_clock_init<double>(p, t, st));
    } else {
        FwdParams<float> p = fwd_params<float>(g, 0.0);
        if (!check) p.err = nullptr;
        TRY(fwd_launch_clock_init<float>(p, t, st));
    }
    g->state_set = 1;
    return SWA_OK;
}

int swa_set_state(swa_grid *g, const double *eta, const double *hu, const double *hv,
                  double t, int where, void *stream) {
    return set_state_impl(g, eta, hu, hv, t, where, stream, true);
}

int swa_get_state(swa_grid *g, double *h, double *hu, double *hv, double *eta, int where,
                  void *stream) {
    if (!g) return set_error(SWA_EINVAL, "null grid");
    if (where != SWA_HOST && where != SWA_DEVICE) return set_error(SWA_EINVAL, "bad where");
    cudaStream_t st = S(stream);
    DevClock clk;
    TRY(cuda_check(cudaMemcpyAsync(&clk, g->clk, sizeof(clk), cudaMemcpyDeviceToHost, st),
                   "clock read"));
    TRY(cuda_check(cudaStreamSynchronize(st), "clock read"));
    const int cur = clk.cur;
    double *dst[4] = {h, hu, hv, eta};
    for (int k = 0; k < 4; k++) {
        if (!dst[k]) continue;
        if (k == 2 && g->d.ndim == 1) {
            if (where == SWA_HOST) memset(dst[k], 0, g->n * 8);
            else TRY(cuda_check(cudaMemsetAsync(dst[k], 0, g->n * 8, st), "hv clear"));
            continue;
        }
        double *d = where == SWA_HOST ? g->staging : dst[k];
        const int field = k == 3 ? 0 : k;
        int mode = 0;
        if (g->d.precision == SWA_FP64) {
            mode = (k == 3) ? 1 : 0;  // eta = h + B
            TRY(conv_out<double>((const double *)g->q[cur][field], (const double *)g->bath, d,
                                 mode, g->n, st));
        } else {
            mode = (k == 0) ? 1 : 0;  // h = eta + hbar
            TRY(conv_out<float>((const float *)g->q[cur][field], (const float *)g->bath, d,
                                mode, g->n, st));
        }
        if (where == SWA_HOST) {
            TRY(cuda_check(cudaMemcpyAsync(dst[k], g->staging, g->n * 8,
                                           cudaMemcpyDeviceToHost, st), "state download"));
            TRY(cuda_check(cudaStreamSynchronize(st), "state download"));
        }
    }
    return SWA_OK;
}

int swa_step_forward(swa_grid *g, int max_steps, double t_end, void *stream) {
    if (!g) return set_error(SWA_EINVAL, "null grid");
    if (max_steps < 0) return set_error(SWA_EINVAL, "max_steps < 0");
    if (!g->state_set) return set_error(SWA_ESTATE, "state not set");
    cudaStream_t st = S(stream);
    const bool ctu = g->scheme == SWA_SCHEME_CTU && g->d.ndim == 2;
    if (ctu && g->wetdry)
        return set_error(SWA_EINVAL, "the wet/dry option needs the split scheme");
    if (g->d.precision == SWA_FP64) {
        const FwdParams<double> p = fwd_params<double>(g, t_end);
        for (int k = 0; k < max_steps; k++)
            TRY(ctu ? fwd_launch_ctu<double>(p, st)
                    : g->wetdry ? fwd_launch_wd<double>(p, st) : fwd_launch_step<double>(p, st));
    } else {
        const FwdParams<float> p = fwd_params<float>(g, t_end);
        for (int k = 0; k < max_steps; k++)
            TRY(ctu ? fwd_launch_ctu<float>(p, st)
                    : g->wetdry ? fwd_launch_wd<float>(p, st) : fwd_launch_step<float>(p, st));
    }
    return SWA_OK;
}

int swa_get_time(swa_grid *g, double *t, double *dt_next, long long *nsteps, void *stream) {
    if (!g) return set_error(SWA_EINVAL, "null grid");
    DevClock clk;
    TRY(cuda_check(cudaMemcpyAsync(&clk, g->clk, sizeof(clk), cudaMemcpyDeviceToHost,
                                   S(stream)), "clock read"));
    TRY(cuda_check(cudaStreamSynchronize(S(stream)), "clock read"));
    if (t) *t = clk.t;
    if (dt_next) *dt_next = clk.dt_cfl;
    if (nsteps) *nsteps = clk.nsteps;
    return SWA_OK;
}

int swa_grid_set_strip_rows(swa_grid *g, int rows) {
    if (!g) return set_error(SWA_EINVAL, "null grid");
    if (rows != 0 && rows != 16 && rows != 32 && rows != 64)
        return set_error(SWA_EINVAL, "strip rows must be 0, 16, 32 or 64");
    g->strip_rows = rows;
    return SWA_OK;
}

int swa_grid_set_rest_skip(swa_grid *g, int on) {
    if (!g) return set_error(SWA_EINVAL, "null grid");
    if (on != 0 && on != 1) return set_error(SWA_EINVAL, "rest skip must be 0 or 1");
    g->keep_rest = !on;
    return SWA_OK;
}

int swa_grid_set_wetdry(swa_grid *g, int on) {
    if (!g) return set_error(SWA_EINVAL, "null grid");
    if (on != 0 && on != 1) return set_error(SWA_EINVAL, "wet/dry must be 0 or 1");
    g->wetdry = on;
    return SWA_OK;
}

int swa_grid_set_scheme(swa_grid *g, int scheme) {
    if (!g) return set_error(SWA_EINVAL, "null grid");
    if (scheme != SWA_SCHEME_SPLIT && scheme != SWA_SCHEME_CTU)
        return set_error(SWA_EINVAL, "scheme must be SWA_SCHEME_SPLIT or SWA_SCHEME_CTU");
    g->scheme = scheme;
    return SWA_OK;
}

int swa_grid_arrays(swa_grid *g, const void **q0, const void **q1, const void **q2,
                    const void **bath, void *stream) {
    if (!g) return set_error(SWA_EINVAL, "null grid");
    DevClock clk;
    TRY(cuda_check(cudaMemcpyAsync(&clk, g->clk, sizeof(clk), cudaMemcpyDeviceToHost,
                                   S(stream)), "clock read"));
    TRY(cuda_check(cudaStreamSynchronize(S(stream)), "clock read"));
    if (q0) *q0 = g->q[clk.cur][0];
    if (q1) *q1 = g->q[clk.cur][1];
    if (q2) *q2 = g->q[clk.cur][2];
    if (bath) *bath = g->bath;
    return SWA_OK;
}

}  // extern "C"

// ----------------------------------------------------------------- adjoint
struct swa_adjoint {
    swa_grid_desc d;
    size_t n;
    size_t esz;
    int nc;
    void *q[2][3];
    void *c;
    double *staging;
    double *smax_dev;
    long long N;
    double dt;
    long long steps_done;
    int cur;
    int steps_per_pass;   // FP32 2D: 1 or 2 adjoint steps per launch
    int all_wet;          // no cell with hbar <= dry_tol (no wall edges)
    double t_f;
    unsigned char *umap;  // FP32 2D: units that have had a nonzero value (quiet-unit hint)
    int umap_n;
};

static void adj_layout(const swa_grid_desc *d, Carve &c, swa_adjoint *a) {
    const size_t n = (size_t)d->nx * d->ny;
    const size_t esz = d->precision == SWA_FP64 ? 8 : 4;
    void *q[2][3];
    for (int b = 0; b < 2; b++)
        for (int k = 0; k < 3; k++) q[b][k] = c.take(n * esz);
    void *cc = c.take(n * esz);
    double *staging = (double *)c.take(n * 8);
    double *smax = (double *)c.take(8);
    unsigned char *umap = nullptr;
    int umap_n = 0;
    if (d->precision == SWA_FP32 && d->ndim == 2) {
        umap_n = adj_f32_unit_map_bytes(d->nx, d->ny);
        umap = (unsigned char *)c.take((size_t)umap_n);
    }
    if (a) {
        for (int b = 0; b < 2; b++)
            for (int k = 0; k < 3; k++) a->q[b][k] = q[b][k];
        a->umap = umap;
        a->umap_n = umap_n;
        a->c = cc;
        a->staging = staging;
        a->smax_dev = smax;
    }
}

template <typename R>
static AdjParams<R> adj_params(const swa_adjoint *a) {
    AdjParams<R> p{};
    p.nx = a->d.nx; p.ny = a->d.ny; p.two_d = a->d.ndim == 2; p.order = a->d.order;
    p.bc = BcSpec{a->d.bc[0], a->d.bc[1], a->d.bc[2], a->d.bc[3]};
    p.nux = (R)(a->dt / a->d.dx);
    p.nuy = (R)(a->dt / a->d.dy);
    p.g = (R)a->d.g;
    p.dry_tol = (R)a->d.dry_tol;
    for (int k = 0; k < 3; k++) {
        p.src[k] = (const R *)a->q[a->cur][k];
        p.dst[k] = (R *)a->q[a->cur ^ 1][k];
    }
    p.c = (const R *)a->c;
    p.all_wet = a->all_wet;
    p.umap = a->umap;
    p.umap_n = a->umap_n;
    return p;
}

// ---------------------------------------------------------------- snapshots
struct swa_snapstore {
    const swa_adjoint *adj;
    int prec;
    int max_snaps;
    int count;
    size_t na;
    int nc;
    void *data;
    double *tau_dev;
    uint8_t *wet;
    float *env;   // snapshot envelope (FP32 2D stores with nx % 4 == 0), else null
    std::vector<double> tau_host;
};

// FP32 snapshots of a 2D grid whose rows split into quads of 4 cells carry an
// envelope: per group of kEnvGroup snapshots and per quad, the maximum
// |component| of each component, which lets the flag pass skip groups.
static bool snap_has_env(const swa_grid_desc *d, int prec) {
    return prec == SWA_FP32 && d->ndim == 2 && d->nx % 4 == 0;
}

static void snap_layout(const swa_grid_desc *d, int max_snaps, int prec, Carve &c,
                        swa_snapstore *s) {
    const size_t na = (size_t)d->nx * d->ny;
    const int nc = d->ndim + 1;
    const size_t esz = prec == SWA_FP64 ? 8 : 4;
    void *data = c.take((size_t)max_snaps * nc * na * esz);
    double *tau = (double *)c.take((size_t)max_snaps * 8);
    uint8_t *wet = (uint8_t *)c.take(na);
    float *env = nullptr;
    if (snap_has_env(d, prec)) {
        const size_t groups = (size_t)(max_snaps + kEnvGroup - 1) / kEnvGroup;
        env = (float *)c.take(groups * 3 * (na / 4) * sizeof(float));
    }
    if (s) { s->data = data; s->tau_dev = tau; s->wet = wet; s->env = env; }
}

// Fold snapshot slot k (just written on stream st) into its envelope group.
static int env_fold(swa_snapstore *s, int k, cudaStream_t st) {
    if (!s->env) return SWA_OK;
    const float *slot = (const float *)s->data + (size_t)k * s->nc * s->na;
    float *grp = s->env + (size_t)(k / kEnvGroup) * 3 * (s->na / 4);
    return env_launch_update(slot, s->na, grp, k % kEnvGroup == 0, st);
}

static int store_into(swa_adjoint *a, swa_snapstore *s, cudaStream_t st) {
    if (s->count >= s->max_snaps)
        return set_error(SWA_ENOMEM, "snapshot store full (%d)", s->max_snaps);
    const double tau = a->t_f - (double)a->steps_done * a->dt;
    const size_t esz = s->prec == SWA_FP64 ? 8 : 4;
    char *slot = (char *)s->data + (size_t)s->count * s->nc * s->na * esz;
    float *sf = s->prec == SWA_FP32 ? (float *)slot : nullptr;
    double *sd = s->prec == SWA_FP64 ? (double *)slot : nullptr;
    if (a->d.precision == SWA_FP64) {
        const double *src[3] = {(const double *)a->q[a->cur][0], (const double *)a->q[a->cur][1],
                                (const double *)a->q[a->cur][2]};
        TRY(adj_launch_store<double>(src, a->nc, a->n, sf, sd, a->n, s->tau_dev + s->count, tau, st));
    } else {
        const float *src[3] = {(const float *)a->q[a->cur][0], (const float *)a->q[a->cur][1],
                               (const float *)a->q[a->cur][2]};
        TRY(adj_launch_store<float>(src, a->nc, a->n, sf, sd, a->n, s->tau_dev + s->count, tau, st));
    }
    TRY(env_fold(s, s->count, st));
    s->tau_host.push_back(tau);
    s->count++;
    return SWA_OK;
}

// ns (1 or 2) adjoint steps in one launch; s: store a snapshot of the state
// after them.
static int adj_steps(swa_adjoint *a, swa_snapstore *s, int ns, cudaStream_t st) {
    double tau = 0.0;
    float *sf = nullptr;
    double *sd = nullptr;
    if (s) {
        if (s->count >= s->max_snaps)
            return set_error(SWA_ENOMEM, "snapshot store full (%d)", s->max_snaps);
        tau = a->t_f - (double)(a->steps_done + ns) * a->dt;
        const size_t esz = s->prec == SWA_FP64 ? 8 : 4;
        char *slot = (char *)s->data + (size_t)s->count * s->nc * s->na * esz;
        if (s->prec == SWA_FP32) sf = (float *)slot;
        else sd = (double *)slot;
    }
    if (a->d.precision == SWA_FP64) {
        AdjParams<double> p = adj_params<double>(a);
        p.snap_f = sf; p.snap_d = sd; p.snap_comp_stride = a->n;
        p.tau_dev = s ? s->tau_dev + s->count : nullptr;
        p.tau_val = tau;
        TRY(adj_launch_step<double>(p, st));
    } else {
        AdjParams<float> p = adj_params<float>(a);
        p.snap_f = sf; p.snap_d = sd; p.snap_comp_stride = a->n;
        p.tau_dev = s ? s->tau_dev + s->count : nullptr;
        p.tau_val = tau;
        p.two_steps = ns == 2;
        TRY(adj_launch_step<float>(p, st));
    }
    if (s) TRY(env_fold(s, s->count, st));
    a->cur ^= 1;
    a->steps_done += ns;
    if (s) { s->tau_host.push_back(tau); s->count++; }
    return SWA_OK;
}

extern "C" {

size_t swa_adjoint_workspace_bytes(const swa_grid_desc *desc) {
    if (check_desc(desc) != SWA_OK) return 0;
    Carve c(nullptr);
    adj_layout(desc, c, nullptr);
    return c.off + 256;
}

int swa_create_adjoint(const swa_grid_desc *desc, const double *bathy_host,
                       const double *phi_host, double t_f, void *ws, size_t ws_bytes,
                       void *stream, swa_adjoint **out) {
    TRY(check_desc(desc));
    if (!bathy_host || !phi_host || !ws || !out) return set_error(SWA_EINVAL, "null argument");
    if (!(t_f > 0)) return set_error(SWA_EINVAL, "t_f must be > 0");
    if (((uintptr_t)ws & 255) != 0) return set_error(SWA_EINVAL, "workspace must be 256-byte aligned");
    const size_t need = swa_adjoint_workspace_bytes(desc);
    if (ws_bytes < need)
        return set_error(SWA_ENOMEM, "adjoint workspace %zu bytes < %zu needed", ws_bytes, need);
    swa_adjoint *a = new (std::nothrow) swa_adjoint();
    if (!a) return set_error(SWA_ENOMEM, "host allocation failed");
    a->d = *desc;
    a->n = (size_t)desc->nx * desc->ny;
    a->esz = desc->precision == SWA_FP64 ? 8 : 4;
    a->nc = desc->ndim + 1;
    a->t_f = t_f;
    // the kernels' dry rule (hbar = max(-B, 0) <= dry_tol) on the host
    a->all_wet = 1;
    for (size_t k = 0; k < a->n && a->all_wet; k++) {
        const double hb = bathy_host[k] < 0.0 ? -bathy_host[k] : 0.0;
        if (!(hb > desc->dry_tol)) a->all_wet = 0;
    }
    Carve c(ws);
    adj_layout(desc, c, a);
    cudaStream_t st = S(stream);
    int rc = cuda_check(cudaMemsetAsync(ws, 0, need - 256, st), "workspace clear");
    if (rc == SWA_OK)
        rc = cuda_check(cudaMemcpyAsync(a->staging, bathy_host, a->n * 8,
                                        cudaMemcpyHostToDevice, st), "bathymetry upload");
    if (rc == SWA_OK) {
        if (desc->precision == SWA_FP64)
            rc = adj_launch_init<double>(a->staging, (double *)a->c, a->n, desc->ndim == 2,
                                         desc->g, desc->dx, desc->dy, desc->dry_tol,
                                         a->smax_dev, st);
        else
            rc = adj_launch_init<float>(a->staging, (float *)a->c, a->n, desc->ndim == 2,
                                        desc->g, desc->dx, desc->dy, desc->dry_tol,
                                        a->smax_dev, st);
    }
    for (int k = 0; k < a->nc && rc == SWA_OK; k++) {
        rc = cuda_check(cudaMemcpyAsync(a->staging, phi_host + (size_t)k * a->n, a->n * 8,
                                        cudaMemcpyHostToDevice, st), "phi upload");
        if (rc != SWA_OK) break;
        if (desc->precision == SWA_FP64)
            rc = conv_in<double>(a->staging, (double *)a->q[0][k], nullptr, 0, a->n, st);
        else
            rc = conv_in<float>(a->staging, (float *)a->q[0][k], nullptr, 0, a->n, st);
    }
    double smax = 0.0;
    if (rc == SWA_OK)
        rc = cuda_check(cudaMemcpyAsync(&smax, a->smax_dev, 8, cudaMemcpyDeviceToHost, st),
                        "smax read");
    if (rc == SWA_OK) rc = cuda_check(cudaStreamSynchronize(st), "create_adjoint");
    if (rc == SWA_OK && !(smax > 0))
        rc = set_error(SWA_EINVAL, "adjoint grid has no wet cell");
    if (rc != SWA_OK) { delete a; return rc; }
    long long N = (long long)ceil(t_f * smax / desc->cfl);
    if (N < 1) N = 1;
    a->N = N;
    a->dt = t_f / (double)N;
    a->steps_done = 0;
    a->cur = 0;
    *out = a;
    return SWA_OK;
}

int swa_destroy_adjoint(swa_adjoint *adj) {
    delete adj;
    return SWA_OK;
}

int swa_adjoint_info(const swa_adjoint *a, long long *n_steps, double *dt,
                     long long *steps_done) {
    if (!a) return set_error(SWA_EINVAL, "null adjoint");
    if (n_steps) *n_steps = a->N;
    if (dt) *dt = a->dt;
    if (steps_done) *steps_done = a->steps_done;
    return SWA_OK;
}

int swa_step_adjoint(swa_adjoint *a, int nsteps, void *stream) {
    if (!a) return set_error(SWA_EINVAL, "null adjoint");
    if (nsteps < 0) return set_error(SWA_EINVAL, "nsteps < 0");
    long long left = a->N - a->steps_done;
    if (nsteps > left) nsteps = (int)left;
    for (int k = 0; k < nsteps;) {
        const int ns = (a->steps_per_pass == 2 && k + 2 <= nsteps) ? 2 : 1;
        TRY(adj_steps(a, nullptr, ns, S(stream)));
        k += ns;
    }
    return SWA_OK;
}

int swa_adjoint_set_steps_per_pass(swa_adjoint *a, int k) {
    if (!a) return set_error(SWA_EINVAL, "null adjoint");
    if (k != 1 && k != 2) return set_error(SWA_EINVAL, "steps per pass must be 1 or 2");
    if (k == 2 && (a->d.precision != SWA_FP32 || a->d.ndim != 2))
        return set_error(SWA_EINVAL, "two steps per pass need a 2D FP32 adjoint");
    a->steps_per_pass = k;
    return SWA_OK;
}

int swa_get_adjoint_state(swa_adjoint *a, double *q, int where, void *stream) {
    if (!a || !q) return set_error(SWA_EINVAL, "null argument");
    cudaStream_t st = S(stream);
    for (int k = 0; k < a->nc; k++) {
        double *d = where == SWA_HOST ? a->staging : q + (size_t)k * a->n;
        if (a->d.precision == SWA_FP64)
            TRY(conv_out<double>((const double *)a->q[a->cur][k], nullptr, d, 0, a->n, st));
        else
            TRY(conv_out<float>((const float *)a->q[a->cur][k], nullptr, d, 0, a->n, st));
        if (where == SWA_HOST) {
            TRY(cuda_check(cudaMemcpyAsync(q + (size_t)k * a->n, a->staging, a->n * 8,
                                           cudaMemcpyDeviceToHost, st), "adjoint download"));
            TRY(cuda_check(cudaStreamSynchronize(st), "adjoint download"));
        }
    }
    return SWA_OK;
}

int swa_set_adjoint_state(swa_adjoint *a, const double *phi, int where, void *stream) {
    if (!a || !phi) return set_error(SWA_EINVAL, "null argument");
    if (where != SWA_HOST && where != SWA_DEVICE) return set_error(SWA_EINVAL, "bad where");
    cudaStream_t st = S(stream);
    for (int k = 0; k < a->nc; k++) {
        const double *src = phi + (size_t)k * a->n;
        if (where == SWA_HOST) {
            TRY(cuda_check(cudaMemcpyAsync(a->staging, src, a->n * 8, cudaMemcpyHostToDevice, st),
                           "phi upload"));
            src = a->staging;
        }
        if (a->d.precision == SWA_FP64)
            TRY(conv_in<double>(src, (double *)a->q[0][k], nullptr, 0, a->n, st));
        else
            TRY(conv_in<float>(src, (float *)a->q[0][k], nullptr, 0, a->n, st));
    }
    if (a->umap)   // a new state: no unit has had a nonzero value yet
        TRY(cuda_check(cudaMemsetAsync(a->umap, 0, (size_t)a->umap_n, st), "unit map clear"));
    a->cur = 0;
    a->steps_done = 0;
    return SWA_OK;
}

size_t swa_snapstore_workspace_bytes(const swa_grid_desc *adj_desc, int max_snaps,
                                     int precision) {
    if (check_desc(adj_desc) != SWA_OK || max_snaps < 1) return 0;
    if (precision != SWA_FP64 && precision != SWA_FP32) return 0;
    Carve c(nullptr);
    snap_layout(adj_desc, max_snaps, precision, c, nullptr);
    return c.off + 256;
}

int swa_create_snapstore(const swa_adjoint *adj, int max_snaps, int precision, void *ws,
                         size_t ws_bytes, swa_snapstore **out) {
    if (!adj || !ws || !out) return set_error(SWA_EINVAL, "null argument");
    if (max_snaps < 1) return set_error(SWA_EINVAL, "max_snaps must be >= 1");
    if (precision != SWA_FP64 && precision != SWA_FP32)
        return set_error(SWA_EINVAL, "bad snapshot precision");
    if (((uintptr_t)ws & 255) != 0) return set_error(SWA_EINVAL, "workspace must be 256-byte aligned");
    const size_t need = swa_snapstore_workspace_bytes(&adj->d, max_snaps, precision);
    if (ws_bytes < need)
        return set_error(SWA_ENOMEM, "snapshot workspace %zu bytes < %zu needed", ws_bytes, need);
    swa_snapstore *s = new (std::nothrow) swa_snapstore();
    if (!s) return set_error(SWA_ENOMEM, "host allocation failed");
    s->adj = adj;
    s->prec = precision;
    s->max_snaps = max_snaps;
    s->count = 0;
    s->na = adj->n;
    s->nc = adj->nc;
    Carve c(ws);
    snap_layout(&adj->d, max_snaps, precision, c, s);
    if (adj->d.precision == SWA_FP64)
        wet_mask_kernel<double><<<ew_blocks(s->na), 256>>>((const double *)adj->c,
                                                           adj->d.dry_tol, s->wet, s->na);
    else
        wet_mask_kernel<float><<<ew_blocks(s->na), 256>>>((const float *)adj->c, 0.0f,
                                                          s->wet, s->na);
    int rc = cuda_check(cudaGetLastError(), "wet_mask_kernel");
    if (rc == SWA_OK) rc = cuda_check(cudaDeviceSynchronize(), "create_snapstore");
    if (rc != SWA_OK) { delete s; return rc; }
    *out = s;
    return SWA_OK;
}

int swa_destroy_snapstore(swa_snapstore *store) {
    delete store;
    return SWA_OK;
}

int swa_store_snapshot(swa_adjoint *a, swa_snapstore *s, void *stream) {
    if (!a || !s) return set_error(SWA_EINVAL, "null argument");
    if (s->adj != a) return set_error(SWA_EINVAL, "store belongs to another adjoint");
    if (!s->tau_host.empty()) {
        const double tau = a->t_f - (double)a->steps_done * a->dt;
        if (!(tau < s->tau_host.back()))
            return set_error(SWA_ESTATE, "snapshot times must strictly decrease");
    }
    return store_into(a, s, S(stream));
}

int swa_run_adjoint(swa_adjoint *a, swa_snapstore *s, int every, void *stream) {
    if (!a || !s) return set_error(SWA_EINVAL, "null argument");
    if (s->adj != a) return set_error(SWA_EINVAL, "store belongs to another adjoint");
    if (every < 1) return set_error(SWA_EINVAL, "every must be >= 1");
    const bool first = s->tau_host.empty() ||
                       a->t_f - (double)a->steps_done * a->dt < s->tau_host.back();
    long long need = first ? 1 : 0;
    for (long long k = a->steps_done + 1; k <= a->N; k++)
        if (k % every == 0 || k == a->N) need++;
    if (need > s->max_snaps - s->count)
        return set_error(SWA_ENOMEM, "snapshot store needs %lld more slots, has %d", need,
                         s->max_snaps - s->count);
    cudaStream_t st = S(stream);
    if (first) TRY(store_into(a, s, st));
    while (a->steps_done < a->N) {
        const long long k = a->steps_done + 1;
        const bool snap1 = (k % every == 0) || (k == a->N);
        // two steps in one pass when no snapshot falls between them
        const int ns = (a->steps_per_pass == 2 && !snap1 && k + 1 <= a->N) ? 2 : 1;
        const long long kl = k + ns - 1;
        const bool snap = (kl % every == 0) || (kl == a->N);
        TRY(adj_steps(a, snap ? s : nullptr, ns, st));
    }
    return SWA_OK;
}

int swa_snapstore_clear(swa_snapstore *s) {
    if (!s) return set_error(SWA_EINVAL, "null store");
    s->count = 0;
    s->tau_host.clear();
    return SWA_OK;
}

int swa_snapstore_info(const swa_snapstore *s, int *count, double *tau_host, int tau_cap) {
    if (!s) return set_error(SWA_EINVAL, "null store");
    if (count) *count = s->count;
    if (tau_host)
        for (int k = 0; k < s->count && k < tau_cap; k++) tau_host[k] = s->tau_host[k];
    return SWA_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- flagging
template <typename R, typename SN>
static int flag_dispatch(const swa_grid *g, const swa_snapstore *s, double t_s, double t_f,
                         double tol, int mode, uint8_t *flags, float *maxip,
                         long long *count, cudaStream_t st) {
    FlagParams<R, SN> p{};
    p.nx = g->d.nx; p.ny = g->d.ny; p.two_d = g->d.ndim == 2;
    p.x_lo = g->d.x_lo; p.y_lo = g->d.y_lo; p.dx = g->d.dx; p.dy = g->d.dy;
    p.dry_tol = (R)g->d.dry_tol;
    for (int b = 0; b < 2; b++)
        for (int k = 0; k < 3; k++) p.q[b][k] = (const R *)g->q[b][k];
    p.bath = (const R *)g->bath;
    p.clk = g->clk;
    const swa_grid_desc &ad = s->adj->d;
    p.anx = ad.nx; p.any = ad.ny;
    p.ax_lo = ad.x_lo; p.ay_lo = ad.y_lo; p.adx = ad.dx; p.ady = ad.dy;
    p.frx = (float)(g->d.dx / ad.dx);
    p.fcx = (float)((g->d.x_lo - ad.x_lo) / ad.dx - 0.5);
    p.fry = (float)(g->d.dy / ad.dy);
    p.fcy = (float)((g->d.y_lo - ad.y_lo) / ad.dy - 0.5);
    p.same_grid = (ad.nx == g->d.nx && ad.ny == g->d.ny && ad.x_lo == g->d.x_lo &&
                   ad.y_lo == g->d.y_lo && ad.dx == g->d.dx && ad.dy == g->d.dy);
    p.awet = s->wet;
    p.snaps = (const SN *)s->data;
    p.na = s->na;
    p.ncomp = s->nc;
    p.snap_stride = (size_t)s->nc * s->na;
    p.tau = s->tau_dev;
    p.K = s->count;
    p.t_s = t_s; p.t_f = t_f; p.tol = tol; p.mode = mode;
    p.flags = flags;
    p.maxip = maxip;
    p.env = s->env;   // the envelope is on the adjoint grid (same or coarser)
    p.count = (unsigned long long *)count;
    return flag_launch<R, SN>(p, st);
}

extern "C" {

int swa_flag_cells(const swa_grid *g, const swa_snapstore *s, double t_s, double t_f,
                   double tol, int mode, uint8_t *flags_dev, float *maxip_dev,
                   long long *count_dev, void *stream) {
    if (!g || !s || !flags_dev || !count_dev) return set_error(SWA_EINVAL, "null argument");
    if (mode != SWA_FLAG_INTERP && mode != SWA_FLAG_BRACKET)
        return set_error(SWA_EINVAL, "bad flag mode");
    if (g->d.ndim != s->adj->d.ndim) return set_error(SWA_EINVAL, "grid/adjoint ndim differ");
    if (!(t_s <= t_f)) return set_error(SWA_EINVAL, "need t_s <= t_f");
    if (s->count < 1) return set_error(SWA_ESTATE, "no snapshots stored");
    cudaStream_t st = S(stream);
    const bool f64 = g->d.precision == SWA_FP64, s64 = s->prec == SWA_FP64;
    if (f64 && s64) return flag_dispatch<double, double>(g, s, t_s, t_f, tol, mode, flags_dev, maxip_dev, count_dev, st);
    if (f64) return flag_dispatch<double, float>(g, s, t_s, t_f, tol, mode, flags_dev, maxip_dev, count_dev, st);
    if (s64) return flag_dispatch<float, double>(g, s, t_s, t_f, tol, mode, flags_dev, maxip_dev, count_dev, st);
    return flag_dispatch<float, float>(g, s, t_s, t_f, tol, mode, flags_dev, maxip_dev, count_dev, st);
}

}  // extern "C"

template <typename R>
static int surface_dispatch(const swa_grid *g, double tol, uint8_t *flags, long long *count,
                            cudaStream_t st) {
    SurfParams<R> p{};
    p.n = g->n;
    for (int b = 0; b < 2; b++)
        for (int k = 0; k < 3; k++) p.q[b][k] = (const R *)g->q[b][k];
    p.bath = (const R *)g->bath;
    p.clk = g->clk;
    p.tol = (R)tol;
    p.dry_tol = (R)g->d.dry_tol;
    p.flags = flags;
    p.count = (unsigned long long *)count;
    return surface_launch<R>(p, st);
}

extern "C" {

int swa_flag_surface(const swa_grid *g, double tol, uint8_t *flags_dev, long long *count_dev,
                     void *stream) {
    if (!g || !flags_dev || !count_dev) return set_error(SWA_EINVAL, "null argument");
    if (!(tol >= 0)) return set_error(SWA_EINVAL, "tol must be >= 0");
    if (g->d.precision == SWA_FP64)
        return surface_dispatch<double>(g, tol, flags_dev, count_dev, S(stream));
    return surface_dispatch<float>(g, tol, flags_dev, count_dev, S(stream));
}

// ------------------------------------------------------------------ gauges
int swa_grid_record_gauges(swa_grid *g, int n, const double *xy_dev, double *series_dev,
                           double *times_dev, long long capacity, void *stream) {
    if (!g) return set_error(SWA_EINVAL, "null grid");
    if (n < 0 || capacity < 0) return set_error(SWA_EINVAL, "n and capacity must be >= 0");
    if (n > 0 && (!xy_dev || !series_dev)) return set_error(SWA_EINVAL, "null argument");
    GaugeRec r{};
    if (n > 0 && capacity > 0) {
        r.n = n;
        r.xy = xy_dev;
        r.series = series_dev;
        r.times = times_dev;
        r.cap = capacity;
        r.row = g->gauge_row;
        r.x_lo = g->d.x_lo; r.y_lo = g->d.y_lo; r.dx = g->d.dx; r.dy = g->d.dy;
    }
    TRY(cuda_check(cudaMemsetAsync(g->gauge_row, 0, sizeof(long long), S(stream)),
                   "gauge row reset"));
    g->gauges = r;
    return SWA_OK;
}

int swa_grid_mass(const swa_grid *g, double *mass_dev, void *stream) {
    if (!g || !mass_dev) return set_error(SWA_EINVAL, "null argument");
    if (!g->state_set) return set_error(SWA_ESTATE, "grid state not set");
    const void *q0[2] = {g->q[0][0], g->q[1][0]};
    const double area = g->d.dx * (g->d.ndim == 2 ? g->d.dy : 1.0);
    return mass_launch(q0, g->bath, g->d.precision == SWA_FP32, g->clk, g->n, area, g->partial,
                       kInitBlocks, mass_dev, S(stream));
}

int swa_grid_gauge_rows(const swa_grid *g, long long *rows, void *stream) {
    if (!g || !rows) return set_error(SWA_EINVAL, "null argument");
    cudaStream_t st = S(stream);
    TRY(cuda_check(cudaMemcpyAsync(rows, g->gauge_row, sizeof(long long),
                                   cudaMemcpyDeviceToHost, st), "gauge rows"));
    return cuda_check(cudaStreamSynchronize(st), "gauge rows");
}

int swa_gauge_sample(const swa_grid *g, int n, const double *xy_dev, double *eta_dev,
                     void *stream) {
    if (!g || (n > 0 && (!xy_dev || !eta_dev))) return set_error(SWA_EINVAL, "null argument");
    if (n < 0) return set_error(SWA_EINVAL, "n < 0");
    if (g->d.precision == SWA_FP64) {
        GaugeParams<double> p{};
        p.nx = g->d.nx; p.ny = g->d.ny; p.two_d = g->d.ndim == 2;
        p.x_lo = g->d.x_lo; p.y_lo = g->d.y_lo; p.dx = g->d.dx; p.dy = g->d.dy;
        for (int b = 0; b < 2; b++)
            for (int k = 0; k < 3; k++) p.q[b][k] = (const double *)g->q[b][k];
        p.bath = (const double *)g->bath;
        p.clk = g->clk; p.n = n; p.xy = xy_dev; p.out = eta_dev;
        return gauge_launch<double>(p, S(stream));
    }
    GaugeParams<float> p{};
    p.nx = g->d.nx; p.ny = g->d.ny; p.two_d = g->d.ndim == 2;
    p.x_lo = g->d.x_lo; p.y_lo = g->d.y_lo; p.dx = g->d.dx; p.dy = g->d.dy;
    for (int b = 0; b < 2; b++)
        for (int k = 0; k < 3; k++) p.q[b][k] = (const float *)g->q[b][k];
    p.bath = (const float *)g->bath;
    p.clk = g->clk; p.n = n; p.xy = xy_dev; p.out = eta_dev;
    return gauge_launch<float>(p, S(stream));
}

}  // extern "C"
