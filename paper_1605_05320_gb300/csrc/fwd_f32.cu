// fwd_f32.cu -- FP32 perturbation-form forward step (Eq. swe, Sec. 5; Roe-type
// f-wave solver per edge, Sec. 6) built for GB300's FP32 pipes.
//
// Storage: eta = h + B, hu, hv and hbar = -B in float.  Depth h = eta + hbar
// enters only wave speeds and Roe averages; the surface jump that drives the
// bathymetry-balanced momentum flux is taken from eta directly, so decimetre
// waves on 4000 m are resolved to float precision of eta, not of h.
//
// Work decomposition: a block owns a strip of SX = 128 columns (one thread
// per column) and walks it along y over H rows.  Along y each thread keeps the
// waves of the last three y-edges of its column in registers (each y-edge is
// solved once, each y-limiter evaluated once).  Along x the row being updated
// is exchanged through shared memory in three barrier-separated phases: cell
// data, x-edge waves, x-edge net fluxes.  Two halo columns on each side are
// loaded by four extra lanes.  Ghost cells are produced by index mapping
// (copy or mirror) while loading.  No FP64 arithmetic runs per cell: the CFL
// maximum is reduced in float (max is exact) and only the last block turns it
// into the next time step in double.
//
// Per edge, the MC-limited correction is formed without a division by the
// wave norm: for Z = b (1, s, vhat) and its upwind neighbour Zu = bu (1, su,
// vu), theta b = bu (1 + su s + vu vhat) / (1 + s^2 + vhat^2), and
// phi(theta) b = sign(b) max(0, min((|b| + sign(b) theta b)/2, 2|b|,
// 2 sign(b) theta b)), which is phi(theta) b for every b including b = 0.
#include "fwd_kernels.cuh"

namespace swadj {

namespace f32 {

constexpr int SX = 128;  // columns per strip = threads per block

struct Cell {            // derived per-cell quantities in an edge's frame
    float h, mn, mt, un, ut, sq, eta;
};

struct EdgeW {           // f-wave data of one edge
    float s1, s3, vh, b1, b2, b3;
};

__device__ __forceinline__ float frcp(float x) { return __fdividef(1.0f, x); }

// derived quantities of a cell: h, velocities, sqrt(h)
__device__ __forceinline__ void derive(float eta, float hbar, float hu, float hv,
                                       float &h, float &u, float &v, float &sq) {
    h = eta + hbar;
    const float r = rsqrtf(h);
    sq = h * r;
    const float ih = r * r;
    u = hu * ih;
    v = hv * ih;
}

__device__ __forceinline__ EdgeW solve(float g, float hL, float mnL, float mtL, float unL,
                                       float utL, float sqL, float etaL, float hR,
                                       float mnR, float mtR, float unR, float utR,
                                       float sqR, float etaR) {
    EdgeW w;
    const float hh = 0.5f * (hL + hR);
    const float rd = frcp(sqL + sqR);
    const float uh = (sqL * unL + sqR * unR) * rd;
    const float vh = (sqL * utL + sqR * utR) * rd;
    const float gh = g * hh;
    const float rc = rsqrtf(gh);
    const float ch = gh * rc;
    const float s1 = uh - ch, s3 = uh + ch;
    const float df1 = mnR - mnL;
    const float df2 = (mnR * unR - mnL * unL) + gh * (etaR - etaL);
    const float df3 = mnR * utR - mnL * utL;
    const float hr = 0.5f * rc;  // 1 / (s3 - s1)
    w.s1 = s1;
    w.s3 = s3;
    w.vh = vh;
    w.b1 = (s3 * df1 - df2) * hr;
    w.b3 = (df2 - s1 * df1) * hr;
    w.b2 = df3 - vh * df1;
    return w;
}

// phi(theta) * b for the MC limiter given r = theta * b
__device__ __forceinline__ float mc_lim(float b, float r) {
    const float sg = b < 0.0f ? -1.0f : 1.0f;
    const float B = fabsf(b), Rr = sg * r;
    float m = fminf(0.5f * (B + Rr), 2.0f * B);
    m = fminf(m, 2.0f * Rr);
    return sg * fmaxf(m, 0.0f);
}

__device__ __forceinline__ float split_pos(float s) {
    return s > 0.0f ? 1.0f : (s < 0.0f ? 0.0f : 0.5f);
}

// Net flux of edge w (neighbours wl, wr) into its left cell (GL) and right
// cell (GR): Q_left -= nu GL, Q_right -= nu GR.
__device__ __forceinline__ void edge_net(const EdgeW &wl, const EdgeW &w, const EdgeW &wr,
                                         float nu, int order, float GL[3], float GR[3]) {
    const float s2 = 0.5f * (w.s1 + w.s3);
    const float p1 = split_pos(w.s1), p2 = split_pos(s2), p3 = split_pos(w.s3);
    // A+dq and the total jump; A-dq = total - A+dq
    const float a1 = p1 * w.b1, a3 = p3 * w.b3;
    float ap0 = a1 + a3;
    float ap1 = a1 * w.s1 + a3 * w.s3;
    float ap2 = (a1 + a3) * w.vh + p2 * w.b2;
    const float t0 = w.b1 + w.b3;
    const float t1 = w.b1 * w.s1 + w.b3 * w.s3;
    const float t2 = t0 * w.vh + w.b2;
    float F0 = 0.0f, F1 = 0.0f, F2 = 0.0f;
    if (order >= 2) {
        // wave 1
        const EdgeW &u1 = w.s1 > 0.0f ? wl : wr;
        const float m1 = fmaf(w.s1, w.s1, fmaf(w.vh, w.vh, 1.0f));
        const float d1 = fmaf(u1.s1, w.s1, fmaf(u1.vh, w.vh, 1.0f));
        const float l1 = mc_lim(w.b1, u1.b1 * d1 * frcp(m1));
        // wave 3
        const EdgeW &u3 = w.s3 > 0.0f ? wl : wr;
        const float m3 = fmaf(w.s3, w.s3, fmaf(w.vh, w.vh, 1.0f));
        const float d3 = fmaf(u3.s3, w.s3, fmaf(u3.vh, w.vh, 1.0f));
        const float l3 = mc_lim(w.b3, u3.b3 * d3 * frcp(m3));
        // wave 2 (shear): vector (0,0,1), theta b = upwind strength
        const EdgeW &u2 = s2 > 0.0f ? wl : wr;
        const float l2 = mc_lim(w.b2, u2.b2);
        const float sg1 = w.s1 > 0.0f ? 0.5f : (w.s1 < 0.0f ? -0.5f : 0.0f);
        const float sg2 = s2 > 0.0f ? 0.5f : (s2 < 0.0f ? -0.5f : 0.0f);
        const float sg3 = w.s3 > 0.0f ? 0.5f : (w.s3 < 0.0f ? -0.5f : 0.0f);
        const float c1 = sg1 * (1.0f - nu * fabsf(w.s1)) * l1;
        const float c2 = sg2 * (1.0f - nu * fabsf(s2)) * l2;
        const float c3 = sg3 * (1.0f - nu * fabsf(w.s3)) * l3;
        F0 = c1 + c3;
        F1 = c1 * w.s1 + c3 * w.s3;
        F2 = F0 * w.vh + c2;
    }
    GL[0] = (t0 - ap0) + F0;
    GL[1] = (t1 - ap1) + F1;
    GL[2] = (t2 - ap2) + F2;
    GR[0] = ap0 - F0;
    GR[1] = ap1 - F1;
    GR[2] = ap2 - F2;
}

struct Slot {            // one cell of the thread's column: raw and derived
    float eta, hu, hv, hb, h, u, v, sq;
};

template <bool TWO_D>
__device__ __forceinline__ Slot load_cell(const FwdParams<float> &p, const float *q0,
                                          const float *q1, const float *q2, int gi, int gj) {
    bool fx, fy = false;
    const int ci = ghost_index(gi, p.nx, p.bc.lo_x, p.bc.hi_x, &fx);
    int cj = 0;
    if (TWO_D) cj = ghost_index(gj, p.ny, p.bc.lo_y, p.bc.hi_y, &fy);
    const size_t o = (size_t)cj * p.nx + ci;
    Slot c;
    c.eta = __ldg(q0 + o);
    c.hu = __ldg(q1 + o);
    c.hv = TWO_D ? __ldg(q2 + o) : 0.0f;
    c.hb = __ldg(p.bath + o);
    if (fx) c.hu = -c.hu;
    if (fy) c.hv = -c.hv;
    derive(c.eta, c.hb, c.hu, c.hv, c.h, c.u, c.v, c.sq);
    return c;
}

// Shared-memory exchange for the x direction of one row.
struct XShared {
    float h[SX + 4], mn[SX + 4], mt[SX + 4], un[SX + 4], ut[SX + 4], sq[SX + 4],
        eta[SX + 4];
    EdgeW w[SX + 3];
    float G0[SX + 2], G1[SX + 2], G2[SX + 2], R0[SX + 2], R1[SX + 2], R2[SX + 2];
};

__device__ __forceinline__ void put_cell(XShared &X, int s, const Slot &c) {
    X.h[s] = c.h; X.mn[s] = c.hu; X.mt[s] = c.hv; X.un[s] = c.u; X.ut[s] = c.v;
    X.sq[s] = c.sq; X.eta[s] = c.eta;
}

__device__ __forceinline__ EdgeW x_solve(const XShared &X, float g, int e) {
    return solve(g, X.h[e], X.mn[e], X.mt[e], X.un[e], X.ut[e], X.sq[e], X.eta[e],
                 X.h[e + 1], X.mn[e + 1], X.mt[e + 1], X.un[e + 1], X.ut[e + 1],
                 X.sq[e + 1], X.eta[e + 1]);
}

__device__ __forceinline__ void x_net(XShared &X, int e, float nu, int order) {
    float GL[3], GR[3];
    edge_net(X.w[e - 1], X.w[e], X.w[e + 1], nu, order, GL, GR);
    X.G0[e - 1] = GL[0]; X.G1[e - 1] = GL[1]; X.G2[e - 1] = GL[2];
    X.R0[e - 1] = GR[0]; X.R1[e - 1] = GR[1]; X.R2[e - 1] = GR[2];
}

// x-direction increment of the thread's cell in row gj (slot t + 2): three
// barrier-separated phases over the block's row.  Slots s = 0 .. SX+3 hold
// columns x0 - 2 + s; edge e lies between slots e and e + 1.
template <bool TWO_D>
__device__ __forceinline__ void x_increment(XShared &X, const FwdParams<float> &p,
                                            const float *q0, const float *q1,
                                            const float *q2, const Slot &own, int x0,
                                            int gj, float nux, float dq[3]) {
    const int t = threadIdx.x;
    put_cell(X, t + 2, own);
    if (t < 4) {
        const int s = t < 2 ? t : SX + t;        // slots 0, 1, SX+2, SX+3
        const Slot h = load_cell<TWO_D>(p, q0, q1, q2, x0 - 2 + s, gj);
        put_cell(X, s, h);
    }
    __syncthreads();
    X.w[t + 1] = x_solve(X, p.g, t + 1);         // edges 1 .. SX
    if (t < 3) {
        const int e = t == 0 ? 0 : SX + t;       // edges 0, SX+1, SX+2
        X.w[e] = x_solve(X, p.g, e);
    }
    __syncthreads();
    x_net(X, t + 1, nux, p.order);               // net fluxes of edges 1 .. SX
    if (t == 3) x_net(X, SX + 1, nux, p.order);
    __syncthreads();
    // cell slot t+2: left edge t+1 (cell is its right cell), right edge t+2
    dq[0] = -nux * (X.R0[t] + X.G0[t + 1]);
    dq[1] = -nux * (X.R1[t] + X.G1[t + 1]);
    dq[2] = -nux * (X.R2[t] + X.G2[t + 1]);
}

// y edge between two cells of the thread's column (normal momentum hv)
__device__ __forceinline__ EdgeW y_solve(float g, const Slot &a, const Slot &b) {
    return solve(g, a.h, a.hv, a.hu, a.v, a.u, a.sq, a.eta, b.h, b.hv, b.hu, b.v, b.u,
                 b.sq, b.eta);
}

template <bool TWO_D>
__global__ void __launch_bounds__(SX) fwd_f32_strip(FwdParams<float> p, int H) {
    __shared__ XShared X;
    __shared__ float s_nu[2];
    __shared__ int s_cur, s_run;
    __shared__ float red[SX / 32];
    __shared__ int am_last;

    const int t = threadIdx.x;
    double t_now = 0.0, dt = 0.0;
    if (t == 0) {
        volatile DevClock *clk = p.clk;
        t_now = clk->t;
        dt = clk->dt_cfl;
        if (p.t_end - t_now < dt) dt = p.t_end - t_now;
        s_run = dt > 0.0;
        s_nu[0] = (float)(dt / (double)p.dx);
        s_nu[1] = (float)(dt / (double)p.dy);
        s_cur = clk->cur;
    }
    __syncthreads();
    if (!s_run) return;  // clock at t_end: no-op step
    const float nux = s_nu[0], nuy = s_nu[1];
    const int cur = s_cur;
    const float *q0 = p.q[cur][0], *q1 = p.q[cur][1], *q2 = p.q[cur][2];
    float *o0 = p.q[cur ^ 1][0], *o1 = p.q[cur ^ 1][1], *o2 = p.q[cur ^ 1][2];
    const float g = p.g;
    const int x0 = blockIdx.x * SX;
    const int gi = x0 + t;
    const bool col_ok = gi < p.nx;
    const float rdx = 1.0f / p.dx, rdy = 1.0f / p.dy;
    float smax = 0.0f;
    bool bad = false;

    auto finish_cell = [&](const Slot &c, int gj, const float dq[3]) {
        const float ne = c.eta + dq[0], nu_ = c.hu + dq[1], nv = c.hv + dq[2];
        if (col_ok) {
            const size_t o = (size_t)gj * p.nx + gi;
            o0[o] = ne;
            o1[o] = nu_;
            if (TWO_D) o2[o] = nv;
            const float h = ne + c.hb;
            bad |= !(h > 0.0f) || !isfinite(nu_) || !isfinite(nv);
            const float r = rsqrtf(h);
            const float cc = p.g * h * rsqrtf(p.g * h);
            float s = (fabsf(nu_) * r * r + cc) * rdx;
            if (TWO_D) s += (fabsf(nv) * r * r + cc) * rdy;
            smax = fmaxf(smax, s);
        }
    };

    if (!TWO_D) {
        const Slot a = load_cell<false>(p, q0, q1, q2, gi, 0);
        float dq[3];
        x_increment<false>(X, p, q0, q1, q2, a, x0, 0, nux, dq);
        finish_cell(a, 0, dq);
    } else {
        const int j0 = blockIdx.y * H;
        const int j1 = min(j0 + H, p.ny);
        Slot A = {}, Bc = {}, C = {};
        EdgeW ym = {}, y0 = {}, yp = {};   // y-edges r-5/2, r-3/2, r-1/2
        float Gl[3] = {0, 0, 0}, Gr[3] = {0, 0, 0};  // edge r-5/2 (prev iteration)
        for (int r = j0 - 2; r <= j1 + 1; r++) {
            A = Bc;
            Bc = C;
            C = load_cell<true>(p, q0, q1, q2, gi, r);
            if (r >= j0 - 1) {           // y-edge r-1/2 between rows r-1 and r
                ym = y0;
                y0 = yp;
                yp = y_solve(g, Bc, C);
            }
            float nl[3] = {0, 0, 0}, nr[3] = {0, 0, 0};
            if (r >= j0 + 1) edge_net(ym, y0, yp, nuy, p.order, nl, nr);  // edge r-3/2
            if (r >= j0 + 2) {           // update row r-2
                float dq[3];
                x_increment<true>(X, p, q0, q1, q2, A, x0, r - 2, nux, dq);
                // row r-2: lower edge r-5/2 (Gr of previous), upper edge r-3/2 (nl)
                // y fluxes are in (h, hv, hu) order
                dq[0] += -nuy * (Gr[0] + nl[0]);
                dq[2] += -nuy * (Gr[1] + nl[1]);
                dq[1] += -nuy * (Gr[2] + nl[2]);
                finish_cell(A, r - 2, dq);
            }
            Gl[0] = nl[0]; Gl[1] = nl[1]; Gl[2] = nl[2];
            Gr[0] = nr[0]; Gr[1] = nr[1]; Gr[2] = nr[2];
        }
        (void)Gl;
    }
    if (bad) atomicOr(p.err, ERR_UNSTABLE);

    // block max of the CFL number (float, exact) -> partial; last block advances
    for (int o = 16; o > 0; o >>= 1) smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    if ((t & 31) == 0) red[t >> 5] = smax;
    __syncthreads();
    const int bid = blockIdx.x + blockIdx.y * gridDim.x;
    if (t == 0) {
        float m = red[0];
        for (int k = 1; k < SX / 32; k++) m = fmaxf(m, red[k]);
        reinterpret_cast<float *>(p.partial)[bid] = m;
        __threadfence();
        const unsigned int tk = atomicAdd(&p.clk->ticket, 1u);
        am_last = (tk == (unsigned int)(p.nblocks - 1));
    }
    __syncthreads();
    if (am_last) {
        __threadfence();
        float m = 0.0f;
        const float *pf = reinterpret_cast<const float *>(p.partial);
        for (int k = t; k < p.nblocks; k += SX) m = fmaxf(m, __ldcg(pf + k));
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((t & 31) == 0) red[t >> 5] = m;
        __syncthreads();
        if (t == 0) {
            for (int k = 1; k < SX / 32; k++) m = fmaxf(m, red[k]);
            m = fmaxf(m, red[0]);
            volatile DevClock *clk = p.clk;
            clk->t = t_now + dt;
            clk->smax = (double)m;
            clk->dt_cfl = p.cfl / (double)m;
            clk->cur = cur ^ 1;
            clk->nsteps = clk->nsteps + 1;
            clk->ticket = 0u;
        }
    }
}

}  // namespace f32

// Strip height: the number of rows a block walks.  Chosen so that the grid
// fills the GPU with whole blocks; swa tuning may override it.
static int strip_rows(const FwdParams<float> &p) {
    if (p.fwd_rows > 0) return p.fwd_rows;
    return 48;
}

template <>
int fwd_launch_step<float>(const FwdParams<float> &p0, cudaStream_t st) {
    FwdParams<float> p = p0;
    if (p.two_d) {
        const int H = strip_rows(p);
        dim3 grid((p.nx + f32::SX - 1) / f32::SX, (p.ny + H - 1) / H);
        p.nblocks = (int)(grid.x * grid.y);
        f32::fwd_f32_strip<true><<<grid, f32::SX, 0, st>>>(p, H);
    } else {
        dim3 grid((p.nx + f32::SX - 1) / f32::SX, 1);
        p.nblocks = (int)grid.x;
        f32::fwd_f32_strip<false><<<grid, f32::SX, 0, st>>>(p, 1);
    }
    return swadj_host::cuda_check(cudaGetLastError(), "fwd_f32_strip");
}

template <>
int fwd_step_blocks<float>(const FwdParams<float> &p) {
    if (p.two_d) {
        const int H = strip_rows(p);
        return ((p.nx + f32::SX - 1) / f32::SX) * ((p.ny + H - 1) / H);
    }
    return (p.nx + f32::SX - 1) / f32::SX;
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
