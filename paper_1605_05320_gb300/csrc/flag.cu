// flag.cu -- adjoint-weighted flagging (Sec. 4.1, 4.2, Sec. 6) and gauges.
//
// For the forward state at its device time t and q = (eta, hu, hv) the pass
// computes m = max over tau in [t, T] of |q^(tau) . q|, T = min(t + (t_f -
// t_s), t_f), the window clipped to the stored snapshot times, with q^
// bilinear in space (component by component, clamped at the outermost
// adjoint cell centres) and either linear in time (INTERP: the maximum of a
// piecewise-linear function sits at a window end or at a snapshot time inside
// it) or taken over every bracketing snapshot (BRACKET, Eq. ip_timepoint).
// m = 0 where the forward cell is dry or a positively weighted adjoint cell
// is dry (Sec. 6).  The pass streams each snapshot once per cell: it is
// bandwidth bound, so the snapshot loop is written for coalesced loads.
#include <type_traits>

#include "flag.cuh"
#include "gauge.cuh"

namespace swadj {

struct Window {
    int empty;
    int k0, k1;          // snapshots read: k0..k1 inclusive
    int ki0, ki1;        // snapshots strictly inside the window (INTERP), or
                         // the whole read range (BRACKET)
    int kh, kl;          // INTERP: bracket index at hi and at lo
    int exact_h, exact_l;
    double ah, al;       // weights on snapshot kh (resp. kl) at hi (lo)
    double lo, hi;
};

// Index k of the snapshot interval holding s: the first k (from 0) whose
// successor is no later than s, i.e. tau[k+1] <= s (K-1 if none).
__device__ __forceinline__ int bracket_index(const double *tau, int K, double s) {
    int a = 1, b = K;  // first j in [1, K) with tau[j] <= s, else K
    while (a < b) {
        const int m = (a + b) >> 1;
        if (tau[m] > s) a = m + 1;
        else b = m;
    }
    return a - 1;
}

__device__ Window make_window(const double *tau, int K, double t, double t_s,
                              double t_f, int mode) {
    Window w;
    double T = t + (t_f - t_s);
    if (T > t_f) T = t_f;
    double lo = t, hi = T;
    w.empty = 1;
    w.k0 = 0; w.k1 = -1; w.ki0 = 0; w.ki1 = -1;
    w.kh = -2; w.kl = -2; w.exact_h = 1; w.exact_l = 1;
    w.ah = 1.0; w.al = 1.0;
    if (K < 1) return w;
    if (lo < tau[K - 1]) lo = tau[K - 1];
    if (hi > tau[0]) hi = tau[0];
    w.lo = lo; w.hi = hi;
    if (lo > hi || t > t_f) return w;
    w.empty = 0;
    if (mode == SWA_FLAG_BRACKET) {
        int kb = K - 1, ke = 0;
        for (int k = 0; k < K; k++) if (tau[k] <= lo) { kb = k; break; }
        for (int k = K - 1; k >= 0; k--) if (tau[k] >= hi) { ke = k; break; }
        w.k0 = ke; w.k1 = kb;
        w.ki0 = ke; w.ki1 = kb;
        return w;
    }
    const int kh = bracket_index(tau, K, hi);
    const int kl = bracket_index(tau, K, lo);
    w.kh = kh; w.kl = kl;
    w.exact_h = (kh + 1 >= K || tau[kh] == hi);
    w.exact_l = (kl + 1 >= K || tau[kl] == lo);
    if (!w.exact_h) w.ah = (hi - tau[kh + 1]) / (tau[kh] - tau[kh + 1]);
    if (!w.exact_l) w.al = (lo - tau[kl + 1]) / (tau[kl] - tau[kl + 1]);
    w.k0 = kh;
    w.k1 = w.exact_l ? kl : kl + 1;
    if (w.k1 < w.k0) w.k1 = w.k0;
    // tau[k] in (lo, hi) exactly for k in [kh + 1, kl], minus an end that
    // coincides with lo or hi
    w.ki0 = kh + 1;
    w.ki1 = kl;
    while (w.ki0 <= w.ki1 && !(tau[w.ki0] < hi)) w.ki0++;
    while (w.ki1 >= w.ki0 && !(tau[w.ki1] > lo)) w.ki1--;
    return w;
}

// Arithmetic of the flag products.  In float every rounding is fixed in the
// source (fmaf and unfused multiplies), so the pruned and the full variant
// form the same numbers; double keeps the plain expressions.
__device__ __forceinline__ float acc(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double acc(double a, double b, double c) { return a * b + c; }
__device__ __forceinline__ float dot3(float a, float x, float b, float y, float c, float z) {
    return fmaf(c, z, fmaf(b, y, __fmul_rn(a, x)));
}
__device__ __forceinline__ double dot3(double a, double x, double b, double y, double c,
                                       double z) {
    return a * x + b * y + c * z;
}
__device__ __forceinline__ float lerp2(float a, float x, float b, float y) {
    return fmaf(a, x, __fmul_rn(b, y));
}
__device__ __forceinline__ double lerp2(double a, double x, double b, double y) {
    return a * x + b * y;
}

// Products are accumulated in float when both the forward state and the
// snapshots are float (the bandwidth-bound FP32 path; GB300's FP64 rate is a
// small fraction of its FP32 rate) and in double otherwise.
//
// PRUNE (float, 2D, adjoint on another grid, envelope present, no maxip
// output): the rule of flag_kernel_f32x4<true> below with the bilinear
// stencil.  The interpolated snapshot value of a component is a convex
// combination of its stencil cells' values, so its magnitude is at most the
// largest envelope entry M_c over the quads holding the stencil cells with
// positive weight; a group is skipped where M_e |eta| + M_u |hu| + M_v |hv|
// < tol (1 - 1e-5).  Flags and count equal the full pass's.
template <typename R, typename S, bool SAME, bool PRUNE>
__global__ void __launch_bounds__(256) flag_kernel(FlagParams<R, S> p) {
    using A = typename std::conditional<sizeof(R) == 4 && sizeof(S) == 4, float,
                                        double>::type;
    __shared__ Window sw;
    if (threadIdx.x == 0) sw = make_window(p.tau, p.K, p.clk->t, p.t_s, p.t_f, p.mode);
    __syncthreads();
    const Window &w = sw;
    const int cur = p.clk->cur;
    const R *q0 = p.q[cur][0], *q1 = p.q[cur][1], *q2 = p.q[cur][2];
    const size_t n = (size_t)p.nx * p.ny;
    int f = 0;
    // persistent grid: each block walks cells i, i + gridDim.x * 256, ...
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        A m = A(0);
        const R a = q0[i], b = p.bath[i];
        R h, eta;
        if (sizeof(R) == 4) { eta = a; h = a + b; }
        else { h = a; eta = a + b; }
        const A qe = (A)eta, qu = (A)q1[i];
        const A qv = p.two_d ? (A)q2[i] : A(0);
        bool dry = !(h > p.dry_tol);
        size_t st[4] = {i, i, i, i};
        A wt[4] = {A(1), A(0), A(0), A(0)};
        if (!SAME && sizeof(A) == 4 && p.two_d) {
            // FP32 pass: the stencil from the float map (FP64 is a small
            // fraction of the FP32 rate on this GPU)
            const int ix = (int)(i % p.nx), jy = (int)(i / p.nx);
            float fx = fmaf((float)ix + 0.5f, p.frx, p.fcx);
            fx = fminf(fmaxf(fx, 0.f), (float)(p.anx - 1));
            int i0 = (int)floorf(fx);
            if (i0 > p.anx - 2) i0 = p.anx - 2;
            if (i0 < 0) i0 = 0;
            float ax = fx - (float)i0;
            const int i1 = p.anx > 1 ? i0 + 1 : i0;
            if (p.anx == 1) ax = 0.f;
            float fy = fmaf((float)jy + 0.5f, p.fry, p.fcy);
            fy = fminf(fmaxf(fy, 0.f), (float)(p.any - 1));
            int j0 = (int)floorf(fy);
            if (j0 > p.any - 2) j0 = p.any - 2;
            if (j0 < 0) j0 = 0;
            float ay = fy - (float)j0;
            const int j1 = p.any > 1 ? j0 + 1 : j0;
            if (p.any == 1) ay = 0.f;
            st[0] = (size_t)j0 * p.anx + i0; wt[0] = (A)__fmul_rn(1.f - ax, 1.f - ay);
            st[1] = (size_t)j0 * p.anx + i1; wt[1] = (A)__fmul_rn(ax, 1.f - ay);
            st[2] = (size_t)j1 * p.anx + i0; wt[2] = (A)__fmul_rn(1.f - ax, ay);
            st[3] = (size_t)j1 * p.anx + i1; wt[3] = (A)__fmul_rn(ax, ay);
        } else if (!SAME) {
            const int ix = (int)(i % p.nx), jy = (int)(i / p.nx);
            const double x = p.x_lo + ((double)ix + 0.5) * p.dx;
            const double y = p.y_lo + ((double)jy + 0.5) * p.dy;
            double fx = (x - p.ax_lo) / p.adx - 0.5;
            fx = fx < 0.0 ? 0.0 : (fx > (double)(p.anx - 1) ? (double)(p.anx - 1) : fx);
            int i0 = (int)floor(fx);
            if (i0 > p.anx - 2) i0 = p.anx - 2;
            if (i0 < 0) i0 = 0;
            double ax = fx - (double)i0;
            const int i1 = p.anx > 1 ? i0 + 1 : i0;
            if (p.anx == 1) ax = 0.0;
            if (!p.two_d) {
                st[0] = i0; st[1] = i1;
                wt[0] = (A)(1.0 - ax); wt[1] = (A)ax;
            } else {
                double fy = (y - p.ay_lo) / p.ady - 0.5;
                fy = fy < 0.0 ? 0.0 : (fy > (double)(p.any - 1) ? (double)(p.any - 1) : fy);
                int j0 = (int)floor(fy);
                if (j0 > p.any - 2) j0 = p.any - 2;
                if (j0 < 0) j0 = 0;
                double ay = fy - (double)j0;
                const int j1 = p.any > 1 ? j0 + 1 : j0;
                if (p.any == 1) ay = 0.0;
                st[0] = (size_t)j0 * p.anx + i0; wt[0] = (A)((1.0 - ax) * (1.0 - ay));
                st[1] = (size_t)j0 * p.anx + i1; wt[1] = (A)(ax * (1.0 - ay));
                st[2] = (size_t)j1 * p.anx + i0; wt[2] = (A)((1.0 - ax) * ay);
                st[3] = (size_t)j1 * p.anx + i1; wt[3] = (A)(ax * ay);
            }
        }
#pragma unroll
        for (int c = 0; c < 4; c++)
            if (wt[c] > A(0) && !p.awet[st[c]]) dry = true;
        // PRUNE: a cell at rest (q = 0) has every product zero, m = 0
        const bool rest = PRUNE && qe == A(0) && qu == A(0) && qv == A(0);
        if (!w.empty && !dry && !rest) {
            const bool interp = p.mode != SWA_FLAG_BRACKET;
            const int gb0 = w.k0 / kEnvGroup, gb1 = w.k1 / kEnvGroup;
            unsigned mask = 0u;
            bool need_h = true, need_l = true;
            if (PRUNE) {
                const size_t na4 = p.na >> 2;
                const float tolp = (float)(p.tol * (1.0 - 1e-5));
                const A ae = fabs(qe), au = fabs(qu), av = fabs(qv);
                const int ng = gb1 - gb0 + 1 < 32 ? gb1 - gb0 + 1 : 32;
                for (int j = 0; j < ng; j++) {
                    const float *eg = p.env + (size_t)(gb0 + j) * 3 * na4;
                    float Me = 0.f, Mu = 0.f, Mv = 0.f;
#pragma unroll
                    for (int c = 0; c < 4; c++) {
                        if (!(wt[c] > A(0))) continue;
                        const size_t q = st[c] >> 2;
                        Me = fmaxf(Me, __ldg(eg + q));
                        Mu = fmaxf(Mu, __ldg(eg + na4 + q));
                        Mv = fmaxf(Mv, __ldg(eg + 2 * na4 + q));
                    }
                    const float bnd = (float)(Me * ae + Mu * au + Mv * av);
                    if (bnd < tolp) mask |= 1u << j;
                }
                // groups past the first 32 of the window are always read
                auto skipped = [&](int gb) -> bool {
                    const int jj = gb - gb0;
                    return jj < 32 && ((mask >> jj) & 1u) != 0u;
                };
                if (interp) {
                    const int kh1 = w.exact_h ? w.kh : w.kh + 1;
                    const int kl1 = w.exact_l ? w.kl : w.kl + 1;
                    need_h = !(skipped(w.kh / kEnvGroup) && skipped(kh1 / kEnvGroup));
                    need_l = !(skipped(w.kl / kEnvGroup) && skipped(kl1 / kEnvGroup));
                }
            }
            A dh0 = A(0), dh1 = A(0), dl0 = A(0), dl1 = A(0);
            for (int gb = gb0; gb <= gb1; gb++) {
                const int jj = gb - gb0;
                const bool gs = PRUNE && jj < 32 && ((mask >> jj) & 1u) != 0u;
                const int ka = w.k0 > gb * kEnvGroup ? w.k0 : gb * kEnvGroup;
                const int kb = w.k1 < gb * kEnvGroup + kEnvGroup - 1 ? w.k1
                                                                    : gb * kEnvGroup + kEnvGroup - 1;
                if (gs) {
                    const bool hh = need_h && w.kh <= kb && w.kh + 1 >= ka;
                    const bool ll = need_l && w.kl <= kb && w.kl + 1 >= ka;
                    if (!interp || !(hh || ll)) continue;
                }
                for (int k = ka; k <= kb; k++) {
                    if (gs && !((need_h && (k == w.kh || k == w.kh + 1)) ||
                                (need_l && (k == w.kl || k == w.kl + 1))))
                        continue;
                    const S *s = p.snaps + (size_t)k * p.snap_stride;
                    A v0, v1, v2 = A(0);
                    if (SAME) {
                        v0 = (A)s[i];
                        v1 = (A)s[p.na + i];
                        if (p.ncomp == 3) v2 = (A)s[2 * p.na + i];
                    } else {
                        v0 = A(0); v1 = A(0);
#pragma unroll
                        for (int c = 0; c < 4; c++) {
                            v0 = acc(wt[c], (A)s[st[c]], v0);
                            v1 = acc(wt[c], (A)s[p.na + st[c]], v1);
                            if (p.ncomp == 3) v2 = acc(wt[c], (A)s[2 * p.na + st[c]], v2);
                        }
                    }
                    const A d = dot3(v0, qe, v1, qu, v2, qv);
                    if (k >= w.ki0 && k <= w.ki1) m = fabs(d) > m ? fabs(d) : m;
                    if (k == w.kh) dh0 = d;
                    if (k == w.kh + 1) dh1 = d;
                    if (k == w.kl) dl0 = d;
                    if (k == w.kl + 1) dl1 = d;
                }
            }
            if (interp) {
                const A ah = (A)w.ah, al = (A)w.al;
                const A vh = w.exact_h ? dh0 : lerp2(ah, dh0, A(1) - ah, dh1);
                const A vl = w.exact_l ? dl0 : lerp2(al, dl0, A(1) - al, dl1);
                m = fabs(vh) > m ? fabs(vh) : m;
                m = fabs(vl) > m ? fabs(vl) : m;
            }
        }
        const int fi = (!w.empty && !dry && m >= (A)p.tol) ? 1 : 0;
        p.flags[i] = (uint8_t)fi;
        if (!PRUNE && p.maxip) p.maxip[i] = (float)m;
        f += fi;
    }
    int cnt = f;
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(p.count, (unsigned long long)cnt);
}

// FP32 forward state and FP32 snapshots on the same grid: the bandwidth-bound
// case.  Each thread takes 4 consecutive cells with 16-byte loads; the window
// (index ranges and end weights) is computed once per block, so the per-cell
// loop has no FP64 work at all.
//
// PRUNE (no maxip output requested, envelope present): a group of snapshots
// is read only where it can matter.  For a cell with forward state q and a
// group whose per-component maxima over the cell's quad are (Me, Mu, Mv),
// every product satisfies |q^ . q| <= Me |eta| + Mu |hu| + Mv |hv| =: bnd.
// If bnd < tol (1 - 1e-5) for every wet cell of the quad, no product of the
// group can reach tol even after float rounding (the products and bnd carry
// relative errors of a few 1e-7), and neither can a time-interpolated end
// value built from two such products; the group is skipped.  An end value
// (INTERP) is computed from both of its snapshots whenever either of their
// groups is read.  Every product that is formed is the one the unpruned pass
// forms, so the flags and the count are identical to the unpruned pass; only
// m differs (it may omit values below tol), hence PRUNE only without maxip.
// Ahead of the forward wave q = 0 exactly: such a quad reads its state only.
template <bool PRUNE>
__global__ void __launch_bounds__(256, 4) flag_kernel_f32x4(FlagParams<float, float> p) {
    __shared__ Window sw;
    if (threadIdx.x == 0) sw = make_window(p.tau, p.K, p.clk->t, p.t_s, p.t_f, p.mode);
    __syncthreads();
    const Window &w = sw;   // read from shared memory where used
    const int cur = p.clk->cur;
    const size_t n4 = ((size_t)p.nx * p.ny) >> 2;
    const bool interp = p.mode != SWA_FLAG_BRACKET;
    const float tol = (float)p.tol;
    const float tolp = (float)(p.tol * (1.0 - 1e-5));
    const int gb0 = w.k0 / kEnvGroup, gb1 = w.k1 / kEnvGroup;
    const size_t cs = p.na >> 2, ks = p.snap_stride >> 2;
    int f = 0;
    // persistent grid: each block walks quads i, i + gridDim.x * 256, ...
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
         i += (size_t)gridDim.x * blockDim.x) {
        const float4 e = reinterpret_cast<const float4 *>(p.q[cur][0])[i];
        const float4 u = reinterpret_cast<const float4 *>(p.q[cur][1])[i];
        const float4 v = reinterpret_cast<const float4 *>(p.q[cur][2])[i];
        const float4 hb = reinterpret_cast<const float4 *>(p.bath)[i];
        const uchar4 wet = reinterpret_cast<const uchar4 *>(p.awet)[i];
        const float dt = p.dry_tol;
        const bool ok0 = e.x + hb.x > dt && wet.x, ok1 = e.y + hb.y > dt && wet.y;
        const bool ok2 = e.z + hb.z > dt && wet.z, ok3 = e.w + hb.w > dt && wet.w;
        float4 m = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 dh0 = m, dh1 = m, dl0 = m, dl1 = m;
        // envelope test of group gb (PRUNE only): true when no product of the
        // group can reach tol in any wet cell of the quad
        auto skip = [&](int gb) -> bool {
            const float *eg = p.env + (size_t)gb * 3 * n4;
            const float Me = __ldg(eg + i), Mu = __ldg(eg + n4 + i), Mv = __ldg(eg + 2 * n4 + i);
            const float b0 = Me * fabsf(e.x) + Mu * fabsf(u.x) + Mv * fabsf(v.x);
            const float b1 = Me * fabsf(e.y) + Mu * fabsf(u.y) + Mv * fabsf(v.y);
            const float b2 = Me * fabsf(e.z) + Mu * fabsf(u.z) + Mv * fabsf(v.z);
            const float b3 = Me * fabsf(e.w) + Mu * fabsf(u.w) + Mv * fabsf(v.w);
            return (!ok0 || b0 < tolp) && (!ok1 || b1 < tolp) && (!ok2 || b2 < tolp) &&
                   (!ok3 || b3 < tolp);
        };
        // PRUNE: a quad whose forward state is exactly zero (the ocean at rest
        // ahead of the wave) has every product exactly zero, m = 0 as in the
        // full pass, so even its envelope is not read
        const bool rest = e.x == 0.f && e.y == 0.f && e.z == 0.f && e.w == 0.f &&
                          u.x == 0.f && u.y == 0.f && u.z == 0.f && u.w == 0.f &&
                          v.x == 0.f && v.y == 0.f && v.z == 0.f && v.w == 0.f;
        if (!w.empty && (!PRUNE || ((ok0 || ok1 || ok2 || ok3) && !rest))) {
            const float4 *s0 = reinterpret_cast<const float4 *>(p.snaps) + i;
            // skip bits of the first 32 groups of the window (256 snapshots),
            // their loads issued independently of one another
            unsigned mask = 0u;
            if (PRUNE) {
                const int ng = gb1 - gb0 + 1 < 32 ? gb1 - gb0 + 1 : 32;
#pragma unroll 2
                for (int j = 0; j < ng; j++)
                    if (skip(gb0 + j)) mask |= 1u << j;
            }
            // groups past the first 32 of the window are always read
            auto skipped = [&](int gb) -> bool {
                const int j = gb - gb0;
                return j < 32 && ((mask >> j) & 1u) != 0u;
            };
            bool need_h = true, need_l = true;
            if (PRUNE && interp) {
                const int kh1 = w.exact_h ? w.kh : w.kh + 1;
                const int kl1 = w.exact_l ? w.kl : w.kl + 1;
                need_h = !(skipped(w.kh / kEnvGroup) && skipped(kh1 / kEnvGroup));
                need_l = !(skipped(w.kl / kEnvGroup) && skipped(kl1 / kEnvGroup));
            }
            for (int gb = gb0; gb <= gb1; gb++) {
                const bool gs = PRUNE && skipped(gb);
                const int ka = w.k0 > gb * kEnvGroup ? w.k0 : gb * kEnvGroup;
                const int kb = w.k1 < gb * kEnvGroup + kEnvGroup - 1 ? w.k1
                                                                    : gb * kEnvGroup + kEnvGroup - 1;
                if (gs) {
                    // a skipped group can only supply the snapshots of a
                    // needed end pair
                    const bool hh = need_h && w.kh <= kb && w.kh + 1 >= ka;
                    const bool ll = need_l && w.kl <= kb && w.kl + 1 >= ka;
                    if (!interp || !(hh || ll)) continue;
                }
#pragma unroll 2
                for (int k = ka; k <= kb; k++) {
                    if (gs && !((need_h && (k == w.kh || k == w.kh + 1)) ||
                                (need_l && (k == w.kl || k == w.kl + 1))))
                        continue;
                    const float4 a = __ldcs(s0 + (size_t)k * ks);
                    const float4 b = __ldcs(s0 + (size_t)k * ks + cs);
                    const float4 c = __ldcs(s0 + (size_t)k * ks + 2 * cs);
                    float4 d;
                    // rounding fixed in the source, identical in both variants
                    d.x = fmaf(c.x, v.x, fmaf(b.x, u.x, __fmul_rn(a.x, e.x)));
                    d.y = fmaf(c.y, v.y, fmaf(b.y, u.y, __fmul_rn(a.y, e.y)));
                    d.z = fmaf(c.z, v.z, fmaf(b.z, u.z, __fmul_rn(a.z, e.z)));
                    d.w = fmaf(c.w, v.w, fmaf(b.w, u.w, __fmul_rn(a.w, e.w)));
                    if (k >= w.ki0 && k <= w.ki1) {
                        m.x = fmaxf(m.x, fabsf(d.x)); m.y = fmaxf(m.y, fabsf(d.y));
                        m.z = fmaxf(m.z, fabsf(d.z)); m.w = fmaxf(m.w, fabsf(d.w));
                    }
                    if (k == w.kh) dh0 = d;
                    if (k == w.kh + 1) dh1 = d;
                    if (k == w.kl) dl0 = d;
                    if (k == w.kl + 1) dl1 = d;
                }
            }
            if (interp) {
                const float ah = (float)w.ah, al = (float)w.al;
                const float bh = 1.f - ah, bl = 1.f - al;
#define SWADJ_ENDS(c)                                                          \
    {                                                                          \
        const float vh = w.exact_h ? dh0.c : fmaf(ah, dh0.c, __fmul_rn(bh, dh1.c)); \
        const float vl = w.exact_l ? dl0.c : fmaf(al, dl0.c, __fmul_rn(bl, dl1.c)); \
        m.c = fmaxf(m.c, fmaxf(fabsf(vh), fabsf(vl)));                         \
    }
                SWADJ_ENDS(x) SWADJ_ENDS(y) SWADJ_ENDS(z) SWADJ_ENDS(w)
#undef SWADJ_ENDS
            }
        }
        const int f0 = (!w.empty && ok0 && m.x >= tol), f1 = (!w.empty && ok1 && m.y >= tol);
        const int f2 = (!w.empty && ok2 && m.z >= tol), f3 = (!w.empty && ok3 && m.w >= tol);
        reinterpret_cast<uchar4 *>(p.flags)[i] = make_uchar4(f0, f1, f2, f3);
        if (!PRUNE && p.maxip) {
            const float4 mm = make_float4(ok0 ? m.x : 0.f, ok1 ? m.y : 0.f,
                                          ok2 ? m.z : 0.f, ok3 ? m.w : 0.f);
            reinterpret_cast<float4 *>(p.maxip)[i] = w.empty ? make_float4(0.f, 0.f, 0.f, 0.f) : mm;
        }
        f += f0 + f1 + f2 + f3;
    }
    int cnt = f;
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(p.count, (unsigned long long)cnt);
}

// Envelope of one stored snapshot, folded into its group: one thread per
// quad of 4 consecutive cells.
__global__ void __launch_bounds__(256) env_update_kernel(const float *slot, size_t na,
                                                         float *env, int first) {
    const size_t n4 = na >> 2;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4;
         q += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float4 a = __ldcg(reinterpret_cast<const float4 *>(slot + c * na) + q);
            const float mx = fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(a.w)));
            float *o = env + c * n4 + q;
            *o = first ? mx : fmaxf(*o, mx);
        }
    }
}

int env_launch_update(const float *slot, size_t na, float *env_group, int first,
                      cudaStream_t st) {
    const size_t n4 = na >> 2;
    size_t blocks = (n4 + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    env_update_kernel<<<(unsigned)blocks, 256, 0, st>>>(slot, na, env_group, first);
    return swadj_host::cuda_check(cudaGetLastError(), "env_update_kernel");
}

// Blocks of the persistent FP32 flag pass: every SM filled with as many
// blocks as fit.
template <bool PRUNE>
static size_t persistent_flag_blocks() {
    static int per_sm = 0, sms = 0;
    if (per_sm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, flag_kernel_f32x4<PRUNE>, 256, 0);
        if (per_sm < 1) per_sm = 1;
        if (sms < 1) sms = 1;
    }
    return (size_t)per_sm * (size_t)sms;
}

// Blocks of a persistent generic flag pass, per instantiation.
template <typename R, typename S, bool SAME, bool PRUNE>
static unsigned generic_flag_blocks(size_t n) {
    static int per_sm = 0, sms = 0;
    if (per_sm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, flag_kernel<R, S, SAME, PRUNE>,
                                                      256, 0);
        if (per_sm < 1) per_sm = 1;
        if (sms < 1) sms = 1;
    }
    const size_t need = (n + 255) / 256, b = (size_t)per_sm * (size_t)sms;
    return (unsigned)(need < b ? need : b);
}

template <typename R, typename S>
int flag_launch(const FlagParams<R, S> &p, cudaStream_t st) {
    const size_t n = (size_t)p.nx * p.ny;
    cudaError_t e = cudaMemsetAsync(p.count, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return swadj_host::cuda_check(e, "flag count reset");
    if (sizeof(R) == 4 && sizeof(S) == 4 && p.same_grid && p.two_d && (n & 3) == 0) {
        const size_t n4 = n >> 2;
        const FlagParams<float, float> &pf = *reinterpret_cast<const FlagParams<float, float> *>(&p);
        const size_t need = (n4 + 255) / 256;
        if (p.env && !p.maxip) {
            const size_t b = persistent_flag_blocks<true>();
            flag_kernel_f32x4<true><<<(unsigned)(need < b ? need : b), 256, 0, st>>>(pf);
        } else {
            const size_t b = persistent_flag_blocks<false>();
            flag_kernel_f32x4<false><<<(unsigned)(need < b ? need : b), 256, 0, st>>>(pf);
        }
    } else if (p.same_grid) {
        flag_kernel<R, S, true, false>
            <<<generic_flag_blocks<R, S, true, false>(n), 256, 0, st>>>(p);
    } else if (sizeof(R) == 4 && sizeof(S) == 4 && p.two_d && p.env && !p.maxip) {
        flag_kernel<float, float, false, true>
            <<<generic_flag_blocks<float, float, false, true>(n), 256, 0, st>>>(
                *reinterpret_cast<const FlagParams<float, float> *>(&p));
    } else {
        flag_kernel<R, S, false, false>
            <<<generic_flag_blocks<R, S, false, false>(n), 256, 0, st>>>(p);
    }
    return swadj_host::cuda_check(cudaGetLastError(), "flag_kernel");
}

template int flag_launch<double, double>(const FlagParams<double, double> &, cudaStream_t);
template int flag_launch<double, float>(const FlagParams<double, float> &, cudaStream_t);
template int flag_launch<float, float>(const FlagParams<float, float> &, cudaStream_t);
template int flag_launch<float, double>(const FlagParams<float, double> &, cudaStream_t);

// |eta| > tol on wet cells, eta stored (float) or h + B (double).
template <typename R>
__global__ void __launch_bounds__(256) surface_kernel(SurfParams<R> p) {
    const int cur = p.clk->cur;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    int f = 0;
    if (i < p.n) {
        const R a = p.q[cur][0][i], b = p.bath[i];
        R h, eta;
        if (sizeof(R) == 4) { eta = a; h = a + b; }
        else { h = a; eta = a + b; }
        f = (h > p.dry_tol && fabs(eta) > p.tol) ? 1 : 0;
        p.flags[i] = (uint8_t)f;
    }
    const int cnt = __syncthreads_count(f);
    if (threadIdx.x == 0 && cnt) atomicAdd(p.count, (unsigned long long)cnt);
}

template <typename R>
int surface_launch(const SurfParams<R> &p, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(p.count, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return swadj_host::cuda_check(e, "surface count reset");
    surface_kernel<R><<<(unsigned)((p.n + 255) / 256), 256, 0, st>>>(p);
    return swadj_host::cuda_check(cudaGetLastError(), "surface_kernel");
}

template int surface_launch<double>(const SurfParams<double> &, cudaStream_t);
template int surface_launch<float>(const SurfParams<float> &, cudaStream_t);

template <typename R>
__global__ void gauge_kernel(GaugeParams<R> p) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= p.n) return;
    const int cur = p.clk->cur;
    p.out[k] = gauge_eta<R>(p.q[cur][0], p.bath, p.nx, p.ny, p.two_d, p.x_lo, p.y_lo, p.dx,
                            p.dy, p.xy[2 * k], p.xy[2 * k + 1]);
}

template <typename R>
int gauge_launch(const GaugeParams<R> &p, cudaStream_t st) {
    if (p.n <= 0) return 0;
    gauge_kernel<R><<<(p.n + 127) / 128, 128, 0, st>>>(p);
    return swadj_host::cuda_check(cudaGetLastError(), "gauge_kernel");
}

template int gauge_launch<double>(const GaugeParams<double> &, cudaStream_t);
template int gauge_launch<float>(const GaugeParams<float> &, cudaStream_t);

}  // namespace swadj
