// Host-only check of the AMR glue's map builder (no GPU needed): the fill,
// average and coarse-fine edge maps that build_maps produces from random
// patch layouts equal those of a brute-force search over every patch, and
// bad geometry is rejected.  Built and run by tests/test_amr_host.py.
#include "patches.cu"

#include <algorithm>
#include <cstdio>
#include <random>
#include <tuple>

namespace {

struct Box {
    long long I0, J0;
    int nx, ny;
    bool interior(long long I, long long J) const {
        return I >= I0 + 2 && I < I0 + nx - 2 && J >= J0 + 2 && J < J0 + ny - 2;
    }
};

// The maps by definition: for each ring cell, search every patch in index
// order; for each covered coarse cell, the first patch in index order; for
// each uncovered coarse cell, its neighbours (+x, -x, +y, -y) that some
// patch covers, with the first such patch's fine cells along the edge.
void brute_maps(const GridRefs &c, const swa_patchset *ps, int level, int r,
                std::vector<int4> &fill, std::vector<int4> &avg, std::vector<int4> &cf,
                std::vector<int4> &cfu) {
    const swa_grid_desc &d = c.d;
    std::vector<int> ids;
    std::vector<Box> box;
    for (int k = 0; k < ps->n; k++) {
        const swa_patch_desc &q = ps->pd[k];
        if (q.level != level) continue;
        const long long i0 = llround((q.x_lo + 2 * q.dx - d.x_lo) / d.dx);
        const long long j0 = llround((q.y_lo + 2 * q.dy - d.y_lo) / d.dy);
        ids.push_back(k);
        box.push_back(Box{i0 * r - 2, j0 * r - 2, q.nx, q.ny});
    }
    const int np = (int)ids.size();
    for (int a = 0; a < np; a++) {
        const Box &b = box[a];
        for (int j = 0; j < b.ny; j++)
            for (int i = 0; i < b.nx; i++) {
                if (i >= 2 && i < b.nx - 2 && j >= 2 && j < b.ny - 2) continue;
                const long long I = b.I0 + i, J = b.J0 + j;
                int4 m = make_int4(ids[a], j * b.nx + i, 0, 0);
                int src = -1;
                for (int q = 0; q < np && src < 0; q++)
                    if (q != a && box[q].interior(I, J)) src = q;
                if (src >= 0) {
                    m.z = ids[src];
                    m.w = (int)((J - box[src].J0) * box[src].nx + (I - box[src].I0));
                } else {
                    const long long ic = I / r, jc = J / r;
                    m.z = -1 - (int)((I - ic * r) + r * (J - jc * r));
                    m.w = (int)(jc * d.nx + ic);
                }
                fill.push_back(m);
            }
    }
    for (int jc = 0; jc < d.ny; jc++)
        for (int ic = 0; ic < d.nx; ic++)
            for (int a = 0; a < np; a++)
                if (box[a].interior((long long)ic * r, (long long)jc * r)) {
                    const Box &b = box[a];
                    avg.push_back(make_int4(jc * d.nx + ic, ids[a],
                                            (int)((jc * r - b.J0) * b.nx + (ic * r - b.I0)), 0));
                    break;
                }
    auto cover = [&](long long ic, long long jc) {
        for (int a = 0; a < np; a++)
            if (box[a].interior(ic * r, jc * r)) return a;
        return -1;
    };
    for (int jc = 0; jc < d.ny; jc++)
        for (int ic = 0; ic < d.nx; ic++) {
            if (cover(ic, jc) >= 0) continue;
            const int first = (int)cf.size();
            const int step[4][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 1}, {0, -1, 1}};
            for (const auto &s : step) {
                const int iv = ic + s[0], jv = jc + s[1], axis = s[2];
                if (iv < 0 || iv >= d.nx || jv < 0 || jv >= d.ny) continue;
                const int a = cover(iv, jv);
                if (a < 0) continue;
                const Box &b = box[a];
                const bool hi = s[0] + s[1] > 0;
                // the fine cell of V touching U with the lowest coordinate
                // along the edge, then steps of one fine cell along it
                const long long I = axis == 0 ? (long long)iv * r + (hi ? 0 : r - 1) : (long long)iv * r;
                const long long J = axis == 1 ? (long long)jv * r + (hi ? 0 : r - 1) : (long long)jv * r;
                const int stride = axis == 0 ? b.nx : 1;
                cf.push_back(make_int4(jc * d.nx + ic, ids[a],
                                       (int)((J - b.J0) * b.nx + (I - b.I0)),
                                       axis + 2 * (hi ? 1 : 0) + 4 * stride));
            }
            if ((int)cf.size() > first)
                cfu.push_back(make_int4(jc * d.nx + ic, first, (int)cf.size() - first, 0));
        }
}

bool same_in_order(const std::vector<int4> &u, const std::vector<int4> &v) {
    if (u.size() != v.size()) return false;
    for (size_t i = 0; i < u.size(); i++)
        if (u[i].x != v[i].x || u[i].y != v[i].y || u[i].z != v[i].z || u[i].w != v[i].w)
            return false;
    return true;
}

bool same(std::vector<int4> u, std::vector<int4> v) {
    auto key = [](const int4 &a, const int4 &b) {
        return std::tie(a.x, a.y, a.z, a.w) < std::tie(b.x, b.y, b.z, b.w);
    };
    std::sort(u.begin(), u.end(), key);
    std::sort(v.begin(), v.end(), key);
    if (u.size() != v.size()) return false;
    for (size_t i = 0; i < u.size(); i++)
        if (u[i].x != v[i].x || u[i].y != v[i].y || u[i].z != v[i].z || u[i].w != v[i].w)
            return false;
    return true;
}

swa_patch_desc patch(const GridRefs &c, int level, int r, int i0, int j0, int mx, int my) {
    swa_patch_desc q;
    q.level = level;
    q.nx = mx * r + 4;
    q.ny = my * r + 4;
    q.dx = c.d.dx / r;
    q.dy = c.d.dy / r;
    q.x_lo = c.d.x_lo + i0 * c.d.dx - 2 * q.dx;
    q.y_lo = c.d.y_lo + j0 * c.d.dy - 2 * q.dy;
    return q;
}

void set_patches(swa_patchset &ps, const std::vector<swa_patch_desc> &pd) {
    ps.pd = pd;
    ps.n = (int)pd.size();
    ps.common = swa_grid_desc{};
    for (int k = 0; k < 4; k++) ps.common.bc[k] = SWA_BC_EXTRAP;
    for (int l = 0; l <= SWA_MAX_LEVELS; l++) ps.lev[l].npatches = 0;
    for (const auto &q : pd) ps.lev[q.level].npatches++;
}

}  // namespace

int main() {
    std::mt19937 rng(1605);
    int checked = 0, failures = 0;
    long long edges = 0;
    for (int trial = 0; trial < 300; trial++) {
        GridRefs c{};
        c.d.ndim = 2;
        c.d.precision = SWA_FP32;
        c.d.nx = 12 + (int)(rng() % 40);
        c.d.ny = 12 + (int)(rng() % 40);
        c.d.x_lo = 1000.0;
        c.d.y_lo = -500.0;
        c.d.dx = 10.0;
        c.d.dy = 7.0;
        const int r = 1 + (int)(rng() % 5);
        const int lift = (r == 1) ? 2 : 1;   // keep rings inside the domain
        std::vector<swa_patch_desc> pd;
        const int np = 1 + (int)(rng() % 12);
        for (int k = 0; k < np; k++) {
            const int mx = 1 + (int)(rng() % 8), my = 1 + (int)(rng() % 8);
            const int sx = c.d.nx - mx - 2 * lift, sy = c.d.ny - my - 2 * lift;
            if (sx < 1 || sy < 1) continue;
            const int i0 = lift + (int)(rng() % sx), j0 = lift + (int)(rng() % sy);
            pd.push_back(patch(c, (rng() % 4 == 0) ? 2 : 1, r, i0, j0, mx, my));
        }
        swa_patchset ps;
        set_patches(ps, pd);
        if (ps.lev[1].npatches == 0) continue;
        std::vector<int4> f1, a1, e1, u1, f2, a2, e2, u2;
        if (amr::build_maps(c, &ps, 1, r, f1, a1, e1, u1) != SWA_OK) {
            printf("trial %d rejected a valid layout: %s\n", trial, swa_last_error());
            failures++;
            continue;
        }
        brute_maps(c, &ps, 1, r, f2, a2, e2, u2);
        checked++;
        edges += (long long)e1.size();
        if (!same(f1, f2) || !same(a1, a2)) {
            printf("trial %d: maps differ\n", trial);
            failures++;
        }
        if (!same_in_order(e1, e2) || !same_in_order(u1, u2)) {
            printf("trial %d: edge maps differ (%zu vs %zu edges)\n", trial, e1.size(), e2.size());
            failures++;
        }
    }
    // geometry that must be rejected
    GridRefs c{};
    c.d.ndim = 2; c.d.precision = SWA_FP32; c.d.nx = 20; c.d.ny = 20;
    c.d.dx = 10.0; c.d.dy = 10.0;
    struct Bad { const char *what; swa_patch_desc q; int r; } bad[] = {
        {"ring outside the domain", patch(c, 1, 2, 0, 5, 4, 4), 2},
        {"interior off the coarse corners", patch(c, 1, 2, 5, 5, 4, 4), 2},
        {"cell size not coarse / r", patch(c, 1, 2, 5, 5, 4, 4), 3},
        {"interior not whole coarse cells", patch(c, 1, 2, 5, 5, 4, 4), 2},
    };
    bad[1].q.x_lo += 0.5 * bad[1].q.dx;
    bad[3].q.nx += 1;
    for (auto &b : bad) {
        swa_patchset ps;
        set_patches(ps, {b.q});
        std::vector<int4> f, a, e, u;
        if (amr::build_maps(c, &ps, 1, b.r, f, a, e, u) != SWA_EINVAL) {
            printf("not rejected: %s\n", b.what);
            failures++;
        }
    }
    GridRefs c64 = c;
    c64.d.precision = SWA_FP64;
    {
        swa_patchset ps;
        set_patches(ps, {patch(c, 1, 2, 5, 5, 4, 4)});
        std::vector<int4> f, a, e, u;
        if (amr::build_maps(c64, &ps, 1, 2, f, a, e, u) != SWA_EINVAL) {
            printf("not rejected: FP64 coarse grid\n");
            failures++;
        }
    }
    {
        // a fine level with a wall: the ring fills assume extrapolation
        swa_patchset ps;
        set_patches(ps, {patch(c, 1, 2, 5, 5, 4, 4)});
        ps.common.bc[2] = SWA_BC_WALL;
        std::vector<int4> f, a, e, u;
        if (amr::build_maps(c, &ps, 1, 2, f, a, e, u) != SWA_EINVAL) {
            printf("not rejected: fine patch set with a wall\n");
            failures++;
        }
    }
    printf("layouts checked %d, coarse-fine edges %lld, failures %d\n", checked, edges, failures);
    return failures == 0 && checked >= 100 && edges > 1000 ? 0 : 1;
}
