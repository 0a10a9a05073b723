// Host-only check of the AMR glue's map builder (no GPU needed): the fill,
// average and coarse-fine edge maps that build_maps produces from random
// layouts of one and two nested levels equal those of a brute-force search
// over every patch, and bad geometry is rejected.  Built and run by
// tests/test_amr_host.py.
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
    int local(long long I, long long J) const { return (int)((J - J0) * nx + (I - I0)); }
};

struct Lev {
    std::vector<int> ids;
    std::vector<Box> box;
    int r = 1;
    long long per = 1;
    // first patch in index order (other than skip) whose interior holds (I, J)
    int owner(long long I, long long J, int skip = -1) const {
        for (int a = 0; a < (int)box.size(); a++)
            if (a != skip && box[a].interior(I, J)) return a;
        return -1;
    }
};

// The maps by definition, every query a search over all patches of a level.
void brute_maps(const GridRefs &c, const swa_patchset *ps, int L, const int *levels,
                const int *ratios, std::vector<amr::HostMaps> &out) {
    const swa_grid_desc &d = c.d;
    std::vector<Lev> G(L + 1);
    double dx = d.dx, dy = d.dy;
    for (int l = 1; l <= L; l++) {
        G[l].r = ratios[l - 1];
        G[l].per = G[l - 1].per * G[l].r;
        for (int k = 0; k < ps->n; k++) {
            const swa_patch_desc &q = ps->pd[k];
            if (q.level != levels[l - 1]) continue;
            const long long i0 = llround((q.x_lo + 2 * q.dx - d.x_lo) / dx);
            const long long j0 = llround((q.y_lo + 2 * q.dy - d.y_lo) / dy);
            G[l].ids.push_back(k);
            G[l].box.push_back(Box{i0 * G[l].r - 2, j0 * G[l].r - 2, q.nx, q.ny});
        }
        dx /= G[l].r;
        dy /= G[l].r;
    }
    out.assign(L + 1, amr::HostMaps());
    for (int l = 1; l <= L; l++) {
        const Lev &g = G[l], &gp = G[l - 1];
        const int r = g.r;
        amr::HostMaps &M = out[l];
        M.base.assign(ps->n, -1);
        for (int a = 0; a < (int)g.box.size(); a++) {
            const Box &b = g.box[a];
            M.base[g.ids[a]] = (int)M.fill.size();
            for (int j = 0; j < b.ny; j++)
                for (int i = 0; i < b.nx; i++) {
                    if (i >= 2 && i < b.nx - 2 && j >= 2 && j < b.ny - 2) continue;
                    const long long I = b.I0 + i, J = b.J0 + j;
                    int4 m = make_int4(g.ids[a], j * b.nx + i, 0, 0);
                    int par = -1;
                    const int src = g.owner(I, J, a);
                    if (src >= 0) {
                        m.z = g.ids[src];
                        m.w = g.box[src].local(I, J);
                    } else {
                        const long long Ip = I / r, Jp = J / r;
                        m.z = -1 - (int)((I - Ip * r) + r * (J - Jp * r));
                        if (l == 1) {
                            m.w = (int)(Jp * d.nx + Ip);
                        } else {
                            const int pb = gp.owner(Ip, Jp);
                            m.w = gp.box[pb].local(Ip, Jp);
                            par = gp.ids[pb];
                        }
                    }
                    M.fill.push_back(m);
                    M.par.push_back(par);
                }
        }
        // copies of the parent's interior cells: (patch or -1, cell, I, J)
        std::vector<std::tuple<int, int, long long, long long>> copies;
        if (l == 1) {
            for (int jc = 0; jc < d.ny; jc++)
                for (int ic = 0; ic < d.nx; ic++) copies.emplace_back(-1, jc * d.nx + ic, ic, jc);
        } else {
            for (int b = 0; b < (int)gp.box.size(); b++) {
                const Box &B = gp.box[b];
                for (int j = 2; j < B.ny - 2; j++)
                    for (int i = 2; i < B.nx - 2; i++)
                        copies.emplace_back(gp.ids[b], j * B.nx + i, B.I0 + i, B.J0 + j);
            }
        }
        const long long gnx = (long long)d.nx * gp.per, gny = (long long)d.ny * gp.per;
        for (const auto &cp : copies) {
            const int pu = std::get<0>(cp), u = std::get<1>(cp);
            const long long I = std::get<2>(cp), J = std::get<3>(cp);
            const int a = g.owner(I * r, J * r);
            if (a >= 0) {
                M.avg.push_back(make_int4(pu, u, g.ids[a], g.box[a].local(I * r, J * r)));
                continue;
            }
            const int first = (int)M.cf.size();
            const int step[4][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 1}, {0, -1, 1}};
            for (const auto &s : step) {
                const long long Iv = I + s[0], Jv = J + s[1];
                const int axis = s[2];
                if (Iv < 0 || Iv >= gnx || Jv < 0 || Jv >= gny) continue;
                const int q = g.owner(Iv * r, Jv * r);
                if (q < 0) continue;
                const bool hi = s[0] + s[1] > 0;
                // the cell of V touching U with the lowest coordinate along
                // the edge, then steps of one cell along it
                const long long If = axis == 0 ? Iv * r + (hi ? 0 : r - 1) : Iv * r;
                const long long Jf = axis == 1 ? Jv * r + (hi ? 0 : r - 1) : Jv * r;
                M.cf.push_back(make_int4(pu, u, g.ids[q], g.box[q].local(If, Jf)));
                M.cfw.push_back(axis + 2 * (hi ? 1 : 0) + 4 * (axis == 0 ? g.box[q].nx : 1));
            }
            if ((int)M.cf.size() > first)
                M.cfu.push_back(make_int4(pu, u, first, (int)M.cf.size() - first));
        }
    }
}

bool same4(std::vector<int4> u, std::vector<int4> v, bool sorted) {
    auto key = [](const int4 &a, const int4 &b) {
        return std::tie(a.x, a.y, a.z, a.w) < std::tie(b.x, b.y, b.z, b.w);
    };
    if (sorted) {
        std::sort(u.begin(), u.end(), key);
        std::sort(v.begin(), v.end(), key);
    }
    if (u.size() != v.size()) return false;
    for (size_t i = 0; i < u.size(); i++)
        if (u[i].x != v[i].x || u[i].y != v[i].y || u[i].z != v[i].z || u[i].w != v[i].w)
            return false;
    return true;
}

bool same_maps(const amr::HostMaps &a, const amr::HostMaps &b) {
    return same4(a.fill, b.fill, false) && a.par == b.par && a.base == b.base &&
           same4(a.avg, b.avg, false) &&
           same4(a.cf, b.cf, false) && a.cfw == b.cfw && same4(a.cfu, b.cfu, false);
}

// A patch whose interior is mx x my parent cells from parent cell (i0, j0),
// dxp the parent cell width.
swa_patch_desc patch(const GridRefs &c, int level, int r, double dxp, double dyp, long long i0,
                     long long j0, int mx, int my) {
    swa_patch_desc q;
    q.level = level;
    q.nx = mx * r + 4;
    q.ny = my * r + 4;
    q.dx = dxp / r;
    q.dy = dyp / r;
    q.x_lo = c.d.x_lo + i0 * dxp - 2 * q.dx;
    q.y_lo = c.d.y_lo + j0 * dyp - 2 * q.dy;
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
    int checked = 0, checked2 = 0, failures = 0;
    long long edges = 0, edges2 = 0;
    for (int trial = 0; trial < 400; trial++) {
        GridRefs c{};
        c.d.ndim = 2;
        c.d.precision = SWA_FP32;
        c.d.nx = 12 + (int)(rng() % 40);
        c.d.ny = 12 + (int)(rng() % 40);
        c.d.x_lo = 1000.0;
        c.d.y_lo = -500.0;
        c.d.dx = 10.0;
        c.d.dy = 7.0;
        const bool two = trial % 2 == 1;
        const int r1 = 1 + (int)(rng() % 5), r2 = 1 + (int)(rng() % 4);
        const int lift = (r1 == 1) ? 2 : 1;   // keep rings inside the domain
        std::vector<swa_patch_desc> pd;
        // level 1 (patch-set level 1) and, for two levels, patch-set level 3;
        // patch-set level 2 holds distractors the hierarchy ignores
        const int np = 1 + (int)(rng() % 10);
        struct Int { long long i0, j0; int mx, my; };
        std::vector<Int> l1;
        for (int k = 0; k < np; k++) {
            const int mx = 1 + (int)(rng() % 8), my = 1 + (int)(rng() % 8);
            const int sx = c.d.nx - mx - 2 * lift, sy = c.d.ny - my - 2 * lift;
            if (sx < 1 || sy < 1) continue;
            const int i0 = lift + (int)(rng() % sx), j0 = lift + (int)(rng() % sy);
            const int lev = (rng() % 5 == 0) ? 2 : 1;
            pd.push_back(patch(c, lev, r1, c.d.dx, c.d.dy, i0, j0, mx, my));
            if (lev == 1) l1.push_back({i0, j0, mx, my});
        }
        if (two && !l1.empty()) {
            // level-2 patches nested in level-1 interiors: their level-1
            // cells (ring included) stay inside one level-1 interior
            const int m2 = 1 + (int)(rng() % 5);
            for (int k = 0; k < m2; k++) {
                const Int &p = l1[rng() % l1.size()];
                const long long w = (long long)p.mx * r1, h = (long long)p.my * r1;
                const long long margin = r2 == 1 ? 2 : 1;
                if (w < 2 * margin + 1 || h < 2 * margin + 1) continue;
                const int mx = 1 + (int)(rng() % (w - 2 * margin));
                const int my = 1 + (int)(rng() % (h - 2 * margin));
                const long long i0 = p.i0 * r1 + margin + (long long)(rng() % (w - 2 * margin - mx + 1));
                const long long j0 = p.j0 * r1 + margin + (long long)(rng() % (h - 2 * margin - my + 1));
                pd.push_back(patch(c, 3, r2, c.d.dx / r1, c.d.dy / r1, i0, j0, mx, my));
            }
        }
        swa_patchset ps;
        set_patches(ps, pd);
        if (ps.lev[1].npatches == 0 || (two && ps.lev[3].npatches == 0)) continue;
        const int L = two ? 2 : 1;
        const int levels[2] = {1, 3}, ratios[2] = {r1, r2};
        std::vector<amr::HostMaps> M1, M2;
        if (amr::build_maps(c, &ps, L, levels, ratios, M1) != SWA_OK) {
            printf("trial %d rejected a valid layout: %s\n", trial, swa_last_error());
            failures++;
            continue;
        }
        brute_maps(c, &ps, L, levels, ratios, M2);
        (two ? checked2 : checked)++;
        for (int l = 1; l <= L; l++) {
            // a ring cell's entry is its patch's base plus its ring index
            // (what a level launch filling its own rings looks up)
            for (size_t e = 0; e < M1[l].fill.size(); e++) {
                const int4 m = M1[l].fill[e];
                const swa_patch_desc &q = ps.pd[m.x];
                const int i = m.y % q.nx, j = m.y / q.nx;
                if (!patches::ring_cell(i, j, q.nx, q.ny) ||
                    M1[l].base[m.x] + patches::ring_index(i, j, q.nx, q.ny) != (int)e) {
                    printf("trial %d level %d: entry %zu is not at its ring index\n", trial, l, e);
                    failures++;
                    break;
                }
            }
            (l == 2 ? edges2 : edges) += (long long)M1[l].cf.size();
            if (!same_maps(M1[l], M2[l])) {
                printf("trial %d level %d: maps differ (%zu vs %zu edges)\n", trial, l,
                       M1[l].cf.size(), M2[l].cf.size());
                failures++;
            }
        }
    }
    // geometry that must be rejected
    GridRefs c{};
    c.d.ndim = 2; c.d.precision = SWA_FP32; c.d.nx = 20; c.d.ny = 20;
    c.d.dx = 10.0; c.d.dy = 10.0;
    const int one = 1;
    int two = 2;
    struct Bad { const char *what; swa_patch_desc q; int r; } bad[] = {
        {"ring outside the domain", patch(c, 1, 2, 10, 10, 0, 5, 4, 4), 2},
        {"interior off the coarse corners", patch(c, 1, 2, 10, 10, 5, 5, 4, 4), 2},
        {"cell size not coarse / r", patch(c, 1, 2, 10, 10, 5, 5, 4, 4), 3},
        {"interior not whole coarse cells", patch(c, 1, 2, 10, 10, 5, 5, 4, 4), 2},
    };
    bad[1].q.x_lo += 0.5 * bad[1].q.dx;
    bad[3].q.nx += 1;
    for (auto &b : bad) {
        swa_patchset ps;
        set_patches(ps, {b.q});
        std::vector<amr::HostMaps> M;
        if (amr::build_maps(c, &ps, 1, &one, &b.r, M) != SWA_EINVAL) {
            printf("not rejected: %s\n", b.what);
            failures++;
        }
    }
    GridRefs c64 = c;
    c64.d.precision = SWA_FP64;
    {
        swa_patchset ps;
        set_patches(ps, {patch(c, 1, 2, 10, 10, 5, 5, 4, 4)});
        std::vector<amr::HostMaps> M;
        if (amr::build_maps(c64, &ps, 1, &one, &two, M) != SWA_EINVAL) {
            printf("not rejected: FP64 coarse grid\n");
            failures++;
        }
    }
    {
        // a fine level with a wall: the ring fills assume extrapolation
        swa_patchset ps;
        set_patches(ps, {patch(c, 1, 2, 10, 10, 5, 5, 4, 4)});
        ps.common.bc[2] = SWA_BC_WALL;
        std::vector<amr::HostMaps> M;
        if (amr::build_maps(c, &ps, 1, &one, &two, M) != SWA_EINVAL) {
            printf("not rejected: fine patch set with a wall\n");
            failures++;
        }
    }
    {
        // a level-2 patch whose ring leaves the level-1 interior (level-1
        // interior: coarse cells 5..8, level-1 cells 10..17; the level-2
        // patch's ring reaches level-1 cell 9)
        swa_patchset ps;
        set_patches(ps, {patch(c, 1, 2, 10, 10, 5, 5, 4, 4), patch(c, 2, 2, 5, 5, 10, 11, 3, 3)});
        const int lv[2] = {1, 2}, rr[2] = {2, 2};
        std::vector<amr::HostMaps> M;
        if (amr::build_maps(c, &ps, 2, lv, rr, M) != SWA_EINVAL) {
            printf("not rejected: a level-2 patch outside level 1\n");
            failures++;
        }
        // the same patch one level-1 cell further in is accepted
        set_patches(ps, {patch(c, 1, 2, 10, 10, 5, 5, 4, 4), patch(c, 2, 2, 5, 5, 11, 11, 3, 3)});
        if (amr::build_maps(c, &ps, 2, lv, rr, M) != SWA_OK) {
            printf("rejected a nested level-2 patch: %s\n", swa_last_error());
            failures++;
        }
    }
    printf("layouts checked: %d one-level (%lld edges), %d two-level (%lld level-2 edges), "
           "failures %d\n", checked, edges, checked2, edges2, failures);
    return failures == 0 && checked >= 100 && checked2 >= 100 && edges > 1000 && edges2 > 500
               ? 0 : 1;
}
