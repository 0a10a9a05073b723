"""Batched uneven patches (one persistent launch per level step) against the
FP64 oracle, stepped level by level with the level's shared time step
dt_l = cfl / max over the level's cells, and against the single-grid path."""
import numpy as np
import pytest

import oracle as O
from paper_1605_05320_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def S():
    from paper_1605_05320_gb300 import build
    build.build()
    from paper_1605_05320_gb300 import swadj
    swadj.load()
    return swadj


def bf(B):
    return -(np.float32(-B).astype(np.float64))


def make_patches(seed=3):
    rng = np.random.default_rng(seed)
    sizes = [(2, 2), (17, 40), (33, 5), (70, 70), (16, 16), (5, 129), (64, 48), (31, 33)]
    out = []
    for k, (nx, ny) in enumerate(sizes):
        lev = 1 + (k % 2)
        d = 4000.0 / 4 ** (lev - 1)
        x0 = rng.uniform(300e3, 900e3)
        y0 = rng.uniform(700e3, 1200e3)
        out.append((lev, x0, y0, nx, ny, d, d))
    return out


def test_patches_match_oracle(S):
    patches = make_patches()
    fields = [synth.patch_fields(p, src=(600e3, 950e3), amp=0.5, width=60e3) for p in patches]
    rng = np.random.default_rng(4)
    mom = [(rng.uniform(-2, 2, p[3] * p[4]), rng.uniform(-2, 2, p[3] * p[4])) for p in patches]
    common = S.make_desc(2, 2, 2, 0, 0, 1, 1, precision=S.SWA_FP32)
    ps = S.PatchSet(patches, [f[0] for f in fields], common)
    for k, (B, eta) in enumerate(fields):
        ps.set_state(k, eta, mom[k][0], mom[k][1])
    steps = {1: 6, 2: 9}
    for lev in steps:
        ps.start(lev)
        ps.step(lev, steps[lev])
    torch.cuda.synchronize()
    assert S.swa_sync_status() == 0
    # oracle: level by level with the level-wide dt
    for lev, nst in steps.items():
        ks = [k for k, p in enumerate(patches) if p[0] == lev]
        grids = {k: O.Grid(2, patches[k][3], patches[k][4], patches[k][1], patches[k][2],
                           patches[k][5], patches[k][6]) for k in ks}
        st = {k: [fields[k][1] - bf(fields[k][0]), mom[k][0].copy(), mom[k][1].copy()] for k in ks}
        t = 0.0
        for _ in range(nst):
            smax = max(O.fwd_smax(grids[k], *st[k]) for k in ks)
            dt = 0.75 / smax
            for k in ks:
                st[k] = list(O.fwd_step(grids[k], st[k][0], st[k][1], st[k][2], bf(fields[k][0]), dt))
            t += dt
        tg, _, ng = ps.time(lev)
        assert ng == nst and abs(tg - t) <= 1e-5 * t
        for k in ks:
            got = ps.get_state(k)
            assert np.abs(got["eta"] - (st[k][0] + bf(fields[k][0]))).max() <= 2e-5
            assert np.abs(got["hu"] - st[k][1]).max() <= 2e-4
            assert np.abs(got["hv"] - st[k][2]).max() <= 2e-4


def test_single_patch_is_bit_identical_to_grid(S):
    p = (1, 500e3, 800e3, 150, 97, 2000.0, 2000.0)
    B, eta = synth.patch_fields(p, src=(600e3, 900e3), amp=0.8, width=40e3)
    common = S.make_desc(2, 2, 2, 0, 0, 1, 1, precision=S.SWA_FP32)
    ps = S.PatchSet([p], [B], common)
    z = np.zeros(p[3] * p[4])
    ps.set_state(0, eta, z, z)
    ps.start(1)
    ps.step(1, 25)
    d = S.make_desc(2, p[3], p[4], p[1], p[2], p[5], p[6], precision=S.SWA_FP32)
    g = S.Grid(d, B)
    g.set_state(eta, z, z, 0.0)
    g.step(25, 1e300)
    a, b = ps.get_state(0), g.get_state()
    for f in ("eta", "hu", "hv"):
        assert np.array_equal(a[f], b[f]), f
    assert ps.time(1)[0] == g.time()[0]


def test_quiet_strips_of_patch_and_grid_match_the_full_path(S):
    """A compact source on an ocean at rest, so that most strips are quiet
    at first: one patch (quiet strips, rest CFL terms formed from hbar), the
    same grid (quiet units, rest CFL terms from the grid's table) and the
    grid with the shortcuts off give the same state, and the same time after
    every step (the CFL maximum over cells at rest is exact on each path)."""
    p = (1, 500e3, 800e3, 150, 97, 2000.0, 2000.0)
    B, eta = synth.patch_fields(p, src=(650e3, 890e3), amp=0.8, width=8e3)
    eta = np.where(np.abs(eta) < 1e-6, 0.0, eta)
    z = np.zeros(p[3] * p[4])
    common = S.make_desc(2, 2, 2, 0, 0, 1, 1, precision=S.SWA_FP32)
    ps = S.PatchSet([p], [B], common)
    ps.set_state(0, eta, z, z)
    ps.start(1)
    d = S.make_desc(2, p[3], p[4], p[1], p[2], p[5], p[6], precision=S.SWA_FP32)
    grids = []
    for skip in (1, 0):
        g = S.Grid(d, B)
        S.swa_grid_set_rest_skip(g.h, skip)
        g.set_state(eta, z, z, 0.0)
        grids.append(g)
    for _ in range(30):
        ps.step(1, 1)
        for g in grids:
            g.step(1, 1e300)
        t = [ps.time(1)[0]] + [g.time()[0] for g in grids]
        assert t[0] == t[1] == t[2], t
    assert S.swa_sync_status() == 0
    a = ps.get_state(0)
    for g in grids:
        b = g.get_state()
        for f in ("eta", "hu", "hv"):
            assert np.array_equal(a[f], b[f]), f
    assert np.abs(a["eta"]).max() > 1e-3 and (a["eta"] == 0).mean() > 0.2   # both parts present


def test_single_patch_matches_grid_with_supersonic_band(S):
    """Shallow (10 m) water with a band flowing at 1.5 c among subsonic cells,
    stepped as a grid (strips of 64 rows) and as one patch (strips of 16
    rows): warps group subsonic and supersonic edges differently, and each
    edge's arithmetic must not depend on that."""
    nx, ny = 150, 97
    p = (1, 0.0, 0.0, nx, ny, 1000.0, 1000.0)
    rng = np.random.default_rng(17)
    B = np.full(nx * ny, -10.0)
    eta = 0.2 * rng.standard_normal(nx * ny)
    hu = 2.0 * rng.standard_normal(nx * ny)
    hv = 2.0 * rng.standard_normal(nx * ny)
    band = (np.arange(nx * ny) % nx >= 40) & (np.arange(nx * ny) % nx < 75)
    hu[band] += 1.5 * 10.0 * np.sqrt(9.81 * 10.0)
    common = S.make_desc(2, 2, 2, 0, 0, 1, 1, precision=S.SWA_FP32)
    ps = S.PatchSet([p], [B], common)
    S.swa_patches_set_tile_rows(ps.h, 1, 16)
    ps.set_state(0, eta, hu, hv)
    ps.start(1)
    ps.step(1, 20)
    d = S.make_desc(2, nx, ny, 0.0, 0.0, 1000.0, 1000.0, precision=S.SWA_FP32)
    g = S.Grid(d, B)
    S.swa_grid_set_strip_rows(g.h, 64)
    g.set_state(eta, hu, hv, 0.0)
    g.step(20, 1e300)
    assert S.swa_sync_status() == 0
    a, b = ps.get_state(0), g.get_state()
    for f in ("eta", "hu", "hv"):
        assert np.array_equal(a[f], b[f]), f
    assert ps.time(1)[0] == g.time()[0]


def test_grid_strip_height_does_not_change_results(S):
    """Strip heights 16, 32 and 64 on a ragged grid with walls and momenta."""
    sc = synth.small_2d(97, 45, seed=21)
    res = []
    for rows in (16, 32, 64):
        d = S.make_desc(2, 97, 45, 0.0, 0.0, sc.grid.dx, sc.grid.dy, precision=S.SWA_FP32,
                        bc=(1, 0, 1, 0))
        g = S.Grid(d, sc.B)
        S.swa_grid_set_strip_rows(g.h, rows)
        g.set_state(sc.eta0, sc.hu0, sc.hv0, 0.0)
        g.step(40, 1e300)
        res.append((g.get_state(), g.time()))
    assert S.swa_sync_status() == 0
    for st, t in res[1:]:
        for f in ("eta", "hu", "hv"):
            assert np.array_equal(st[f], res[0][0][f]), f
        assert t == res[0][1]


def test_strip_height_does_not_change_results(S):
    patches = make_patches(seed=5)
    fields = [synth.patch_fields(p, src=(600e3, 950e3), amp=0.5, width=60e3) for p in patches]
    common = S.make_desc(2, 2, 2, 0, 0, 1, 1, precision=S.SWA_FP32)
    res = []
    for rows in (32, 16):
        ps = S.PatchSet(patches, [f[0] for f in fields], common)
        for k, (B, eta) in enumerate(fields):
            z = np.zeros(B.size)
            ps.set_state(k, eta, z, z)
        for lev in (1, 2):
            S.swa_patches_set_tile_rows(ps.h, lev, rows)
            ps.start(lev)
            ps.step(lev, 7)
        res.append([ps.get_state(k)["eta"] for k in range(len(patches))])
    for a, b in zip(*res):
        assert np.array_equal(a, b)


def test_level_steps_replay_in_a_cuda_graph(S):
    patches = make_patches(seed=6)
    fields = [synth.patch_fields(p, src=(600e3, 950e3), amp=0.5, width=60e3) for p in patches]
    common = S.make_desc(2, 2, 2, 0, 0, 1, 1, precision=S.SWA_FP32)

    def fresh():
        ps = S.PatchSet(patches, [f[0] for f in fields], common)
        for k, (B, eta) in enumerate(fields):
            z = np.zeros(B.size)
            ps.set_state(k, eta, z, z)
        for lev in (1, 2):
            ps.start(lev)
        return ps

    ref = fresh()
    for _ in range(3):
        ref.step(1, 4)
        ref.step(2, 4)
    ps = fresh()
    ps.step(1, 1)  # warm-up outside the capture, then undo by restarting
    for k, (B, eta) in enumerate(fields):
        z = np.zeros(B.size)
        ps.set_state(k, eta, z, z)
    for lev in (1, 2):
        ps.start(lev)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        ps.step(1, 4, stream=s)
        ps.step(2, 4, stream=s)
    # capture records without running: replay 3 times = 12 steps per level
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    for k in range(len(patches)):
        assert np.array_equal(ps.get_state(k)["eta"], ref.get_state(k)["eta"])
    assert ps.time(1)[2] == 12 and ps.time(2)[2] == 12
