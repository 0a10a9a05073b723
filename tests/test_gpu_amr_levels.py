"""GPU parity of the AMR glue over nested levels (swa_create_amr_levels,
swa_amr_step) against the oracle's hierarchy (oracle/amr_levels.py), through
the C ABI.

Tolerances as for two levels: eta within 2e-5 m (a 0.5 m hump over 80-120
m), momenta within 2e-5 of their maximum, on every level's interiors, with
refluxing on and off.  Exact where FP32 is exact: ratios 1 at every level
against the single grid, a level-2 patch cut in two, the ocean at rest.
Mass (FP64 audit of the coarse grid, whose covered cells hold the means of
the levels below): within 1e-9 of its start with refluxing, drifting by more
than 1e-7 without.
"""
import numpy as np
import pytest

import oracle as O
from oracle.amr_levels import LevelHierarchy, Patch
from paper_1605_05320_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def S():
    from paper_1605_05320_gb300 import build
    build.build()
    from paper_1605_05320_gb300 import swadj
    swadj.load()
    assert torch.cuda.is_available()
    return swadj


def bath32(B):
    return -(np.float32(-B).astype(np.float64))


def coarse_desc(S, case):
    nc, dx = case["nc"], case["dx"]
    return S.make_desc(2, nc, nc, 0.0, 0.0, dx, dx, precision=S.SWA_FP32, bc=(1, 1, 1, 1))


def gpu_levels(S, case):
    grid = S.Grid(coarse_desc(S, case), case["coarse"]["B"])
    c = case["coarse"]
    grid.set_state(c["eta"], c["hu"], c["hv"], 0.0)
    nc, dx = case["nc"], case["dx"]
    common = S.make_desc(2, nc, nc, 0.0, 0.0, dx, dx, precision=S.SWA_FP32)
    pats = [p for lv in case["levels"] for p in lv["patches"]]
    ps = S.PatchSet([p["desc"] for p in pats], [p["B"] for p in pats], common)
    for k, p in enumerate(pats):
        ps.set_state(k, p["eta"], p["hu"], p["hv"])
    L = len(case["levels"])
    for l in range(1, L + 1):
        ps.start(l, 0.0)
    amr = S.Amr(grid, ps, list(range(1, L + 1)), [lv["r"] for lv in case["levels"]])
    return grid, ps, amr


def oracle_levels(case, reflux=True):
    nc, dx = case["nc"], case["dx"]
    cg = O.Grid(2, nc, nc, 0.0, 0.0, dx, dx, order=2, bc=(1, 1, 1, 1))
    c = case["coarse"]
    Bc = bath32(c["B"])
    spec, fine = [], []
    for lv in case["levels"]:
        spec.append(([Patch(*p["box"]) for p in lv["patches"]], lv["r"],
                     [bath32(p["B"]) for p in lv["patches"]]))
        fine.append([(p["eta"] - bath32(p["B"]), p["hu"], p["hv"]) for p in lv["patches"]])
    H = LevelHierarchy(cg, Bc, spec, reflux=reflux)
    H.set_state(c["eta"] - Bc, c["hu"], c["hv"], fine, 0.0)
    return H


def dt_coarse(dx):
    return 0.6 * 0.75 * dx / np.sqrt(9.81 * 130.0)


LAYOUTS = [
    [(2, [(6, 6, 12, 12)]), (2, [(20, 20, 8, 8)])],
    # two level-1 patches side by side, level 2 across their edge at ratio 3
    [(2, [(5, 6, 7, 12), (12, 6, 6, 12)]), (3, [(14, 16, 6, 8), (20, 16, 5, 8)])],
    # three levels below the coarse grid
    [(2, [(6, 6, 12, 12)]), (2, [(18, 18, 12, 12)]), (2, [(44, 44, 8, 8)])],
]


def patch_index(case):
    """(level, k within level) -> patch-set index."""
    idx, n = {}, 0
    for l, lv in enumerate(case["levels"], start=1):
        for k in range(len(lv["patches"])):
            idx[(l, k)] = n
            n += 1
    return idx


@pytest.mark.parametrize("layout", range(len(LAYOUTS)))
@pytest.mark.parametrize("reflux", [True, False])
def test_levels_match_the_oracle(S, layout, reflux):
    case = synth.amr_levels_basin(24, LAYOUTS[layout])
    grid, ps, amr = gpu_levels(S, case)
    amr.set_reflux(reflux)
    H = oracle_levels(case, reflux)
    for l in range(1, len(case["levels"]) + 1):
        assert amr.info(l)[2] == len(H.edges[l])
    dt, t = dt_coarse(case["dx"]), 0.0
    for _ in range(4):
        amr.step(t, dt)
        assert H.step(t, dt)
        t = t + dt
    assert S.swa_sync_status() == 0
    st = grid.get_state()
    assert np.abs(st["eta"] - (H.h + H.B)).max() <= 2e-5
    for a, b in ((st["hu"], H.hu), (st["hv"], H.hv)):
        assert np.abs(a - b).max() <= 2e-5 * np.abs(b).max()
    idx = patch_index(case)
    for l in range(1, len(case["levels"]) + 1):
        for k, g in enumerate(H.G[l]):
            f = ps.get_state(idx[(l, k)])
            fh, fu, fv = H.q[l][k]
            inner = np.zeros((g.ny, g.nx), bool)
            inner[2:-2, 2:-2] = True
            inner = inner.ravel()
            assert np.abs(f["eta"] - (fh + H.Bf[l][k]))[inner].max() <= 2e-5, (l, k)
            assert np.abs(f["hu"] - fu)[inner].max() <= 2e-5 * np.abs(fu).max(), (l, k)
            assert np.abs(f["hv"] - fv)[inner].max() <= 2e-5 * np.abs(fv).max(), (l, k)
        assert abs(ps.time(l)[0] - t) <= 1e-12 * t


@pytest.mark.parametrize("layout", range(len(LAYOUTS)))
def test_fills_in_the_level_launch_equal_the_fill_kernel(S, layout):
    """The rings filled by the level launches themselves (the default) and by
    a fill kernel before each launch give the same hierarchy bit for bit."""
    out = []
    for mode in (S.SWA_AMR_FILL_FUSED, S.SWA_AMR_FILL_KERNEL):
        case = synth.amr_levels_basin(24, LAYOUTS[layout])
        grid, ps, amr = gpu_levels(S, case)
        amr.set_fill_mode(mode)
        dt, t = dt_coarse(case["dx"]), 0.0
        for _ in range(4):
            amr.step(t, dt)
            t = t + dt
        assert S.swa_sync_status() == 0
        npat = sum(len(lv["patches"]) for lv in case["levels"])
        out.append([grid.get_state()] + [ps.get_state(k) for k in range(npat)])
    for a, b in zip(*out):
        for k in ("eta", "hu", "hv"):
            assert np.array_equal(a[k], b[k]), k


def coarse_mass(S, grid):
    m = torch.zeros(1, dtype=torch.float64, device="cuda")
    S.swa_grid_mass(grid.h, m)
    torch.cuda.synchronize()
    return m.item()


@pytest.mark.parametrize("layout", range(len(LAYOUTS)))
def test_levels_conserve_mass(S, layout):
    drift = {}
    for reflux in (True, False):
        case = synth.amr_levels_basin(24, LAYOUTS[layout], mean_coarse=True)
        grid, ps, amr = gpu_levels(S, case)
        amr.set_reflux(reflux)
        dt, t = dt_coarse(case["dx"]), 0.0
        m0 = coarse_mass(S, grid)
        for _ in range(6):
            amr.step(t, dt)
            t = t + dt
        assert S.swa_sync_status() == 0
        drift[reflux] = abs(coarse_mass(S, grid) - m0) / m0
    assert drift[True] <= 1e-9, drift
    assert drift[False] > 1e-7, drift
    print(f"layout {layout}: relative mass drift {drift[True]:.1e} with refluxing, "
          f"{drift[False]:.1e} without")


def test_ratios_one_are_the_single_grid_bit_for_bit(S):
    layout = [(1, [(4, 5, 14, 12), (15, 3, 6, 8)]),
              (1, [(7, 8, 6, 5), (11, 10, 5, 5), (17, 5, 2, 4)])]
    case = synth.amr_levels_basin(24, layout, seed=1)
    grid, ps, amr = gpu_levels(S, case)
    plain = S.Grid(coarse_desc(S, case), case["coarse"]["B"])
    c = case["coarse"]
    plain.set_state(c["eta"], c["hu"], c["hv"], 0.0)
    dt, t = dt_coarse(case["dx"]), 0.0
    for _ in range(8):
        amr.step(t, dt)
        plain.step(1, t + dt)
        t = t + dt
    assert S.swa_sync_status() == 0
    a, b = grid.get_state(), plain.get_state()
    for k in ("eta", "hu", "hv"):
        assert np.array_equal(a[k], b[k]), k


def test_ocean_at_rest_stays_at_rest(S):
    case = synth.amr_levels_basin(16, [(4, [(4, 4, 8, 8)]), (2, [(18, 18, 4, 5)])], rest=True)
    grid, ps, amr = gpu_levels(S, case)
    dt, t = dt_coarse(case["dx"]), 0.0
    for _ in range(3):
        amr.step(t, dt)
        t = t + dt
    assert S.swa_sync_status() == 0
    st = grid.get_state()
    assert np.all(st["eta"] == 0) and np.all(st["hu"] == 0) and np.all(st["hv"] == 0)
    for k in range(2):
        f = ps.get_state(k)
        assert np.all(f["eta"] == 0) and np.all(f["hu"] == 0) and np.all(f["hv"] == 0)


def test_a_level_two_patch_cut_in_two_gives_the_patch_bit_for_bit(S):
    one = synth.amr_levels_basin(24, [(2, [(6, 6, 12, 12)]), (2, [(20, 20, 8, 8)])])
    two = synth.amr_levels_basin(24, [(2, [(6, 6, 12, 12)]), (2, [(20, 20, 3, 8), (23, 20, 5, 8)])])
    g1, p1, a1 = gpu_levels(S, one)
    g2, p2, a2 = gpu_levels(S, two)
    dt, t = dt_coarse(one["dx"]), 0.0
    for _ in range(4):
        a1.step(t, dt)
        a2.step(t, dt)
        t = t + dt
    assert S.swa_sync_status() == 0
    s1, s2 = g1.get_state(), g2.get_state()
    for k in ("eta", "hu", "hv"):
        assert np.array_equal(s1[k], s2[k]), k
        assert np.array_equal(p1.get_state(0)[k], p2.get_state(0)[k]), k
    whole = p1.get_state(1)["eta"].reshape(20, 20)
    left = p2.get_state(1)["eta"].reshape(20, 10)
    right = p2.get_state(2)["eta"].reshape(20, 14)
    assert np.array_equal(left[2:-2, 2:-2], whole[2:-2, 2:8])
    assert np.array_equal(right[2:-2, 2:-2], whole[2:-2, 8:18])


def test_a_level_outside_its_parent_is_rejected(S):
    case = synth.amr_levels_basin(24, [(2, [(6, 6, 12, 12)]), (2, [(12, 20, 6, 6)])])
    with pytest.raises(S.SwaError):
        gpu_levels(S, case)


def test_levels_off_their_start_time_are_reported(S):
    """A level stepped on its own before the hierarchy step starts it away
    from t_n: the next status call says so (no device fault)."""
    case = synth.amr_levels_basin(24, LAYOUTS[0])
    grid, ps, amr = gpu_levels(S, case)
    ps.step(2, 1, 10.0)
    amr.step(0.0, dt_coarse(case["dx"]))
    assert S.swa_sync_status() == S.SWA_ESTATE
    assert S.swa_sync_status() == 0
