"""GPU parity of the two-level AMR glue (swa_amr_step) against the oracle's
hierarchy (oracle/amr.py), through the C ABI.

Tolerances: the GPU levels are FP32 (perturbation form), the oracle FP64:
eta within 2e-5 m (a 0.5 m hump over 80-120 m), momenta within 2e-5 of their
maximum, after the steps each test takes, with refluxing on and off.  Exact
where FP32 is exact: the ocean at rest, r = 1 against the single grid, a
patch cut in two.  Mass (FP64 audit of the coarse grid, whose covered cells
hold the fine means): with refluxing it stays within 1e-9 of its start
(relative; FP32 rounding of the updates is near 1e-11), without it drifts by
more than 1e-7 (the oracle drifts by 7e-7 to 2e-6 on these layouts).
"""
import numpy as np
import pytest

import oracle as O
from oracle.amr import Hierarchy, Patch
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


def coarse_desc(S, case):
    nc, dx = case["nc"], case["dx"]
    return S.make_desc(2, nc, nc, 0.0, 0.0, dx, dx, precision=S.SWA_FP32, bc=(1, 1, 1, 1))


def gpu_hierarchy(S, case):
    grid = S.Grid(coarse_desc(S, case), case["coarse"]["B"])
    c = case["coarse"]
    grid.set_state(c["eta"], c["hu"], c["hv"], 0.0)
    nc, dx = case["nc"], case["dx"]
    # the fine level extrapolates beyond its rings, as the oracle's patches do
    common = S.make_desc(2, nc, nc, 0.0, 0.0, dx, dx, precision=S.SWA_FP32)
    descs = [p["desc"] for p in case["patches"]]
    ps = S.PatchSet(descs, [p["B"] for p in case["patches"]], common)
    for k, p in enumerate(case["patches"]):
        ps.set_state(k, p["eta"], p["hu"], p["hv"])
    ps.start(1, 0.0)
    amr = S.Amr(grid, ps, 1, case["r"])
    return grid, ps, amr


def oracle_hierarchy(case, reflux=True):
    nc, dx, r = case["nc"], case["dx"], case["r"]
    cg = O.Grid(2, nc, nc, 0.0, 0.0, dx, dx, order=2, bc=(1, 1, 1, 1))
    c = case["coarse"]
    patches = [Patch(*p["box"]) for p in case["patches"]]
    H = Hierarchy(cg, c["B"], patches, r, [p["B"] for p in case["patches"]], reflux=reflux)
    H.set_state(c["eta"] - c["B"], c["hu"], c["hv"],
                [(p["eta"] - p["B"], p["hu"], p["hv"]) for p in case["patches"]], 0.0)
    return H, cg


def bath32(B):
    # the FP32 levels store hbar = float(-B): give the oracle B = -hbar
    return -(np.float32(-B).astype(np.float64))


def case32(case):
    out = dict(case)
    out["coarse"] = dict(case["coarse"], B=bath32(case["coarse"]["B"]))
    out["patches"] = [dict(p, B=bath32(p["B"])) for p in case["patches"]]
    return out


def dt_coarse(dx):
    return 0.6 * 0.75 * dx / np.sqrt(9.81 * 130.0)


def run_both(S, case, steps, m=1, reflux=True):
    grid, ps, amr = gpu_hierarchy(S, case)
    amr.set_reflux(reflux)
    H, cg = oracle_hierarchy(case32(case), reflux=reflux)
    assert amr.info()[2] == len(H.cf_edges)
    dt, t = dt_coarse(case["dx"]), 0.0
    for _ in range(steps):
        amr.step(t, dt, m)
        assert H.step(t, dt, m)
        t = t + dt
    assert S.swa_sync_status() == 0
    return grid, ps, H, t


@pytest.mark.parametrize("r,boxes", [
    (2, [(8, 8, 8, 8)]),
    (4, [(6, 7, 5, 6), (10, 9, 6, 5), (15, 4, 3, 3)]),   # overlapping, adjacent, apart
    (3, [(7, 8, 4, 7), (11, 8, 5, 7)]),                   # odd ratio, siblings side by side
])
@pytest.mark.parametrize("reflux", [True, False])
def test_hierarchy_matches_the_oracle(S, r, boxes, reflux):
    case = synth.amr_basin(24, r, boxes)
    grid, ps, H, t = run_both(S, case, 6, reflux=reflux)
    st = grid.get_state()
    Bc = case32(case)["coarse"]["B"]
    assert np.abs(st["eta"] - (H.h + Bc)).max() <= 2e-5
    for a, b in ((st["hu"], H.hu), (st["hv"], H.hv)):
        assert np.abs(a - b).max() <= 2e-5 * np.abs(b).max()
    for k, p in enumerate(case32(case)["patches"]):
        f = ps.get_state(k)
        fh, fu, fv = H.fine[k]
        g = H.grids[k]
        inner = np.zeros((g.ny, g.nx), bool)
        inner[2:-2, 2:-2] = True
        inner = inner.ravel()
        assert np.abs(f["eta"] - (fh + p["B"]))[inner].max() <= 2e-5
        assert np.abs(f["hu"] - fu)[inner].max() <= 2e-5 * np.abs(fu).max()
        assert np.abs(f["hv"] - fv)[inner].max() <= 2e-5 * np.abs(fv).max()
    assert abs(grid.time()[0] - t) <= 1e-12 * t and abs(ps.time(1)[0] - t) <= 1e-12 * t


MASS_SETS = [(2, [(8, 8, 8, 8)]),
             (4, [(6, 6, 5, 7), (11, 9, 6, 4)]),
             (3, [(4, 4, 6, 6), (10, 4, 4, 6), (12, 7, 5, 5)])]


def coarse_mass(S, grid):
    m = torch.zeros(1, dtype=torch.float64, device="cuda")
    S.swa_grid_mass(grid.h, m)
    torch.cuda.synchronize()
    return m.item()


@pytest.mark.parametrize("r,boxes", MASS_SETS)
def test_refluxing_conserves_mass(S, r, boxes):
    """Walls all round, coarse bottom and surface the means of the fine
    samples: the coarse grid's mass (its covered cells hold the fine means)
    stays constant over 10 coarse steps with refluxing and drifts without."""
    drift = {}
    for reflux in (True, False):
        case = synth.amr_basin(24, r, boxes, mean_coarse=True)
        grid, ps, amr = gpu_hierarchy(S, case)
        amr.set_reflux(reflux)
        dt, t = dt_coarse(case["dx"]), 0.0
        m0 = coarse_mass(S, grid)
        for _ in range(10):
            amr.step(t, dt)
            t = t + dt
        assert S.swa_sync_status() == 0
        drift[reflux] = abs(coarse_mass(S, grid) - m0) / m0
    assert drift[True] <= 1e-9, drift
    assert drift[False] > 1e-7, drift
    print(f"r={r}: relative mass drift {drift[True]:.1e} with refluxing, "
          f"{drift[False]:.1e} without")


def test_refluxing_needs_the_split_scheme(S):
    case = synth.amr_basin(16, 2, [(5, 5, 4, 4)])
    grid, ps, amr = gpu_hierarchy(S, case)
    grid.set_scheme(S.SWA_SCHEME_CTU)
    with pytest.raises(S.SwaError):
        amr.step(0.0, dt_coarse(case["dx"]))
    amr.set_reflux(False)
    amr.step(0.0, dt_coarse(case["dx"]))
    assert S.swa_sync_status() == 0


def test_ratio_one_is_the_single_grid_bit_for_bit(S):
    case = synth.amr_basin(24, 1, [(5, 6, 6, 5), (9, 8, 5, 7), (14, 3, 4, 4)], seed=1)
    grid, ps, amr = gpu_hierarchy(S, case)
    plain = S.Grid(coarse_desc(S, case), case["coarse"]["B"])
    c = case["coarse"]
    plain.set_state(c["eta"], c["hu"], c["hv"], 0.0)
    dt, t = dt_coarse(case["dx"]), 0.0
    for _ in range(10):
        amr.step(t, dt)
        plain.step(1, t + dt)
        t = t + dt
    assert S.swa_sync_status() == 0
    a, b = grid.get_state(), plain.get_state()
    for k in ("eta", "hu", "hv"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("r", [2, 4])
def test_ocean_at_rest_stays_at_rest(S, r):
    case = synth.amr_basin(16, r, [(4, 4, 5, 6), (7, 8, 4, 4)], rest=True)
    grid, ps, amr = gpu_hierarchy(S, case)
    dt, t = dt_coarse(case["dx"]), 0.0
    for _ in range(4):
        amr.step(t, dt)
        t = t + dt
    assert S.swa_sync_status() == 0
    st = grid.get_state()
    assert np.all(st["eta"] == 0) and np.all(st["hu"] == 0) and np.all(st["hv"] == 0)
    for k in range(2):
        f = ps.get_state(k)
        assert np.all(f["eta"] == 0) and np.all(f["hu"] == 0) and np.all(f["hv"] == 0)


def test_a_patch_cut_in_two_gives_the_patch_bit_for_bit(S):
    one = synth.amr_basin(24, 2, [(8, 8, 8, 8)])
    two = synth.amr_basin(24, 2, [(8, 8, 3, 8), (11, 8, 5, 8)])
    g1, p1, a1 = gpu_hierarchy(S, one)
    g2, p2, a2 = gpu_hierarchy(S, two)
    dt, t = dt_coarse(one["dx"]), 0.0
    for _ in range(6):
        a1.step(t, dt)
        a2.step(t, dt)
        t = t + dt
    assert S.swa_sync_status() == 0
    s1, s2 = g1.get_state(), g2.get_state()
    for k in ("eta", "hu", "hv"):
        assert np.array_equal(s1[k], s2[k]), k
    whole = p1.get_state(0)["eta"].reshape(20, 20)
    left = p2.get_state(0)["eta"].reshape(20, 10)
    right = p2.get_state(1)["eta"].reshape(20, 14)
    assert np.array_equal(left[2:-2, 2:-2], whole[2:-2, 2:8])
    assert np.array_equal(right[2:-2, 2:-2], whole[2:-2, 8:18])


def test_a_coarse_step_above_its_cfl_step_is_reported(S):
    """dt_c beyond the coarse CFL step: the coarse grid falls short of
    t_n + dt_c and the next status call says so (no device fault)."""
    case = synth.amr_basin(16, 2, [(5, 5, 4, 4)])
    grid, ps, amr = gpu_hierarchy(S, case)
    amr.step(0.0, 5.0 * dt_coarse(case["dx"]))
    assert S.swa_sync_status() == S.SWA_ESTATE
    assert S.swa_sync_status() == 0   # the word was cleared


def test_misaligned_patches_are_rejected(S):
    case = synth.amr_basin(16, 2, [(5, 5, 4, 4)])
    grid = S.Grid(coarse_desc(S, case), case["coarse"]["B"])
    lev, x0, y0, nx, ny, dx, dy = case["patches"][0]["desc"]
    bad = [(lev, x0 + 0.5 * dx, y0, nx, ny, dx, dy)]
    ps = S.PatchSet(bad, [case["patches"][0]["B"]], coarse_desc(S, case))
    with pytest.raises(S.SwaError):
        S.Amr(grid, ps, 1, 2)
