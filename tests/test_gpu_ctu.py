"""GPU parity of the unsplit 2D step with transverse waves (SWA_SCHEME_CTU)
against the oracle's scheme 1, through the C ABI.

Tolerances (as for the split step):
  * FP64: bit-identical to the oracle (built without contraction, same
    evaluation order), identical step count and time;
  * FP32 perturbation form: eta within 1e-5 m, momenta within 1e-5 of their
    maximum after 200 steps (decimetre waves over 4000 m depth).
"""
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
    assert torch.cuda.is_available()
    return swadj


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)


def bath_seen(B, fp32):
    # the FP32 path stores hbar = float(-B): give the oracle B = -hbar
    return -(np.float32(-B).astype(np.float64)) if fp32 else B


def gpu_ctu(S, sc, precision, order, bc, nsteps, t_end=1e12, hu=None, hv=None, cfl=0.75):
    gs = sc.grid
    d = S.make_desc(gs.ndim, gs.nx, gs.ny, gs.x_lo, gs.y_lo, gs.dx, gs.dy,
                    precision=precision, order=order, bc=bc, cfl=cfl)
    g = S.Grid(d, sc.B)
    g.set_scheme(S.SWA_SCHEME_CTU)
    g.set_state(sc.eta0, sc.hu0 if hu is None else hu,
                (sc.hv0 if hv is None else hv) if gs.ndim == 2 else None, 0.0)
    g.step(nsteps, t_end)
    st = g.get_state()
    t, _, n = g.time()
    assert S.swa_sync_status() == 0
    return st, t, n


def oracle_ctu(sc, order, bc, nsteps, t_end=1e12, B=None, hu=None, hv=None, cfl=0.75):
    og = O.Grid.from_spec(sc.grid, order=order, bc=bc, cfl=cfl, scheme=O.SCHEME_CTU)
    B = sc.B if B is None else B
    return O.fwd_run(og, sc.eta0 - B, sc.hu0 if hu is None else hu,
                     sc.hv0 if hv is None else hv, B, nsteps, t_end)


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 1, 1, 1), (1, 0, 0, 1)])
def test_fp64_ctu_bit_identical_to_the_oracle(S, order, bc):
    # 150 x 97: 16 x 8 tiles with ragged edges in both directions
    sc = synth.small_2d(150, 97, seed=21)
    st, t, n = gpu_ctu(S, sc, S.SWA_FP64, order, bc, 300)
    h, hu, hv, t_ref, n_ref = oracle_ctu(sc, order, bc, 300)
    assert n == n_ref == 300 and t == t_ref
    assert np.array_equal(st["h"], h)
    assert np.array_equal(st["hu"], hu)
    assert np.array_equal(st["hv"], hv)


def test_fp64_ctu_fast_flow_and_courant_near_one(S):
    """Strong currents (|u| up to a third of c, so the Roe speeds of both
    signs and the transverse splits all take part) at Courant number 0.95,
    which the unsplit step without transverse terms would not survive."""
    sc = synth.small_2d(61, 45, seed=22)
    rng = np.random.default_rng(22)
    h = sc.eta0 - sc.B
    m = 0.3 * np.sqrt(9.81 * h) * h
    hu = rng.uniform(-1, 1, sc.grid.n) * m
    hv = rng.uniform(-1, 1, sc.grid.n) * m
    st, t, n = gpu_ctu(S, sc, S.SWA_FP64, 2, (1, 0, 1, 0), 120, hu=hu, hv=hv, cfl=0.95)
    h, uu, vv, t_ref, n_ref = oracle_ctu(sc, 2, (1, 0, 1, 0), 120, hu=hu, hv=hv, cfl=0.95)
    assert n == n_ref == 120 and t == t_ref
    assert np.array_equal(st["h"], h) and np.array_equal(st["hu"], uu)
    assert np.array_equal(st["hv"], vv)


def test_ctu_stops_at_t_end(S):
    sc = synth.small_2d(40, 33, seed=23)
    st, t, n = gpu_ctu(S, sc, S.SWA_FP64, 2, (0, 0, 0, 0), 500, 37.5)
    h, _, _, t_ref, n_ref = oracle_ctu(sc, 2, (0, 0, 0, 0), 500, 37.5)
    assert t == t_ref == 37.5 and n == n_ref < 500
    assert np.array_equal(st["h"], h)


def test_fp32_ctu_vs_oracle(S):
    sc = synth.small_2d(130, 90, seed=24, amp=0.5)
    st, t, n = gpu_ctu(S, sc, S.SWA_FP32, 2, (0, 0, 0, 0), 200)
    Bf = bath_seen(sc.B, True)
    h, hu, hv, t_ref, n_ref = oracle_ctu(sc, 2, (0, 0, 0, 0), 200, B=Bf)
    assert n == n_ref
    assert abs(t - t_ref) <= 1e-5 * t_ref
    assert np.abs(st["eta"] - (h + Bf)).max() <= 1e-5
    assert rel(st["hu"], hu) <= 1e-5 and rel(st["hv"], hv) <= 1e-5


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_ctu_ocean_at_rest(S, precision):
    sc = synth.small_2d(70, 45, seed=25)
    p = S.SWA_FP64 if precision == "fp64" else S.SWA_FP32
    d = S.make_desc(2, 70, 45, 0.0, 0.0, sc.grid.dx, sc.grid.dy, precision=p,
                    bc=(1, 0, 1, 0))
    g = S.Grid(d, sc.B)
    g.set_scheme(S.SWA_SCHEME_CTU)
    z = np.zeros(sc.grid.n)
    g.set_state(z, z, z, 0.0)
    g.step(300, 1e12)
    st = g.get_state()
    assert np.all(st["eta"] == 0.0) and np.all(st["hu"] == 0) and np.all(st["hv"] == 0)
    assert g.time()[2] == 300 and S.swa_sync_status() == 0


def test_ctu_on_a_1d_grid_is_the_split_step(S):
    sc = synth.config1()
    gs = sc.grid
    out = []
    for scheme in (S.SWA_SCHEME_SPLIT, S.SWA_SCHEME_CTU):
        d = S.make_desc(1, gs.nx, 1, gs.x_lo, 0.0, gs.dx, gs.dy, precision=S.SWA_FP64)
        g = S.Grid(d, sc.B)
        g.set_scheme(scheme)
        g.set_state(sc.eta0, sc.hu0, None, 0.0)
        g.step(200, 1e12)
        out.append(g.get_state())
    assert np.array_equal(out[0]["h"], out[1]["h"])
    assert np.array_equal(out[0]["hu"], out[1]["hu"])


@pytest.mark.parametrize("nx,ny", [(2, 2), (3, 5), (17, 2), (5, 9), (33, 3)])
@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 1, 1, 1)])
def test_ctu_degenerate_grids(S, nx, ny, bc):
    """Grids narrower or lower than one tile, a few cells across."""
    sc = synth.small_2d(nx, ny, seed=26)
    st, t, n = gpu_ctu(S, sc, S.SWA_FP64, 2, bc, 40)
    h, hu, hv, t_ref, n_ref = oracle_ctu(sc, 2, bc, 40)
    assert n == n_ref == 40 and t == t_ref
    assert np.array_equal(st["h"], h) and np.array_equal(st["hu"], hu)
    assert np.array_equal(st["hv"], hv)
    st, t, n = gpu_ctu(S, sc, S.SWA_FP32, 2, bc, 40)
    Bf = bath_seen(sc.B, True)
    h, hu, hv, t_ref, n_ref = oracle_ctu(sc, 2, bc, 40, B=Bf)
    assert n == n_ref
    assert np.abs(st["eta"] - (h + Bf)).max() <= 1e-5
    scale = max(np.abs(hu).max(), np.abs(hv).max(), 1.0)
    assert np.abs(st["hu"] - hu).max() <= 1e-5 * scale
    assert np.abs(st["hv"] - hv).max() <= 1e-5 * scale


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_ctu_full_size_step_sampled_against_oracle_windows(S, precision):
    """2048^2 (the basin of the scenario benchmark): one unsplit step from a
    perturbed state, sampled cells compared with the oracle on 9 x 9 windows
    around them (a cell's update reads cells within 2 of it, corners
    included)."""
    sc = synth.config2()
    rng = np.random.default_rng(27)
    hu = rng.uniform(-20, 20, sc.grid.n)
    hv = rng.uniform(-20, 20, sc.grid.n)
    p = S.SWA_FP64 if precision == "fp64" else S.SWA_FP32
    fp32 = p == S.SWA_FP32
    gs = sc.grid
    d = S.make_desc(2, gs.nx, gs.ny, gs.x_lo, gs.y_lo, gs.dx, gs.dy, precision=p)
    g = S.Grid(d, sc.B)
    g.set_scheme(S.SWA_SCHEME_CTU)
    g.set_state(sc.eta0, hu, hv, 0.0)
    g.step(1, 1e12)
    s1 = g.get_state()
    assert S.swa_sync_status() == 0
    Bs = bath_seen(sc.B, fp32)
    if fp32:
        eta = np.float32(sc.eta0).astype(np.float64)
        hu = np.float32(hu).astype(np.float64)
        hv = np.float32(hv).astype(np.float64)
    else:
        eta = sc.eta0
    s0 = {"h": eta - Bs, "hu": hu, "hv": hv}
    og = O.Grid.from_spec(gs)
    dt = og.cfl / O.fwd_smax(og, s0["h"], s0["hu"], s0["hv"])
    nx = gs.nx
    cells = [(int(i), int(j)) for i, j in zip(rng.integers(0, nx, 150), rng.integers(0, nx, 150))]
    cells += [(0, 0), (nx - 1, 5), (7, nx - 1), (nx - 1, nx - 1), (16, 8), (15, 7)]
    for (i, j) in cells:
        ii = np.clip(np.arange(i - 4, i + 5), 0, nx - 1)
        jj = np.clip(np.arange(j - 4, j + 5), 0, nx - 1)
        idx = (jj[:, None] * nx + ii[None, :]).ravel()
        wg = O.Grid(2, 9, 9, 0.0, 0.0, gs.dx, gs.dy, order=2, scheme=O.SCHEME_CTU)
        h, u, v = O.fwd_step(wg, s0["h"][idx], s0["hu"][idx], s0["hv"][idx], Bs[idx], dt)
        o = j * nx + i
        if not fp32:
            assert abs(s1["h"][o] - h[40]) <= 1e-12 * 4000
            assert abs(s1["hu"][o] - u[40]) <= 1e-12 * 200
            assert abs(s1["hv"][o] - v[40]) <= 1e-12 * 200
        else:
            assert abs(s1["eta"][o] - (h[40] + Bs[o])) <= 2e-6
            assert abs(s1["hu"][o] - u[40]) <= 2e-5 and abs(s1["hv"][o] - v[40]) <= 2e-5
