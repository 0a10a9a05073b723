"""GPU parity of the wet/dry option (swa_grid_set_wetdry: the shore solver at
dry and transonic edges) against the oracle's shore solver, through the C
ABI.

Tolerances: FP64 bit for bit (the FP64 kernels evaluate the reference's
expressions in its order without contraction).  FP32 (perturbation form):
depth within 2 dry_tol of the oracle (a cell near dry_tol may fall on the
other side of it in FP32 and keep or lose its momentum), the ocean at rest
against land exactly at rest, mass to 1e-6 relative.
"""
import numpy as np
import pytest

import oracle as O
from paper_1605_05320_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

G = 9.81
TOL = 1e-3


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


def ritter_case():
    n, L = 400, 100.0
    x = -L + (np.arange(n) + 0.5) * 2 * L / n
    B = np.zeros(n)
    h = np.where(x < 0, 1.0, 0.0)
    return dict(ndim=1, nx=n, ny=1, x0=-L, dx=2 * L / n, dy=1.0, B=B, h=h, eta=h.copy(),
                hu=np.zeros(n), hv=None, cfl=0.75, steps=200, t_end=6.0)


def island_case():
    n, L = 48, 1000.0
    xc = (np.arange(n) + 0.5) * L / n
    X, Y = np.meshgrid(xc, xc)
    B = (-2.0 + 3.0 * np.exp(-((X - 500) ** 2 + (Y - 450) ** 2) / 150 ** 2) + 0.002 * X).ravel()
    return dict(ndim=2, nx=n, ny=n, x0=0.0, dx=L / n, dy=L / n, B=B, h=np.maximum(0.0, -B),
                eta=np.zeros(n * n), hu=np.zeros(n * n), hv=np.zeros(n * n), cfl=0.75,
                steps=150, t_end=1e9)


def runup_case(nx=48, ny=40):
    L = 1000.0
    xc = (np.arange(nx) + 0.5) * L / nx
    yc = (np.arange(ny) + 0.5) * L / nx
    X, Y = np.meshgrid(xc, yc)
    B = (-2.0 + 3.0 * X / L + 0.2 * np.cos(Y / 90)).ravel()
    eta = (0.4 * np.exp(-((X - 250) ** 2 + (Y - 500) ** 2) / 80 ** 2)).ravel()
    return dict(ndim=2, nx=nx, ny=ny, x0=0.0, dx=L / nx, dy=L / nx, B=B,
                h=np.maximum(0.0, eta - B), eta=eta, hu=np.zeros(nx * ny),
                hv=np.zeros(nx * ny), cfl=0.5, steps=150, t_end=1e9)


CASES = {"ritter": ritter_case, "island": island_case, "runup": runup_case}


def gpu_run(S, c, precision):
    """The case on the GPU; returns the final state, the clock and the depth
    the state set gave the grid (as its precision stores it), the oracle's
    start."""
    d = S.make_desc(c["ndim"], c["nx"], c["ny"], c["x0"], 0.0, c["dx"], c["dy"],
                    precision=precision, bc=(1, 1, 1, 1), cfl=c["cfl"])
    g = S.Grid(d, c["B"])
    g.set_wetdry(True)
    Bs = c["B"] if precision == S.SWA_FP64 else bath32(c["B"])
    eta = np.where(c["h"] > 0, c["eta"], Bs)   # land: eta = B, h = 0
    g.set_state(eta, c["hu"], c["hv"] if c["hv"] is not None else np.zeros_like(c["hu"]), 0.0)
    if precision == S.SWA_FP64:
        h_start = eta - c["B"]
    else:
        h_start = np.float32(eta).astype(np.float64) - Bs
    g.step(c["steps"], c["t_end"])
    st = g.get_state()
    assert S.swa_sync_status() == 0
    return st, g.time(), h_start


def oracle_run(c, h, B):
    grid = O.Grid(c["ndim"], c["nx"], c["ny"], c["x0"], 0.0, c["dx"], c["dy"], order=2,
                  bc=(1, 1, 1, 1), cfl=c["cfl"], wetdry=1)
    return O.fwd_run(grid, h, c["hu"], c["hv"], B, c["steps"], c["t_end"])


@pytest.mark.parametrize("case", sorted(CASES))
def test_fp64_matches_the_oracle_bit_for_bit(S, case):
    c = CASES[case]()
    st, (t, _, nsteps), h0 = gpu_run(S, c, S.SWA_FP64)
    h, hu, hv, t_ref, k = oracle_run(c, h0, c["B"])
    assert nsteps == k and t == t_ref
    assert np.array_equal(st["h"], h)
    assert np.array_equal(st["hu"], hu)
    if hv is not None:
        assert np.array_equal(st["hv"], hv)
    assert st["h"].min() >= 0.0


@pytest.mark.parametrize("case", sorted(CASES))
def test_fp32_matches_the_oracle(S, case):
    c = CASES[case]()
    st, (t, _, nsteps), h0 = gpu_run(S, c, S.SWA_FP32)
    h, hu, hv, t_ref, k = oracle_run(c, h0, bath32(c["B"]))
    if c["t_end"] < 1e9:
        assert abs(t - t_ref) <= 1e-12 * t_ref
    else:
        assert nsteps == k
    assert np.abs(st["h"] - h).max() <= 2 * TOL, np.abs(st["h"] - h).max()
    assert st["h"].min() >= 0.0
    if case == "island":
        assert np.all(st["hu"] == 0) and np.all(st["hv"] == 0)
        assert np.all(st["eta"][c["h"] > 0] == 0.0)
    if case == "runup":
        m0 = h0.sum()
        assert abs(st["h"].sum() - m0) <= 1e-6 * m0


def test_without_dry_cells_fp64_is_the_plain_step(S):
    sc = synth.small_2d(60, 44, seed=3)
    out = []
    for wd in (False, True):
        d = S.make_desc(2, 60, 44, 0.0, 0.0, sc.grid.dx, sc.grid.dy, precision=S.SWA_FP64,
                        bc=(1, 0, 0, 1))
        g = S.Grid(d, sc.B)
        g.set_wetdry(wd)
        g.set_state(sc.eta0, sc.hu0, sc.hv0, 0.0)
        g.step(40, 1e12)
        out.append(g.get_state())
    assert S.swa_sync_status() == 0
    for k in ("h", "hu", "hv"):
        assert np.array_equal(out[0][k], out[1][k]), k


def test_wetdry_with_the_unsplit_scheme_is_refused(S):
    c = island_case()
    d = S.make_desc(2, c["nx"], c["ny"], 0.0, 0.0, c["dx"], c["dy"], precision=S.SWA_FP64,
                    bc=(1, 1, 1, 1))
    g = S.Grid(d, c["B"])
    g.set_wetdry(True)
    g.set_scheme(S.SWA_SCHEME_CTU)
    with pytest.raises(S.SwaError):
        g.step(1, 1e9)


def test_land_without_the_option_is_reported(S):
    c = island_case()
    d = S.make_desc(2, c["nx"], c["ny"], 0.0, 0.0, c["dx"], c["dy"], precision=S.SWA_FP64,
                    bc=(1, 1, 1, 1))
    g = S.Grid(d, c["B"])
    assert S.swa_sync_status() == 0          # a new grid reports nothing
    eta = np.where(c["h"] > 0, 0.0, c["B"])
    g.set_state(eta, c["hu"], c["hv"], 0.0)
    assert S.swa_sync_status() == S.SWA_EUNSTABLE
    g.set_wetdry(True)
    g.set_state(eta, c["hu"], c["hv"], 0.0)
    g.step(5, 1e9)
    assert S.swa_sync_status() == 0
