"""swa_step_forward_static: the forward step for callers that cannot allocate
device memory (their memory belongs to a host framework, or allocation is not
allowed where they run).  It takes its reduction scratch from a static array
inside the library; here it is checked against the workspace-based
swa_step_forward on the same inputs, two calls in a row, in both precisions.

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

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


def _storage(S, sc, precision, ndim=2):
    """The caller's own device arrays, in the library's storage layout (the
    third momentum array is absent in 1D)."""
    if precision == S.SWA_FP64:
        dt = torch.float64
        q = [sc.eta0 - sc.B, sc.hu0, sc.hv0]
        bath = sc.B
    else:
        dt = torch.float32
        q = [sc.eta0, sc.hu0, sc.hv0]
        bath = -sc.B
    dev = [torch.tensor(np.asarray(a, dtype=np.float64), device="cuda").to(dt) for a in q]
    if ndim == 1:
        dev[2] = None
    return dev, torch.tensor(np.asarray(bath, dtype=np.float64), device="cuda").to(dt)


def _check_two_calls(S, sc, d, precision, ndim):
    """Two static steps in a row against two workspace steps on a grid made
    from the same inputs."""
    g = S.Grid(d, sc.B)
    g.set_state(sc.eta0, sc.hu0, sc.hv0 if ndim == 2 else None, 0.0)
    q_in, bath = _storage(S, sc, d.precision, ndim)
    tol = 1e-12 if precision == "fp64" else 1e-6
    for call in range(2):
        _, dt, _ = g.time()
        q_out = [None if x is None else torch.empty_like(x) for x in q_in]
        smax = torch.zeros(1, dtype=torch.float64, device="cuda")
        S.swa_step_forward_static(d, q_in, q_out, bath, dt, smax)
        g.step(1, 1e300)
        torch.cuda.synchronize()
        assert S.swa_sync_status() == 0
        ref = g.get_state()
        r0 = ref["h"] if precision == "fp64" else ref["eta"]
        refs = (r0, ref["hu"], ref["hv"])[:ndim + 1]
        got = [x.double().cpu().numpy() for x in q_out[:ndim + 1]]
        for a, b in zip(got, refs):
            assert np.abs(a - b).max() <= tol * max(np.abs(b).max(), 1.0)
        _, dt_next, _ = g.time()
        assert abs(d.cfl / smax.item() - dt_next) <= 1e-12 * dt_next
        q_in = q_out


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_static_step_matches_workspace_step_twice(S, precision):
    p = S.SWA_FP64 if precision == "fp64" else S.SWA_FP32
    sc = synth.small_2d(150, 97, seed=21)
    d = S.make_desc(2, sc.grid.nx, sc.grid.ny, 0.0, 0.0, sc.grid.dx, sc.grid.dy,
                    precision=p)
    _check_two_calls(S, sc, d, precision, 2)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_static_step_1d_matches_workspace_step_twice(S, precision):
    """1D grid (2000 cells, step shelf): the third arrays are absent."""
    p = S.SWA_FP64 if precision == "fp64" else S.SWA_FP32
    sc = synth.config1()
    d = S.make_desc(1, sc.grid.nx, 1, sc.grid.x_lo, 0.0, sc.grid.dx, 1.0, precision=p)
    _check_two_calls(S, sc, d, precision, 1)


def test_static_step_at_the_slot_limit(S):
    """A 2048 x 2048 FP64 grid needs exactly SWA_STATIC_MAX_BLOCKS reduction
    slots: accepted, and equal to the workspace step."""
    sc = synth.small_2d(2048, 2048, seed=22, L=2048e3)
    d = S.make_desc(2, 2048, 2048, 0.0, 0.0, sc.grid.dx, sc.grid.dy, precision=S.SWA_FP64)
    _check_two_calls(S, sc, d, "fp64", 2)


def test_static_step_rejects_oversized_grid(S):
    d = S.make_desc(2, 4096, 2048, 0.0, 0.0, 1e3, 1e3, precision=S.SWA_FP64)
    dummy = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in range(3)]
    out = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in range(3)]
    with pytest.raises(S.SwaError) as e:
        S.swa_step_forward_static(d, dummy, out, dummy[0], 1.0, None)
    assert e.value.code == S.SWA_ENOMEM
    assert "static scratch" in str(e.value)
