"""Temporal blocking of the fixed-dt FP32 adjoint (two steps per pass,
swa_adjoint_set_steps_per_pass): every snapshot and the final state are
bit-identical to one step per launch, on grids ragged in both strip
directions, with walls, extrapolation and a mix, orders 1 and 2, an island
of dry cells (wet/dry walls), a snapshot spacing that forces single steps
between pairs, and an odd number of steps."""
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


def _island(sc):
    xc, yc = sc.adj_grid.centres()
    X, Y = np.meshgrid(xc, yc)
    cx, cy = 0.45 * xc[-1], 0.5 * yc[-1]
    land = ((X - cx) ** 2 + (Y - cy) ** 2).ravel() < (0.08 * xc[-1]) ** 2
    sc.B_adj = np.where(land, 5.0, sc.B_adj)
    return sc


def _run(S, sc, bc, order, every, k, steps=None):
    d = S.make_desc(2, sc.adj_grid.nx, sc.adj_grid.ny, 0.0, 0.0, sc.adj_grid.dx,
                    sc.adj_grid.dy, precision=S.SWA_FP32, order=order, bc=bc)
    adj = S.Adjoint(d, sc.B_adj, sc.phi, sc.t_f)
    S.swa_adjoint_set_steps_per_pass(adj.h, k)
    if steps is not None:
        adj.step(steps)
        torch.cuda.synchronize()
        return adj.get_state(), None
    N, _, _ = adj.info()
    store = S.SnapStore(adj, N // every + 3, S.SWA_FP32)
    store.run_adjoint(every)
    K, tau = store.info()
    n = sc.adj_grid.n
    snaps = store.ws[: K * 3 * n * 4].cpu().numpy().view(np.float32).reshape(K, 3, n).copy()
    return snaps, np.array(tau[:K])


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 1, 1, 1), (1, 0, 0, 1)])
@pytest.mark.parametrize("order", [1, 2])
def test_two_steps_per_pass_equal_one_step(S, bc, order):
    sc = _island(synth.small_2d(97, 70, seed=17))
    sc.phi[0] = synth.gaussian_field(sc.adj_grid, 0.7 * sc.adj_grid.nx * sc.adj_grid.dx,
                                     0.4 * sc.adj_grid.ny * sc.adj_grid.dy, 1.0,
                                     5 * sc.adj_grid.dx)
    a, ta = _run(S, sc, bc, order, 5, 1)
    b, tb = _run(S, sc, bc, order, 5, 2)
    assert S.swa_sync_status() == 0
    assert a.shape == b.shape and np.array_equal(ta, tb)
    assert np.array_equal(a, b)
    assert np.abs(a[-1]).max() > 1e-3


@pytest.mark.parametrize("shape", [(2, 2), (5, 3), (24, 33), (49, 2), (130, 96)])
def test_two_steps_per_pass_small_and_ragged(S, shape):
    """Grids narrower than a strip, a few rows high, and a multiple of the
    strip sizes; an odd number of steps (the last one single)."""
    nx, ny = shape
    sc = synth.small_2d(nx, ny, seed=5)
    sc.phi[0] = np.random.default_rng(3).uniform(0.0, 1.0, sc.adj_grid.n)
    for bc in [(0, 0, 0, 0), (1, 1, 1, 1)]:
        a, _ = _run(S, sc, bc, 2, 1, 1, steps=21)
        b, _ = _run(S, sc, bc, 2, 1, 2, steps=21)
        assert np.array_equal(a, b), (shape, bc)
    assert S.swa_sync_status() == 0


def test_two_steps_per_pass_rejected_where_not_built(S):
    sc = synth.config1()
    d = S.make_desc(1, sc.grid.nx, 1, sc.grid.x_lo, 0.0, sc.grid.dx, 1.0,
                    precision=S.SWA_FP32)
    adj = S.Adjoint(d, sc.B_adj, sc.phi, sc.t_f)
    with pytest.raises(S.SwaError):
        S.swa_adjoint_set_steps_per_pass(adj.h, 2)
    S.swa_adjoint_set_steps_per_pass(adj.h, 1)
