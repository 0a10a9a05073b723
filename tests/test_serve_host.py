"""Host logic of the serving loop, without a GPU: which arrived request is
admitted next (shortest job first with a wait bound, or first come first
served), the device-memory budget check, and the config-5 request trace
(Poisson arrivals at the stated rate, grid sizes from the stated set)."""
import numpy as np
import pytest

from paper_1605_05320_gb300 import build as B
from paper_1605_05320_gb300 import serve
from paper_1605_05320_gb300 import swadj as S


def req(i, arrival, n):
    return serve.Request(i, arrival, n, 1.0, 30e3, 0.5, 0.5)


def test_sjf_takes_the_smallest_grid_then_the_earliest():
    arrived = [req(0, 0.0, 2048), req(1, 0.1, 512), req(2, 0.2, 512), req(3, 0.3, 1024)]
    assert serve.pick_next(arrived, 1.0, "sjf", 30.0).id == 1


def test_a_request_past_the_wait_bound_goes_first():
    arrived = [req(0, 0.0, 4096), req(1, 5.0, 4096), req(2, 40.0, 512)]
    # at t = 41 s requests 0 and 1 have waited more than 30 s: the first of them
    assert serve.pick_next(arrived, 41.0, "sjf", 30.0).id == 0
    # before the bound, the smallest grid
    assert serve.pick_next(arrived, 20.0, "sjf", 30.0).id == 2
    # waits are measured on the replay clock: arrival 100 s at time scale
    # 0.01 comes at 1 s, so at 40 s it has waited 39 s
    late = [req(5, 100.0, 4096), req(6, 1000.0, 512)]
    assert serve.pick_next(late, 40.0, "sjf", 30.0, time_scale=0.01).id == 5
    assert serve.pick_next(late, 20.0, "sjf", 30.0, time_scale=0.01).id == 6


def test_fifo_takes_the_first_arrived():
    arrived = [req(0, 0.0, 4096), req(1, 0.1, 512)]
    assert serve.pick_next(arrived, 1.0, "fifo").id == 0
    assert serve.pick_next([], 1.0, "sjf") is None


@pytest.fixture(scope="module")
def lib():
    B.build()
    return S.load()


def test_budget_check_uses_the_grid_workspace(lib):
    for n in (512, 1024, 2048):
        fp = serve.Server.footprint(n)
        d = S.make_desc(2, n, n, 0.0, 0.0, 1.0, 1.0, precision=S.SWA_FP32)
        ws = S.swa_grid_workspace_bytes(d)
        # the grid's workspace (7 float arrays and the FP64 staging array at
        # least) plus one flag byte per cell
        assert fp == ws + n * n and ws >= n * n * (7 * 4 + 8)
        assert serve.fits(0.0, n, fp)
        assert not serve.fits(1.0, n, fp)
    assert serve.Server.footprint(2048) > 3.9 * serve.Server.footprint(1024)


def test_config5_trace():
    reqs = serve.trace_from_config(n_req=512, rate=20.0)
    t = np.array([r.arrival for r in reqs])
    assert len(reqs) == 512 and np.all(np.diff(t) > 0)
    # Poisson arrivals at 20 per second: exponential gaps of mean 0.05 s
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 0.05) < 0.05 * 4 / np.sqrt(512)
    assert {r.n for r in reqs} == {512, 1024, 2048, 4096}
    assert all(0.1 <= r.amp <= 2.0 and 10e3 <= r.width <= 60e3 for r in reqs)
