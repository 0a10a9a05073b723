"""Serving loop: scenarios admitted by HBM budget and slots, overlapping on
the device on their own streams, against one resident adjoint.  Each
request's result (gauge series, flag counts, step count) is the same when it
runs alone and when it runs in a mix with others (bit-identical: every
scenario's arithmetic is independent of its co-runners)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def serve():
    from paper_1605_05320_gb300 import build
    build.build()
    from paper_1605_05320_gb300 import serve as srv
    from paper_1605_05320_gb300 import swadj
    swadj.load()
    L = 384e3
    adj = srv.ResidentAdjoint(n=96, L=L, t_f=900.0, t_s=300.0, tol=1e-4,
                              target=(0.9 * L, 0.5 * L), snaps=20, n_seamounts=6)
    return srv, adj


def _reqs(srv):
    sizes = [64, 96, 128, 64, 128, 96]
    rng = np.random.default_rng(9)
    return [srv.Request(i, 0.0, n, float(rng.uniform(0.1, 2.0)), float(rng.uniform(10e3, 60e3)),
                        float(rng.uniform()), float(rng.uniform())) for i, n in enumerate(sizes)]


def test_same_result_alone_and_in_the_mix(serve):
    srv, adj = serve
    reqs = _reqs(srv)
    alone = {}
    for r in reqs:
        res, _ = srv.Server(adj, n_gauges=8).run([r])
        alone[r.id] = res[0]
    mixed, stats = srv.Server(adj, n_gauges=8, max_slots=6).run(reqs)
    assert stats["requests"] == len(reqs) and stats["peak_active"] >= 2
    for m in mixed:
        a = alone[m.id]
        assert m.steps == a.steps > 0
        assert np.array_equal(m.gauges, a.gauges)
        assert np.array_equal(m.flag_counts, a.flag_counts)
    assert sum(int(m.flag_counts.sum()) for m in mixed) > 0


def test_admission_respects_budget_and_slots(serve):
    srv, adj = serve
    reqs = _reqs(srv)
    foot = max(srv.Server.footprint(r.n) for r in reqs)
    budget = adj.bytes + 1.5 * foot
    res, stats = srv.Server(adj, n_gauges=4, budget_bytes=budget, max_slots=8).run(reqs)
    assert stats["requests"] == len(reqs)
    assert stats["peak_bytes"] <= budget
    assert stats["peak_active"] < len(reqs)
    res, stats = srv.Server(adj, n_gauges=4, max_slots=1).run(reqs)
    assert stats["peak_active"] == 1 and stats["requests"] == len(reqs)


def test_requests_arriving_later_are_admitted_while_others_run(serve):
    srv, adj = serve
    reqs = _reqs(srv)
    big = srv.Request(100, 0.0, 384, 1.0, 30e3, 0.3, 0.5)
    for k, r in enumerate(reqs):
        r.arrival = 0.001 * (k + 1)
    res, stats = srv.Server(adj, n_gauges=4).run([big] + reqs)
    assert stats["requests"] == len(reqs) + 1
    first = next(r for r in res if r.id == 100)
    later = [r for r in res if r.id != 100]
    # admitted while the first scenario was still running on the device
    assert any(r.admitted < first.done for r in later)
    assert stats["peak_active"] >= 2
    assert all(r.latency >= 0 for r in res)
