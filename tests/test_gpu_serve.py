"""Serving loop: scenarios admitted by HBM budget and slots, overlapping on
the device on their own streams, against one resident adjoint.  Each
request's result (gauge series, flag counts, step count) is the same when it
runs alone and when it runs in a mix with others (bit-identical: every
scenario's arithmetic is independent of its co-runners), and a served
request's gauges and flag counts match the FP64 oracle run on the same
seeded inputs (gauges within 1e-4 m; flag counts within the cells whose m
lies within 1e-3 tol of tol)."""
import math

import numpy as np
import pytest

import oracle as O

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


def test_served_request_matches_the_oracle(serve):
    """Two requests served together; each one's gauge series and flag counts
    against the oracle: the forward run of the same seeded state on the same
    bathymetry (as FP32 storage holds it), in blocks of 10 steps, a gauge
    sample and a flag pass against the oracle's adjoint snapshots after each
    block."""
    from paper_1605_05320_gb300 import synth
    srv, adj = serve
    reqs = [r for r in _reqs(srv) if r.n in (96, 128)][:2]
    server = srv.Server(adj, n_gauges=8, max_slots=4)
    res, stats = server.run(reqs)
    assert stats["requests"] == 2
    L = adj.L
    na = adj.desc.nx
    da = L / na
    aspec = synth.GridSpec(2, na, na, 0.0, 0.0, da, da)
    sm = synth.seamounts(L, adj.seed + 1, adj.n_seamounts, 1600.0 / 2048.0)
    Ba = synth.basin_bathymetry(aspec, L, adj.seed, adj.n_seamounts, seamount_params=sm)
    phi = np.zeros((3, aspec.n))
    target = (0.9 * L, 0.5 * L)
    phi[0] = synth.gaussian_field(aspec, target[0], target[1], 1.0, 10e3)
    agrid = O.Grid.from_spec(aspec)
    hbar_a = np.maximum(-Ba, 0.0)
    N, _, _ = adj.adj.info()
    every = max(1, math.ceil(N / (20 - 1)))
    snaps, tau, N_ref, _ = O.adj_run(agrid, hbar_a, phi, adj.t_f, every)
    assert N == N_ref
    for r in reqs:
        out = next(x for x in res if x.id == r.id)
        n = r.n
        dx = L / n
        spec = synth.GridSpec(2, n, n, 0.0, 0.0, dx, dx)
        Bf = -(np.float32(-server.bathymetry(n)).astype(np.float64))
        eta = synth.gaussian_field(spec, (0.1 + 0.6 * r.src_u) * L, (0.1 + 0.8 * r.src_v) * L,
                                   r.amp, r.width)
        og = O.Grid.from_spec(spec)
        h, hu, hv, t = eta - Bf, np.zeros(spec.n), np.zeros(spec.n), 0.0
        gerr, slack = 0.0, 0
        for k in range(len(out.flag_counts)):
            h, hu, hv, t, _ = O.fwd_run(og, h, hu, hv, Bf, srv.MACRO, adj.t_f, t)
            gerr = max(gerr, float(np.abs(out.gauges[k] - O.gauge(og, h, Bf, server.gauges)).max()))
            _, m_ref, c_ref = O.flag(og, h, hu, hv, Bf, t, agrid, hbar_a, snaps, tau, adj.t_s,
                                     adj.t_f, adj.tol, O.FLAG_INTERP)
            near = int((np.abs(m_ref - adj.tol) <= 1e-3 * adj.tol).sum())
            assert abs(int(out.flag_counts[k]) - c_ref) <= near, (r.id, k)
            slack += near
        assert gerr <= 1e-4, (r.id, gerr)
        assert int(out.flag_counts.sum()) > 0
