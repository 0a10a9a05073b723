"""Serving loop: many forward tsunami scenarios against one resident adjoint.

One adjoint problem per target location (Sec. 2: one adjoint answers every
forward problem with the same functional; Sec. 4: its snapshots are stored
once) is solved at start-up and kept on the device with its snapshots.
Scenario requests (grid size, source position, amplitude, width) arrive over
time.  The loop admits a request when a slot is free and its device memory
fits the HBM budget, gives each admitted scenario its own CUDA stream, and
keeps enqueuing "macro steps" (10 forward steps, a gauge sample, one adjoint-
weighted flag pass) round-robin over the active scenarios, so the work of
requests that arrived at different times overlaps on the GPU (continuous
batching).  Admission takes the arrived request with the least work first
(a request that has waited longer than max_wait_s goes ahead of it); small
grids run on high-priority streams and keep more macro steps queued (the
host tops queues up only between its passes over the active scenarios).
Completion is detected by polling CUDA events, never by a device-wide
synchronisation.  Results per request: gauge time series, flag
counts per pass, latency (completion minus arrival).

Everything on the numerical path runs in libswadj's kernels; this module only
allocates workspaces (torch), orders work on streams and measures time.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import swadj as S
from . import synth

MACRO = 10          # forward steps per macro step (one flag pass each)
AHEAD = 2           # macro steps kept in flight per scenario, at least
# cell-steps kept in flight per scenario: a small grid's macro step is short,
# so it keeps more of them queued than a large grid (the host tops queues up
# only between its passes over the active scenarios)
AHEAD_CELL_STEPS = 2 * 2048 * 2048 * MACRO
SMALL = 1024        # grids up to SMALL^2 run on high-priority streams


@dataclass
class Request:
    id: int
    arrival: float
    n: int
    amp: float
    width: float
    src_u: float
    src_v: float


@dataclass
class Result:
    id: int
    n: int
    arrival: float
    admitted: float
    done: float
    steps: int
    gauges: np.ndarray
    flag_counts: np.ndarray
    latency: float = field(init=False)

    def __post_init__(self):
        self.latency = self.done - self.arrival


def pick_next(arrived, now, policy="sjf", max_wait_s=30.0, time_scale=1.0):
    """The request to admit next among `arrived` (requests that have arrived
    by `now`, in arrival order): "fifo" takes the first; "sjf" takes the one
    with the least work (the smallest grid, then the earliest), unless some
    have waited longer than max_wait_s, of which it takes the first."""
    if not arrived:
        return None
    if policy == "fifo":
        return arrived[0]
    old = [r for r in arrived if now - r.arrival * time_scale > max_wait_s]
    return old[0] if old else min(arrived, key=lambda q: (q.n, q.arrival))


def fits(used_bytes, n, budget_bytes, precision=S.SWA_FP32):
    """Whether an n x n scenario fits next to used_bytes of device memory."""
    return used_bytes + Server.footprint(n, precision) <= budget_bytes


class ResidentAdjoint:
    """The adjoint for one target, solved once, snapshots kept on device."""

    def __init__(self, n, L, t_f, t_s, tol, target, snaps=150, precision=S.SWA_FP32,
                 seed=1605, n_seamounts=20, width=10e3):
        dx = L / n
        spec = synth.GridSpec(2, n, n, 0.0, 0.0, dx, dx)
        sm = synth.seamounts(L, seed + 1, n_seamounts, 1600.0 / 2048.0)
        B = synth.basin_bathymetry(spec, L, seed, n_seamounts, seamount_params=sm)
        phi = np.zeros((3, spec.n))
        phi[0] = synth.gaussian_field(spec, target[0], target[1], 1.0, width)
        self.desc = S.make_desc(2, n, n, 0.0, 0.0, dx, dx, precision=precision)
        self.adj = S.Adjoint(self.desc, B, phi, t_f)
        N, dt, _ = self.adj.info()
        every = max(1, math.ceil(N / (snaps - 1)))
        self.store = S.SnapStore(self.adj, N // every + 3, precision)
        self.store.run_adjoint(every)
        self.t_f, self.t_s, self.tol = t_f, t_s, tol
        self.L, self.seed, self.n_seamounts = L, seed, n_seamounts
        self.bytes = self.adj.nbytes + self.store.nbytes


class Scenario:
    def __init__(self, req: Request, server: "Server", device):
        import torch
        self.req = req
        L = server.adjoint.L
        n = req.n
        dx = L / n
        self.desc = S.make_desc(2, n, n, 0.0, 0.0, dx, dx, precision=server.precision)
        B = server.bathymetry(n)
        # shortest jobs first: a small scenario's kernels go ahead of a large
        # one's when the GPU frees up (results do not depend on the order)
        self.stream = torch.cuda.Stream(device=device, priority=-1 if n <= SMALL else 0)
        self.ahead = max(AHEAD, math.ceil(AHEAD_CELL_STEPS / (n * n * MACRO)))
        self.grid = S.Grid(self.desc, B, stream=self.stream)
        self.t_f = server.adjoint.t_f
        spec = synth.GridSpec(2, n, n, 0.0, 0.0, dx, dx)
        eta = server.initial_surface(req)
        z = np.zeros(spec.n)
        self.grid.set_state(eta, z, z, 0.0, stream=self.stream)
        _, dt0, _ = S.swa_get_time(self.grid.h, self.stream)
        # macro steps to reach t_f with margin (steps past t_f are device no-ops)
        self.n_macro = int(math.ceil(self.t_f / dt0 * 1.05 / MACRO)) + 1
        ng = server.gauges.shape[0]
        f64 = dict(dtype=torch.float64, device=device)
        self.xy = torch.tensor(server.gauges, **f64)
        self.series = torch.zeros((self.n_macro, ng), **f64)
        self.counts = torch.zeros(self.n_macro, dtype=torch.int64, device=device)
        self.flags = torch.zeros(spec.n, dtype=torch.uint8, device=device)
        self.enqueued = 0
        self.events = []
        self.bytes = self.grid.nbytes + spec.n + self.series.numel() * 8

    def enqueue_macro(self, server):
        import torch
        k = self.enqueued
        st = self.stream
        S.swa_step_forward(self.grid.h, MACRO, self.t_f, st)
        S.swa_gauge_sample(self.grid.h, self.xy.shape[0], self.xy, self.series[k], st)
        a = server.adjoint
        S.swa_flag_cells(self.grid.h, a.store.h, a.t_s, a.t_f, a.tol, S.SWA_FLAG_INTERP,
                         self.flags, None, self.counts[k], st)
        ev = torch.cuda.Event()
        ev.record(st)
        self.events.append(ev)
        self.enqueued += 1

    def in_flight(self):
        while self.events and self.events[0].query():
            self.events.pop(0)
        return len(self.events)

    def finished(self):
        return self.enqueued >= self.n_macro and self.in_flight() == 0


class Server:
    def __init__(self, adjoint: ResidentAdjoint, budget_bytes: float = 80e9,
                 max_slots: int = 16, precision=S.SWA_FP32, n_gauges: int = 16,
                 device="cuda", seed: int = 2026, policy: str = "sjf",
                 max_wait_s: float = 30.0):
        self.adjoint = adjoint
        self.budget = budget_bytes
        self.max_slots = max_slots
        if policy not in ("sjf", "fifo"):
            raise ValueError("policy must be 'sjf' or 'fifo'")
        self.policy = policy
        self.max_wait_s = max_wait_s
        self.precision = precision
        self.device = device
        self._bathy = {}
        self._eta = {}
        rng = np.random.default_rng(seed)
        L = adjoint.L
        self.gauges = np.stack([rng.uniform(0.1 * L, 0.9 * L, n_gauges),
                                rng.uniform(0.1 * L, 0.9 * L, n_gauges)], axis=1)

    def bathymetry(self, n):
        if n not in self._bathy:
            a = self.adjoint
            dx = a.L / n
            spec = synth.GridSpec(2, n, n, 0.0, 0.0, dx, dx)
            sm = synth.seamounts(a.L, a.seed + 1, a.n_seamounts, 1600.0 / 2048.0)
            self._bathy[n] = synth.basin_bathymetry(spec, a.L, a.seed, a.n_seamounts,
                                                    seamount_params=sm)
        return self._bathy[n]

    def initial_surface(self, req):
        """The request's initial surface (its payload): prepared by prepare(),
        else formed here."""
        eta = self._eta.pop(req.id, None)
        if eta is not None:
            return eta
        L = self.adjoint.L
        n = req.n
        spec = synth.GridSpec(2, n, n, 0.0, 0.0, L / n, L / n)
        return synth.gaussian_field(spec, (0.1 + 0.6 * req.src_u) * L,
                                    (0.1 + 0.8 * req.src_v) * L, req.amp, req.width)

    def prepare(self, requests, max_bytes: float = 4e9):
        """Host data outside the serving clock: the bathymetry at every grid
        size of the trace (the server's static data) and the initial surface
        each request arrives with, in arrival order while they fit in
        max_bytes of host memory (later ones are formed at admission)."""
        for r in requests:
            self.bathymetry(r.n)
        held = 0.0
        for r in sorted(requests, key=lambda r: r.arrival):
            if r.id in self._eta:
                continue
            held += 8.0 * r.n * r.n
            if held > max_bytes:
                break
            self._eta[r.id] = self.initial_surface(r)

    @staticmethod
    def footprint(n, precision=S.SWA_FP32):
        d = S.make_desc(2, n, n, 0.0, 0.0, 1.0, 1.0, precision=precision)
        return S.swa_grid_workspace_bytes(d) + n * n

    def run(self, requests, time_scale: float = 1.0, log=None):
        """Serve `requests` (arrival times in seconds, compressed by
        time_scale); returns (results, stats).  The host data of prepare()
        is formed before the clock starts."""
        import torch
        self.prepare(requests)
        pending = sorted(requests, key=lambda r: r.arrival)
        active = []
        results = []
        used = self.adjoint.bytes
        t0 = time.perf_counter()
        peak_active = 0
        peak_bytes = used
        while pending or active:
            now = time.perf_counter() - t0
            # admit: the arrived request with the least work first (shortest
            # job first), unless one has waited longer than max_wait_s (then
            # the longest-waiting one), while a slot and the budget allow
            while pending and len(active) < self.max_slots:
                now = time.perf_counter() - t0
                arrived = [r for r in pending if r.arrival * time_scale <= now]
                if not arrived:
                    break
                r = pick_next(arrived, now, self.policy, self.max_wait_s, time_scale)
                if not fits(used, r.n, self.budget, self.precision):
                    break
                pending.remove(r)
                sc = Scenario(r, self, self.device)
                sc.admitted = time.perf_counter() - t0
                used += sc.bytes
                active.append(sc)
            peak_active = max(peak_active, len(active))
            peak_bytes = max(peak_bytes, used)
            # keep every active scenario's queue topped up
            progressed = False
            for sc in active:
                while sc.enqueued < sc.n_macro and sc.in_flight() < sc.ahead:
                    sc.enqueue_macro(self)
                    progressed = True
            # retire finished scenarios
            still = []
            for sc in active:
                if sc.finished():
                    done = time.perf_counter() - t0
                    _, _, steps = S.swa_get_time(sc.grid.h, sc.stream)
                    results.append(Result(sc.req.id, sc.req.n, sc.req.arrival * time_scale,
                                          sc.admitted, done, steps,
                                          sc.series.cpu().numpy(), sc.counts.cpu().numpy()))
                    used -= sc.bytes
                    if log:
                        log(f"done {sc.req.id} n={sc.req.n} steps={steps} "
                            f"latency={done - sc.req.arrival * time_scale:.3f}s")
                else:
                    still.append(sc)
            active = still
            if not progressed:
                if active:
                    active[0].events[0].synchronize() if active[0].events else None
                elif pending:
                    wait = pending[0].arrival * time_scale - (time.perf_counter() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.05))
        wall = time.perf_counter() - t0
        lat = np.array([r.latency for r in results])
        stats = {"requests": len(results), "wall_s": wall,
                 "scenarios_per_s": len(results) / wall if wall > 0 else 0.0,
                 "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
                 "p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
                 "peak_active": peak_active, "peak_bytes": peak_bytes,
                 "cell_updates": float(sum(r.steps * r.n * r.n for r in results))}
        stats["cell_updates_per_s"] = stats["cell_updates"] / wall if wall > 0 else 0.0
        return results, stats


def trace_from_config(n_req=512, rate=20.0, sizes=(512, 1024, 2048, 4096), seed=2026):
    return [Request(r["id"], r["arrival"], r["n"], r["amp"], r["width"], r["src_u"],
                    r["src_v"])
            for r in synth.config5_requests(seed=seed, n=n_req, rate=rate, sizes=sizes)]


def run_plain(adjoint: ResidentAdjoint, requests, precision=S.SWA_FP64, n_gauges=16,
              device="cuda"):
    """Plain per-grid runs, one request after another on one stream (no
    admission, no overlap), in `precision`; returns (results, stats)."""
    import torch
    srv = Server(adjoint, precision=precision, n_gauges=n_gauges, device=device)
    srv.prepare(requests)
    results = []
    t0 = time.perf_counter()
    for r in sorted(requests, key=lambda r: r.arrival):
        sc = Scenario(r, srv, device)
        while sc.enqueued < sc.n_macro:
            sc.enqueue_macro(srv)
        sc.stream.synchronize()
        _, _, steps = S.swa_get_time(sc.grid.h, sc.stream)
        done = time.perf_counter() - t0
        results.append(Result(r.id, r.n, 0.0, 0.0, done, steps, sc.series.cpu().numpy(),
                              sc.counts.cpu().numpy()))
        del sc
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    cu = float(sum(x.steps * x.n * x.n for x in results))
    return results, {"requests": len(results), "wall_s": wall,
                     "scenarios_per_s": len(results) / wall, "cell_updates": cu,
                     "cell_updates_per_s": cu / wall}


def main(argv=None):
    """Serving benchmark: the served FP32 continuous-batching loop and the
    plain per-grid FP64 form on the same request trace (basin workload,
    resident 2048^2 adjoint with 150 FP32 snapshots).  Prints one JSON line."""
    import argparse
    import json

    import torch
    from . import build
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=24)
    ap.add_argument("--rate", type=float, default=20.0)
    ap.add_argument("--sizes", default="512,1024")
    ap.add_argument("--adjoint-n", type=int, default=2048)
    ap.add_argument("--plain-requests", type=int, default=8)
    ap.add_argument("--prepare-gb", type=float, default=4.0,
                    help="host memory for request payloads formed before the clock")
    a = ap.parse_args(argv)
    build.build()
    S.load()
    sizes = tuple(int(x) for x in a.sizes.split(","))
    L = 2048e3
    # tol and target of the basin workload; its time window is the one of the
    # 1 km grid (t_f = 2000 basin CFL steps of 1 km cells), whatever the
    # size of the grid built here to read them
    sc2 = synth.config2(n=256, L=L)
    sc2.t_f = 2000.0 * 0.75 * 1e3 / np.sqrt(synth.G * 4000.0)
    sc2.t_s = 0.32 * sc2.t_f
    t0 = time.perf_counter()
    adj = ResidentAdjoint(a.adjoint_n, L, sc2.t_f, sc2.t_s, sc2.tol, sc2.meta["target"])
    torch.cuda.synchronize()
    adj_s = time.perf_counter() - t0
    reqs = trace_from_config(a.requests, a.rate, sizes)
    server = Server(adj)
    t0 = time.perf_counter()
    server.prepare(reqs, max_bytes=a.prepare_gb * 1e9)
    prep_s = time.perf_counter() - t0
    res, st = server.run(reqs)
    st["host_prepare_s"] = prep_s
    lat_by = {}
    for r in res:
        lat_by.setdefault(r.n, []).append(r.latency)
    st["p50_by_size_s"] = {str(k): float(np.percentile(v, 50)) for k, v in lat_by.items()}
    out = {"metric": "served scenarios/s (FP32 continuous batching) vs plain per-grid FP64",
           "adjoint_setup_s": adj_s, "served": st,
           "trace": {"requests": a.requests, "rate_per_s": a.rate, "sizes": sizes}}
    if a.plain_requests > 0:   # 0 skips the (slow) per-grid FP64 comparison
        sub = reqs[: a.plain_requests]
        served_sub, sst = Server(adj).run([Request(r.id, 0.0, r.n, r.amp, r.width, r.src_u,
                                                   r.src_v) for r in sub])
        _, pst = run_plain(adj, sub, precision=S.SWA_FP64)
        # gauge error of the FP32 served results against the FP64 per-grid ones
        plain64, _ = run_plain(adj, sub[:2], precision=S.SWA_FP64)
        gerr = 0.0
        for r in plain64:
            s = next(x for x in served_sub if x.id == r.id)
            k = min(len(s.gauges), len(r.gauges))
            gerr = max(gerr, float(np.abs(s.gauges[:k] - r.gauges[:k]).max()))
        out.update({"same_requests_served_fp32": sst, "plain_fp64": pst,
                    "served_over_plain": sst["scenarios_per_s"] / pst["scenarios_per_s"],
                    "gauge_max_abs_err_fp32_vs_fp64_m": gerr})
    print(json.dumps(out))


if __name__ == "__main__":
    main()
