#!/usr/bin/env python3
"""Benchmark of the adjoint-guided shallow-water hot path on one GB300.

One step = one whole tsunami scenario of the 2048 x 2048 basin workload
(1 km cells, seeded synthetic bathymetry with a tanh shelf and 20 seamounts,
1 m Gaussian source, 10 km Gaussian target on the shelf):
  * the adjoint solved backward over [0, t_f] with a snapshot every 20 steps
    (snapshot copy fused into the step kernel),
  * the forward run to t_f (about 2000 CFL steps, time step reduced on the
    device inside the step kernel),
  * a gauge sample at every forward step (recorded by the step kernel) and
    of the final state,
  * an adjoint-weighted flag pass every 10 forward steps over the time window
    [t, min(t + t_f - t_s, t_f)], t_s = 0.32 t_f.
The metric is cell-updates per second of the SWE steps (forward + adjoint)
over the whole scenario time, flag passes and gauges included.

`--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload instead (host cores, OpenMP).  Multi-GPU (torchrun): every rank runs
its own scenario (independent problems, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FWD_BLOCK = 10      # forward steps between flag passes
SNAP_EVERY = 20     # adjoint steps between snapshots
N_GAUGES = 2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-patches", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the untimed side measurements (flag comparison, schemes, "
                         "fully active step, FP64 kernels, AMR): for profiler launch lists")
    return ap.parse_args()


def max_over_ranks(x: float, world: int, device=None) -> float:
    """Maximum of a per-rank number over all ranks (a timing taken on every
    rank; the job takes as long as its slowest rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, steps: int, world: int, ms_max: float) -> float:
    """Units processed by all ranks per second of the slowest rank (weak
    scaling: every rank processes the same independent workload)."""
    return units_per_rank * steps * world / (ms_max * 1e-3)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"swadj_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        with open(self.path) as f:
            return summarize_clocks(f)


def summarize_clocks(lines):
    """Median SM clock under load, the maximum clock and the throttle reasons
    seen, from nvidia-smi CSV lines of ClockSampler.Q (noheader, nounits);
    None without a sample."""
    sms, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sms.append(float(parts[1]))
            mx = float(parts[2])
        except ValueError:
            continue
        for nm, v in zip(names, parts[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    if not sms:
        return None
    return {"sm_mhz": statistics.median(sms), "sm_max_mhz": mx,
            "reasons": sorted(reasons), "samples": len(sms)}


# ------------------------------------------------------------------ our arm
class Scenario:
    def __init__(self, S, torch, sc, precision, device):
        self.S, self.torch, self.sc = S, torch, sc
        p = S.SWA_FP32 if precision == "fp32" else S.SWA_FP64
        self.p = p
        self.desc = S.make_desc(2, sc.grid.nx, sc.grid.ny, 0.0, 0.0, sc.grid.dx,
                                sc.grid.dy, precision=p)
        self.adesc = S.make_desc(2, sc.adj_grid.nx, sc.adj_grid.ny, 0.0, 0.0,
                                 sc.adj_grid.dx, sc.adj_grid.dy, precision=p)
        self.grid = S.Grid(self.desc, sc.B)
        self.adj = S.Adjoint(self.adesc, sc.B_adj, sc.phi, sc.t_f)
        self.N_adj, self.dt_adj, _ = self.adj.info()
        self.K_max = self.N_adj // SNAP_EVERY + 3
        self.store = S.SnapStore(self.adj, self.K_max, p)
        n = sc.grid.n
        f64 = dict(dtype=torch.float64, device=device)
        self.eta_d = torch.tensor(sc.eta0, **f64)
        self.hu_d = torch.tensor(sc.hu0, **f64)
        self.hv_d = torch.tensor(sc.hv0, **f64)
        self.phi_d = torch.tensor(sc.phi.reshape(-1), **f64)
        def pinned(a):
            return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).pin_memory()
        self.eta_h = pinned(sc.eta0)
        self.hu_h = pinned(sc.hu0)
        self.hv_h = pinned(sc.hv0)
        self.phi_h = pinned(sc.phi.reshape(-1))
        self.xy = torch.tensor(sc.gauges, **f64)
        self.flags = torch.zeros(n, dtype=torch.uint8, device=device)
        self.n = n
        self.n_fwd = None

    def measure_steps(self):
        """Untimed: run the forward to t_f once to learn the step count and
        the device time at each flag pass (for the snapshot window sizes)."""
        S = self.S
        self.grid.set_state(self.eta_d, self.hu_d, self.hv_d, 0.0)
        ts = []
        while True:
            t, dt, ns = self.grid.time()
            if ns % FWD_BLOCK == 0 and ns > 0:
                ts.append(t)
            if not (t < self.sc.t_f):
                break
            self.grid.step(1, self.sc.t_f)
        self.n_fwd = ns
        self.flag_times = ts
        S.swa_sync_status()

    def alloc_series(self):
        torch = self.torch
        self.series = torch.zeros((self.n_fwd + 1, N_GAUGES), dtype=torch.float64,
                                  device=self.flags.device)
        self.counts = torch.zeros(self.n_fwd // FWD_BLOCK + 1, dtype=torch.int64,
                                  device=self.flags.device)

    def run(self, tstream, host_io=False, ev=None):
        """One scenario on torch stream `tstream`.  ev: optional dict of event
        lists for kernel timing (recorded on the same stream)."""
        S, torch = self.S, self.torch
        stream = tstream.cuda_stream
        g, sc = self.grid, self.sc
        launches = 0
        if host_io:
            S.swa_set_state(g.h, self.eta_h, self.hu_h, self.hv_h, 0.0, S.SWA_HOST, stream)
            S.swa_set_adjoint_state(self.adj.h, self.phi_h, S.SWA_HOST, stream)
        else:
            S.swa_set_state(g.h, self.eta_d, self.hu_d, self.hv_d, 0.0, S.SWA_DEVICE, stream)
            S.swa_set_adjoint_state(self.adj.h, self.phi_d, S.SWA_DEVICE, stream)
        launches += 3 + 1 + 3
        S.swa_snapstore_clear(self.store.h)
        if ev is not None:
            ev["adj"][0].record(tstream)
        S.swa_run_adjoint(self.adj.h, self.store.h, SNAP_EVERY, stream)
        if ev is not None:
            ev["adj"][1].record(tstream)
        launches += self.N_adj + 1
        fp = 0
        # gauges are sampled by the step kernels themselves (the state each
        # step starts from); the final state is sampled after the loop
        S.swa_grid_record_gauges(g.h, N_GAUGES, self.xy, self.series, None, self.n_fwd,
                                 stream)
        for s in range(self.n_fwd):
            # forward launches are timed in blocks of FWD_BLOCK (between flag
            # passes), so the events do not separate consecutive steps
            if ev is not None and s % FWD_BLOCK == 0:
                ev["fwd"][s // FWD_BLOCK][0].record(tstream)
            S.swa_step_forward(g.h, 1, sc.t_f, stream)
            if ev is not None and ((s + 1) % FWD_BLOCK == 0 or s == self.n_fwd - 1):
                ev["fwd"][s // FWD_BLOCK][1].record(tstream)
            launches += 1
            if (s + 1) % FWD_BLOCK == 0:
                if ev is not None:
                    ev["flag"][fp][0].record(tstream)
                S.swa_flag_cells(g.h, self.store.h, sc.t_s, sc.t_f, sc.tol,
                                 S.SWA_FLAG_INTERP, self.flags, None,
                                 self.counts[fp], stream)
                if ev is not None:
                    ev["flag"][fp][1].record(tstream)
                fp += 1
                launches += 1
        S.swa_gauge_sample(g.h, N_GAUGES, self.xy, self.series[self.n_fwd], stream)
        launches += 1
        if host_io:
            out_series = self.series.to("cpu", non_blocking=True)
            out_counts = self.counts.to("cpu", non_blocking=True)
            return launches, out_series, out_counts
        return launches, None, None


SURFACE_TOLS = (0.14, 0.09)   # the paper's two surface-flagging tolerances (Sec. 6), metres


def compare_flags(scen, tstream):
    """Untimed: one more scenario with, every FWD_BLOCK forward steps, the
    adjoint-weighted flag pass and surface flagging (|eta| > tol) at the
    paper's two tolerances; returns the flagged-cell counts per pass
    (mean, max, and the fraction of passes with any flag)."""
    S, torch = scen.S, scen.torch
    stream = tstream.cuda_stream
    g, sc = scen.grid, scen.sc
    S.swa_set_state(g.h, scen.eta_d, scen.hu_d, scen.hv_d, 0.0, S.SWA_DEVICE, stream)
    S.swa_set_adjoint_state(scen.adj.h, scen.phi_d, S.SWA_DEVICE, stream)
    S.swa_snapstore_clear(scen.store.h)
    S.swa_run_adjoint(scen.adj.h, scen.store.h, SNAP_EVERY, stream)
    npass = scen.n_fwd // FWD_BLOCK
    dev = scen.flags.device
    cnt = torch.zeros((1 + len(SURFACE_TOLS), npass), dtype=torch.int64, device=dev)
    for k in range(npass):
        S.swa_step_forward(g.h, FWD_BLOCK, sc.t_f, stream)
        S.swa_flag_cells(g.h, scen.store.h, sc.t_s, sc.t_f, sc.tol, S.SWA_FLAG_INTERP,
                         scen.flags, None, cnt[0, k], stream)
        for j, tol in enumerate(SURFACE_TOLS):
            S.swa_flag_surface(g.h, tol, scen.flags, cnt[1 + j, k], stream)
    torch.cuda.synchronize()
    c = cnt.cpu().numpy()
    names = [f"adjoint_tol_{sc.tol:g}"] + [f"surface_tol_{t:g}_m" for t in SURFACE_TOLS]
    return {"passes": npass, "every_steps": FWD_BLOCK,
            "counts": {nm: {"mean": float(c[i].mean()), "max": int(c[i].max()),
                            "passes_with_flags": float((c[i] > 0).mean())}
                       for i, nm in enumerate(names)}}


def compare_schemes(scen, stream, steps=100):
    """Outside the timed region: the basin's 2D forward step under both
    updates (dimensionally split, the scenario's; unsplit with transverse
    waves), each on a fresh grid from the scenario's initial state, 3 warm-up
    launches, then `steps` launches between CUDA events on the launching
    stream.  The state (28 B per cell in FP32) fits in L2 here; both are
    timed alike."""
    S, torch = scen.S, scen.torch
    hs = stream.cuda_stream
    w = 4 if scen.p == S.SWA_FP32 else 8
    out = {"steps": steps}
    for name, scheme in (("split", S.SWA_SCHEME_SPLIT), ("ctu", S.SWA_SCHEME_CTU)):
        g = S.Grid(scen.desc, scen.sc.B)
        g.set_scheme(scheme)
        g.set_state(scen.eta_d, scen.hu_d, scen.hv_d, 0.0, hs)
        g.step(3, 1e12, hs)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.step(steps, 1e12, hs)
        e1.record(stream)
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / steps
        out[name] = {"us_per_step": round(us, 2),
                     "cell_updates_per_s": scen.n / (us * 1e-6),
                     "hbm_gbs_algorithmic": round(7 * w * scen.n / (us * 1e-6) / 1e9, 1)}
        del g
    if S.swa_sync_status(hs) != 0:
        raise RuntimeError("device status nonzero after the scheme comparison")
    return out


def measure_active_forward(scen, stream, steps=100, seed=7):
    """Outside the timed region: the FP32 forward step on a state with no
    cell at rest (the basin's initial surface plus seeded random momenta of
    +-5 m^2/s everywhere), so no row can skip its wave arithmetic: the
    step's cost where the whole ocean moves.  3 warm-up launches, then
    `steps` launches between CUDA events on the launching stream."""
    S, torch = scen.S, scen.torch
    hs = stream.cuda_stream
    rng = np.random.default_rng(seed)
    n = scen.n
    g = S.Grid(scen.desc, scen.sc.B)
    g.set_state(scen.sc.eta0, rng.uniform(-5.0, 5.0, n), rng.uniform(-5.0, 5.0, n), 0.0, hs)
    g.step(3, 1e12, hs)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.step(steps, 1e12, hs)
    e1.record(stream)
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) * 1e3 / steps
    peak, _ = load_peaks()
    if S.swa_sync_status(hs) != 0:
        raise RuntimeError("device status nonzero after the active-state forward steps")
    del g
    return {"steps": steps, "us_per_step": round(us, 2),
            "cell_updates_per_s": n / (us * 1e-6),
            "hbm_frac_of_measured": round(28.0 * n / (us * 1e-6) / 1e9 / peak, 4)}


def measure_fp64(scen, stream, alu, steps=10):
    """Outside the timed region: the FP64 forward and adjoint steps on the
    same basin (the plain per-grid FP64 form), 2 warm-up launches then
    `steps` launches each, against the measured FP64 FMA rate (counted
    method flops per cell; a division or square root costs several FMA-pipe
    slots, so the fraction is an upper bound of the real pipe use)."""
    S, torch = scen.S, scen.torch
    hs = stream.cuda_stream
    sc = scen.sc
    d = S.make_desc(2, sc.grid.nx, sc.grid.ny, 0.0, 0.0, sc.grid.dx, sc.grid.dy,
                    precision=S.SWA_FP64)
    g = S.Grid(d, sc.B)
    g.set_state(sc.eta0, sc.hu0, sc.hv0, 0.0, hs)
    g.step(2, 1e12, hs)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.step(steps, 1e12, hs)
    e1.record(stream)
    torch.cuda.synchronize()
    fwd_us = e0.elapsed_time(e1) * 1e3 / steps
    del g
    adj = S.Adjoint(d, sc.B_adj, sc.phi, sc.t_f)
    adj.step(2, hs)
    e0.record(stream)
    adj.step(steps, hs)
    e1.record(stream)
    torch.cuda.synchronize()
    adj_us = e0.elapsed_time(e1) * 1e3 / steps
    del adj
    if S.swa_sync_status(hs) != 0:
        raise RuntimeError("device status nonzero after the FP64 steps")
    n = sc.grid.n
    pk = alu["fp64_fma_flops"]
    out = {"peak_fp64_tflops_measured": round(pk / 1e12, 3), "steps": steps}
    for name, us, fl in (("fwd_step", fwd_us, FP64_FWD_FLOPS_PER_CELL),
                         ("adj_step", adj_us, FP64_ADJ_FLOPS_PER_CELL)):
        rate = fl * n / (us * 1e-6)
        out[name] = {"us_per_step": round(us, 1), "flops_per_cell": fl,
                     "tflops": round(rate / 1e12, 3), "frac_of_fp64_peak": round(rate / pk, 4),
                     "hbm_gbs": round(56.0 * n / (us * 1e-6) / 1e9, 1)}
    return out


def measure_amr(stream, steps=20, ratio=4, side=32, tiles=8):
    """Outside the timed region: the two-level AMR glue on the basin.  The
    coarse level is the 2048^2 basin (1 km cells); the fine level is
    tiles x tiles patches of side x side coarse cells refined by `ratio`,
    tiling a square around the source (the basin fields sampled at 250 m).
    Times `steps` hierarchy steps (coarse step, `ratio` fine substeps each
    with its ring fill, averaging down, refluxing) after 3 warm-up steps, the
    same without refluxing, and the coarse step and the fine launch on their
    own, with CUDA events on the stream."""
    import torch
    from paper_1605_05320_gb300 import swadj as S
    from paper_1605_05320_gb300 import synth
    hs = stream.cuda_stream
    B, eta, n, dx, descs, fields = synth.amr_basin_2048(ratio, side, tiles)
    d = S.make_desc(2, n, n, 0.0, 0.0, dx, dx, precision=S.SWA_FP32)
    fine_cells = sum(q[3] * q[4] for q in descs)
    dt_c = 0.9 * 0.75 * dx / np.sqrt(9.81 * float(np.max(-B)))

    def hierarchy():
        g = S.Grid(d, B)
        g.set_state(eta, np.zeros(n * n), np.zeros(n * n), 0.0, hs)
        ps = S.PatchSet(descs, [f[0] for f in fields], d, stream=hs)
        for k, f in enumerate(fields):
            z = np.zeros_like(f[1])
            ps.set_state(k, f[1], z, z, hs)
        ps.start(1, 0.0, hs)
        return g, ps, S.Amr(g, ps, 1, ratio, stream=hs)

    def timed(fn, k):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e3 / k

    # the fine level's strip height, tuned on a copy (tuning steps it)
    from paper_1605_05320_gb300 import tune
    g2, ps2, _ = hierarchy()
    with torch.cuda.stream(stream):
        rows = tune.tune_patches(ps2)[1]
    g, ps, amr = hierarchy()
    S.swa_patches_set_tile_rows(ps.h, 1, rows)
    clock = {"t": 0.0}

    def one_step():
        amr.step(clock["t"], dt_c, 1, hs)
        clock["t"] = clock["t"] + dt_c

    for _ in range(3):
        one_step()
    us_step = timed(one_step, steps)
    amr.set_reflux(False)
    us_plain = timed(one_step, steps)
    amr.set_reflux(True)
    amr.set_fill_mode(S.SWA_AMR_FILL_FUSED)
    us_fused = timed(one_step, steps)
    amr.set_fill_mode(S.SWA_AMR_FILL_KERNEL)
    if S.swa_sync_status(hs) != 0:
        raise RuntimeError("AMR hierarchy step reported an error")
    nfill, navg, nedges = amr.info()
    us_coarse = timed(lambda: g2.step(1, 1e12, hs), steps)
    us_fine = timed(lambda: ps2.step(1, 1, 1e300, hs), steps * ratio)
    if S.swa_sync_status(hs) != 0:
        raise RuntimeError("device status nonzero after the AMR measurement")
    updates = n * n + ratio * fine_cells
    return {"coarse": f"{n}^2, {dx:g} m cells", "patches": len(descs), "ratio": ratio,
            "fine_cells": fine_cells, "steps": steps,
            "us_per_step": round(us_step, 1), "coarse_step_us": round(us_coarse, 1),
            "fine_launch_us": round(us_fine, 1),
            "glue_us_per_step": round(us_step - us_coarse - ratio * us_fine, 1),
            "ring_cells": nfill, "covered_coarse_cells": navg, "coarse_fine_edges": nedges,
            "fine_strip_rows": rows,
            "us_per_step_without_refluxing": round(us_plain, 1),
            "us_per_step_fills_in_the_level_launch": round(us_fused, 1),
            "cell_updates_per_s": updates / (us_step * 1e-6)}


def measure_amr_nested(stream, steps=10, ratio=4):
    """Outside the timed region: the AMR glue over two nested patch levels on
    the basin (the 2048^2 coarse grid, level 1 as in measure_amr, level 2:
    16 patches of 32 x 32 level-1 cells refined by `ratio` again around the
    source).  Times `steps` hierarchy steps (each: the coarse step, 4 level-1
    substeps, each with 4 level-2 substeps, averaging and refluxing at both
    levels) after 3 warm-up steps, with the strip heights tuned per level."""
    import torch
    from paper_1605_05320_gb300 import swadj as S
    from paper_1605_05320_gb300 import synth, tune
    hs = stream.cuda_stream
    B, eta, n, dx, descs, fields = synth.amr_basin_2048_nested(ratio)
    d = S.make_desc(2, n, n, 0.0, 0.0, dx, dx, precision=S.SWA_FP32)
    cells = {lv: sum(q[3] * q[4] for q in descs if q[0] == lv) for lv in (1, 2)}
    dt_c = 0.9 * 0.75 * dx / np.sqrt(9.81 * float(np.max(-B)))

    def hierarchy():
        g = S.Grid(d, B)
        g.set_state(eta, np.zeros(n * n), np.zeros(n * n), 0.0, hs)
        ps = S.PatchSet(descs, [f[0] for f in fields], d, stream=hs)
        for k, f in enumerate(fields):
            z = np.zeros_like(f[1])
            ps.set_state(k, f[1], z, z, hs)
        ps.start(1, 0.0, hs)
        ps.start(2, 0.0, hs)
        return g, ps

    g2, ps2 = hierarchy()
    with torch.cuda.stream(stream):
        rows = tune.tune_patches(ps2)
    g, ps = hierarchy()
    for lv in (1, 2):
        S.swa_patches_set_tile_rows(ps.h, lv, rows[lv])
    amr = S.Amr(g, ps, [1, 2], [ratio, ratio], stream=hs)
    clock = {"t": 0.0}

    def one_step():
        amr.step(clock["t"], dt_c, 1, hs)
        clock["t"] = clock["t"] + dt_c

    for _ in range(3):
        one_step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        one_step()
    e1.record(stream)
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) * 1e3 / steps
    if S.swa_sync_status(hs) != 0:
        raise RuntimeError("nested AMR hierarchy step reported an error")
    updates = n * n + ratio * cells[1] + ratio * ratio * cells[2]
    return {"coarse": f"{n}^2, {dx:g} m cells", "ratios": [ratio, ratio],
            "patches": [sum(1 for q in descs if q[0] == lv) for lv in (1, 2)],
            "cells": [cells[1], cells[2]], "strip_rows": [rows[1], rows[2]],
            "coarse_fine_edges": [amr.info(1)[2], amr.info(2)[2]], "steps": steps,
            "us_per_step": round(us, 1), "cell_updates_per_s": updates / (us * 1e-6)}


def cell_updates(sc_obj):
    return (sc_obj.n_fwd * sc_obj.n + sc_obj.N_adj * sc_obj.adj.n)


def flag_bytes(sc_obj):
    """Per flag pass: (bytes every pass reads, bytes of the full pass).  Every
    pass reads the forward q (3 words), hbar or B (1 word), the adjoint wet
    mask (1 byte) and writes the flag byte; the full pass also reads every
    snapshot in the window (3 words each), the envelope-pruned pass reads the
    window's envelope groups (3 floats per quad of 4 cells each) and only the
    snapshot groups whose bound reaches tol, which depends on the data."""
    tau = np.array([sc_obj.sc.t_f - k * SNAP_EVERY * sc_obj.dt_adj
                    for k in range(sc_obj.N_adj // SNAP_EVERY + 1)] + [0.0])
    tau = np.unique(tau)[::-1]
    w = 4 if sc_obj.p == sc_obj.S.SWA_FP32 else 8
    lo_b, full_b = [], []
    t_f, t_s = sc_obj.sc.t_f, sc_obj.sc.t_s
    K = len(tau)
    for t in sc_obj.flag_times:
        T = min(t + (t_f - t_s), t_f)
        lo, hi = max(t, tau[-1]), min(T, tau[0])
        if lo > hi:
            k0, k_eff = 0, 0
        else:
            kh = next((k for k in range(K - 1) if tau[k + 1] <= hi), K - 1)
            kl = next((k for k in range(K - 1) if tau[k + 1] <= lo), K - 1)
            exact_l = kl + 1 >= K or tau[kl] == lo
            k0, k1 = kh, (kl if exact_l else kl + 1)
            k_eff = k1 - k0 + 1
        base = sc_obj.n * (4 * w + 1 + 1)
        groups = 0 if k_eff == 0 else (k0 + k_eff - 1) // ENV_GROUP - k0 // ENV_GROUP + 1
        lo_b.append(base + groups * 3 * 4 * (sc_obj.adj.n // 4))
        full_b.append(base + sc_obj.adj.n * 3 * w * k_eff)
    return lo_b, full_b


# FP32 operations of one forward cell-update of the split order-2 step, each
# add, multiply, fma, min, max, select and special-function op counted once,
# every edge solved and limited once (no halo recomputation): staging 6,
# x-sweep 122 (Roe f-wave solve 29, net fluxes with MC limiter 78, update 10,
# derived cell data 5), y-sweep 117, CFL term 12.
# FP32 operations per cell-update of the forward step in its subsonic form,
# counted in the source (each add, mul, fma, min, max, select and special
# function once; every edge solved and limited once): x-sweep 104 (cell
# data 7, Roe solve 25, fluctuations and MC-limited net fluxes 62, update
# 10), y-sweep 103, CFL term 11.
FWD_OPS_PER_CELL = 218
# FP64 operations per cell-update of the FP64 kernels, counted from the
# oracle's formulas (division and square root as one): forward ~320 (per
# sweep: Roe solve 49, fluctuations and limited corrections of three waves
# 90, update 15; CFL 8), adjoint ~210 (per sweep: solve 20, two waves 78,
# update 7).
FP64_FWD_FLOPS_PER_CELL = 320
FP64_ADJ_FLOPS_PER_CELL = 210
ENV_GROUP = 8


def run_ours(args, rank, world, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    device = torch.device("cuda", local_rank)
    from paper_1605_05320_gb300 import build as B
    B.build()
    from paper_1605_05320_gb300 import swadj as S
    from paper_1605_05320_gb300 import synth
    S.load()
    sc = synth.config2(n=args.n, L=args.n * 1e3)
    scen = Scenario(S, torch, sc, args.precision, device)
    scen.measure_steps()
    scen.alloc_series()
    stream = torch.cuda.current_stream(device)
    hs = stream.cuda_stream

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        scen.run(stream)
    torch.cuda.synchronize()
    assert S.swa_sync_status(hs) == 0

    # timed region: K scenarios, device-resident inputs, kernel events
    n_flag = scen.n_fwd // FWD_BLOCK
    evs = []
    for _ in range(args.steps):
        E = torch.cuda.Event
        evs.append({"adj": (E(enable_timing=True), E(enable_timing=True)),
                    "fwd": [(E(enable_timing=True), E(enable_timing=True))
                            for _ in range((scen.n_fwd + FWD_BLOCK - 1) // FWD_BLOCK)],
                    "flag": [(E(enable_timing=True), E(enable_timing=True))
                             for _ in range(n_flag)]})
    clocks = ClockSampler(local_rank)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    launches = 0
    for k in range(args.steps):
        nl, _, _ = scen.run(stream, ev=evs[k])
        launches += nl
    end.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    ms = max_over_ranks(start.elapsed_time(end), world, device)
    assert S.swa_sync_status(hs) == 0
    ms_step = ms / args.steps
    cu = cell_updates(scen)
    value = whole_job_rate(cu, args.steps, world, ms)

    # kernel timings
    fwd_ms = [e[0].elapsed_time(e[1]) for d in evs for e in d["fwd"]]   # per block
    adj_ms = [d["adj"][0].elapsed_time(d["adj"][1]) for d in evs]
    flag_ms = [e[0].elapsed_time(e[1]) for d in evs for e in d["flag"]]
    w = 4 if args.precision == "fp32" else 8
    fb = flag_bytes(scen)
    peak, peak_kind = load_peaks()
    kern = {
        "fwd_step": {"launches": scen.n_fwd * args.steps,
                     "avg_us": 1e3 * float(np.sum(fwd_ms)) / (scen.n_fwd * args.steps),
                     "timing": f"CUDA events around each block of {FWD_BLOCK} launches",
                     "bytes_per_launch": 7 * w * scen.n,
                     "total_ms": float(np.sum(fwd_ms)) / args.steps},
        "adj_step": {"launches": scen.N_adj * args.steps,
                     "avg_us": 1e3 * np.mean(adj_ms) / scen.N_adj,
                     "bytes_per_launch": 7 * w * scen.adj.n
                     + 3 * w * scen.adj.n / SNAP_EVERY,
                     "total_ms": float(np.sum(adj_ms)) / args.steps},
        "flag": {"launches": len(flag_ms), "avg_us": 1e3 * np.mean(flag_ms),
                 "bytes_per_launch": float(np.mean(fb[0])) if fb[0] else 0.0,
                 "bytes_note": "lower bound: state, mask, flags and envelope; the pruned "
                               "pass also reads the snapshot groups that can reach tol",
                 "full_pass_bytes_per_launch": float(np.mean(fb[1])) if fb[1] else 0.0,
                 "total_ms": float(np.sum(flag_ms)) / args.steps},
    }
    for k, v in kern.items():
        v["gbs"] = v["bytes_per_launch"] / (v["avg_us"] * 1e-6) / 1e9 if v["avg_us"] > 0 else 0.0
        v["frac"] = v["gbs"] / peak
    dom = max(kern, key=lambda k: kern[k]["total_ms"])
    traffic = None
    tr_path = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tr_path):
        try:
            tr = json.load(open(tr_path))
            key = f"{dom}_{args.precision}_{args.n}"
            traffic = tr.get(key)
        except Exception:
            traffic = None
    roofline = {"bound": "hbm", "kernel": dom,
                "achieved": round(kern[dom]["gbs"], 1), "peak": peak,
                "peak_kind": f"{peak_kind} hbm_gbs", "unit": "GB/s",
                "frac": round(kern[dom]["frac"], 4), "traffic": traffic,
                "bytes_per_launch": kern[dom]["bytes_per_launch"]}
    if args.precision == "fp32":
        # the FP32 forward step is compute-bound (it stays near its time with
        # the loads taken out): its operation rate against the measured FP32
        # peak, beside the HBM fraction the roofline object reports
        fw = kern["fwd_step"]
        ops = FWD_OPS_PER_CELL * scen.n
        alu = S.measure_alu_peaks(local_rank)
        fp32_ops_peak = alu["fp32_fma_flops"] / 2.0   # one lane operation per FMA-pipe slot
        fw["ops_per_launch"] = ops
        fw["tops"] = ops / (fw["avg_us"] * 1e-6) / 1e12
        fw["alu_frac"] = fw["tops"] * 1e12 / fp32_ops_peak
        fw["t_min_us"] = {"hbm": fw["bytes_per_launch"] / (peak * 1e9) * 1e6,
                          "alu": ops / fp32_ops_peak * 1e6}
        roofline["alu"] = {"ops_per_cell": FWD_OPS_PER_CELL, "achieved_tops": round(fw["tops"], 3),
                           "peak_tops": round(fp32_ops_peak / 1e12, 2),
                           "peak_kind": "measured: FP32 FMA probe (swa_alu_probe), one op per "
                                        "FMA slot", "frac": round(fw["alu_frac"], 4)}
        roofline["measured_alu_peaks_tflops"] = {k: round(v / 1e12, 3) for k, v in alu.items()}

    # end-to-end through the C ABI with host buffers
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for k in range(args.steps):
        _, s_out, c_out = scen.run(stream, host_io=True)
        stream.synchronize()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(e0.elapsed_time(e1), world, device)
    h2d = 3 * scen.n * 8 + 3 * scen.adj.n * 8
    d2h = scen.series.numel() * 8 + scen.counts.numel() * 8
    e2e = {"value": whole_job_rate(cu, args.steps, world, ms_e2e), "unit": "cell-updates/s",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "ms_per_step": ms_e2e / args.steps}

    out = {
        "metric": "SWE cell-updates/s (forward + adjoint steps, whole scenario incl. flag passes and gauges)",
        "value": value, "unit": "cell-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "f64",
        "data": "synthetic (seeded basin bathymetry, Gaussian source and target)",
        "config": workload_config(args.n, world),
        "scenario": {"precision": args.precision, "forward_steps": scen.n_fwd,
                     "adjoint_steps": scen.N_adj, "snapshots": scen.store.info()[0],
                     "flag_passes": n_flag},
        "roofline": roofline,
        "kernels": {k: {kk: (round(vv, 3) if isinstance(vv, float) else vv)
                        for kk, vv in v.items()} for k, v in kern.items()},
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "flagged_cells_per_pass_mean": float(scen.counts.double().mean().item()),
    }
    if rank == 0 and not args.no_extras:
        with torch.cuda.stream(stream):
            out["flag_comparison"] = compare_flags(scen, stream)
            out["forward_schemes"] = compare_schemes(scen, stream)
            out["forward_active"] = measure_active_forward(scen, stream)
            out["fp64"] = measure_fp64(scen, stream, alu=S.measure_alu_peaks(local_rank))
            out["amr"] = measure_amr(stream)
            out["amr_nested"] = measure_amr_nested(stream)
    return out


# ------------------------------------------------------- batched patches
def run_patches(level_steps=100, graph_steps=10, seed=5320):
    """The batched uneven-patch workload: 1500 patches on 3 levels (sides
    16..256, cell size 1 km / 4^(level-1)), FP32, bathymetry and source from
    the basin fields; strip height autotuned per level; each level's steps
    replayed from a captured CUDA graph.  Returns per-level throughput."""
    import torch
    from paper_1605_05320_gb300 import swadj as S
    from paper_1605_05320_gb300 import synth, tune
    patches = [(lev, x0, y0, nx, ny, d, d)
               for (lev, x0, y0, nx, ny, d) in synth.config3_patches(seed=seed)]
    t0 = time.perf_counter()
    fields = [synth.patch_fields(p) for p in patches]
    gen_s = time.perf_counter() - t0
    common = S.make_desc(2, 2, 2, 0, 0, 1, 1, precision=S.SWA_FP32)
    ps = S.PatchSet(patches, [f[0] for f in fields], common)

    def reset():
        for k, (B, eta) in enumerate(fields):
            z = np.zeros(B.size)
            ps.set_state(k, eta, z, z)
        for lev in ps.levels:
            ps.start(lev)

    reset()
    rows = tune.tune_patches(ps)
    reset()
    stream = torch.cuda.Stream()
    out = {"patches": len(patches), "levels": {}, "graph_steps": graph_steps,
           "level_steps": level_steps, "setup_s": round(gen_s, 1)}
    graphs = {}
    for lev in ps.levels:
        ps.step(lev, 2, stream=stream)  # warm up outside capture
    torch.cuda.synchronize()
    for lev in ps.levels:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            ps.step(lev, graph_steps, stream=stream)
        graphs[lev] = g
    for lev in ps.levels:
        npat, nstrips, ncells = S.swa_patches_level_info(ps.h, lev)
        reps = max(1, level_steps // graph_steps)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):  # replays and events on one stream
            graphs[lev].replay()
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                graphs[lev].replay()
            e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        nst = reps * graph_steps
        out["levels"][str(lev)] = {
            "patches": npat, "strips": nstrips, "cells": ncells, "strip_rows": rows[lev],
            "us_per_level_step": round(1e3 * ms / nst, 2),
            "cell_updates_per_s": ncells * nst / (ms * 1e-3),
            "hbm_frac_of_measured": (28.0 * ncells * nst / (ms * 1e-3)) / 1e9 / load_peaks()[0]}
    assert S.swa_sync_status() == 0
    tot_cells = sum(v["cells"] for v in out["levels"].values())
    tot_us = sum(v["us_per_level_step"] for v in out["levels"].values())
    out["cell_updates_per_s_all_levels"] = tot_cells / (tot_us * 1e-6)
    return out


# ------------------------------------------------------------ oracle timing
_ORACLE_CASE = {}


def oracle_sample(n, steps):
    """The FP64 oracle on a bounded sample of the same workload, OpenMP on
    all host cores: `steps` forward and `steps` adjoint steps on the n x n
    basin, plus the flag work those forward steps carry in the scenario (one
    pass per FWD_BLOCK forward steps), i.e. one pass over a band of
    steps / FWD_BLOCK of the basin's rows, against the scenario's number of
    snapshots (seeded values: the oracle's cost does not depend on them).
    Returns (cell-updates/s, seconds, threads, description)."""
    import oracle as O
    from paper_1605_05320_gb300 import synth
    O.build()
    O.set_threads(os.cpu_count() or 1)
    if n not in _ORACLE_CASE:
        sc = synth.config2(n=n, L=n * 1e3)
        og = O.Grid.from_spec(sc.grid)
        hbar = np.maximum(-sc.B_adj, 0.0)
        smax = O.adj_smax(og, hbar)
        N_adj = int(np.ceil(sc.t_f * smax / og.cfl))
        K = N_adj // SNAP_EVERY + 2
        rows = max(1, int(round(n * steps / FWD_BLOCK)))
        j0 = (n - rows) // 2
        bg = O.Grid(2, n, rows, sc.grid.x_lo, sc.grid.y_lo + j0 * sc.grid.dy,
                    sc.grid.dx, sc.grid.dy)
        sl = slice(j0 * n, (j0 + rows) * n)
        rng = np.random.default_rng(2048)
        snaps = 1e-3 * rng.standard_normal((K, 3, rows * n))
        tau = np.linspace(sc.t_f, 0.0, K)
        band = (bg, sl, snaps, tau)
        _ORACLE_CASE[n] = (sc, og, hbar, sc.t_f / N_adj, band)
    sc, og, hbar, dt_adj, (bg, sl, snaps, tau) = _ORACLE_CASE[n]
    h0 = sc.eta0 - sc.B
    t0 = time.perf_counter()
    O.fwd_run(og, h0, sc.hu0, sc.hv0, sc.B, steps, sc.t_f)
    e, m, gm = sc.phi[0], sc.phi[1], sc.phi[2]
    for _ in range(steps):
        e, m, gm = O.adj_step(og, e, m, gm, hbar, dt_adj)
    O.flag(bg, h0[sl], sc.hu0[sl], sc.hv0[sl], sc.B[sl], 0.5 * sc.t_f, bg, hbar[sl], snaps,
           tau, sc.t_s, sc.t_f, sc.tol, O.FLAG_INTERP)
    sec = time.perf_counter() - t0
    what = (f"{steps} forward + {steps} adjoint FP64 oracle steps on the {n}x{n} basin and "
            f"a flag pass over {bg.ny} of its rows against {snaps.shape[0]} snapshots "
            f"(the flag work of {steps} forward steps)")
    return 2 * steps * sc.grid.n / sec, sec, O.num_threads(), what


def precision_vs_oracle(n=256, L=2048e3, every=20, n_gauges=16, tol=1e-4):
    """Oracle leg (host cores): the FP32 GPU path against the FP64 oracle over
    a whole basin scenario on an n x n grid of the same generator (2048 km,
    2000 CFL steps to t_f): a gauge sample and an adjoint-weighted flag pass
    after every FWD_BLOCK forward steps on both sides, and the FP64 mass
    audit (swa_grid_mass) of the FP32 state against the oracle's mass.  The
    oracle is given the bathymetry FP32 storage holds.  At 8 km cells the
    10 km target is coarsely resolved and m stays below 3e-4, so the flag
    threshold is `tol` = 1e-4, inside the range m takes."""
    import torch
    import oracle as O
    from paper_1605_05320_gb300 import swadj as S
    from paper_1605_05320_gb300 import synth
    O.build()
    O.set_threads(os.cpu_count() or 1)
    sc = synth.config2(n=n, L=L, n_gauges=n_gauges)
    sc.tol = tol
    Bf = -(np.float32(-sc.B).astype(np.float64))
    d = S.make_desc(2, n, n, 0.0, 0.0, sc.grid.dx, sc.grid.dy, precision=S.SWA_FP32)
    g = S.Grid(d, sc.B)
    g.set_state(sc.eta0, sc.hu0, sc.hv0, 0.0)
    adj = S.Adjoint(d, sc.B_adj, sc.phi, sc.t_f)
    N, _, _ = adj.info()
    store = S.SnapStore(adj, N // every + 3, S.SWA_FP32)
    store.run_adjoint(every)
    og = O.Grid.from_spec(sc.grid)
    hbar = np.maximum(-sc.B_adj, 0.0)
    snaps, tau, _, _ = O.adj_run(og, hbar, sc.phi, sc.t_f, every)
    xy = torch.tensor(sc.gauges, dtype=torch.float64, device="cuda")
    gout = torch.zeros(len(sc.gauges), dtype=torch.float64, device="cuda")
    flags = torch.zeros(sc.grid.n, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    mass = torch.zeros(1, dtype=torch.float64, device="cuda")
    S.swa_grid_mass(g.h, mass)
    m0 = float(mass.item())
    area = sc.grid.dx * sc.grid.dy
    h, hu, hv, t = sc.eta0 - Bf, sc.hu0.copy(), sc.hv0.copy(), 0.0
    gerr, gmax, passes, differ, outside, flagged = 0.0, 0.0, 0, 0, 0, 0
    while t < sc.t_f:
        g.step(FWD_BLOCK, sc.t_f)
        h, hu, hv, t, _ = O.fwd_run(og, h, hu, hv, Bf, FWD_BLOCK, sc.t_f, t)
        S.swa_gauge_sample(g.h, len(sc.gauges), xy, gout)
        S.swa_flag_cells(g.h, store.h, sc.t_s, sc.t_f, sc.tol, S.SWA_FLAG_INTERP, flags, None,
                         cnt)
        torch.cuda.synchronize()
        g_ref = O.gauge(og, h, Bf, sc.gauges)
        gerr = max(gerr, float(np.abs(gout.cpu().numpy() - g_ref).max()))
        gmax = max(gmax, float(np.abs(g_ref).max()))
        f_ref, m_ref, c_ref = O.flag(og, h, hu, hv, Bf, t, og, hbar, snaps, tau, sc.t_s,
                                     sc.t_f, sc.tol, O.FLAG_INTERP)
        f = flags.cpu().numpy()
        near = np.abs(m_ref - sc.tol) <= 1e-3 * sc.tol
        differ += int((f != f_ref).sum())
        outside += int((f[~near] != f_ref[~near]).sum())
        flagged += c_ref
        passes += 1
    S.swa_grid_mass(g.h, mass)
    torch.cuda.synchronize()
    if S.swa_sync_status() != 0:
        raise RuntimeError("device status nonzero after the precision run")
    m_ref = float(h.sum()) * area
    return {"grid": f"{n}x{n} basin, {L / n / 1e3:.0f} km cells, FP32 perturbation form vs "
                    f"FP64 oracle, whole run to t_f",
            "forward_steps": int(g.time()[2]), "flag_passes": passes,
            "gauges": len(sc.gauges), "gauge_max_abs_err_m": gerr,
            "gauge_max_abs_m": gmax, "flag_cells_differing": differ,
            "flag_cells_differing_outside_band": outside,
            "flagged_cells_oracle": flagged, "tol": tol,
            "mass_fp64_audit": {"initial": m0, "final": float(mass.item()),
                                "drift_rel": abs(float(mass.item()) - m0) / m0,
                                "oracle_final": m_ref,
                                "rel_diff_vs_oracle": abs(float(mass.item()) - m_ref) / m_ref}}


def serving_vs_plain(n_req=24, n_plain=4, rate=20.0, with_oracle=True):
    """Served FP32 continuous batching on the first n_req requests of the
    serving trace (Poisson at `rate`, sizes 512^2 .. 4096^2 over 2048 km)
    against one resident 2048^2 adjoint with 150 FP32 snapshots, and the
    plain per-grid FP64 form on the first n_plain requests of 512^2 or
    1024^2 (an FP64 4096^2 scenario alone takes minutes), served again in
    FP32 for the same-trace ratio; the gauge error of the served FP32
    results against plain FP64, and of one served 512^2 request against
    the FP64 oracle (oracle leg, host cores)."""
    import torch
    from paper_1605_05320_gb300 import serve as srv
    from paper_1605_05320_gb300 import swadj as S
    from paper_1605_05320_gb300 import synth
    L = 2048e3
    sc2 = synth.config2(n=256, L=L)
    sc2.t_f = 2000.0 * 0.75 * 1e3 / np.sqrt(synth.G * 4000.0)
    sc2.t_s = 0.32 * sc2.t_f
    t0 = time.perf_counter()
    adj = srv.ResidentAdjoint(2048, L, sc2.t_f, sc2.t_s, sc2.tol, sc2.meta["target"])
    torch.cuda.synchronize()
    adj_s = time.perf_counter() - t0
    reqs = srv.trace_from_config(n_req, rate, (512, 1024, 2048, 4096))
    res, st = srv.Server(adj).run(reqs)
    small = [srv.Request(r.id, 0.0, r.n, r.amp, r.width, r.src_u, r.src_v)
             for r in reqs if r.n <= 1024][:n_plain]
    served_sub, sst = srv.Server(adj).run(small)
    plain, pst = srv.run_plain(adj, small, precision=S.SWA_FP64)
    gerr = 0.0
    for p in plain:
        q = next(x for x in served_sub if x.id == p.id)
        k = min(len(q.gauges), len(p.gauges))
        gerr = max(gerr, float(np.abs(q.gauges[:k] - p.gauges[:k]).max()))
    # one served 512^2 request against the oracle (oracle leg)
    orc = None
    r512 = next((r for r in small if r.n == 512), None)
    if r512 is not None and with_oracle:
        import oracle as O
        O.build()
        O.set_threads(os.cpu_count() or 1)
        out = next(x for x in served_sub if x.id == r512.id)
        srv_ = srv.Server(adj)
        n = 512
        dx = L / n
        spec = synth.GridSpec(2, n, n, 0.0, 0.0, dx, dx)
        Bf = -(np.float32(-srv_.bathymetry(n)).astype(np.float64))
        eta = synth.gaussian_field(spec, (0.1 + 0.6 * r512.src_u) * L,
                                   (0.1 + 0.8 * r512.src_v) * L, r512.amp, r512.width)
        og = O.Grid.from_spec(spec)
        h, hu, hv, t = eta - Bf, np.zeros(spec.n), np.zeros(spec.n), 0.0
        oerr = 0.0
        for k in range(len(out.gauges)):
            h, hu, hv, t, _ = O.fwd_run(og, h, hu, hv, Bf, srv.MACRO, adj.t_f, t)
            oerr = max(oerr, float(np.abs(out.gauges[k] - O.gauge(og, h, Bf, srv_.gauges)).max()))
        orc = {"request": r512.id, "gauges": len(srv_.gauges), "samples": len(out.gauges),
               "gauge_max_abs_err_m": oerr}
    lat_by = {}
    for r in res:
        lat_by.setdefault(r.n, []).append(r.latency)
    return {"trace": {"requests": n_req, "rate_per_s": rate, "sizes": [512, 1024, 2048, 4096],
                      "counts_by_size": {str(k): len(v) for k, v in sorted(lat_by.items())}},
            "adjoint": {"grid": "2048x2048", "snapshots_fp32": adj.store.info()[0],
                        "setup_s": round(adj_s, 3)},
            "served_fp32": {k: (round(v, 4) if isinstance(v, float) else v) for k, v in st.items()},
            "p50_by_size_s": {str(k): round(float(np.percentile(v, 50)), 4)
                              for k, v in sorted(lat_by.items())},
            "same_requests": {"ids": [r.id for r in small], "sizes": [r.n for r in small],
                              "served_fp32_scenarios_per_s": sst["scenarios_per_s"],
                              "plain_fp64_scenarios_per_s": pst["scenarios_per_s"],
                              "served_over_plain": sst["scenarios_per_s"] / pst["scenarios_per_s"],
                              "gauge_max_abs_err_fp32_vs_fp64_m": gerr},
            "vs_oracle": orc}


def workload_config(n, world):
    """The workload both arms report (the reference arm times a bounded
    sample of it)."""
    return {"workload": f"basin {n}x{n} 1 km, forward to t_f + adjoint (snapshot every "
                        f"{SNAP_EVERY} steps) + adjoint-weighted flag pass every "
                        f"{FWD_BLOCK} forward steps + {N_GAUGES} gauges",
            "cells": n * n,
            "l2": "inputs larger than L2 (snapshot store streamed by every flag pass)",
            "parallelism": f"replicas x{world} (independent scenarios)"}


def run_reference(args, world=1):
    cores = os.cpu_count() or 1
    n = args.n
    per = 2
    for _ in range(args.warmup):
        oracle_sample(n, per)
    t0 = time.perf_counter()
    cells = 0
    for _ in range(args.steps):
        v, sec, thr, what = oracle_sample(n, per)
        cells += 2 * per * n * n
    sec = time.perf_counter() - t0
    value = cells / sec
    sample = f"per step: {what} (OpenMP, {thr} threads)"
    return {
        "impl": "reference",
        "metric": "SWE cell-updates/s (forward + adjoint steps, whole scenario incl. flag passes and gauges)",
        "value": value, "unit": "cell-updates/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded basin bathymetry, Gaussian source and target)",
        "config": workload_config(n, world),
        "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": thr,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, world)))
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    out = run_ours(args, rank, world, local_rank)
    if rank == 0 and not args.no_patches:
        out["patches"] = run_patches()
    if rank == 0:
        if not args.no_cpu_baseline:
            v, sec, thr, what = oracle_sample(args.n, 2)
            out["cpu_baseline"] = {
                "value": v, "unit": "cell-updates/s", "cores": thr, "kind": "oracle",
                "sample": f"{what} ({sec:.1f} s, OpenMP)"}
            # the rest of the oracle leg: precision of the FP32 path and the
            # served form, each against the FP64 oracle on the host cores
            out["precision"] = precision_vs_oracle()
        if not args.no_serving:
            out["serving"] = serving_vs_plain(with_oracle=not args.no_cpu_baseline)
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
