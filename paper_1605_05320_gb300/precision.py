"""Precision study: the FP32 perturbation form against FP64.

Workload: 4096 x 4096 basin on [0, 4096 km]^2 (1 km cells, 40 seamounts,
shelf at 0.85 L), 0.2 m Gaussian source placed so that its first arrival at
the target falls inside [t_s, t_f], 5000 forward steps, 16 gauges (8 in the
basin, 8 within 100 km of the target), adjoint on a coarser 1024 x 1024 grid
(4 km) with a snapshot every 20 adjoint steps, a flag pass every 10 forward
steps.  Both precisions run on the GPU in lockstep.  The FP64 GPU
path rounds exactly like the FP64 CPU oracle (its kernels evaluate the
oracle's expressions in the oracle's order without contraction; the GPU
tests check this on sampled cells of the 2048^2 grid), so its series stand in
for the oracle at a size the oracle cannot run in reasonable time.

Output (one JSON line): max |eta_fp32 - eta_fp64| over all gauge samples and
the flag-set differences per pass (all, and outside a 1e-3 relative band
around the tolerance).
"""
from __future__ import annotations

import json
import time

import numpy as np

from . import swadj as S
from . import synth

FLAG_EVERY = 10
SNAP_EVERY = 20


class Run:
    def __init__(self, precision, sc):
        import torch
        p = S.SWA_FP32 if precision == "fp32" else S.SWA_FP64
        d = S.make_desc(2, sc.grid.nx, sc.grid.ny, 0.0, 0.0, sc.grid.dx, sc.grid.dy,
                        precision=p)
        ad = S.make_desc(2, sc.adj_grid.nx, sc.adj_grid.ny, 0.0, 0.0, sc.adj_grid.dx,
                         sc.adj_grid.dy, precision=p)
        self.adj = S.Adjoint(ad, sc.B_adj, sc.phi, sc.t_f)
        N, _, _ = self.adj.info()
        self.store = S.SnapStore(self.adj, N // SNAP_EVERY + 3, p)
        self.store.run_adjoint(SNAP_EVERY)
        self.g = S.Grid(d, sc.B)
        self.g.set_state(sc.eta0, sc.hu0, sc.hv0, 0.0)
        self.flags = torch.zeros(sc.grid.n, dtype=torch.uint8, device="cuda")
        self.m = torch.zeros(sc.grid.n, dtype=torch.float32, device="cuda")
        self.cnt = torch.zeros(1, dtype=torch.int64, device="cuda")


def main(argv=None):
    import argparse

    import torch
    from . import build
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--adj-n", type=int, default=1024)
    ap.add_argument("--steps", type=int, default=5000)
    a = ap.parse_args(argv)
    build.build()
    S.load()
    sc = synth.config4(n=a.n, adj_n=a.adj_n, steps=a.steps)
    t0 = time.perf_counter()
    runs = {k: Run(k, sc) for k in ("fp32", "fp64")}
    ng = sc.gauges.shape[0]
    xy = torch.tensor(sc.gauges, dtype=torch.float64, device="cuda")
    series = {k: torch.zeros((a.steps, ng), dtype=torch.float64, device="cuda") for k in runs}
    diffs, outside, nflags = [], [], []
    lo, hi = sc.tol * (1 - 1e-3), sc.tol * (1 + 1e-3)
    for s in range(a.steps):
        for k, r in runs.items():
            r.g.step(1, sc.t_f)
            S.swa_gauge_sample(r.g.h, ng, xy, series[k][s])
            if (s + 1) % FLAG_EVERY == 0:
                S.swa_flag_cells(r.g.h, r.store.h, sc.t_s, sc.t_f, sc.tol, S.SWA_FLAG_INTERP,
                                 r.flags, r.m, r.cnt)
        if (s + 1) % FLAG_EVERY == 0:
            d = runs["fp32"].flags != runs["fp64"].flags
            m64 = runs["fp64"].m
            near = (m64 >= lo) & (m64 <= hi)
            diffs.append(d.sum())
            outside.append((d & ~near).sum())
            nflags.append(runs["fp64"].cnt.clone())
    torch.cuda.synchronize()
    assert S.swa_sync_status() == 0
    s32, s64 = series["fp32"].cpu().numpy(), series["fp64"].cpu().numpy()
    diffs = torch.stack(diffs).cpu().numpy() if diffs else np.zeros(1)
    outside = torch.stack(outside).cpu().numpy() if outside else np.zeros(1)
    nflags = torch.cat(nflags).cpu().numpy() if nflags else np.zeros(1)
    t32, t64 = runs["fp32"].g.time()[0], runs["fp64"].g.time()[0]
    out = {"workload": f"basin {a.n}^2 (1 km), 40 seamounts, 0.2 m source "
                       f"{np.hypot(*np.subtract(sc.meta['source'], sc.meta['target'])) / 1e3:.0f}"
                       f" km from the target, adjoint {a.adj_n}^2, {a.steps} steps, 16 gauges",
           "gauge_max_abs_err_m": float(np.abs(s32 - s64).max()),
           "gauge_max_abs_m": float(np.abs(s64).max()),
           "t_end_fp32_s": t32, "t_end_fp64_s": t64,
           "flag_passes": int(len(diffs)),
           "flag_cells_fp64_mean": float(nflags.mean()),
           "flag_cells_fp64_max": int(nflags.max()),
           "flag_cells_differing_max": int(diffs.max()),
           "flag_cells_differing_outside_1e-3_band_max": int(outside.max()),
           "wall_s": time.perf_counter() - t0}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
