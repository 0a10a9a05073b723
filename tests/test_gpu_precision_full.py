"""The FP32 perturbation form against the FP64 oracle on the full 2048^2
basin scenario (1 km cells, 2000 forward steps to t_f, the adjoint with a
snapshot every 20 steps, a flag pass and 16 gauge samples after every 10
forward steps): the precision study at the scenario's own size.

It runs the oracle for the whole scenario on the host cores (about ten
minutes on 16 cores, 10 GB of snapshots in host memory), so it runs only
when SWA_FULL_PRECISION=1 is set; the 128^2 version of the same comparison
runs in test_gpu_precision.py every time.  Tolerances as there: gauges within
1e-4 m, flag sets identical outside the cells whose oracle m lies within
1e-3 tol of tol.
"""
import json
import os
import time

import numpy as np
import pytest

import oracle as O
from paper_1605_05320_gb300 import synth

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(os.environ.get("SWA_FULL_PRECISION") != "1",
                                 reason="full-size oracle run: set SWA_FULL_PRECISION=1")]
torch = pytest.importorskip("torch")

EVERY = 20
BLOCK = 10


def test_fp32_full_basin_run_against_the_oracle():
    from paper_1605_05320_gb300 import build
    build.build()
    from paper_1605_05320_gb300 import swadj as S
    S.load()
    t_start = time.time()
    sc = synth.config2(n_gauges=16)
    n = sc.grid.n
    Bf = -(np.float32(-sc.B).astype(np.float64))
    d = S.make_desc(2, sc.grid.nx, sc.grid.ny, 0.0, 0.0, sc.grid.dx, sc.grid.dy,
                    precision=S.SWA_FP32)
    g = S.Grid(d, sc.B)
    g.set_state(sc.eta0, sc.hu0, sc.hv0, 0.0)
    adj = S.Adjoint(d, sc.B_adj, sc.phi, sc.t_f)
    N, _, _ = adj.info()
    store = S.SnapStore(adj, N // EVERY + 3, S.SWA_FP32)
    store.run_adjoint(EVERY)
    og = O.Grid.from_spec(sc.grid)
    hbar = np.maximum(-sc.B_adj, 0.0)
    snaps, tau, N_ref, _ = O.adj_run(og, hbar, sc.phi, sc.t_f, EVERY)
    assert N == N_ref
    xy = torch.tensor(sc.gauges, dtype=torch.float64, device="cuda")
    gout = torch.zeros(len(sc.gauges), dtype=torch.float64, device="cuda")
    flags = torch.zeros(n, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    h, hu, hv, t = sc.eta0 - Bf, sc.hu0.copy(), sc.hv0.copy(), 0.0
    gerr, gmax, passes, differ, outside, flagged, steps = 0.0, 0.0, 0, 0, 0, 0, 0
    while t < sc.t_f:
        g.step(BLOCK, sc.t_f)
        h, hu, hv, t, k = O.fwd_run(og, h, hu, hv, Bf, BLOCK, sc.t_f, t)
        steps += k
        S.swa_gauge_sample(g.h, len(sc.gauges), xy, gout)
        S.swa_flag_cells(g.h, store.h, sc.t_s, sc.t_f, sc.tol, S.SWA_FLAG_INTERP, flags, None,
                         cnt)
        torch.cuda.synchronize()
        t_gpu = g.time()[0]
        assert abs(t_gpu - t) <= 1e-5 * t
        g_ref = O.gauge(og, h, Bf, sc.gauges)
        gerr = max(gerr, float(np.abs(gout.cpu().numpy() - g_ref).max()))
        gmax = max(gmax, float(np.abs(g_ref).max()))
        f_ref, m_ref, c_ref = O.flag(og, h, hu, hv, Bf, t, og, hbar, snaps, tau, sc.t_s, sc.t_f,
                                     sc.tol, O.FLAG_INTERP)
        near = np.abs(m_ref - sc.tol) <= 1e-3 * sc.tol
        f = flags.cpu().numpy()
        differ += int((f != f_ref).sum())
        outside += int((f[~near] != f_ref[~near]).sum())
        flagged += c_ref
        passes += 1
    assert S.swa_sync_status() == 0
    result = {"grid": "2048x2048", "forward_steps": steps, "adjoint_steps": N, "passes": passes,
              "gauges": len(sc.gauges), "gauge_max_abs_err_m": gerr, "gauge_max_abs_m": gmax,
              "flag_cells_differing": differ, "flag_cells_differing_outside_band": outside,
              "flagged_cells_oracle": flagged, "wall_s": round(time.time() - t_start, 1)}
    print(json.dumps(result))
    out = os.environ.get("SWA_FULL_PRECISION_OUT")
    if out:
        with open(out, "w") as fh:
            fh.write(json.dumps(result) + "\n")
    assert passes >= 190 and flagged > 0
    assert outside == 0
    assert gerr <= 1e-4
