"""Small fixed cases of each hot kernel, sized for profiler captures.

Each case runs one kernel family of the scenario path on the 2048 x 2048
basin (1 km cells) through the public binding, with far less device memory
than the full scenario (no 101-snapshot store), so that a capture that saves
and restores device memory between passes stays small:

  fwd   FP32 forward steps (fwd_f32_strips), ~120 MB on the device; the
        basin's initial state (the ocean at rest outside the source), or with
        `--active` seeded random momenta everywhere (no cell at rest)
  ctu   FP32 unsplit forward steps with transverse waves (fwd_ctu_kernel),
        ~120 MB
  amr   two-level AMR steps on the basin: the 2048^2 coarse grid and 64
        patches refined by 4 around the source (coarse fluxes for the
        refluxing, fills, fine launches, averaging with the refluxing),
        ~200 MB; `--rows 16` sets the fine level's strip height
  adj   the full FP32 adjoint run (adj_f32_strips, ~2000 launches) with a
        fused snapshot every 100 steps, ~1.3 GB
  flag  FP32 adjoint-weighted flag passes without the m output (the
        envelope-pruned flag_kernel_f32x4) against a store of one snapshot
        every 100 adjoint steps, ~1.3 GB; `--full` requests m as well, which
        runs the full pass; `--adj-n 1024` puts the adjoint on a coarser
        1024^2 grid (the pruned bilinear flag_kernel)

Launch counts (for a profiler's -s / -c): `fwd` and `ctu` run 1 initial-CFL
launch then `--steps` step launches; `amr` runs its set-up launches, then 11
per step (coarse fluxes, coarse step, 4 x (fill, fine launch), averaging); `adj` runs 1 init launch then every adjoint step to
t_f; `flag` runs `--steps` flag passes after its set-up launches.

    python -m paper_1605_05320_gb300.profcase fwd --steps 120
"""
from __future__ import annotations

import argparse


def main(argv=None):
    import numpy as np
    import torch

    from . import build
    from . import swadj as S
    from . import synth
    ap = argparse.ArgumentParser()
    ap.add_argument("kernel", choices=["fwd", "ctu", "amr", "adj", "flag"])
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--steps", type=int, default=120)
    ap.add_argument("--full", action="store_true")
    ap.add_argument("--active", action="store_true",
                    help="fwd/ctu: random momenta of +-5 m^2/s in every cell")
    ap.add_argument("--adj-n", type=int, default=0,
                    help="flag: adjoint on a coarser adj_n^2 grid (bilinear stencil)")
    ap.add_argument("--rows", type=int, default=0,
                    help="amr: strip height of the fine level (16 or 32; 0 = default)")
    a = ap.parse_args(argv)
    build.build()
    S.load()
    n = a.n
    sc = synth.config2(n=n, L=n * 1e3)
    d = S.make_desc(2, n, n, 0.0, 0.0, sc.grid.dx, sc.grid.dy, precision=S.SWA_FP32)
    out = {}
    if a.kernel in ("fwd", "ctu"):
        g = S.Grid(d, sc.B)
        if a.kernel == "ctu":
            g.set_scheme(S.SWA_SCHEME_CTU)
        hu, hv = sc.hu0, sc.hv0
        if a.active:
            rng = np.random.default_rng(7)
            hu, hv = rng.uniform(-5.0, 5.0, sc.grid.n), rng.uniform(-5.0, 5.0, sc.grid.n)
        g.set_state(sc.eta0, hu, hv, 0.0)
        g.step(a.steps, sc.t_f)
        out["t"] = g.time()[0]
    elif a.kernel == "amr":
        B, eta, n2, dx, descs, fields = synth.amr_basin_2048()
        d2 = S.make_desc(2, n2, n2, 0.0, 0.0, dx, dx, precision=S.SWA_FP32)
        g = S.Grid(d2, B)
        z = np.zeros(n2 * n2)
        g.set_state(eta, z, z, 0.0)
        ps = S.PatchSet(descs, [f[0] for f in fields], d2)
        for k, f in enumerate(fields):
            ps.set_state(k, f[1], np.zeros_like(f[1]), np.zeros_like(f[1]))
        ps.start(1, 0.0)
        if a.rows:
            S.swa_patches_set_tile_rows(ps.h, 1, a.rows)
        amr = S.Amr(g, ps, 1, 4)
        dt_c = 0.9 * 0.75 * dx / np.sqrt(9.81 * float(np.max(-B)))
        t = 0.0
        for _ in range(a.steps):
            amr.step(t, dt_c)
            t = t + dt_c
        out["t"] = g.time()[0]
    elif a.kernel == "adj":
        adj = S.Adjoint(d, sc.B_adj, sc.phi, sc.t_f)
        N, _, _ = adj.info()
        st = S.SnapStore(adj, N // 100 + 3, S.SWA_FP32)
        st.run_adjoint(100)
        out["steps"] = N
        out["snaps"] = st.info()[0]
    else:
        ad = d
        if a.adj_n:
            sc = synth.config2(n=n, L=n * 1e3, adj_n=a.adj_n)
            ad = S.make_desc(2, a.adj_n, a.adj_n, 0.0, 0.0, sc.adj_grid.dx, sc.adj_grid.dy,
                             precision=S.SWA_FP32)
        adj = S.Adjoint(ad, sc.B_adj, sc.phi, sc.t_f)
        N, _, _ = adj.info()
        st = S.SnapStore(adj, N // 100 + 3, S.SWA_FP32)
        st.run_adjoint(100)
        g = S.Grid(d, sc.B)
        g.set_state(sc.eta0, sc.hu0, sc.hv0, 0.0)
        g.step(300, sc.t_f)
        fl = torch.zeros(n * n, dtype=torch.uint8, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        m = torch.zeros(n * n, dtype=torch.float32, device="cuda") if a.full else None
        for _ in range(a.steps):
            S.swa_flag_cells(g.h, st.h, sc.t_s, sc.t_f, sc.tol, S.SWA_FLAG_INTERP, fl,
                             m, cnt)
        out["snaps"] = st.info()[0]
        out["flags"] = cnt
    torch.cuda.synchronize()
    if S.swa_sync_status() != 0:
        raise RuntimeError("device status nonzero after the profiling case")
    print(a.kernel, {k: (int(v.item()) if hasattr(v, "item") else v) for k, v in out.items()})


if __name__ == "__main__":
    main()
