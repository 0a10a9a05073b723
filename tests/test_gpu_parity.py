"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

Tolerances (error metric: per field max|gpu - ref| / max|ref|):
  * FP64 forward: <= 1e-12 in h, hu, hv after 1000 steps; identical step
    count and time (the CFL reduction is exact)
  * FP64 adjoint: <= 1e-12 per component for every snapshot; identical tau
  * FP64 flags: identical except cells with |m - tol| <= 1e-6 tol; m to 1e-12
  * FP32 perturbation form: eta within 1e-5 m, momenta within 1e-5 of their
    maximum, after 200 steps (decimetre waves, 4000 m depth)
"""
import numpy as np
import pytest

import oracle as O
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


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)


def bath_seen(B, precision_fp32):
    """The bathymetry the GPU path works with: the FP32 path stores
    hbar = float(-B), so the oracle is given B = -hbar to compare like with
    like (eta is then exactly the same number on both sides)."""
    if not precision_fp32:
        return B
    return -(np.float32(-B).astype(np.float64))


def desc_of(S, spec, precision, order=2, bc=(0, 0, 0, 0)):
    return S.make_desc(spec.ndim, spec.nx, spec.ny, spec.x_lo, spec.y_lo, spec.dx,
                       spec.dy, precision=precision, order=order, bc=bc)


def run_gpu_forward(S, sc, precision, order, bc, nsteps, t_end=1e12):
    g = S.Grid(desc_of(S, sc.grid, precision, order, bc), sc.B)
    g.set_state(sc.eta0, sc.hu0, sc.hv0 if sc.grid.ndim == 2 else None, 0.0)
    g.step(nsteps, t_end)
    st = g.get_state()
    t, dt, n = g.time()
    assert S.swa_sync_status() == 0
    return st, t, n


def run_oracle_forward(sc, order, bc, nsteps, t_end=1e12, B=None):
    og = O.Grid.from_spec(sc.grid, order=order, bc=bc)
    B = sc.B if B is None else B
    h0 = sc.eta0 - B
    hv = sc.hv0 if sc.grid.ndim == 2 else None
    return O.fwd_run(og, h0, sc.hu0, hv, B, nsteps, t_end)


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 1, 1, 1), (1, 0, 0, 1)])
def test_fp64_forward_2d_1000_steps(S, order, bc):
    # 150 x 97: several 32 x 4 tiles with ragged edges in both directions
    sc = synth.small_2d(150, 97, seed=3)
    st, t, n = run_gpu_forward(S, sc, S.SWA_FP64, order, bc, 1000)
    h, hu, hv, t_ref, n_ref = run_oracle_forward(sc, order, bc, 1000)
    assert n == n_ref == 1000
    assert abs(t - t_ref) <= 1e-12 * t_ref
    assert rel(st["h"], h) <= 1e-12
    assert rel(st["hu"], hu) <= 1e-12
    assert rel(st["hv"], hv) <= 1e-12


def test_fp64_forward_rounds_like_the_oracle(S):
    """The FP64 kernels are built without contraction and evaluate in the
    oracle's order: the result is bit-identical, which is what the 1e-12
    bound needs in (h, hu) form (one ulp of a 4000 m depth moves hu by ~1e-11
    per step through g hhat d_eta)."""
    sc = synth.small_2d(150, 97, seed=13)
    st, t, n = run_gpu_forward(S, sc, S.SWA_FP64, 2, (1, 0, 0, 1), 300)
    h, hu, hv, t_ref, n_ref = run_oracle_forward(sc, 2, (1, 0, 0, 1), 300)
    assert t == t_ref
    assert np.array_equal(st["h"], h) and np.array_equal(st["hu"], hu)
    assert np.array_equal(st["hv"], hv)


def test_fp64_forward_1d_config1(S):
    sc = synth.config1()
    st, t, n = run_gpu_forward(S, sc, S.SWA_FP64, 2, (0, 0, 0, 0), 1000)
    h, hu, _, t_ref, n_ref = run_oracle_forward(sc, 2, (0, 0, 0, 0), 1000)
    assert n == n_ref
    assert abs(t - t_ref) <= 1e-12 * t_ref
    assert rel(st["h"], h) <= 1e-12 and rel(st["hu"], hu) <= 1e-12


def test_forward_stops_at_t_end(S):
    sc = synth.small_2d(40, 33, seed=4)
    t_end = 37.5
    st, t, n = run_gpu_forward(S, sc, S.SWA_FP64, 2, (0, 0, 0, 0), 500, t_end)
    h, hu, hv, t_ref, n_ref = run_oracle_forward(sc, 2, (0, 0, 0, 0), 500, t_end)
    assert t == t_end and t_ref == t_end and n == n_ref < 500
    assert rel(st["h"], h) <= 1e-12


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_lake_at_rest_bit_exact(S, precision):
    sc = synth.small_2d(70, 45, seed=5)
    p = S.SWA_FP64 if precision == "fp64" else S.SWA_FP32
    g = S.Grid(desc_of(S, sc.grid, p, 2, (1, 0, 1, 0)), sc.B)
    z = np.zeros(sc.grid.n)
    g.set_state(z, z, z, 0.0)
    g.step(300, 1e12)
    st = g.get_state()
    assert np.all(st["eta"] == 0.0) and np.all(st["hu"] == 0) and np.all(st["hv"] == 0)
    assert g.time()[2] == 300


def test_fp32_perturbation_forward_vs_fp64_oracle(S):
    sc = synth.small_2d(130, 90, seed=6, amp=0.5)
    st, t, n = run_gpu_forward(S, sc, S.SWA_FP32, 2, (0, 0, 0, 0), 200)
    Bf = bath_seen(sc.B, True)
    h, hu, hv, t_ref, n_ref = run_oracle_forward(sc, 2, (0, 0, 0, 0), 200, B=Bf)
    assert n == n_ref
    assert abs(t - t_ref) <= 1e-5 * t_ref
    eta_ref = h + Bf
    assert np.abs(st["eta"] - eta_ref).max() <= 1e-5
    assert rel(st["hu"], hu) <= 1e-5 and rel(st["hv"], hv) <= 1e-5


def _adjoint_pair(S, sc, precision, every, bc=(0, 0, 0, 0), order=2):
    ad = desc_of(S, sc.adj_grid, precision, order, bc)
    adj = S.Adjoint(ad, sc.B_adj, sc.phi, sc.t_f)
    N, dt, _ = adj.info()
    store = S.SnapStore(adj, N // every + 3, precision)
    store.run_adjoint(every)
    K, tau = store.info()
    og = O.Grid.from_spec(sc.adj_grid, order=order, bc=bc)
    hbar = np.maximum(-sc.B_adj, 0.0)
    snaps, tau_ref, N_ref, dt_ref = O.adj_run(og, hbar, sc.phi, sc.t_f, every)
    return adj, store, (N, dt, K, tau), (snaps, tau_ref, N_ref, dt_ref)


def _read_snaps(S, store, precision, nc, n):
    K = store.info()[0]
    dt = np.float64 if precision == S.SWA_FP64 else np.float32
    esz = 8 if precision == S.SWA_FP64 else 4
    raw = store.ws[: K * nc * n * esz].cpu().numpy().view(dt)
    return raw.reshape(K, nc, n).astype(np.float64)


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 1, 1, 1)])
def test_fp64_adjoint_snapshots(S, bc):
    sc = synth.small_2d(96, 70, seed=7)
    adj, store, (N, dt, K, tau), (snaps, tau_ref, N_ref, dt_ref) = \
        _adjoint_pair(S, sc, S.SWA_FP64, 5, bc)
    assert N == N_ref and dt == dt_ref
    assert K == len(tau_ref) and np.array_equal(tau, tau_ref)
    got = _read_snaps(S, store, S.SWA_FP64, 3, sc.adj_grid.n)
    for k in range(K):
        for c in range(3):
            ref = snaps[k, c]
            if np.abs(ref).max() == 0:
                assert np.all(got[k, c] == 0)
            else:
                assert rel(got[k, c], ref) <= 1e-12, (k, c)


def test_fp64_adjoint_1d_with_dry_cells(S):
    sc = synth.config1(nx=600)
    B = sc.B.copy()
    B[550:] = 5.0   # land beyond x = 333 km: wet/dry wall
    sc.B_adj = B
    sc.phi[:, 550:] = 0.0
    sc.t_f = 1800.0
    adj, store, (N, dt, K, tau), (snaps, tau_ref, N_ref, dt_ref) = \
        _adjoint_pair(S, sc, S.SWA_FP64, 10)
    assert N == N_ref and np.array_equal(tau, tau_ref)
    got = _read_snaps(S, store, S.SWA_FP64, 2, sc.adj_grid.n)
    assert rel(got, snaps) <= 1e-12


def _with_island(sc):
    """Dry adjoint cells (B > 0) in a disc of radius 8 cells in mid-basin: the
    edges around it are wet/dry walls of the adjoint (Sec. 5)."""
    xc, yc = sc.adj_grid.centres()
    X, Y = np.meshgrid(xc, yc)
    L, Ly = sc.adj_grid.nx * sc.adj_grid.dx, sc.adj_grid.ny * sc.adj_grid.dy
    r = np.hypot(X - 0.6 * L, Y - 0.5 * Ly).ravel()
    sc.B_adj = np.where(r < 8 * sc.adj_grid.dx, 10.0, sc.B_adj)
    sc.phi[:, r < 8 * sc.adj_grid.dx] = 0.0
    return sc


def test_fp64_adjoint_2d_with_island(S):
    sc = _with_island(synth.small_2d(96, 70, seed=7))
    adj, store, (N, dt, K, tau), (snaps, tau_ref, N_ref, dt_ref) = \
        _adjoint_pair(S, sc, S.SWA_FP64, 5, (1, 0, 0, 1))
    assert N == N_ref and np.array_equal(tau, tau_ref)
    got = _read_snaps(S, store, S.SWA_FP64, 3, sc.adj_grid.n)
    for c in range(3):
        assert rel(got[:, c], snaps[:, c]) <= 1e-12, c


def test_adjoint_with_indicator_target(S):
    """Adjoint data an indicator of a disc (discontinuous, as the target
    regions of the paper's examples): FP64 snapshots within 1e-12 of the
    oracle, FP32 within 5e-5 of each component's maximum over the run."""
    sc = synth.small_2d(96, 70, seed=7)
    L = sc.adj_grid.nx * sc.adj_grid.dx
    Ly = sc.adj_grid.ny * sc.adj_grid.dy
    sc.phi[:] = 0.0
    sc.phi[0] = synth.disc_indicator(sc.adj_grid, 0.8 * L, 0.5 * Ly, 6 * sc.adj_grid.dx)
    for prec, bound in ((S.SWA_FP64, 1e-12), (S.SWA_FP32, 5e-5)):
        adj, store, (N, dt, K, tau), (snaps, tau_ref, N_ref, dt_ref) = \
            _adjoint_pair(S, sc, prec, 5, (1, 1, 1, 1))
        assert N == N_ref and np.array_equal(tau, tau_ref)
        got = _read_snaps(S, store, prec, 3, sc.adj_grid.n)
        for c in range(3):
            assert rel(got[:, c], snaps[:, c]) <= bound, (prec, c, rel(got[:, c], snaps[:, c]))


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 1, 1, 1), (1, 0, 0, 1)])
def test_fp32_adjoint_snapshots_vs_oracle(S, order, bc):
    """FP32 adjoint (c = sqrt(g hbar) rounded to float, float arithmetic)
    against the FP64 oracle on a 96 x 70 grid (ragged in both tile
    directions) with an island: every snapshot, every component, within
    2e-5 of the component's maximum over the run."""
    sc = _with_island(synth.small_2d(96, 70, seed=7))
    adj, store, (N, dt, K, tau), (snaps, tau_ref, N_ref, dt_ref) = \
        _adjoint_pair(S, sc, S.SWA_FP32, 5, bc, order)
    assert N == N_ref and np.array_equal(tau, tau_ref)
    got = _read_snaps(S, store, S.SWA_FP32, 3, sc.adj_grid.n)
    dry = sc.B_adj > 0
    for c in range(3):
        err = rel(got[:, c], snaps[:, c])
        assert err <= 2e-5, (c, err)
        assert np.all(got[:, c][:, dry] == 0)


def _flag_compare(S, sc, precision, mode, t_s, nsteps, every=5, with_m=True):
    """Both sides compute everything from the seeded inputs: adjoint with
    snapshots, nsteps forward steps, then the flag pass."""
    fp32 = precision == S.SWA_FP32
    adj, store, (N, dt, K, tau), (snaps, tau_ref, _, _) = \
        _adjoint_pair(S, sc, precision, every)
    g = S.Grid(desc_of(S, sc.grid, precision), sc.B)
    g.set_state(sc.eta0, sc.hu0, sc.hv0, 0.0)
    g.step(nsteps, sc.t_f)
    n = sc.grid.n
    flags = torch.zeros(n, dtype=torch.uint8, device="cuda")
    m = torch.zeros(n, dtype=torch.float32, device="cuda") if with_m else None
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    S.swa_flag_cells(g.h, store.h, t_s, sc.t_f, sc.tol, mode, flags, m, cnt)
    torch.cuda.synchronize()
    # oracle side
    Bs = bath_seen(sc.B, fp32)
    h, hu, hv, t_ref, _ = run_oracle_forward(sc, 2, (0, 0, 0, 0), nsteps, sc.t_f, B=Bs)
    og = O.Grid.from_spec(sc.grid)
    ag = O.Grid.from_spec(sc.adj_grid)
    f_ref, m_ref, c_ref = O.flag(og, h, hu, hv, Bs, t_ref, ag,
                                 np.maximum(-sc.B_adj, 0), snaps, tau_ref, t_s,
                                 sc.t_f, sc.tol, mode)
    m = None if m is None else m.cpu().numpy()
    return flags.cpu().numpy(), m, int(cnt.item()), f_ref, m_ref, c_ref


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("t_s_frac", [0.32, 1.0])
def test_fp64_flags_match_oracle(S, mode, t_s_frac):
    sc = synth.small_2d(88, 61, seed=8)
    f, m, c, f_ref, m_ref, c_ref = _flag_compare(S, sc, S.SWA_FP64, mode,
                                                 t_s_frac * sc.t_f, 150)
    near = np.abs(m_ref - sc.tol) <= 1e-6 * sc.tol
    assert np.array_equal(f[~near], f_ref[~near])
    assert c_ref > 0 and abs(c - c_ref) <= near.sum()
    assert np.abs(m - m_ref).max() <= 1e-6 * m_ref.max() + 1e-30  # m is stored as float
    assert f.sum() == c


def test_fp32_flags_close_to_oracle(S):
    sc = synth.small_2d(88, 61, seed=9)
    f, m, c, f_ref, m_ref, c_ref = _flag_compare(S, sc, S.SWA_FP32, 0, 0.32 * sc.t_f, 150)
    near = np.abs(m_ref - sc.tol) <= 1e-3 * sc.tol
    assert np.array_equal(f[~near], f_ref[~near])
    assert np.abs(m - m_ref).max() <= 1e-4 * m_ref.max()


def _flags_pruned_and_full(S, g, store, t_s, t_f, tol, mode):
    n = g.desc.nx * g.desc.ny
    out = []
    for with_m in (False, True):
        flags = torch.zeros(n, dtype=torch.uint8, device="cuda")
        m = torch.zeros(n, dtype=torch.float32, device="cuda") if with_m else None
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        S.swa_flag_cells(g.h, store.h, t_s, t_f, tol, mode, flags, m, cnt)
        torch.cuda.synchronize()
        out.append((flags.cpu().numpy(), int(cnt.item()), None if m is None else m.cpu().numpy()))
    assert S.swa_sync_status() == 0
    return out


@pytest.mark.parametrize("mode", [0, 1])
def test_pruned_flag_pass_identical_to_full_pass(S, mode):
    """The envelope-pruned pass (no m output) against the full pass (m
    requested) on the same device data: identical flags and count at several
    forward times, window widths down to less than one snapshot interval, and
    tolerances spanning the range of m.  The source is a bump on an ocean at
    rest, so most of the grid is quiet ahead of the wave front."""
    sc = synth.small_2d(256, 160, seed=12)
    sc.hu0[:] = 0.0
    sc.hv0[:] = 0.0
    d = desc_of(S, sc.grid, S.SWA_FP32)
    adj = S.Adjoint(d, sc.B_adj, sc.phi, sc.t_f)
    N, dt, _ = adj.info()
    store = S.SnapStore(adj, N // 5 + 3, S.SWA_FP32)
    store.run_adjoint(5)
    g = S.Grid(d, sc.B)
    g.set_state(sc.eta0, sc.hu0, sc.hv0, 0.0)
    done, checked = 0, 0
    for target in (10, 60, 140, 260, 400):
        g.step(target - done, sc.t_f)
        done = target
        for t_s in (0.32 * sc.t_f, 0.95 * sc.t_f, sc.t_f - 0.5 * dt):
            (fp, cp, _), (ff, cf, m) = _flags_pruned_and_full(S, g, store, t_s, sc.t_f,
                                                                sc.tol, mode)
            assert np.array_equal(fp, ff) and cp == cf, (target, t_s)
            pos = m[m > 0]
            for tol in (np.quantile(pos, [0.1, 0.5, 0.9, 0.999]) if pos.size else []):
                (fp, cp, _), (ff, cf, _) = _flags_pruned_and_full(S, g, store, t_s, sc.t_f,
                                                                  float(tol), mode)
                assert np.array_equal(fp, ff) and cp == cf and cf > 0, (target, t_s, tol)
                checked += 1
    # flagged sets were compared at most (time, window) pairs
    assert checked >= 20


def test_pruned_flags_on_a_coarser_adjoint_grid(S):
    """FP32 forward grid with the adjoint on a coarser grid (bilinear
    stencil): the envelope-pruned pass equals the full pass bit for bit at
    several times, windows and tolerances, and matches the oracle."""
    sc = synth.config2(n=96, L=96e3 * 4, adj_n=40, seed=11)
    sc.hu0[:] = 0.0
    sc.hv0[:] = 0.0
    d = desc_of(S, sc.grid, S.SWA_FP32)
    ad = desc_of(S, sc.adj_grid, S.SWA_FP32)
    adj = S.Adjoint(ad, sc.B_adj, sc.phi, sc.t_f)
    N, dt, _ = adj.info()
    store = S.SnapStore(adj, N // 5 + 3, S.SWA_FP32)
    store.run_adjoint(5)
    g = S.Grid(d, sc.B)
    g.set_state(sc.eta0, sc.hu0, sc.hv0, 0.0)
    done, checked = 0, 0
    for target in (10, 60, 140):
        g.step(target - done, sc.t_f)
        done = target
        for t_s in (sc.t_s, 0.95 * sc.t_f, sc.t_f - 0.5 * dt):
            for mode in (0, 1):
                (fp, cp, _), (ff, cf, m) = _flags_pruned_and_full(S, g, store, t_s, sc.t_f,
                                                                    sc.tol, mode)
                assert np.array_equal(fp, ff) and cp == cf, (target, t_s, mode)
                pos = m[m > 0]
                for tol in (np.quantile(pos, [0.1, 0.5, 0.9]) if pos.size else []):
                    (fp, cp, _), (ff, cf, _) = _flags_pruned_and_full(
                        S, g, store, t_s, sc.t_f, float(tol), mode)
                    assert np.array_equal(fp, ff) and cp == cf and cf > 0
                    checked += 1
    assert checked >= 12
    # against the oracle, from the seeded inputs
    f, _, c, f_ref, m_ref, c_ref = _flag_compare(S, sc, S.SWA_FP32, 0, sc.t_s, 100,
                                                 with_m=False)
    near = np.abs(m_ref - sc.tol) <= 1e-3 * sc.tol
    assert np.array_equal(f[~near], f_ref[~near])
    assert f.sum() == c


def test_pruned_flags_match_oracle(S):
    """The pruned pass (no m output) against the oracle's flags."""
    sc = synth.small_2d(88, 60, seed=9)
    sc.hu0[:] = 0.0
    sc.hv0[:] = 0.0
    f, _, c, f_ref, m_ref, c_ref = _flag_compare(S, sc, S.SWA_FP32, 0, 0.32 * sc.t_f, 150,
                                                 with_m=False)
    near = np.abs(m_ref - sc.tol) <= 1e-3 * sc.tol
    assert c_ref > 0
    assert np.array_equal(f[~near], f_ref[~near])
    assert f.sum() == c


def test_coarse_adjoint_grid_flags(S):
    """Adjoint on a coarser grid: bilinear interpolation onto forward cells."""
    sc = synth.config2(n=96, L=96e3 * 4, adj_n=40, seed=11)
    f, m, c, f_ref, m_ref, c_ref = _flag_compare(S, sc, S.SWA_FP64, 0, sc.t_s, 100)
    near = np.abs(m_ref - sc.tol) <= 1e-6 * sc.tol
    assert np.array_equal(f[~near], f_ref[~near])
    assert np.abs(m - m_ref).max() <= 1e-6 * m_ref.max()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_gauges_match_oracle(S, precision):
    sc = synth.small_2d(60, 50, seed=10)
    p = S.SWA_FP64 if precision == "fp64" else S.SWA_FP32
    g = S.Grid(desc_of(S, sc.grid, p), sc.B)
    g.set_state(sc.eta0, sc.hu0, sc.hv0, 0.0)
    g.step(20, 1e12)
    xy = np.array([[1.3e5, 2.2e5], [-5.0, 9e9], [5e5, 1e5], [3.333e5, 4.1e5]])
    xy_d = torch.tensor(xy, dtype=torch.float64, device="cuda")
    out = torch.zeros(len(xy), dtype=torch.float64, device="cuda")
    S.swa_gauge_sample(g.h, len(xy), xy_d, out)
    Bs = bath_seen(sc.B, p == S.SWA_FP32)
    h, hu, hv, _, _ = run_oracle_forward(sc, 2, (0, 0, 0, 0), 20, B=Bs)
    ref = O.gauge(O.Grid.from_spec(sc.grid), h, Bs, xy)
    tol = 1e-12 if precision == "fp64" else 1e-5
    assert np.abs(out.cpu().numpy() - ref).max() <= tol


def test_mass_conserved_walls_fp64_full_size(S):
    """Property at the full 2048^2 size: with walls the FP64 step conserves
    mass to roundoff."""
    sc = synth.config2()
    g = S.Grid(desc_of(S, sc.grid, S.SWA_FP64, 2, (1, 1, 1, 1)), sc.B)
    g.set_state(sc.eta0, sc.hu0, sc.hv0, 0.0)
    m0 = g.get_state()["h"].sum()
    g.step(20, 1e12)
    m1 = g.get_state()["h"].sum()
    assert abs(m1 - m0) / m0 <= 1e-13


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_full_size_step_sampled_against_oracle_windows(S, precision):
    """2048^2, the bench's launch configuration: one step from a perturbed
    state, sampled cells compared with the oracle run on 9 x 9 windows around
    them (a cell's update depends only on cells within 2 of it)."""
    sc = synth.config2()
    rng = np.random.default_rng(12)
    hu = rng.uniform(-20, 20, sc.grid.n)
    hv = rng.uniform(-20, 20, sc.grid.n)
    p = S.SWA_FP64 if precision == "fp64" else S.SWA_FP32
    fp32 = p == S.SWA_FP32
    g = S.Grid(desc_of(S, sc.grid, p), sc.B)
    g.set_state(sc.eta0, hu, hv, 0.0)
    g.step(1, 1e12)
    s1 = g.get_state()
    # the oracle's inputs: the seeded state as the storage precision holds it
    Bs = bath_seen(sc.B, fp32)
    if fp32:
        eta = np.float32(sc.eta0).astype(np.float64)
        hu = np.float32(hu).astype(np.float64)
        hv = np.float32(hv).astype(np.float64)
    else:
        eta = sc.eta0
    s0 = {"h": eta - Bs, "hu": hu, "hv": hv}
    og = O.Grid.from_spec(sc.grid)
    dt = og.cfl / O.fwd_smax(og, s0["h"], s0["hu"], s0["hv"])
    nx = sc.grid.nx
    cells = [(int(i), int(j)) for i, j in zip(rng.integers(0, nx, 200), rng.integers(0, nx, 200))]
    cells += [(0, 0), (nx - 1, 5), (7, nx - 1), (nx - 1, nx - 1)]
    for (i, j) in cells:
        ii = np.clip(np.arange(i - 4, i + 5), 0, nx - 1)
        jj = np.clip(np.arange(j - 4, j + 5), 0, nx - 1)
        idx = (jj[:, None] * nx + ii[None, :]).ravel()
        wg = O.Grid(2, 9, 9, 0.0, 0.0, sc.grid.dx, sc.grid.dy, order=2)
        h, u, v = O.fwd_step(wg, s0["h"][idx], s0["hu"][idx], s0["hv"][idx], Bs[idx], dt)
        o = (j * nx + i)
        if precision == "fp64":
            assert abs(s1["h"][o] - h[40]) <= 1e-12 * 4000
            assert abs(s1["hu"][o] - u[40]) <= 1e-12 * 200
            assert abs(s1["hv"][o] - v[40]) <= 1e-12 * 200
        else:
            assert abs(s1["eta"][o] - (h[40] + Bs[o])) <= 2e-6
            assert abs(s1["hu"][o] - u[40]) <= 2e-5 and abs(s1["hv"][o] - v[40]) <= 2e-5


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_surface_flags_match_oracle(S, precision):
    sc = synth.small_2d(120, 80, seed=14, amp=0.6)
    p = S.SWA_FP64 if precision == "fp64" else S.SWA_FP32
    g = S.Grid(desc_of(S, sc.grid, p), sc.B)
    g.set_state(sc.eta0, sc.hu0, sc.hv0, 0.0)
    g.step(30, 1e12)
    flags = torch.zeros(sc.grid.n, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    S.swa_flag_surface(g.h, 0.09, flags, cnt)
    torch.cuda.synchronize()
    Bs = bath_seen(sc.B, p == S.SWA_FP32)
    h, hu, hv, _, _ = run_oracle_forward(sc, 2, (0, 0, 0, 0), 30, B=Bs)
    f_ref, c_ref = O.flag_surface(O.Grid.from_spec(sc.grid), h, Bs, 0.09)
    f = flags.cpu().numpy()
    eta = h + Bs
    near = np.abs(np.abs(eta) - 0.09) <= (1e-12 if precision == "fp64" else 1e-5)
    assert np.array_equal(f[~near], f_ref[~near])
    assert c_ref > 0 and int(cnt.item()) == int(f.sum())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fused_gauge_recording_matches_per_step_sampling(S, precision):
    """Gauges recorded by the step kernel (the state each step starts from)
    equal swa_gauge_sample before each step; rows stop at capacity; steps
    past t_end record nothing."""
    sc = synth.small_2d(90, 64, seed=31)
    p = S.SWA_FP64 if precision == "fp64" else S.SWA_FP32
    d = desc_of(S, sc.grid, p)
    xy = torch.tensor(np.concatenate([sc.gauges, [[0.5e6, 0.2e6], [0.01e6, 0.6e6]]]),
                      dtype=torch.float64, device="cuda")
    ng, nsteps, cap = xy.shape[0], 30, 25
    # reference: one sample after every step
    g1 = S.Grid(d, sc.B)
    g1.set_state(sc.eta0, sc.hu0, sc.hv0, 0.0)
    ref = torch.zeros((nsteps, ng), dtype=torch.float64, device="cuda")
    tref = []
    for s in range(nsteps):
        S.swa_gauge_sample(g1.h, ng, xy, ref[s])
        tref.append(g1.time()[0])
        g1.step(1, 1e300)
    # fused
    g2 = S.Grid(d, sc.B)
    g2.set_state(sc.eta0, sc.hu0, sc.hv0, 0.0)
    series = torch.full((cap, ng), -7.0, dtype=torch.float64, device="cuda")
    times = torch.zeros(cap, dtype=torch.float64, device="cuda")
    S.swa_grid_record_gauges(g2.h, ng, xy, series, times, cap)
    g2.step(nsteps, 1e300)
    assert S.swa_grid_gauge_rows(g2.h) == nsteps
    torch.cuda.synchronize()
    assert torch.equal(series, ref[:cap])
    assert np.array_equal(times.cpu().numpy(), np.array(tref[:cap]))
    # steps past t_end are no-ops and record nothing
    S.swa_grid_record_gauges(g2.h, ng, xy, series, times, cap)
    t_now = g2.time()[0]
    g2.step(5, t_now)
    assert S.swa_grid_gauge_rows(g2.h) == 0
    # off
    S.swa_grid_record_gauges(g2.h, 0, None, None, None, 0)
    g2.step(2, 1e300)
    assert S.swa_grid_gauge_rows(g2.h) == 0
    assert S.swa_sync_status() == 0


@pytest.mark.parametrize("nx,ny", [(2, 2), (3, 5), (29, 2), (5, 31), (33, 3)])
@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 1, 1, 1)])
def test_degenerate_grids_forward_and_adjoint(S, nx, ny, bc):
    """Grids narrower than a warp strip and only a few rows high: every
    strip lane and row beyond the grid is index-mapped to a ghost cell.
    FP64 forward and adjoint within 1e-12 of the oracle, the FP32 forward
    within the perturbation-form tolerance after 40 steps, the FP32 adjoint
    within 2e-5 of each component's maximum."""
    sc = synth.small_2d(nx, ny, seed=40 + nx + ny, L=nx * 5e3)
    st, t, n = run_gpu_forward(S, sc, S.SWA_FP64, 2, bc, 40)
    h, hu, hv, t_ref, n_ref = run_oracle_forward(sc, 2, bc, 40)
    assert n == n_ref == 40 and abs(t - t_ref) <= 1e-12 * t_ref
    for got, ref in ((st["h"], h), (st["hu"], hu), (st["hv"], hv)):
        assert np.abs(got - ref).max() <= 1e-12 * max(np.abs(ref).max(), 1.0)
    st32, t32, n32 = run_gpu_forward(S, sc, S.SWA_FP32, 2, bc, 40)
    Bf = bath_seen(sc.B, True)
    h, hu, hv, _, _ = run_oracle_forward(sc, 2, bc, 40, B=Bf)
    assert n32 == 40
    assert np.abs(st32["eta"] - (h + Bf)).max() <= 1e-5
    assert np.abs(st32["hu"] - hu).max() <= 1e-4 * max(np.abs(hu).max(), 1.0)
    assert np.abs(st32["hv"] - hv).max() <= 1e-4 * max(np.abs(hv).max(), 1.0)
    adj, store, (N, dt, K, tau), (snaps, tau_ref, N_ref, dt_ref) = \
        _adjoint_pair(S, sc, S.SWA_FP64, 5, bc)
    assert N == N_ref and np.array_equal(tau, tau_ref)
    got = _read_snaps(S, store, S.SWA_FP64, 3, sc.adj_grid.n)
    assert np.abs(got - snaps).max() <= 1e-12 * max(np.abs(snaps).max(), 1.0)
    adj32, store32, (N32, _, _, tau32), _ = _adjoint_pair(S, sc, S.SWA_FP32, 5, bc)
    assert N32 == N_ref and np.array_equal(tau32, tau_ref)
    got32 = _read_snaps(S, store32, S.SWA_FP32, 3, sc.adj_grid.n)
    for c in range(3):
        assert np.abs(got32[:, c] - snaps[:, c]).max() <= \
            2e-5 * max(np.abs(snaps[:, c]).max(), 1e-30) + 1e-30
    assert S.swa_sync_status() == 0


@pytest.mark.parametrize("nx,ny", [(3, 5), (4, 3), (29, 2), (33, 3), (8, 6)])
def test_degenerate_grids_flags(S, nx, ny):
    """Flag passes on grids of a few cells (cell counts that are and are not
    multiples of 4 take the generic and the 4-cell kernels), against the
    oracle in FP64 and FP32, pruned (no m output) in FP32."""
    sc = synth.small_2d(nx, ny, seed=60 + nx + ny, L=nx * 5e3)
    sc.tol = 1e-7
    f, m, c, f_ref, m_ref, c_ref = _flag_compare(S, sc, S.SWA_FP64, 0, 0.32 * sc.t_f, 20)
    near = np.abs(m_ref - sc.tol) <= 1e-6 * sc.tol
    assert np.array_equal(f[~near], f_ref[~near]) and f.sum() == c
    assert np.abs(m - m_ref).max() <= 1e-6 * max(m_ref.max(), 1e-30)
    for with_m in (True, False):
        f, m, c, f_ref, m_ref, c_ref = _flag_compare(S, sc, S.SWA_FP32, 0, 0.32 * sc.t_f, 20,
                                                     with_m=with_m)
        near = np.abs(m_ref - sc.tol) <= 1e-3 * sc.tol
        assert np.array_equal(f[~near], f_ref[~near]) and f.sum() == c
    assert c_ref > 0


@pytest.mark.parametrize("bc,rows", [((0, 0, 0, 0), 32), ((1, 0, 1, 0), 32),
                                     ((1, 1, 0, 1), 16), ((0, 1, 1, 0), 64)])
def test_rest_skip_is_exact(S, bc, rows):
    """Skipping the wave arithmetic of rows exactly at rest, and the copy of
    quiet units (every cell of the unit's stencil window at rest), gives the
    same state, time and step count as computing them in full: a compact
    source on an ocean at rest (most units quiet at first, fewer as the wave
    spreads and reaches the walls), 150 steps each way, compared value for
    value (an exact zero may differ in sign)."""
    sc = synth.small_2d(300, 260, seed=31)
    eta0 = np.where(np.abs(sc.eta0) < 1e-6, 0.0, sc.eta0)
    z = np.zeros_like(eta0)
    out = []
    for on in (1, 0):
        g = S.Grid(desc_of(S, sc.grid, S.SWA_FP32, 2, bc), sc.B)
        S.swa_grid_set_strip_rows(g.h, rows)
        S.swa_grid_set_rest_skip(g.h, on)
        g.set_state(eta0, z, z, 0.0)
        g.step(150, 1e12)
        out.append((g.get_state(), g.time()))
    assert S.swa_sync_status() == 0
    (a, ta), (b, tb) = out
    assert ta == tb
    for f in ("eta", "hu", "hv"):
        assert np.array_equal(a[f], b[f]), f
    assert np.abs(a["eta"]).max() > 1e-3 and (a["eta"] == 0).mean() > 0.1   # both parts present
