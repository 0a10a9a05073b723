"""Thin ctypes binding of libswadj.so (see include/swadj.h).

Functions here carry the C names and only marshal arguments: every step of
the method runs in the CUDA kernels of the library.  Device memory comes
from PyTorch (CUDA tensors used as workspaces and buffers); streams are
passed as raw cudaStream_t handles.  Importing this module on a machine
without the built library raises; there is no CPU fallback.

The small classes at the bottom (Grid, Adjoint, SnapStore) only allocate the
workspaces with torch and keep them alive next to the handles.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libswadj.so")

SWA_OK, SWA_EINVAL, SWA_ENOMEM, SWA_ECUDA, SWA_ESTATE, SWA_EUNSTABLE, SWA_ETIMEOUT = \
    0, -1, -2, -3, -4, -5, -6
SWA_FP64, SWA_FP32 = 0, 1
SWA_BC_EXTRAP, SWA_BC_WALL = 0, 1
SWA_FLAG_INTERP, SWA_FLAG_BRACKET = 0, 1
SWA_HOST, SWA_DEVICE = 0, 1
SWA_SCHEME_SPLIT, SWA_SCHEME_CTU = 0, 1

# Every symbol declared in include/swadj.h.
EXPORTS = [
    "swa_version", "swa_last_error", "swa_sync_status",
    "swa_grid_workspace_bytes", "swa_create_grid", "swa_destroy_grid",
    "swa_set_state", "swa_get_state", "swa_step_forward", "swa_get_time",
    "swa_grid_set_strip_rows",
    "swa_grid_set_scheme",
    "swa_grid_set_rest_skip",
    "swa_grid_arrays",
    "swa_adjoint_workspace_bytes", "swa_create_adjoint", "swa_destroy_adjoint",
    "swa_adjoint_info", "swa_step_adjoint", "swa_adjoint_set_steps_per_pass", "swa_get_adjoint_state",
    "swa_set_adjoint_state", "swa_snapstore_clear",
    "swa_snapstore_workspace_bytes", "swa_create_snapstore",
    "swa_destroy_snapstore", "swa_store_snapshot", "swa_run_adjoint",
    "swa_snapstore_info",
    "swa_flag_cells", "swa_flag_surface", "swa_gauge_sample",
    "swa_grid_record_gauges", "swa_grid_gauge_rows",
    "swa_step_forward_static",
    "swa_patches_workspace_bytes", "swa_create_patches", "swa_destroy_patches",
    "swa_patches_set_state", "swa_patches_start_level", "swa_patches_get_state",
    "swa_step_level", "swa_patches_get_time", "swa_patches_level_info",
    "swa_patches_set_tile_rows",
    "swa_amr_workspace_bytes", "swa_create_amr", "swa_destroy_amr", "swa_amr_step",
    "swa_amr_set_reflux", "swa_amr_info", "swa_grid_set_wetdry", "swa_amr_set_fill_mode", "swa_amr_levels_workspace_bytes",
    "swa_create_amr_levels",
    "swa_alu_probe_ops", "swa_alu_probe",
    "swa_grid_mass",
]


class SwaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"swadj error {code}: {msg}")
        self.code = code


class swa_grid_desc(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("x_lo", ctypes.c_double), ("y_lo", ctypes.c_double),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("precision", ctypes.c_int), ("order", ctypes.c_int),
                ("bc", ctypes.c_int * 4),
                ("g", ctypes.c_double), ("cfl", ctypes.c_double),
                ("dry_tol", ctypes.c_double)]


class swa_patch_desc(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("x_lo", ctypes.c_double), ("y_lo", ctypes.c_double),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double)]


def make_desc(ndim, nx, ny, x_lo, y_lo, dx, dy, precision=SWA_FP64, order=2,
              bc=(SWA_BC_EXTRAP,) * 4, g=9.81, cfl=0.75, dry_tol=1e-3):
    d = swa_grid_desc()
    d.ndim, d.nx, d.ny = int(ndim), int(nx), int(ny)
    d.x_lo, d.y_lo, d.dx, d.dy = float(x_lo), float(y_lo), float(dx), float(dy)
    d.precision, d.order = int(precision), int(order)
    for k in range(4):
        d.bc[k] = int(bc[k])
    d.g, d.cfl, d.dry_tol = float(g), float(cfl), float(dry_tol)
    return d


_lib = None
_V = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_SZ = ctypes.c_size_t
_P = ctypes.POINTER


def load(path: str = LIB_PATH):
    """Load the library (built beforehand by build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libswadj.so not built at {path}; run "
                          "paper_1605_05320_gb300.build.build() first")
    lib = ctypes.CDLL(path)
    D = _P(swa_grid_desc)
    sig = {
        "swa_version": ([], ctypes.c_char_p),
        "swa_last_error": ([], ctypes.c_char_p),
        "swa_sync_status": ([_V], _I),
        "swa_grid_workspace_bytes": ([D], _SZ),
        "swa_create_grid": ([D, _V, _V, _SZ, _V, _P(_V)], _I),
        "swa_destroy_grid": ([_V], _I),
        "swa_set_state": ([_V, _V, _V, _V, _D, _I, _V], _I),
        "swa_get_state": ([_V, _V, _V, _V, _V, _I, _V], _I),
        "swa_step_forward": ([_V, _I, _D, _V], _I),
        "swa_get_time": ([_V, _P(_D), _P(_D), _P(ctypes.c_longlong), _V], _I),
        "swa_grid_arrays": ([_V, _P(_V), _P(_V), _P(_V), _P(_V), _V], _I),
        "swa_grid_set_strip_rows": ([_V, _I], _I),
        "swa_grid_set_scheme": ([_V, _I], _I),
        "swa_grid_set_rest_skip": ([_V, _I], _I),
        "swa_adjoint_workspace_bytes": ([D], _SZ),
        "swa_create_adjoint": ([D, _V, _V, _D, _V, _SZ, _V, _P(_V)], _I),
        "swa_destroy_adjoint": ([_V], _I),
        "swa_adjoint_info": ([_V, _P(ctypes.c_longlong), _P(_D), _P(ctypes.c_longlong)], _I),
        "swa_step_adjoint": ([_V, _I, _V], _I),
        "swa_adjoint_set_steps_per_pass": ([_V, _I], _I),
        "swa_get_adjoint_state": ([_V, _V, _I, _V], _I),
        "swa_set_adjoint_state": ([_V, _V, _I, _V], _I),
        "swa_snapstore_clear": ([_V], _I),
        "swa_snapstore_workspace_bytes": ([D, _I, _I], _SZ),
        "swa_create_snapstore": ([_V, _I, _I, _V, _SZ, _P(_V)], _I),
        "swa_destroy_snapstore": ([_V], _I),
        "swa_store_snapshot": ([_V, _V, _V], _I),
        "swa_run_adjoint": ([_V, _V, _I, _V], _I),
        "swa_snapstore_info": ([_V, _P(_I), _V, _I], _I),
        "swa_flag_cells": ([_V, _V, _D, _D, _D, _I, _V, _V, _V, _V], _I),
        "swa_gauge_sample": ([_V, _I, _V, _V, _V], _I),
        "swa_grid_record_gauges": ([_V, _I, _V, _V, _V, ctypes.c_longlong, _V], _I),
        "swa_grid_gauge_rows": ([_V, _P(ctypes.c_longlong), _V], _I),
        "swa_flag_surface": ([_V, _D, _V, _V, _V], _I),
        "swa_step_forward_static": ([D, _P(_V), _P(_V), _V, _D, _V, _V], _I),
        "swa_patches_workspace_bytes": ([_I, _V, D], _SZ),
        "swa_create_patches": ([_I, _V, _P(_V), D, _V, _SZ, _V, _P(_V)], _I),
        "swa_destroy_patches": ([_V], _I),
        "swa_patches_set_state": ([_V, _I, _V, _V, _V, _I, _V], _I),
        "swa_patches_start_level": ([_V, _I, _D, _V], _I),
        "swa_patches_get_state": ([_V, _I, _V, _V, _V, _V, _I, _V], _I),
        "swa_step_level": ([_V, _I, _I, _D, _V], _I),
        "swa_patches_get_time": ([_V, _I, _P(_D), _P(_D), _P(ctypes.c_longlong), _V], _I),
        "swa_patches_level_info": ([_V, _I, _P(_I), _P(_I), _P(ctypes.c_longlong)], _I),
        "swa_patches_set_tile_rows": ([_V, _I, _I], _I),
        "swa_amr_workspace_bytes": ([_V, _V, _I, _I], _SZ),
        "swa_create_amr": ([_V, _V, _I, _I, _V, _SZ, _V, _P(_V)], _I),
        "swa_destroy_amr": ([_V], _I),
        "swa_amr_step": ([_V, _D, _D, _I, _V], _I),
        "swa_amr_set_reflux": ([_V, _I], _I),
        "swa_grid_set_wetdry": ([_V, _I], _I),
        "swa_amr_set_fill_mode": ([_V, _I], _I),
        "swa_amr_info": ([_V, _I, _P(_I), _P(_I), _P(_I)], _I),
        "swa_amr_levels_workspace_bytes": ([_V, _V, _I, _P(_I), _P(_I)], _SZ),
        "swa_create_amr_levels": ([_V, _V, _I, _P(_I), _P(_I), _V, _SZ, _V, _P(_V)], _I),
        "swa_alu_probe_ops": ([_I, _I, _I, _I], _D),
        "swa_grid_mass": ([_V, _V, _V], _I),
        "swa_alu_probe": ([_I, _I, _I, _I, _V, _V], _I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _chk(rc):
    if rc != SWA_OK:
        raise SwaError(rc, load().swa_last_error().decode())
    return rc


def _ptr(x):
    """Device or host pointer of a torch tensor / numpy array / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        assert x.flags.c_contiguous
        return x.ctypes.data
    assert x.is_contiguous()
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ------------------------------------------------------------ same-name calls
def swa_version():
    return load().swa_version().decode()


def swa_last_error():
    return load().swa_last_error().decode()


def swa_sync_status(stream=None):
    return load().swa_sync_status(_stream(stream))


def swa_grid_workspace_bytes(desc):
    return int(load().swa_grid_workspace_bytes(ctypes.byref(desc)))


def swa_create_grid(desc, bathy_host, ws, ws_bytes, stream=None):
    out = _V()
    _chk(load().swa_create_grid(ctypes.byref(desc), _ptr(bathy_host), _ptr(ws),
                                ws_bytes, _stream(stream), ctypes.byref(out)))
    return out.value


def swa_destroy_grid(h):
    return _chk(load().swa_destroy_grid(h))


def swa_set_state(h, eta, hu, hv, t, where, stream=None):
    return _chk(load().swa_set_state(h, _ptr(eta), _ptr(hu), _ptr(hv), float(t),
                                     where, _stream(stream)))


def swa_get_state(h, hh, hu, hv, eta, where, stream=None):
    return _chk(load().swa_get_state(h, _ptr(hh), _ptr(hu), _ptr(hv), _ptr(eta),
                                     where, _stream(stream)))


def swa_step_forward(h, max_steps, t_end, stream=None):
    return _chk(load().swa_step_forward(h, int(max_steps), float(t_end), _stream(stream)))


def swa_get_time(h, stream=None):
    t, dt, n = _D(), _D(), ctypes.c_longlong()
    _chk(load().swa_get_time(h, ctypes.byref(t), ctypes.byref(dt), ctypes.byref(n),
                             _stream(stream)))
    return t.value, dt.value, n.value


def swa_grid_set_strip_rows(h, rows):
    return _chk(load().swa_grid_set_strip_rows(h, int(rows)))


def swa_grid_set_rest_skip(h, on):
    return _chk(load().swa_grid_set_rest_skip(h, int(on)))


def swa_grid_set_scheme(h, scheme):
    return _chk(load().swa_grid_set_scheme(h, int(scheme)))


def swa_grid_set_wetdry(h, on):
    return _chk(load().swa_grid_set_wetdry(h, int(bool(on))))


def swa_grid_arrays(h, stream=None):
    a = [_V() for _ in range(4)]
    _chk(load().swa_grid_arrays(h, *[ctypes.byref(x) for x in a], _stream(stream)))
    return [x.value for x in a]


def swa_adjoint_workspace_bytes(desc):
    return int(load().swa_adjoint_workspace_bytes(ctypes.byref(desc)))


def swa_create_adjoint(desc, bathy_host, phi_host, t_f, ws, ws_bytes, stream=None):
    out = _V()
    _chk(load().swa_create_adjoint(ctypes.byref(desc), _ptr(bathy_host), _ptr(phi_host),
                                   float(t_f), _ptr(ws), ws_bytes, _stream(stream),
                                   ctypes.byref(out)))
    return out.value


def swa_destroy_adjoint(h):
    return _chk(load().swa_destroy_adjoint(h))


def swa_adjoint_info(h):
    n, dt, s = ctypes.c_longlong(), _D(), ctypes.c_longlong()
    _chk(load().swa_adjoint_info(h, ctypes.byref(n), ctypes.byref(dt), ctypes.byref(s)))
    return n.value, dt.value, s.value


def swa_step_adjoint(h, nsteps, stream=None):
    return _chk(load().swa_step_adjoint(h, int(nsteps), _stream(stream)))


def swa_adjoint_set_steps_per_pass(h, k):
    return _chk(load().swa_adjoint_set_steps_per_pass(h, int(k)))


def swa_get_adjoint_state(h, q, where, stream=None):
    return _chk(load().swa_get_adjoint_state(h, _ptr(q), where, _stream(stream)))


def swa_set_adjoint_state(h, phi, where, stream=None):
    return _chk(load().swa_set_adjoint_state(h, _ptr(phi), where, _stream(stream)))


def swa_snapstore_clear(h):
    return _chk(load().swa_snapstore_clear(h))


def swa_snapstore_workspace_bytes(adj_desc, max_snaps, precision):
    return int(load().swa_snapstore_workspace_bytes(ctypes.byref(adj_desc), int(max_snaps),
                                                    int(precision)))


def swa_create_snapstore(adj, max_snaps, precision, ws, ws_bytes):
    out = _V()
    _chk(load().swa_create_snapstore(adj, int(max_snaps), int(precision), _ptr(ws),
                                     ws_bytes, ctypes.byref(out)))
    return out.value


def swa_destroy_snapstore(h):
    return _chk(load().swa_destroy_snapstore(h))


def swa_store_snapshot(adj, store, stream=None):
    return _chk(load().swa_store_snapshot(adj, store, _stream(stream)))


def swa_run_adjoint(adj, store, every, stream=None):
    return _chk(load().swa_run_adjoint(adj, store, int(every), _stream(stream)))


def swa_snapstore_info(store, cap=0):
    cnt = _I()
    buf = np.zeros(max(cap, 1))
    _chk(load().swa_snapstore_info(store, ctypes.byref(cnt), buf.ctypes.data if cap else None,
                                   int(cap)))
    return cnt.value, buf[:min(cap, cnt.value)].copy()


def swa_flag_cells(grid, store, t_s, t_f, tol, mode, flags_dev, maxip_dev, count_dev,
                   stream=None):
    return _chk(load().swa_flag_cells(grid, store, float(t_s), float(t_f), float(tol),
                                      int(mode), _ptr(flags_dev), _ptr(maxip_dev),
                                      _ptr(count_dev), _stream(stream)))


def swa_flag_surface(grid, tol, flags_dev, count_dev, stream=None):
    return _chk(load().swa_flag_surface(grid, float(tol), _ptr(flags_dev), _ptr(count_dev),
                                        _stream(stream)))


def swa_gauge_sample(grid, n, xy_dev, eta_dev, stream=None):
    return _chk(load().swa_gauge_sample(grid, int(n), _ptr(xy_dev), _ptr(eta_dev),
                                        _stream(stream)))


def swa_grid_record_gauges(grid, n, xy_dev, series_dev, times_dev, capacity, stream=None):
    return _chk(load().swa_grid_record_gauges(grid, int(n), _ptr(xy_dev), _ptr(series_dev),
                                              _ptr(times_dev), int(capacity), _stream(stream)))


def swa_grid_mass(grid, mass_dev, stream=None):
    """FP64 mass audit of the grid's current state into a device double."""
    return _chk(load().swa_grid_mass(grid, _ptr(mass_dev), _stream(stream)))


def swa_grid_gauge_rows(grid, stream=None):
    r = ctypes.c_longlong()
    _chk(load().swa_grid_gauge_rows(grid, ctypes.byref(r), _stream(stream)))
    return int(r.value)


SWA_PROBE_FFMA64, SWA_PROBE_FFMA32, SWA_PROBE_FFMA32X2, SWA_PROBE_RSQRT32 = 0, 1, 2, 3


def swa_alu_probe_ops(kind, blocks, threads, iters):
    return load().swa_alu_probe_ops(int(kind), int(blocks), int(threads), int(iters))


def swa_alu_probe(kind, blocks, threads, iters, sink_dev, stream=None):
    return _chk(load().swa_alu_probe(int(kind), int(blocks), int(threads), int(iters),
                                     _ptr(sink_dev), _stream(stream)))


def measure_alu_peaks(device=0, iters=4096, reps=3):
    """Measured peaks on the current device, per second: FP64 and FP32 FMA
    flops, packed FP32x2 FMA flops, FP32 reciprocal square roots.  Each probe
    fills every SM (8 blocks of 256 threads per SM), best of `reps`."""
    import torch
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    blocks, threads = 8 * sms, 256
    sink = torch.zeros(blocks, dtype=torch.float32, device="cuda")
    out = {}
    names = {SWA_PROBE_FFMA64: "fp64_fma_flops", SWA_PROBE_FFMA32: "fp32_fma_flops",
             SWA_PROBE_FFMA32X2: "fp32x2_fma_flops", SWA_PROBE_RSQRT32: "fp32_rsqrt_ops"}
    s = torch.cuda.current_stream()
    for kind, name in names.items():
        it = iters // 8 if kind == SWA_PROBE_FFMA64 else iters
        swa_alu_probe(kind, blocks, threads, 16, sink, s)   # warm up
        best = None
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            swa_alu_probe(kind, blocks, threads, it, sink, s)
            e1.record(s)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        out[name] = swa_alu_probe_ops(kind, blocks, threads, it) / (best * 1e-3)
    return out


def swa_step_forward_static(desc, q_in, q_out, bath, dt, smax_out_dev=None, stream=None):
    """One forward step without any device allocation (scratch comes from a
    static array inside the library); q_in / q_out are 3 device buffers each
    (the third may be None in 1D)."""
    qi = (_V * 3)(*[_ptr(x) for x in q_in])
    qo = (_V * 3)(*[_ptr(x) for x in q_out])
    return _chk(load().swa_step_forward_static(ctypes.byref(desc), qi, qo, _ptr(bath),
                                               float(dt), _ptr(smax_out_dev),
                                               _stream(stream)))


def _patch_array(patches):
    arr = (swa_patch_desc * len(patches))()
    for k, p in enumerate(patches):
        lev, x0, y0, nx, ny, dx, dy = p
        arr[k].level, arr[k].nx, arr[k].ny = int(lev), int(nx), int(ny)
        arr[k].x_lo, arr[k].y_lo, arr[k].dx, arr[k].dy = float(x0), float(y0), float(dx), float(dy)
    return arr


def swa_patches_workspace_bytes(patches, common):
    arr = _patch_array(patches)
    return int(load().swa_patches_workspace_bytes(len(patches), ctypes.cast(arr, _V),
                                                  ctypes.byref(common)))


def swa_create_patches(patches, bathy_list, common, ws, ws_bytes, stream=None):
    arr = _patch_array(patches)
    bl = [np.ascontiguousarray(b, dtype=np.float64) for b in bathy_list]
    ptrs = (_V * len(bl))(*[b.ctypes.data for b in bl])
    out = _V()
    _chk(load().swa_create_patches(len(patches), ctypes.cast(arr, _V), ptrs,
                                   ctypes.byref(common), _ptr(ws), ws_bytes,
                                   _stream(stream), ctypes.byref(out)))
    return out.value


def swa_destroy_patches(h):
    return _chk(load().swa_destroy_patches(h))


def swa_patches_set_state(h, k, eta, hu, hv, where, stream=None):
    return _chk(load().swa_patches_set_state(h, int(k), _ptr(eta), _ptr(hu), _ptr(hv), where,
                                             _stream(stream)))


def swa_patches_start_level(h, level, t=0.0, stream=None):
    return _chk(load().swa_patches_start_level(h, int(level), float(t), _stream(stream)))


def swa_patches_get_state(h, k, hh, hu, hv, eta, where, stream=None):
    return _chk(load().swa_patches_get_state(h, int(k), _ptr(hh), _ptr(hu), _ptr(hv),
                                             _ptr(eta), where, _stream(stream)))


def swa_step_level(h, level, nsteps, t_end, stream=None):
    return _chk(load().swa_step_level(h, int(level), int(nsteps), float(t_end),
                                      _stream(stream)))


def swa_patches_get_time(h, level, stream=None):
    t, dt, n = _D(), _D(), ctypes.c_longlong()
    _chk(load().swa_patches_get_time(h, int(level), ctypes.byref(t), ctypes.byref(dt),
                                     ctypes.byref(n), _stream(stream)))
    return t.value, dt.value, n.value


def swa_patches_level_info(h, level):
    a, b, c = _I(), _I(), ctypes.c_longlong()
    _chk(load().swa_patches_level_info(h, int(level), ctypes.byref(a), ctypes.byref(b),
                                       ctypes.byref(c)))
    return a.value, b.value, c.value


def swa_patches_set_tile_rows(h, level, rows):
    return _chk(load().swa_patches_set_tile_rows(h, int(level), int(rows)))


# ------------------------------------------------- workspace-owning helpers
def _workspace(nbytes, device):
    import torch
    return torch.empty(int(nbytes), dtype=torch.uint8, device=device)


class Grid:
    """A forward grid whose workspace is a torch CUDA tensor."""

    def __init__(self, desc, B, device="cuda", stream=None):
        import torch
        self.desc = desc
        self.n = desc.nx * desc.ny
        self.nbytes = swa_grid_workspace_bytes(desc)
        if self.nbytes == 0:
            raise SwaError(SWA_EINVAL, swa_last_error())
        self.ws = _workspace(self.nbytes, device)
        B = np.ascontiguousarray(B, dtype=np.float64)
        self.h = swa_create_grid(desc, B, self.ws, self.nbytes, stream)
        self.device = torch.device(device)

    def set_state(self, eta, hu, hv=None, t=0.0, stream=None):
        if isinstance(eta, np.ndarray):
            arrs = [np.ascontiguousarray(a, dtype=np.float64) if a is not None else None
                    for a in (eta, hu, hv)]
            swa_set_state(self.h, arrs[0], arrs[1], arrs[2], t, SWA_HOST, stream)
        else:
            swa_set_state(self.h, eta, hu, hv, t, SWA_DEVICE, stream)

    def get_state(self, stream=None):
        out = [np.zeros(self.n) for _ in range(4)]
        swa_get_state(self.h, *out, SWA_HOST, stream)
        return dict(h=out[0], hu=out[1], hv=out[2], eta=out[3])

    def step(self, max_steps, t_end, stream=None):
        swa_step_forward(self.h, max_steps, t_end, stream)

    def set_scheme(self, scheme):
        swa_grid_set_scheme(self.h, scheme)

    def set_wetdry(self, on):
        swa_grid_set_wetdry(self.h, on)

    def time(self, stream=None):
        return swa_get_time(self.h, stream)

    def __del__(self):
        try:
            if getattr(self, "h", None):
                swa_destroy_grid(self.h)
                self.h = None
        except Exception:
            pass


class Adjoint:
    def __init__(self, desc, B, phi, t_f, device="cuda", stream=None):
        self.desc = desc
        self.n = desc.nx * desc.ny
        self.nc = desc.ndim + 1
        self.nbytes = swa_adjoint_workspace_bytes(desc)
        if self.nbytes == 0:
            raise SwaError(SWA_EINVAL, swa_last_error())
        self.ws = _workspace(self.nbytes, device)
        B = np.ascontiguousarray(B, dtype=np.float64)
        phi = np.ascontiguousarray(np.asarray(phi, dtype=np.float64).reshape(self.nc, self.n))
        self.h = swa_create_adjoint(desc, B, phi, t_f, self.ws, self.nbytes, stream)
        self.t_f = t_f

    def info(self):
        return swa_adjoint_info(self.h)

    def step(self, nsteps, stream=None):
        swa_step_adjoint(self.h, nsteps, stream)

    def get_state(self, stream=None):
        q = np.zeros((self.nc, self.n))
        swa_get_adjoint_state(self.h, q, SWA_HOST, stream)
        return q

    def __del__(self):
        try:
            if getattr(self, "h", None):
                swa_destroy_adjoint(self.h)
                self.h = None
        except Exception:
            pass


class SnapStore:
    def __init__(self, adj: Adjoint, max_snaps, precision, device="cuda"):
        self.adj = adj
        self.nbytes = swa_snapstore_workspace_bytes(adj.desc, max_snaps, precision)
        if self.nbytes == 0:
            raise SwaError(SWA_EINVAL, swa_last_error())
        self.ws = _workspace(self.nbytes, device)
        self.h = swa_create_snapstore(adj.h, max_snaps, precision, self.ws, self.nbytes)
        self.max_snaps = max_snaps

    def run_adjoint(self, every, stream=None):
        swa_run_adjoint(self.adj.h, self.h, every, stream)

    def store(self, stream=None):
        swa_store_snapshot(self.adj.h, self.h, stream)

    def info(self):
        return swa_snapstore_info(self.h, self.max_snaps)

    def __del__(self):
        try:
            if getattr(self, "h", None):
                swa_destroy_snapstore(self.h)
                self.h = None
        except Exception:
            pass


def swa_amr_workspace_bytes(coarse, fine, level, ratio):
    return int(load().swa_amr_workspace_bytes(coarse, fine, int(level), int(ratio)))


def swa_create_amr(coarse, fine, level, ratio, ws, ws_bytes, stream=None):
    out = _V()
    _chk(load().swa_create_amr(coarse, fine, int(level), int(ratio), _ptr(ws), int(ws_bytes),
                               _stream(stream), ctypes.byref(out)))
    return out


def swa_destroy_amr(h):
    return _chk(load().swa_destroy_amr(h))


def swa_amr_step(h, t_n, dt_c, max_launches=1, stream=None):
    return _chk(load().swa_amr_step(h, float(t_n), float(dt_c), int(max_launches),
                                    _stream(stream)))


def swa_amr_set_reflux(h, on):
    return _chk(load().swa_amr_set_reflux(h, int(bool(on))))


SWA_AMR_FILL_FUSED, SWA_AMR_FILL_KERNEL = 0, 1


def swa_amr_set_fill_mode(h, mode):
    return _chk(load().swa_amr_set_fill_mode(h, int(mode)))


def swa_amr_info(h, level=1):
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _chk(load().swa_amr_info(h, int(level), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def _ints(v):
    return (ctypes.c_int * len(v))(*[int(x) for x in v])


def swa_amr_levels_workspace_bytes(coarse, fine, levels, ratios):
    return int(load().swa_amr_levels_workspace_bytes(coarse, fine, len(levels), _ints(levels),
                                                     _ints(ratios)))


def swa_create_amr_levels(coarse, fine, levels, ratios, ws, ws_bytes, stream=None):
    out = _V()
    _chk(load().swa_create_amr_levels(coarse, fine, len(levels), _ints(levels), _ints(ratios),
                                      _ptr(ws), int(ws_bytes), _stream(stream),
                                      ctypes.byref(out)))
    return out


class PatchSet:
    """Batched patches; `patches` is a list of (level, x_lo, y_lo, nx, ny, dx, dy)."""

    def __init__(self, patches, bathy_list, common, device="cuda", stream=None):
        self.patches = list(patches)
        self.nbytes = swa_patches_workspace_bytes(self.patches, common)
        if self.nbytes == 0:
            raise SwaError(SWA_EINVAL, swa_last_error())
        self.ws = _workspace(self.nbytes, device)
        self.h = swa_create_patches(self.patches, bathy_list, common, self.ws, self.nbytes,
                                    stream)
        self.levels = sorted({p[0] for p in self.patches})

    def set_state(self, k, eta, hu, hv, stream=None):
        if isinstance(eta, np.ndarray):
            a = [np.ascontiguousarray(x, dtype=np.float64) for x in (eta, hu, hv)]
            swa_patches_set_state(self.h, k, *a, SWA_HOST, stream)
        else:
            swa_patches_set_state(self.h, k, eta, hu, hv, SWA_DEVICE, stream)

    def start(self, level, t=0.0, stream=None):
        swa_patches_start_level(self.h, level, t, stream)

    def step(self, level, nsteps, t_end=1e300, stream=None):
        swa_step_level(self.h, level, nsteps, t_end, stream)

    def get_state(self, k, stream=None):
        lev, x0, y0, nx, ny, dx, dy = self.patches[k]
        out = [np.zeros(nx * ny) for _ in range(4)]
        swa_patches_get_state(self.h, k, *out, SWA_HOST, stream)
        return dict(h=out[0], hu=out[1], hv=out[2], eta=out[3])

    def time(self, level, stream=None):
        return swa_patches_get_time(self.h, level, stream)

    def __del__(self):
        try:
            if getattr(self, "h", None):
                swa_destroy_patches(self.h)
                self.h = None
        except Exception:
            pass


class Amr:
    """AMR hierarchy over a Grid (coarse) and levels of a PatchSet (ringed
    patches): `level` and `ratio` are one patch-set level and its ratio (the
    two-level glue) or equal-length sequences, level 1 first; keeps both
    alive."""

    def __init__(self, grid, patchset, level, ratio, device="cuda", stream=None):
        self.grid, self.patchset = grid, patchset
        levels = list(level) if hasattr(level, "__len__") else [level]
        ratios = list(ratio) if hasattr(ratio, "__len__") else [ratio]
        self.levels, self.ratios = levels, ratios
        self.nbytes = swa_amr_levels_workspace_bytes(grid.h, patchset.h, levels, ratios)
        if self.nbytes == 0:
            raise SwaError(SWA_EINVAL, swa_last_error())
        self.ws = _workspace(self.nbytes, device)
        if len(levels) == 1:
            self.h = swa_create_amr(grid.h, patchset.h, levels[0], ratios[0], self.ws,
                                    self.nbytes, stream)
        else:
            self.h = swa_create_amr_levels(grid.h, patchset.h, levels, ratios, self.ws,
                                           self.nbytes, stream)

    def step(self, t_n, dt_c, max_launches=1, stream=None):
        swa_amr_step(self.h, t_n, dt_c, max_launches, stream)

    def set_reflux(self, on):
        swa_amr_set_reflux(self.h, on)

    def set_fill_mode(self, mode):
        swa_amr_set_fill_mode(self.h, mode)

    def info(self, level=1):
        """Hierarchy level `level`: (ring cells filled, covered parent cell
        copies, coarse-fine edges)."""
        return swa_amr_info(self.h, level)

    def __del__(self):
        try:
            if getattr(self, "h", None):
                swa_destroy_amr(self.h)
                self.h = None
        except Exception:
            pass
