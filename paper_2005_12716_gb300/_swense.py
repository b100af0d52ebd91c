"""ctypes binding of ``libswense.so`` (argument marshalling only).

Every ``swense_*`` name here calls the C entry point of the same name in ``include/swense.h``.
The functions accept torch CUDA tensors (their ``data_ptr()`` is passed), host numpy arrays for
the host-side level lists, and raise ``SwenseError`` on a non-zero status. No computation of
the method happens in Python; if the library is missing, ``load()`` raises.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None


class SwenseError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class swense_modes(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("depth", ctypes.c_double),
        ("n_snap", ctypes.c_int32),
        ("A_eta", ctypes.c_void_p), ("A_phi", ctypes.c_void_p), ("A_phit", ctypes.c_void_p),
        ("omega", ctypes.c_void_p), ("t_ref", ctypes.c_double),
    ]


class swense_grid_desc(ctypes.Structure):
    _fields_ = [("pad_n", ctypes.c_int32), ("nz", ctypes.c_int32), ("z_levels", ctypes.c_void_p),
                ("scheme", ctypes.c_int32)]


STREAM_MAX_N = 32


class swense_stream_wave(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("k", ctypes.c_double), ("c", ctypes.c_double),
                ("ubar", ctypes.c_double), ("Q", ctypes.c_double), ("R", ctypes.c_double),
                ("depth", ctypes.c_double), ("g", ctypes.c_double), ("period", ctypes.c_double),
                ("height", ctypes.c_double), ("B", ctypes.c_double * STREAM_MAX_N),
                ("E", ctypes.c_double * (STREAM_MAX_N + 1)),
                ("eta_m", ctypes.c_double * (STREAM_MAX_N + 1))]


class swense_relax_zone(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("inner", ctypes.c_float), ("outer", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float)]


ZONE_X, ZONE_Y, ZONE_RADIAL = 0, 1, 2
MAX_ZONES = 8


class swense_grid(ctypes.Structure):
    _fields_ = [
        ("nodes", ctypes.c_void_p), ("eta", ctypes.c_void_p),
        ("nx_r", ctypes.c_int32), ("ny_r", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("n_tl", ctypes.c_int32),
        ("Lx", ctypes.c_double), ("Ly", ctypes.c_double),
        ("z_levels", ctypes.c_void_p), ("t_levels", ctypes.c_void_p),
        ("scheme", ctypes.c_int32),
    ]


LAGRANGE3, SPLINE3 = 0, 1
SCHEMES = {"lagrange3": LAGRANGE3, "spline3": SPLINE3}
P_DYN, P_PHIT, P_TOTAL = 0, 1, 2
P_MODES = {"dyn": P_DYN, "phit": P_PHIT, "total": P_TOTAL}
MAX_LEVELS, MAX_FFT, MAX_TL = 256, 8192, 4

# C symbol -> (restype, argtypes)
_SIGS = {
    "swense_fields_on_grid": (ctypes.c_int, [ctypes.POINTER(swense_modes), ctypes.c_int32,
                                             ctypes.c_void_p, ctypes.POINTER(swense_grid_desc),
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "swense_fields_on_grid_noalloc": (ctypes.c_int, [ctypes.POINTER(swense_modes), ctypes.c_int32,
                                                     ctypes.c_void_p,
                                                     ctypes.POINTER(swense_grid_desc),
                                                     ctypes.c_void_p, ctypes.c_void_p,
                                                     ctypes.c_void_p]),
    "swense_interp": (ctypes.c_int, [ctypes.POINTER(swense_grid), ctypes.c_double, ctypes.c_void_p,
                                     ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_void_p, ctypes.c_void_p]),
    "swense_direct": (ctypes.c_int, [ctypes.POINTER(swense_modes), ctypes.c_double, ctypes.c_void_p,
                                     ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int32, ctypes.c_void_p]),
    "swense_fv_divergence": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                            ctypes.c_void_p]),
    "swense_relax_cells": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_int64, ctypes.c_void_p, ctypes.c_int32,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p]),
    "swense_stream_solve": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.POINTER(swense_stream_wave)]),
    "swense_stream_eval": (ctypes.c_int, [ctypes.POINTER(swense_stream_wave), ctypes.c_double,
                                          ctypes.c_double, ctypes.c_void_p, ctypes.c_int64,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                          ctypes.c_double, ctypes.c_void_p]),
    "swense_tank_modes": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.POINTER(swense_modes), ctypes.c_void_p]),
    "swense_workspace_bytes": (ctypes.c_int64, []),
    "swense_release": (ctypes.c_int, []),
    "swense_last_error": (ctypes.c_char_p, []),
    "swense_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "swense_version": (ctypes.c_int, []),
    "swense_launches": (ctypes.c_int64, []),
    "swense_async_status": (ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p]),
    "swense_selftest_wait_timeout": (ctypes.c_int, [ctypes.c_void_p]),
    "swense_selftest_direct_wait_timeout": (ctypes.c_int, [ctypes.c_int32]),
    "swense_direct_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "swense_selftest_tc_gemm": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                               ctypes.c_void_p]),
}


def lib_path():
    return _build.LIB


def load(build_if_missing=False):
    """Load (and optionally build) the library; raises if it cannot be loaded."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def exported_symbols():
    return list(_SIGS)


def _check(status):
    if status != 0:
        lib = load()
        raise SwenseError(status, lib.swense_last_error().decode())


def _ptr(t):
    if t is None or isinstance(t, int):
        return t
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def make_modes(nx, ny, Lx, Ly, depth, A_eta, A_phi, A_phit, n_snap=1, omega=None, t_ref=0.0):
    """swense_modes from device tensors (complex64 viewed as float pairs, float64 omega)."""
    m = swense_modes(nx, ny, Lx, Ly, depth, n_snap, _ptr(A_eta), _ptr(A_phi), _ptr(A_phit),
                     _ptr(omega), t_ref)
    m._keep = (A_eta, A_phi, A_phit, omega)
    return m


def make_grid_desc(pad_n, z_levels, scheme=LAGRANGE3):
    z = np.ascontiguousarray(z_levels, np.float32)
    d = swense_grid_desc(pad_n, len(z), z.ctypes.data, scheme)
    d._keep = z
    return d


def make_grid(nodes, eta, nx_r, ny_r, nz, n_tl, Lx, Ly, z_levels, t_levels, scheme=LAGRANGE3):
    z = np.ascontiguousarray(z_levels, np.float32)
    t = np.ascontiguousarray(t_levels, np.float64)
    g = swense_grid(_ptr(nodes), _ptr(eta), nx_r, ny_r, nz, n_tl, Lx, Ly, z.ctypes.data,
                    t.ctypes.data, scheme)
    g._keep = (nodes, eta, z, t)
    return g


def swense_fields_on_grid(modes, n_tl, t, desc, nodes, eta, stream=None):
    lib = load()
    tt = None if t is None else np.ascontiguousarray(t, np.float64)
    _check(lib.swense_fields_on_grid(ctypes.byref(modes), n_tl,
                                     None if tt is None else tt.ctypes.data,
                                     ctypes.byref(desc), _ptr(nodes), _ptr(eta), _stream(stream)))


def swense_fields_on_grid_noalloc(modes, n_tl, t, desc, nodes, eta, stream=None):
    lib = load()
    tt = None if t is None else np.ascontiguousarray(t, np.float64)
    _check(lib.swense_fields_on_grid_noalloc(ctypes.byref(modes), n_tl,
                                             None if tt is None else tt.ctypes.data,
                                             ctypes.byref(desc), _ptr(nodes), _ptr(eta),
                                             _stream(stream)))


def swense_interp(grid, t, pts, np_, eta=None, u=None, v=None, w=None, p=None, p_mode=P_DYN,
                  rho=1000.0, g=9.81, count_out_of_range=False, stream=None):
    lib = load()
    cnt = ctypes.c_int64(-1)
    _check(lib.swense_interp(ctypes.byref(grid), t, _ptr(pts), np_, _ptr(eta), _ptr(u), _ptr(v),
                             _ptr(w), _ptr(p), p_mode, rho, g,
                             ctypes.byref(cnt) if count_out_of_range else None, _stream(stream)))
    return cnt.value if count_out_of_range else None


_SIGS.update({
    "swense_interp_plan_bytes": (ctypes.c_int64, [ctypes.c_int64]),
    "swense_interp_plan": (ctypes.c_int, [ctypes.POINTER(swense_grid), ctypes.c_void_p, ctypes.c_int64,
                                          ctypes.c_void_p, ctypes.c_void_p]),
    "swense_interp_with_plan": (ctypes.c_int, [ctypes.POINTER(swense_grid), ctypes.c_double,
                                               ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                               ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                                               ctypes.c_void_p]),
})


def swense_interp_plan_bytes(np_):
    return int(load().swense_interp_plan_bytes(np_))


def swense_interp_plan(grid, pts, np_, plan, stream=None):
    _check(load().swense_interp_plan(ctypes.byref(grid), _ptr(pts), np_, _ptr(plan), _stream(stream)))


def swense_interp_with_plan(grid, t, pts, np_, plan, eta=None, u=None, v=None, w=None, p=None,
                            p_mode=P_DYN, rho=1000.0, g=9.81, count_out_of_range=False, stream=None):
    cnt = ctypes.c_int64(-1)
    _check(load().swense_interp_with_plan(ctypes.byref(grid), t, _ptr(pts), np_, _ptr(plan), _ptr(eta),
                                          _ptr(u), _ptr(v), _ptr(w), _ptr(p), p_mode, rho, g,
                                          ctypes.byref(cnt) if count_out_of_range else None,
                                          _stream(stream)))
    return cnt.value if count_out_of_range else None


DIRECT_FP32, DIRECT_SPLIT_BF16, DIRECT_SPLIT_BF16_PAIRWISE = 0, 1, 2


def swense_direct(modes, t, pts, np_, eta=None, u=None, v=None, w=None, p=None, p_mode=P_DYN,
                  rho=1000.0, g=9.81, precision=DIRECT_FP32, stream=None):
    lib = load()
    _check(lib.swense_direct(ctypes.byref(modes), t, _ptr(pts), np_, _ptr(eta), _ptr(u), _ptr(v),
                             _ptr(w), _ptr(p), p_mode, rho, g, precision, _stream(stream)))


def swense_fv_divergence(u_face, v_face, w_face, n_faces, area, cell_faces, cell_volume, n_cells,
                         div, stream=None):
    lib = load()
    _check(lib.swense_fv_divergence(_ptr(u_face), _ptr(v_face), _ptr(w_face), n_faces, _ptr(area),
                                    _ptr(cell_faces), _ptr(cell_volume), n_cells, _ptr(div),
                                    _stream(stream)))


def swense_relax_cells(cell_xyz, cell_zext, eta_c, nc, zones, alpha_i=None, alpha=None, u_c=None,
                       weight=None, stream=None):
    """zones: sequence of (kind, inner, outer, cx, cy)."""
    lib = load()
    arr = (swense_relax_zone * max(1, len(zones)))(*[swense_relax_zone(*z) for z in zones])
    _check(lib.swense_relax_cells(_ptr(cell_xyz), _ptr(cell_zext), _ptr(eta_c), nc,
                                  ctypes.cast(arr, ctypes.c_void_p) if zones else None, len(zones),
                                  _ptr(alpha_i), _ptr(alpha), _ptr(u_c), _ptr(weight),
                                  _stream(stream)))


def swense_stream_solve(period, height, depth, g=9.81, n=9, height_steps=4):
    """Host-only solve; returns a swense_stream_wave."""
    w = swense_stream_wave()
    _check(load().swense_stream_solve(period, height, depth, g, n, height_steps, ctypes.byref(w)))
    return w


def swense_stream_eval(wave, t, x0, pts, np_, eta=None, u=None, v=None, w=None, p=None,
                       p_mode=P_DYN, rho=1000.0, stream=None):
    _check(load().swense_stream_eval(ctypes.byref(wave), t, x0, _ptr(pts), np_, _ptr(eta), _ptr(u),
                                     _ptr(v), _ptr(w), _ptr(p), p_mode, rho, _stream(stream)))


def swense_tank_modes(A_eta, A_phi, A_phit, nx_t, ny_t, n_snap, Lx, Ly, depth, out_eta, out_phi,
                      out_phit, stream=None):
    """Returns the swense_modes struct the library filled (pointing at the three outputs)."""
    m = swense_modes()
    _check(load().swense_tank_modes(_ptr(A_eta), _ptr(A_phi), _ptr(A_phit), nx_t, ny_t, n_snap, Lx,
                                    Ly, depth, _ptr(out_eta), _ptr(out_phi), _ptr(out_phit),
                                    ctypes.byref(m), _stream(stream)))
    return m


def swense_workspace_bytes():
    return load().swense_workspace_bytes()


def swense_release():
    _check(load().swense_release())


def swense_strerror(status):
    return load().swense_strerror(status).decode()


def swense_version():
    return load().swense_version()


def swense_launches():
    return load().swense_launches()


def swense_async_status(reset=True, stream=None, raise_on_error=True):
    """Status of the bounded device-side waits since the last reset (synchronises the stream):
    0, or SWENSE_ERR_TIMEOUT (-6) raised as SwenseError unless raise_on_error is False."""
    st = load().swense_async_status(1 if reset else 0, _stream(stream))
    if raise_on_error:
        _check(st)
    return st


def swense_selftest_wait_timeout(stream=None):
    _check(load().swense_selftest_wait_timeout(_stream(stream)))


def swense_selftest_direct_wait_timeout(on):
    _check(load().swense_selftest_direct_wait_timeout(1 if on else 0))


def swense_direct_stats(stream=None):
    """(tiles, fallback_tiles) of the last tensor-core direct sum on the current device."""
    t, f = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(load().swense_direct_stats(ctypes.byref(t), ctypes.byref(f), _stream(stream)))
    return t.value, f.value


def swense_selftest_tc_gemm(A, B, D, N, K, variant=0, stream=None):
    _check(load().swense_selftest_tc_gemm(_ptr(A), _ptr(B), _ptr(D), N, K, variant, _stream(stream)))


# ------------------------------------------------------------------ learned correction (MLP)
MLP_NPARAM, MLP_PACKED_BYTES, MLP_XLD = 8772, 32768, 68

_SIGS.update({
    "swense_mlp_pack": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_float, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    "swense_mlp_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                          ctypes.c_void_p, ctypes.c_void_p]),
    "swense_mlp_features": (ctypes.c_int, [ctypes.POINTER(swense_grid), ctypes.c_double,
                                           ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p]),
    "swense_mlp_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "swense_mlp_train_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_int32, ctypes.c_float, ctypes.c_float,
                                             ctypes.c_float, ctypes.c_float, ctypes.c_void_p,
                                             ctypes.c_void_p]),
    "swense_interp_learned": (ctypes.c_int, [ctypes.POINTER(swense_grid), ctypes.c_double,
                                             ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_int32, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p]),
})


class swense_mlp(ctypes.Structure):
    _fields_ = [("params", ctypes.c_void_p), ("adam_m", ctypes.c_void_p), ("adam_v", ctypes.c_void_p),
                ("packed", ctypes.c_void_p), ("step", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("out_scale", ctypes.c_float)]


_SIGS.update({
    "swense_mlp_targets": (ctypes.c_int, [ctypes.c_void_p] * 6 + [ctypes.c_int64, ctypes.c_void_p,
                                                                  ctypes.c_void_p, ctypes.c_void_p]),
    "swense_mlp_train": (ctypes.c_int, [ctypes.POINTER(swense_mlp), ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_float, ctypes.c_int64, ctypes.c_float, ctypes.c_float,
                                        ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p]),
    "swense_mlp_save": (ctypes.c_int, [ctypes.POINTER(swense_mlp), ctypes.c_char_p, ctypes.c_void_p]),
    "swense_mlp_load": (ctypes.c_int, [ctypes.POINTER(swense_mlp), ctypes.c_char_p, ctypes.c_void_p]),
})


def make_mlp(params, adam_m, adam_v, packed, step=0, seed=0, out_scale=0.0):
    m = swense_mlp(_ptr(params), _ptr(adam_m), _ptr(adam_v), _ptr(packed), step, seed, out_scale)
    m._keep = (params, adam_m, adam_v, packed)
    return m


def swense_mlp_targets(eu, ev, ew, et, lagrange, scale, np_, target, field, stream=None):
    _check(load().swense_mlp_targets(_ptr(eu), _ptr(ev), _ptr(ew), _ptr(et), _ptr(lagrange),
                                     _ptr(scale), np_, _ptr(target), _ptr(field), _stream(stream)))


def swense_mlp_train(mlp, x, field, target, n_rows, steps, B, lr, schedule_steps=0, beta1=0.9,
                     beta2=0.999, eps=1e-8, losses=None, stream=None):
    """mlp: a swense_mlp struct (its step / out_scale are updated in place)."""
    _check(load().swense_mlp_train(ctypes.byref(mlp), _ptr(x), _ptr(field), _ptr(target), n_rows,
                                   steps, B, lr, schedule_steps, beta1, beta2, eps, _ptr(losses),
                                   _stream(stream)))


def swense_mlp_save(mlp, path, stream=None):
    _check(load().swense_mlp_save(ctypes.byref(mlp), os.fsencode(path), _stream(stream)))


def swense_mlp_load(mlp, path, stream=None):
    _check(load().swense_mlp_load(ctypes.byref(mlp), os.fsencode(path), _stream(stream)))


def swense_mlp_pack(params, out_scale, packed, stream=None):
    _check(load().swense_mlp_pack(_ptr(params), out_scale, _ptr(packed), _stream(stream)))


def swense_mlp_forward(packed, x, rows, y, stream=None):
    _check(load().swense_mlp_forward(_ptr(packed), _ptr(x), rows, _ptr(y), _stream(stream)))


def swense_mlp_features(grid, t, pts, np_, x, scale, lagrange, eta=None, stream=None):
    _check(load().swense_mlp_features(ctypes.byref(grid), t, _ptr(pts), np_, _ptr(x), _ptr(scale),
                                      _ptr(lagrange), _ptr(eta), _stream(stream)))


def swense_mlp_grad(packed, x, field, target, batch, B, grad, loss=None, stream=None):
    _check(load().swense_mlp_grad(_ptr(packed), _ptr(x), _ptr(field), _ptr(target), _ptr(batch), B,
                                  _ptr(grad), _ptr(loss), _stream(stream)))


def swense_mlp_train_step(params, adam_m, adam_v, packed, step, x, field, target, batch, B, lr,
                          beta1=0.9, beta2=0.999, eps=1e-8, loss=None, stream=None):
    _check(load().swense_mlp_train_step(_ptr(params), _ptr(adam_m), _ptr(adam_v), _ptr(packed),
                                        step, _ptr(x), _ptr(field), _ptr(target), _ptr(batch), B,
                                        lr, beta1, beta2, eps, _ptr(loss), _stream(stream)))


def swense_interp_learned(grid, t, pts, np_, packed, eta=None, u=None, v=None, w=None, p=None,
                          p_mode=P_DYN, rho=1000.0, g=9.81, count_out_of_range=False,
                          stream=None):
    lib = load()
    cnt = ctypes.c_int64(-1)
    _check(lib.swense_interp_learned(ctypes.byref(grid), t, _ptr(pts), np_, _ptr(eta), _ptr(u),
                                     _ptr(v), _ptr(w), _ptr(p), p_mode, rho, g, _ptr(packed),
                                     ctypes.byref(cnt) if count_out_of_range else None,
                                     _stream(stream)))
    return cnt.value if count_out_of_range else None


# ------------------------------------------------------------------ point binning
_SIGS.update({
    "swense_bin_points": (ctypes.c_int, [ctypes.POINTER(swense_grid), ctypes.c_void_p,
                                         ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p]),
    "swense_interp_permuted": (ctypes.c_int, [ctypes.POINTER(swense_grid), ctypes.c_double,
                                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                              ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                                              ctypes.c_void_p]),
})


def swense_bin_points(grid, pts, np_, perm, pts_sorted, stream=None):
    _check(load().swense_bin_points(ctypes.byref(grid), _ptr(pts), np_, _ptr(perm),
                                    _ptr(pts_sorted), _stream(stream)))


def swense_interp_permuted(grid, t, pts_sorted, perm, np_, eta=None, u=None, v=None, w=None,
                           p=None, p_mode=P_DYN, rho=1000.0, g=9.81, count_out_of_range=False,
                           stream=None):
    lib = load()
    cnt = ctypes.c_int64(-1)
    _check(lib.swense_interp_permuted(ctypes.byref(grid), t, _ptr(pts_sorted), _ptr(perm), np_,
                                      _ptr(eta), _ptr(u), _ptr(v), _ptr(w), _ptr(p), p_mode, rho,
                                      g, ctypes.byref(cnt) if count_out_of_range else None,
                                      _stream(stream)))
    return cnt.value if count_out_of_range else None


# ------------------------------------------------------------------ batches and autotuning
class swense_instance(ctypes.Structure):
    _fields_ = [
        ("modes", swense_modes), ("desc", swense_grid_desc), ("n_tl", ctypes.c_int32),
        ("t_levels", ctypes.c_void_p), ("nodes", ctypes.c_void_p), ("eta", ctypes.c_void_p),
        ("pts", ctypes.c_void_p), ("perm", ctypes.c_void_p), ("np", ctypes.c_int64),
        ("t", ctypes.c_double), ("out_eta", ctypes.c_void_p), ("out_u", ctypes.c_void_p),
        ("out_v", ctypes.c_void_p), ("out_w", ctypes.c_void_p), ("out_p", ctypes.c_void_p),
    ]


_SIGS.update({
    "swense_batch_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_void_p]),
    "swense_autotune_grid": (ctypes.c_int, [ctypes.POINTER(swense_modes), ctypes.c_int32,
                                            ctypes.c_void_p, ctypes.POINTER(swense_grid_desc),
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
})


_SIGS["swense_set_grid_tune"] = (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                                ctypes.c_int32])


def swense_set_grid_tune(nx, ny, pad_n, nz, lpc=-1, chunk_bytes=32 << 20, row_variant=0):
    _check(load().swense_set_grid_tune(nx, ny, pad_n, nz, lpc, chunk_bytes, row_variant))


def swense_batch_run(instances, p_mode=P_DYN, rho=1000.0, g=9.81, stream=None):
    """instances: a ctypes array of swense_instance (kept alive by the caller)."""
    _check(load().swense_batch_run(ctypes.addressof(instances), len(instances), p_mode, rho, g,
                                   _stream(stream)))


def swense_autotune_grid(modes, n_tl, t, desc, nodes, eta, stream=None):
    """Returns (levels per column block (0: shared-memory path), chunk bytes, row variant)."""
    lpc = ctypes.c_int32(0)
    chunk = ctypes.c_int64(0)
    rowv = ctypes.c_int32(0)
    tt = None if t is None else np.ascontiguousarray(t, np.float64)
    _check(load().swense_autotune_grid(ctypes.byref(modes), n_tl,
                                       None if tt is None else tt.ctypes.data,
                                       ctypes.byref(desc), _ptr(nodes), _ptr(eta),
                                       ctypes.byref(lpc), ctypes.byref(chunk), ctypes.byref(rowv),
                                       _stream(stream)))
    return lpc.value, chunk.value, rowv.value
