"""ctypes binding of the C ABI in include/claw.h (argument marshalling only).

Every numerical step runs in the CUDA library ``_build/libclaw.so``; this
module converts Python arguments (numpy arrays, torch CUDA tensors, enums
given as strings) into the C calls and raises ``ClawError`` on any non-OK
status.  There is no fallback: if the library cannot be built or loaded, the
first call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

CLAW_OK, CLAW_EINVAL, CLAW_ENOMEM, CLAW_ECUDA, CLAW_ECFL, CLAW_ENONPHYS, CLAW_ETIMEOUT, CLAW_EBOUNDS = range(8)
STATUS_NAMES = {0: "CLAW_OK", 1: "CLAW_EINVAL", 2: "CLAW_ENOMEM", 3: "CLAW_ECUDA", 4: "CLAW_ECFL",
                5: "CLAW_ENONPHYS", 6: "CLAW_ETIMEOUT", 7: "CLAW_EBOUNDS"}
SYSTEMS = {"acoustics": 0, "acoustics_var": 1, "shallow_water": 2, "shallow_water_bathy": 3,
           "shallow_water_dry": 4}
LIMITERS = {"none": 0, "minmod": 1, "mc": 2, "first_order": 3}
BCS = {"periodic": 0, "extrap": 1, "wall": 2}


class ClawError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")


class claw_grid(C.Structure):
    _fields_ = [("ndim", C.c_int), ("n", C.c_int * 3), ("dx", C.c_double * 3)]


class claw_params(C.Structure):
    _fields_ = [("rho", C.c_double), ("K", C.c_double), ("g", C.c_double),
                ("cfl_desired", C.c_double), ("cfl_max", C.c_double), ("dt_max", C.c_double),
                ("precision", C.c_int), ("max_retries", C.c_int), ("splitting", C.c_int),
                ("dry_tol", C.c_double)]


_vp = C.c_void_p
_dp = C.POINTER(C.c_double)
_SIGS = {
    "claw_create": [C.POINTER(claw_grid), C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int),
                    C.POINTER(claw_params), _vp, C.POINTER(_vp)],
    "claw_destroy": [_vp],
    "claw_set_q": [_vp, _vp, C.c_int],
    "claw_get_q": [_vp, _vp, C.c_int],
    "claw_set_aux": [_vp, _vp, _vp, C.c_int],
    "claw_set_bathymetry": [_vp, _vp, C.c_int],
    "claw_step": [_vp, C.c_double, _dp],
    "claw_advance": [_vp, C.c_double, C.c_double, C.POINTER(C.c_int)],
    "claw_run_steps": [_vp, C.c_int],
    "claw_max_speed": [_vp, _dp],
    "claw_get_time": [_vp, _dp, _dp, C.POINTER(C.c_long)],
    "claw_set_time": [_vp, C.c_double, C.c_double, C.c_long],
    "claw_conservation_sums": [_vp, _dp],
    "claw_get_rejections": [_vp, C.POINTER(C.c_long)],
    "claw_run_fixed_steps": [_vp, C.c_int, C.c_double, _dp],
    "claw_checkpoint": [_vp],
    "claw_rollback": [_vp],
    "claw_get_rows": [_vp, C.c_int, C.c_int, _vp, C.c_int],
    "claw_set_rows": [_vp, C.c_int, C.c_int, _vp, C.c_int],
    "claw_last_error": [],
    "claw_ensemble_create": [C.c_int, C.POINTER(claw_grid), C.c_int, C.c_int, C.POINTER(C.c_int),
                             C.POINTER(claw_params), _vp, C.POINTER(_vp)],
    "claw_ensemble_set_q": [_vp, C.c_int, _vp, C.c_int],
    "claw_ensemble_get_q": [_vp, C.c_int, _vp, C.c_int],
    "claw_ensemble_set_aux": [_vp, C.c_int, _vp, _vp, C.c_int],
    "claw_ensemble_set_bathymetry": [_vp, C.c_int, _vp, C.c_int],
    "claw_ensemble_run_steps": [_vp, C.c_int],
    "claw_ensemble_get_time": [_vp, C.c_int, _dp, _dp, C.POINTER(C.c_long)],
    "claw_ensemble_size": [_vp],
    "claw_profile_steps": [_vp, C.c_int, _dp, _dp, C.POINTER(C.c_long)],
    "claw_set_segment": [_vp, C.c_int, C.c_int],
    "claw_set_tile_shape": [_vp, C.c_int, C.c_int, C.c_int, C.c_int],
    "claw_get_tile_shape": [_vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)],
    "claw_autotune": [_vp, C.c_int, C.POINTER(C.c_int)],
    "claw_probe_fma": [C.c_int, _dp, _vp],
    "claw_max_speed_noalloc": [C.POINTER(claw_grid), C.c_int, C.POINTER(C.c_int),
                               C.POINTER(claw_params), _vp, _vp, _vp, _vp, _vp],
}

_lib = None
_lock = threading.Lock()


def debug_build() -> bool:
    """CLAW_DEBUG=1 in the environment selects the checked library (bounds
    checks of the kernels' global accesses, reported as CLAW_EBOUNDS)."""
    return os.environ.get("CLAW_DEBUG", "") == "1"


def library_path() -> str:
    return _build.LIB_DEBUG if debug_build() else _build.LIB


def lib():
    """Load (building first if the sources are newer) the CUDA library."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build(debug=debug_build())
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library missing: {path}")
            L = C.CDLL(path)
            for name, args in _SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = C.c_int
            L.claw_last_error.restype = C.c_char_p
            L.claw_destroy.restype = None
            _lib = L
    return _lib


def _check(st: int, where: str):
    if st != CLAW_OK:
        raise ClawError(st, where, lib().claw_last_error().decode())


def _array_arg(q, dtype=np.float64):
    """(pointer, on_device, keepalive) for a numpy array or a torch tensor."""
    mod = type(q).__module__
    if mod.startswith("torch"):
        import torch
        if q.dtype != torch.float64:
            raise TypeError("state tensors must be float64")
        if not q.is_contiguous():
            raise ValueError("state tensors must be contiguous")
        return C.c_void_p(q.data_ptr()), int(q.is_cuda), q
    a = np.ascontiguousarray(q, dtype=dtype)
    return C.c_void_p(a.ctypes.data), 0, a


def _stream_arg(stream):
    if stream is None:
        return None
    if stream == "torch":
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


SPLITTINGS = {"godunov": 0, "strang": 1, "unsplit": 2}


def make_params(rho=1.0, K=1.0, g=9.81, cfl_desired=0.9, cfl_max=1.0, dt_max=1e9, precision=64,
                max_retries=8, splitting="godunov", dry_tol=1e-3) -> claw_params:
    sp = SPLITTINGS[splitting] if isinstance(splitting, str) else int(splitting)
    return claw_params(float(rho), float(K), float(g), float(cfl_desired), float(cfl_max),
                       float(dt_max), int(precision), int(max_retries), sp, float(dry_tol))


def make_grid(n, dx) -> claw_grid:
    g = claw_grid()
    g.ndim = len(n)
    for d in range(3):
        g.n[d] = int(n[d]) if d < len(n) else 1
        g.dx[d] = float(dx[d]) if d < len(dx) else 1.0
    return g


def make_bc(bc, ndim):
    if isinstance(bc, str):
        bc = [bc] * (2 * ndim)
    arr = (C.c_int * 6)(*([BCS[b] if isinstance(b, str) else int(b) for b in bc]
                          + [1] * (6 - len(bc))))
    return arr


# ----------------------------------------------------------------- C names

def claw_create(n, dx, m, mwaves, system, limiter, bc, params, stream=None):
    out = _vp()
    g = make_grid(n, dx)
    sysc = SYSTEMS[system] if isinstance(system, str) else int(system)
    limc = LIMITERS[limiter] if isinstance(limiter, str) else int(limiter)
    _check(lib().claw_create(C.byref(g), int(m), int(mwaves), sysc, limc, make_bc(bc, len(n)),
                             C.byref(params), _stream_arg(stream), C.byref(out)), "claw_create")
    return out


def claw_ensemble_create(grids, system, limiter, bc, params, stream=None):
    B = len(grids)
    arr = (claw_grid * max(B, 1))()
    for i, (n, dx) in enumerate(grids):
        arr[i] = make_grid(n, dx)
    out = _vp()
    sysc = SYSTEMS[system] if isinstance(system, str) else int(system)
    limc = LIMITERS[limiter] if isinstance(limiter, str) else int(limiter)
    ndim = len(grids[0][0]) if B else 2
    _check(lib().claw_ensemble_create(B, arr, sysc, limc, make_bc(bc, ndim), C.byref(params),
                                      _stream_arg(stream), C.byref(out)), "claw_ensemble_create")
    return out


def claw_destroy(h):
    if h:
        lib().claw_destroy(h)


def claw_set_q(h, q):
    p, dev, keep = _array_arg(q)
    _check(lib().claw_set_q(h, p, dev), "claw_set_q")


def claw_run_fixed_steps(h, nsteps, dt):
    cfl = C.c_double(0.0)
    _check(lib().claw_run_fixed_steps(h, int(nsteps), float(dt), C.byref(cfl)), "claw_run_fixed_steps")
    return cfl.value


def claw_checkpoint(h):
    _check(lib().claw_checkpoint(h), "claw_checkpoint")


def claw_rollback(h):
    _check(lib().claw_rollback(h), "claw_rollback")


def claw_get_rows(h, y0, out):
    """Rows y0 .. y0 + out.shape[1] - 1 into `out` (m, nrows, nx)."""
    p, dev, keep = _array_arg(out)
    if not dev and keep is not out:
        raise ValueError("host output must be a contiguous float64 numpy array")
    _check(lib().claw_get_rows(h, int(y0), int(out.shape[1]), p, dev), "claw_get_rows")
    return out


def claw_set_rows(h, y0, rows):
    p, dev, keep = _array_arg(rows)
    _check(lib().claw_set_rows(h, int(y0), int(rows.shape[1]), p, dev), "claw_set_rows")


def claw_get_q(h, out):
    p, dev, keep = _array_arg(out)
    if not dev and keep is not out:
        raise ValueError("host output must be a contiguous float64 numpy array")
    _check(lib().claw_get_q(h, p, dev), "claw_get_q")
    return out


def claw_set_aux(h, rho, K):
    pr, dr, kr = _array_arg(rho)
    pk, dk, kk = _array_arg(K)
    _check(lib().claw_set_aux(h, pr, pk, dr), "claw_set_aux")


def claw_set_bathymetry(h, B):
    pb, db, kb = _array_arg(B)
    _check(lib().claw_set_bathymetry(h, pb, db), "claw_set_bathymetry")


def claw_step(h, dt=0.0):
    cfl = C.c_double(0.0)
    _check(lib().claw_step(h, float(dt), C.byref(cfl)), "claw_step")
    return cfl.value


def claw_advance(h, t_final, cfl_target=0.0):
    n = C.c_int(0)
    _check(lib().claw_advance(h, float(t_final), float(cfl_target), C.byref(n)), "claw_advance")
    return n.value


def claw_run_steps(h, nsteps):
    _check(lib().claw_run_steps(h, int(nsteps)), "claw_run_steps")


def claw_max_speed(h):
    v = C.c_double(0.0)
    _check(lib().claw_max_speed(h, C.byref(v)), "claw_max_speed")
    return v.value


def claw_get_time(h):
    t, dt, n = C.c_double(), C.c_double(), C.c_long()
    _check(lib().claw_get_time(h, C.byref(t), C.byref(dt), C.byref(n)), "claw_get_time")
    return t.value, dt.value, n.value


def claw_set_time(h, t, dt, nsteps):
    _check(lib().claw_set_time(h, float(t), float(dt), int(nsteps)), "claw_set_time")


def claw_conservation_sums(h, m):
    out = np.zeros(m)
    _check(lib().claw_conservation_sums(h, out.ctypes.data_as(_dp)), "claw_conservation_sums")
    return out


def claw_get_rejections(h):
    n = C.c_long()
    _check(lib().claw_get_rejections(h, C.byref(n)), "claw_get_rejections")
    return n.value


def claw_ensemble_set_q(h, i, q):
    p, dev, keep = _array_arg(q)
    _check(lib().claw_ensemble_set_q(h, int(i), p, dev), "claw_ensemble_set_q")


def claw_ensemble_get_q(h, i, out):
    p, dev, keep = _array_arg(out)
    _check(lib().claw_ensemble_get_q(h, int(i), p, dev), "claw_ensemble_get_q")
    return out


def claw_ensemble_set_aux(h, i, rho, K):
    pr, dr, kr = _array_arg(rho)
    pk, dk, kk = _array_arg(K)
    _check(lib().claw_ensemble_set_aux(h, int(i), pr, pk, dr), "claw_ensemble_set_aux")


def claw_ensemble_set_bathymetry(h, i, B):
    pb, db, kb = _array_arg(B)
    _check(lib().claw_ensemble_set_bathymetry(h, int(i), pb, db), "claw_ensemble_set_bathymetry")


def claw_ensemble_run_steps(h, nsteps):
    _check(lib().claw_ensemble_run_steps(h, int(nsteps)), "claw_ensemble_run_steps")


def claw_ensemble_get_time(h, i):
    t, dt, n = C.c_double(), C.c_double(), C.c_long()
    _check(lib().claw_ensemble_get_time(h, int(i), C.byref(t), C.byref(dt), C.byref(n)),
           "claw_ensemble_get_time")
    return t.value, dt.value, n.value


def claw_ensemble_size(h):
    return int(lib().claw_ensemble_size(h))


def claw_profile_steps(h, nsteps):
    ms = (C.c_double * 4)()
    tot = C.c_double()
    nl = C.c_long()
    _check(lib().claw_profile_steps(h, int(nsteps), ms, C.byref(tot), C.byref(nl)),
           "claw_profile_steps")
    return list(ms), tot.value, nl.value


def claw_set_segment(h, d, seg_len):
    _check(lib().claw_set_segment(h, int(d), int(seg_len)), "claw_set_segment")


TILE_ORDERS = {"largest_first": 0, "list": 1}


def claw_set_tile_shape(h, d, lines=0, seg_len=0, order=-1):
    o = TILE_ORDERS[order] if isinstance(order, str) else int(order)
    _check(lib().claw_set_tile_shape(h, int(d), int(lines), int(seg_len), o), "claw_set_tile_shape")


def claw_get_tile_shape(h, d):
    lines, seg, order = C.c_int(), C.c_int(), C.c_int()
    _check(lib().claw_get_tile_shape(h, int(d), C.byref(lines), C.byref(seg), C.byref(order)),
           "claw_get_tile_shape")
    return lines.value, seg.value, order.value


def claw_probe_fma(precision, stream=None):
    v = C.c_double(0.0)
    _check(lib().claw_probe_fma(int(precision), C.byref(v), _stream_arg(stream)), "claw_probe_fma")
    return v.value


def claw_autotune(h, trial_steps=3):
    seg = (C.c_int * 3)()
    _check(lib().claw_autotune(h, int(trial_steps), seg), "claw_autotune")
    return list(seg)


def claw_max_speed_noalloc(n, dx, system, bc, params, q_dev, out_dev, rho_dev=None, K_dev=None,
                           stream=None):
    """CFL speed pass over caller-owned device tensors, allocating nothing:
    ``q_dev`` (float64 CUDA tensor, SoA), ``out_dev`` (one float64 on the
    device) receives max_d(max|s| / dx_d) asynchronously on ``stream``."""
    g = make_grid(n, dx)
    sysc = SYSTEMS[system] if isinstance(system, str) else int(system)
    ptr = lambda t: None if t is None else C.c_void_p(t.data_ptr())
    _check(lib().claw_max_speed_noalloc(C.byref(g), sysc, make_bc(bc, len(n)), C.byref(params),
                                        ptr(q_dev), ptr(rho_dev), ptr(K_dev), ptr(out_dev),
                                        _stream_arg(stream)), "claw_max_speed_noalloc")
