"""CPU oracle for the dimension-split wave-propagation step (CUDACLAW Sec. 3).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and
the benchmark's CPU-baseline leg may import this package.  It wraps the plain
FP64 C implementation in this directory through ctypes and shares no code
with the CUDA library.

Functions take ``paper_1805_08846_gb300.inputs.Problem``-like objects (any
object with the same attributes) and numpy float64 arrays in the
structure-of-arrays layout ``q[field, (z,) y, x]``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_SYSTEMS = {"acoustics": 0, "acoustics_var": 1, "shallow_water": 2, "shallow_water_bathy": 3,
            "shallow_water_dry": 4}
_LIMITERS = {"none": 0, "minmod": 1, "mc": 2, "first_order": 3}
_BCS = {"periodic": 0, "extrap": 1, "wall": 2}
_SPLITTINGS = {"godunov": 0, "strang": 1, "unsplit": 2}

_dp = C.POINTER(C.c_double)


class _Problem(C.Structure):
    _fields_ = [
        ("ndim", C.c_int), ("n", C.c_int * 3), ("dx", C.c_double * 3),
        ("system", C.c_int), ("limiter", C.c_int), ("bc", C.c_int * 6),
        ("rho", C.c_double), ("K", C.c_double), ("g", C.c_double),
        ("cfl_desired", C.c_double), ("cfl_max", C.c_double), ("dt_max", C.c_double),
        ("max_retries", C.c_int), ("rho_cell", _dp), ("K_cell", _dp),
        ("splitting", C.c_int), ("B_cell", _dp), ("dry_tol", C.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        # ORC_LIB selects another build of these same sources (the mutation
        # test loads deliberately broken copies through it).
        path = os.environ.get("ORC_LIB") or _build.build()
        L = C.CDLL(path)
        L.orc_sweep.restype = C.c_double
        L.orc_sweep.argtypes = [C.POINTER(_Problem), C.c_int, _dp, _dp, C.c_double,
                                C.c_long, C.c_long]
        L.orc_max_speed_dir.restype = C.c_double
        L.orc_max_speed_dir.argtypes = [C.POINTER(_Problem), C.c_int, _dp]
        L.orc_nlines.restype = C.c_long
        L.orc_nlines.argtypes = [C.POINTER(_Problem), C.c_int]
        L.orc_run.restype = C.c_int
        L.orc_run.argtypes = [C.POINTER(_Problem), _dp, C.c_int, C.c_long, C.c_double,
                              C.c_double, _dp, _dp, C.POINTER(C.c_long),
                              C.POINTER(C.c_long), _dp]
        L.orc_phi.restype = C.c_double
        L.orc_phi.argtypes = [C.c_int, C.c_double]
        L.orc_rp_acoustics.restype = None
        L.orc_rp_acoustics.argtypes = [_dp, _dp, C.c_double, C.c_double, C.c_double,
                                       C.c_double, _dp, _dp, _dp, _dp]
        L.orc_rp_shallow_water.restype = None
        L.orc_rp_shallow_water.argtypes = [_dp, _dp, C.c_double, _dp, _dp, _dp, _dp]
        L.orc_rp_shallow_water_bathy.restype = None
        L.orc_rp_shallow_water_bathy.argtypes = [_dp, _dp, C.c_double, C.c_double, C.c_double,
                                                 _dp, _dp, _dp, _dp]
        L.orc_rp_shallow_water_dry.restype = None
        L.orc_rp_shallow_water_dry.argtypes = [_dp, _dp, C.c_double, C.c_double, C.c_double,
                                               C.c_double, _dp, _dp, _dp, _dp]
        L.orc_tr_acoustics.restype = None
        L.orc_tr_acoustics.argtypes = [_dp] + [C.c_double] * 6 + [_dp, _dp]
        L.orc_tr_shallow_water.restype = None
        L.orc_tr_shallow_water.argtypes = [_dp, _dp, _dp, _dp, C.c_double, _dp, _dp]
        L.orc_threads.restype = C.c_int
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


class Oracle:
    """Oracle bound to one problem (geometry, physics, boundaries, coefficients)."""

    def __init__(self, prob, dt_max: float = 1e9, max_retries: int = 8):
        self.prob = prob
        P = _Problem()
        P.ndim = prob.ndim
        n = list(prob.n) + [1] * (3 - prob.ndim)
        dx = list(prob.dx) + [1.0] * (3 - prob.ndim)
        for d in range(3):
            P.n[d] = int(n[d])
            P.dx[d] = float(dx[d])
        P.system = _SYSTEMS[prob.system]
        P.limiter = _LIMITERS[prob.limiter]
        bc = list(prob.bc) + ["extrap"] * (6 - len(prob.bc))
        for i in range(6):
            P.bc[i] = _BCS[bc[i]]
        P.rho, P.K, P.g = float(prob.rho), float(prob.K), float(prob.g)
        P.cfl_desired, P.cfl_max = float(prob.cfl_desired), float(prob.cfl_max)
        P.dt_max = float(dt_max)
        P.max_retries = int(max_retries)
        P.splitting = _SPLITTINGS[getattr(prob, "splitting", "godunov")]
        self._keep = []
        if prob.system == "acoustics_var":
            r = np.ascontiguousarray(prob.rho_cell, dtype=np.float64)
            k = np.ascontiguousarray(prob.K_cell, dtype=np.float64)
            self._keep += [r, k]
            P.rho_cell, P.K_cell = _ptr(r), _ptr(k)
        if prob.system in ("shallow_water_bathy", "shallow_water_dry"):
            b = np.ascontiguousarray(prob.B_cell, dtype=np.float64)
            self._keep.append(b)
            P.B_cell = _ptr(b)
        P.dry_tol = float(getattr(prob, "dry_tol", 0.0))
        self.P = P
        self.m = 3 if prob.system.startswith("shallow_water") else prob.ndim + 1
        self.shape = (self.m,) + tuple(reversed(prob.n))

    def _q(self, q):
        q = np.ascontiguousarray(q, dtype=np.float64)
        assert q.shape == self.shape, (q.shape, self.shape)
        return q

    def sweep(self, d: int, q, dt: float, line_lo: int = 0, line_hi: int = -1):
        """One directional sweep q -> new array; returns (qout, max speed)."""
        q = self._q(q)
        out = np.empty_like(q)
        m = lib().orc_sweep(C.byref(self.P), d, _ptr(q), _ptr(out), float(dt),
                            int(line_lo), int(line_hi))
        return out, m

    def nlines(self, d: int) -> int:
        return int(lib().orc_nlines(C.byref(self.P), d))

    def max_speed_dir(self, d: int, q) -> float:
        return lib().orc_max_speed_dir(C.byref(self.P), d, _ptr(self._q(q)))

    def max_speed_over_dx(self, q) -> float:
        q = self._q(q)
        return max(self.max_speed_dir(d, q) / self.prob.dx[d] for d in range(self.prob.ndim))

    def _run(self, q, mode, nsteps, t_final, fixed_dt, t, dt):
        q = self._q(q).copy()
        t_ = C.c_double(t)
        dt_ = C.c_double(dt)
        nacc, nrej = C.c_long(0), C.c_long(0)
        cfl = C.c_double(0.0)
        st = lib().orc_run(C.byref(self.P), _ptr(q), mode, int(nsteps), float(t_final),
                           float(fixed_dt), C.byref(t_), C.byref(dt_), C.byref(nacc),
                           C.byref(nrej), C.byref(cfl))
        if st == -2:
            raise ValueError("the unsplit update covers 2D acoustics and shallow water only")
        return dict(q=q, t=t_.value, dt=dt_.value, nacc=nacc.value, nrej=nrej.value,
                    cfl=cfl.value, status=st)

    def run_steps(self, q, nsteps: int, t: float = 0.0, dt: float = 0.0,
                  fixed_dt: float = 0.0):
        """Take ``nsteps`` accepted steps with the CFL rule (or ``fixed_dt``)."""
        return self._run(q, 0, nsteps, 0.0, fixed_dt, t, dt)

    def advance(self, q, t_final: float, t: float = 0.0, dt: float = 0.0,
                fixed_dt: float = 0.0):
        """Advance to ``t_final`` with the CFL rule, the last step clipped."""
        return self._run(q, 1, 0, t_final, fixed_dt, t, dt)


def riemann(system: str, ql, qr, rho_l=1.0, K_l=1.0, rho_r=1.0, K_r=1.0, g=9.81, B_l=0.0, B_r=0.0,
            dry_tol=1e-3):
    """Waves W[p][c] (f-waves for shallow_water_bathy and shallow_water_dry),
    speeds s[p], A-dQ, A+dQ at one interface (reduced states)."""
    ql = np.ascontiguousarray(np.pad(np.asarray(ql, dtype=np.float64), (0, 3 - len(ql))))
    qr = np.ascontiguousarray(np.pad(np.asarray(qr, dtype=np.float64), (0, 3 - len(qr))))
    W = np.zeros((3, 3))
    s = np.zeros(3)
    am = np.zeros(3)
    ap = np.zeros(3)
    if system == "shallow_water":
        lib().orc_rp_shallow_water(_ptr(ql), _ptr(qr), float(g), _ptr(W), _ptr(s),
                                   _ptr(am), _ptr(ap))
        return W, s, am, ap
    if system == "shallow_water_bathy":
        lib().orc_rp_shallow_water_bathy(_ptr(ql), _ptr(qr), float(B_l), float(B_r), float(g),
                                         _ptr(W), _ptr(s), _ptr(am), _ptr(ap))
        return W, s, am, ap
    if system == "shallow_water_dry":
        lib().orc_rp_shallow_water_dry(_ptr(ql), _ptr(qr), float(B_l), float(B_r), float(g),
                                       float(dry_tol), _ptr(W), _ptr(s), _ptr(am), _ptr(ap))
        return W, s, am, ap
    lib().orc_rp_acoustics(_ptr(ql), _ptr(qr), float(rho_l), float(K_l), float(rho_r),
                           float(K_r), _ptr(W), _ptr(s), _ptr(am), _ptr(ap))
    return W[:2, :2], s[:2], am[:2], ap[:2]


def transverse(system: str, a, qd=None, qc=None, qu=None, rho=(1.0, 1.0, 1.0), K=(1.0, 1.0, 1.0),
               g=9.81):
    """Transverse split of a reduced fluctuation a (cell below d, cell c,
    cell above u): the parts crossing the lower and upper interfaces."""
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    bm, bp = np.zeros(3), np.zeros(3)
    if system == "shallow_water":
        qd, qc, qu = (np.ascontiguousarray(np.asarray(v, dtype=np.float64)) for v in (qd, qc, qu))
        lib().orc_tr_shallow_water(_ptr(a), _ptr(qd), _ptr(qc), _ptr(qu), float(g), _ptr(bm), _ptr(bp))
    else:
        lib().orc_tr_acoustics(_ptr(a), float(rho[0]), float(K[0]), float(rho[1]), float(K[1]),
                               float(rho[2]), float(K[2]), _ptr(bm), _ptr(bp))
    return bm, bp


def phi(limiter: str, theta: float) -> float:
    return lib().orc_phi(_LIMITERS[limiter], float(theta))


def threads() -> int:
    return int(lib().orc_threads())


def rel_linf(a, ref) -> float:
    """max|a - ref| / max|ref| (absolute when ref is identically zero)."""
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.max(np.abs(ref))
    num = np.max(np.abs(a - ref))
    return float(num / den) if den > 0 else float(num)


def rel_l2(a, ref) -> float:
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref.ravel())
    num = np.linalg.norm((a - ref).ravel())
    return float(num / den) if den > 0 else float(num)


def rel_l1(a, ref) -> float:
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.sum(np.abs(ref))
    num = np.sum(np.abs(a - ref))
    return float(num / den) if den > 0 else float(num)
