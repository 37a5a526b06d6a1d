"""Object wrappers over the C ABI: ``Solver`` (one grid) and ``Ensemble``.

Marshalling only; each method is one C call (see include/claw.h).
"""
from __future__ import annotations

import numpy as np

from . import _lib as L


def _nm(system: str, ndim: int):
    return (3, 3) if system.startswith("shallow_water") else (ndim + 1, 2)


class Solver:
    """One grid.  ``precision`` 64 (plain FP64 path) or 32 (FP32 state and
    arithmetic, FP64 time step / time / sums)."""

    def __init__(self, n, dx, system, limiter, bc, precision=64, rho=1.0, K=1.0, g=9.81,
                 cfl_desired=0.9, cfl_max=1.0, dt_max=1e9, max_retries=8, stream=None,
                 splitting="godunov", dry_tol=1e-3):
        self.ndim = len(n)
        self.n = tuple(int(v) for v in n)
        self.system = system
        self.m, self.mwaves = _nm(system, self.ndim)
        params = L.make_params(rho, K, g, cfl_desired, cfl_max, dt_max, precision, max_retries,
                               splitting, dry_tol)
        self.h = L.claw_create(self.n, dx, self.m, self.mwaves, system, limiter, bc, params, stream)
        self.shape = (self.m,) + tuple(reversed(self.n))

    @classmethod
    def from_problem(cls, prob, precision=64, stream=None, **kw):
        kw.setdefault("splitting", getattr(prob, "splitting", "godunov"))
        kw.setdefault("dry_tol", getattr(prob, "dry_tol", 1e-3))
        s = cls(prob.n, prob.dx, prob.system, prob.limiter, prob.bc, precision=precision,
                rho=prob.rho, K=prob.K, g=prob.g, cfl_desired=prob.cfl_desired,
                cfl_max=prob.cfl_max, stream=stream, **kw)
        if prob.system == "acoustics_var":
            s.set_aux(prob.rho_cell, prob.K_cell)
        if prob.system in ("shallow_water_bathy", "shallow_water_dry") and prob.B_cell is not None:
            s.set_bathymetry(prob.B_cell)
        s.set_q(prob.q0)
        return s

    def close(self):
        if getattr(self, "h", None):
            L.claw_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_q(self, q):
        if hasattr(q, "shape") and tuple(q.shape) != self.shape:
            raise ValueError(f"state shape {tuple(q.shape)} != {self.shape}")
        L.claw_set_q(self.h, q)

    def get_q(self, out=None):
        if out is None:
            out = np.empty(self.shape, dtype=np.float64)
        return L.claw_get_q(self.h, out)

    def set_aux(self, rho, K):
        L.claw_set_aux(self.h, rho, K)

    def set_bathymetry(self, B):
        L.claw_set_bathymetry(self.h, B)

    def step(self, dt=0.0):
        return L.claw_step(self.h, dt)

    def advance(self, t_final, cfl_target=0.0):
        return L.claw_advance(self.h, t_final, cfl_target)

    def run_steps(self, nsteps):
        L.claw_run_steps(self.h, nsteps)

    def max_speed(self):
        return L.claw_max_speed(self.h)

    def run_fixed_steps(self, nsteps, dt):
        """nsteps kept steps of exactly dt; returns the largest Courant number."""
        return L.claw_run_fixed_steps(self.h, nsteps, dt)

    def checkpoint(self):
        L.claw_checkpoint(self.h)

    def rollback(self):
        L.claw_rollback(self.h)

    def get_rows(self, y0, out):
        return L.claw_get_rows(self.h, y0, out)

    def set_rows(self, y0, rows):
        L.claw_set_rows(self.h, y0, rows)

    def time(self):
        return L.claw_get_time(self.h)

    def set_time(self, t, dt, nsteps):
        L.claw_set_time(self.h, t, dt, nsteps)

    def sums(self):
        return L.claw_conservation_sums(self.h, self.m)

    def rejections(self):
        return L.claw_get_rejections(self.h)

    def profile_steps(self, nsteps):
        return L.claw_profile_steps(self.h, nsteps)

    def set_segment(self, d, seg_len):
        L.claw_set_segment(self.h, d, seg_len)

    def set_tile_shape(self, d, lines=0, seg_len=0, order=-1):
        L.claw_set_tile_shape(self.h, d, lines, seg_len, order)

    def tile_shape(self, d):
        """(lines per tile, segment length, order) of direction d."""
        return L.claw_get_tile_shape(self.h, d)

    def autotune(self, trial_steps=3):
        return L.claw_autotune(self.h, trial_steps)


class Ensemble:
    """B independent grids of one system advanced by shared launches."""

    def __init__(self, grids, system, limiter, bc, precision=32, rho=1.0, K=1.0, g=9.81,
                 cfl_desired=0.9, cfl_max=1.0, dt_max=1e9, max_retries=8, stream=None,
                 splitting="godunov", dry_tol=1e-3):
        self.grids = [(tuple(int(v) for v in n), tuple(dx)) for n, dx in grids]
        self.ndim = len(self.grids[0][0])
        self.system = system
        self.m, self.mwaves = _nm(system, self.ndim)
        params = L.make_params(rho, K, g, cfl_desired, cfl_max, dt_max, precision, max_retries,
                               splitting, dry_tol)
        self.h = L.claw_ensemble_create(self.grids, system, limiter, bc, params, stream)

    @classmethod
    def from_problems(cls, probs, precision=32, stream=None, **kw):
        p0 = probs[0]
        kw.setdefault("splitting", getattr(p0, "splitting", "godunov"))
        kw.setdefault("dry_tol", getattr(p0, "dry_tol", 1e-3))
        e = cls([(p.n, p.dx) for p in probs], p0.system, p0.limiter, p0.bc, precision=precision,
                rho=p0.rho, K=p0.K, g=p0.g, cfl_desired=p0.cfl_desired, cfl_max=p0.cfl_max,
                stream=stream, **kw)
        for i, p in enumerate(probs):
            if p.system == "acoustics_var":
                e.set_aux(i, p.rho_cell, p.K_cell)
            if p.system in ("shallow_water_bathy", "shallow_water_dry") and p.B_cell is not None:
                e.set_bathymetry(i, p.B_cell)
            e.set_q(i, p.q0)
        return e

    def __len__(self):
        return len(self.grids)

    def shape(self, i):
        return (self.m,) + tuple(reversed(self.grids[i][0]))

    def close(self):
        if getattr(self, "h", None):
            L.claw_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_q(self, i, q):
        L.claw_ensemble_set_q(self.h, i, q)

    def get_q(self, i, out=None):
        if out is None:
            out = np.empty(self.shape(i), dtype=np.float64)
        return L.claw_ensemble_get_q(self.h, i, out)

    def set_aux(self, i, rho, K):
        L.claw_ensemble_set_aux(self.h, i, rho, K)

    def set_bathymetry(self, i, B):
        L.claw_ensemble_set_bathymetry(self.h, i, B)

    def run_steps(self, nsteps):
        L.claw_ensemble_run_steps(self.h, nsteps)

    def time(self, i):
        return L.claw_ensemble_get_time(self.h, i)

    def profile_steps(self, nsteps):
        return L.claw_profile_steps(self.h, nsteps)

    def set_segment(self, d, seg_len):
        L.claw_set_segment(self.h, d, seg_len)

    def set_tile_shape(self, d, lines=0, seg_len=0, order=-1):
        L.claw_set_tile_shape(self.h, d, lines, seg_len, order)

    def tile_shape(self, d):
        return L.claw_get_tile_shape(self.h, d)

    def autotune(self, trial_steps=3):
        return L.claw_autotune(self.h, trial_steps)
