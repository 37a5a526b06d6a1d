"""Seeded synthetic workloads for the wave-propagation step.

This module only draws and lays out initial data and material parameters.
It holds none of the method's arithmetic (no Riemann solver, limiter,
update or time-step rule), so the CPU oracle and the CUDA path can both be
fed from it without sharing any numerical code.

Every workload restates one of the five benchmark problems (2D acoustics
pulse, 2D radial dam break, 3D two-layer acoustics, 2D shallow-water
ensemble, 3D acoustics ensemble) with these readings where the paper is silent:
cell centres at ``lower + (i + 1/2) dx``, point-sampled initial data,
seed 1805 through ``numpy.random.Generator(PCG64(seed))``.

Array layout is structure-of-arrays, C order: ``q[field, z, y, x]`` (3D)
or ``q[field, y, x]`` (2D), interior cells only, float64.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import List, Optional, Sequence

import numpy as np

SEED = 1805

SYSTEMS = ("acoustics", "acoustics_var", "shallow_water", "shallow_water_bathy", "shallow_water_dry")
LIMITERS = ("none", "minmod", "mc", "first_order")
BCS = ("periodic", "extrap", "wall")
SPLITTINGS = ("godunov", "strang", "unsplit")


@dataclass
class Problem:
    """One grid problem: geometry, physics, boundary kinds and initial state."""

    ndim: int
    n: tuple                      # interior cells (nx, ny[, nz])
    lower: tuple
    upper: tuple
    system: str                   # one of SYSTEMS
    limiter: str                  # one of LIMITERS
    bc: tuple                     # 2*ndim kinds: x-lo, x-hi, y-lo, y-hi[, z-lo, z-hi]
    q0: np.ndarray                # (m, [nz,] ny, nx) float64
    rho: float = 1.0
    K: float = 1.0
    g: float = 9.81
    cfl_desired: float = 0.9
    cfl_max: float = 1.0
    nsteps: int = 1
    rho_cell: Optional[np.ndarray] = None   # ([nz,] ny, nx) for acoustics_var
    K_cell: Optional[np.ndarray] = None
    name: str = ""
    splitting: str = "godunov"    # one of SPLITTINGS
    B_cell: Optional[np.ndarray] = None     # (ny, nx) bottom elevation (shallow_water_bathy / _dry)
    # cell widths given exactly (a piece of a larger grid keeps its parent's
    # widths; recomputing them from the piece's bounds can differ in the last bit)
    cell_width: Optional[tuple] = None
    dry_tol: float = 1e-3         # shallow_water_dry: a cell with h <= dry_tol is dry

    @property
    def m(self) -> int:
        return self.q0.shape[0]

    @property
    def mwaves(self) -> int:
        return 3 if self.system.startswith("shallow_water") else 2

    @property
    def dx(self) -> tuple:
        if self.cell_width is not None:
            return tuple(self.cell_width)
        return tuple((self.upper[d] - self.lower[d]) / self.n[d] for d in range(self.ndim))

    @property
    def ncells(self) -> int:
        return int(np.prod(self.n))

    def with_(self, **kw) -> "Problem":
        return replace(self, **kw)


def centres(n: int, lo: float, hi: float) -> np.ndarray:
    """Cell-centre coordinates lo + (i + 1/2) * dx, i = 0..n-1."""
    dx = (hi - lo) / n
    return lo + (np.arange(n, dtype=np.float64) + 0.5) * dx


# --------------------------------------------------------------------------
# Single-grid workloads
# --------------------------------------------------------------------------

def acoustics_2d_pulse(n: int = 128, ny: Optional[int] = None, rho: float = 1.0,
                       K: float = 4.0, width: float = 200.0, limiter: str = "mc",
                       bc: str = "wall", nsteps: int = 100) -> Problem:
    """2D linear acoustics, m=3 (p,u,v), Gaussian pressure pulse exp(-width r^2)
    centred in [0,1]^2, zero velocity, reflecting walls (128^2, 100 steps)."""
    ny = n if ny is None else ny
    x = centres(n, 0.0, 1.0)
    y = centres(ny, 0.0, 1.0)
    Y, X = np.meshgrid(y, x, indexing="ij")
    r2 = (X - 0.5) ** 2 + (Y - 0.5) ** 2
    q0 = np.zeros((3, ny, n))
    q0[0] = np.exp(-width * r2)
    return Problem(2, (n, ny), (0.0, 0.0), (1.0, 1.0), "acoustics", limiter,
                   (bc,) * 4, q0, rho=rho, K=K, nsteps=nsteps,
                   name=f"acoustics2d_pulse_{n}x{ny}")


def sw_radial_dam_break(n: int = 4096, ny: Optional[int] = None, limiter: str = "minmod",
                        bc: str = "extrap", nsteps: int = 200, h_in: float = 2.0,
                        h_out: float = 1.0, radius: float = 0.5) -> Problem:
    """2D shallow water on [-1,1]^2: h = 2 inside r < 0.5, 1 outside, zero
    momentum, outflow (zeroth-order extrapolation) boundaries (4096^2, 200 steps)."""
    ny = n if ny is None else ny
    x = centres(n, -1.0, 1.0)
    y = centres(ny, -1.0, 1.0)
    Y, X = np.meshgrid(y, x, indexing="ij")
    r = np.sqrt(X * X + Y * Y)
    q0 = np.zeros((3, ny, n))
    q0[0] = np.where(r < radius, h_in, h_out)
    return Problem(2, (n, ny), (-1.0, -1.0), (1.0, 1.0), "shallow_water", limiter,
                   (bc,) * 4, q0, g=9.81, nsteps=nsteps, name=f"sw_radial_dam_break_{n}x{ny}")


def sw_transonic_dam_break(n: int = 120, width: int = 4, axis: int = 0, mirror: bool = False,
                           limiter: str = "mc", h_deep: float = 1.0, h_shallow: float = 0.1,
                           bc: str = "extrap") -> Problem:
    """Planar dam break on [-1,1]^2 whose rarefaction fan spans the jump's
    position: h = h_deep on one side of 0 and h_shallow on the other (depth
    ratio 10), zero momentum.  The jump runs across direction `axis` (n cells
    along it, `width` uniform cells across).  mirror=False puts the deep side
    at negative coordinates, so the 1-wave fan is transonic; mirror=True puts
    it at positive coordinates (the 3-wave fan is transonic)."""
    c = centres(n, -1.0, 1.0)
    prof = np.where(c > 0.0, h_deep, h_shallow) if mirror else np.where(c < 0.0, h_deep, h_shallow)
    if axis == 0:
        shape_xy = (n, width)
        h = np.broadcast_to(prof[None, :], (width, n))
    else:
        shape_xy = (width, n)
        h = np.broadcast_to(prof[:, None], (n, width))
    q0 = np.zeros((3,) + h.shape)
    q0[0] = h
    return Problem(2, shape_xy, (-1.0, -1.0), (1.0, 1.0), "shallow_water", limiter, (bc,) * 4,
                   q0, name=f"sw_transonic_{'xy'[axis]}{'_mirror' if mirror else ''}_{n}")


def sw_bathymetry(n: int = 4096, limiter: str = "minmod", bc: str = "extrap", nsteps: int = 200,
                  bump: float = 0.5, hump: float = 0.2) -> Problem:
    """Shallow water over bathymetry on [-1,1]^2: a Gaussian seamount
    B = bump exp(-20 ((x-0.3)^2 + y^2)) under a surface at rest at 1, with a
    Gaussian surface hump eta = 1 + hump exp(-40 ((x+0.4)^2 + y^2)) that runs
    over it; zero momentum.  B and eta are rounded to multiples of 2^-24, so
    h = eta - B is exact and the resting part of the surface is exactly flat."""
    x = centres(n, -1.0, 1.0)
    Y, X = np.meshgrid(x, x, indexing="ij")
    q = 2.0 ** -24
    B = np.round(bump * np.exp(-20.0 * ((X - 0.3) ** 2 + Y ** 2)) / q) * q
    eta = 1.0 + np.round(hump * np.exp(-40.0 * ((X + 0.4) ** 2 + Y ** 2)) / q) * q
    q0 = np.zeros((3, n, n))
    q0[0] = eta - B
    return Problem(2, (n, n), (-1.0, -1.0), (1.0, 1.0), "shallow_water_bathy", limiter,
                   (bc,) * 4, q0, nsteps=nsteps, B_cell=B, name=f"sw_bathymetry_{n}")


def _round24(a: np.ndarray) -> np.ndarray:
    """Values rounded to multiples of 2^-24 (exact in FP32 for |a| < 1, and
    their differences are exact), so h = eta - B and eta = h + B are exact."""
    q = 2.0 ** -24
    return np.round(np.asarray(a, dtype=np.float64) / q) * q


def sw_dry_dam_break(n: int = 200, width: int = 4, axis: int = 0, h_l: float = 1.0,
                     limiter: str = "mc", bc: str = "extrap") -> Problem:
    """Ritter's dam break on [-1,1]^2: depth h_l at negative coordinates along
    `axis`, a dry bed (h = 0) at positive ones, flat bottom B = 0, zero
    momentum; n cells along `axis`, `width` uniform cells across.  System
    shallow_water_dry (wetting and drying)."""
    c = centres(n, -1.0, 1.0)
    prof = np.where(c < 0.0, h_l, 0.0)
    if axis == 0:
        shape_xy, h = (n, width), np.broadcast_to(prof[None, :], (width, n))
    else:
        shape_xy, h = (width, n), np.broadcast_to(prof[:, None], (n, width))
    q0 = np.zeros((3,) + h.shape)
    q0[0] = h
    return Problem(2, shape_xy, (-1.0, -1.0), (1.0, 1.0), "shallow_water_dry", limiter, (bc,) * 4,
                   q0, B_cell=np.zeros(h.shape), name=f"sw_ritter_{'xy'[axis]}_{n}")


def sw_island(n: int = 4096, ny: Optional[int] = None, limiter: str = "minmod", bc: str = "wall",
              hump: float = 0.2, peak: float = 1.6, nsteps: int = 200) -> Problem:
    """Wetting and drying on [-1,1]^2: a lake whose surface rests at eta = 1
    around an island B = peak exp(-8 ((x - 0.25)^2 + y^2)) that rises above
    it (the island's top, where B > eta, is dry: h = 0), with a Gaussian
    surface hump eta = 1 + hump exp(-40 ((x + 0.5)^2 + y^2)) that runs up the
    island's shore and falls back; zero momentum.  B and eta are rounded to
    multiples of 2^-24, so h = max(eta - B, 0) is exact and, with hump = 0,
    the lake is exactly at rest."""
    ny = n if ny is None else ny
    x = centres(n, -1.0, 1.0)
    y = centres(ny, -1.0, 1.0)
    Y, X = np.meshgrid(y, x, indexing="ij")
    B = _round24(peak * np.exp(-8.0 * ((X - 0.25) ** 2 + Y ** 2)))
    eta = 1.0 + _round24(hump * np.exp(-40.0 * ((X + 0.5) ** 2 + Y ** 2)))
    q0 = np.zeros((3, ny, n))
    q0[0] = np.maximum(eta - B, 0.0)
    return Problem(2, (n, ny), (-1.0, -1.0), (1.0, 1.0), "shallow_water_dry", limiter, (bc,) * 4,
                   q0, nsteps=nsteps, B_cell=B, name=f"sw_island_{n}x{ny}")


def sw_beach(n: int = 200, ny: int = 40, limiter: str = "mc", bc: str = "wall",
             slope: float = 0.8, eta0: float = 0.3, hump: float = 0.15) -> Problem:
    """Run-up on a plane beach on [-1,1]^2: bottom B = slope * x, still water
    at eta0 (dry where B > eta0) with a hump eta0 + hump exp(-30 (x + 0.4)^2),
    uniform across y, zero momentum; walls by default (mass is conserved
    exactly).  B and eta are rounded to multiples of 2^-24."""
    x = centres(n, -1.0, 1.0)
    B = _round24(np.broadcast_to(slope * x[None, :], (ny, n)))
    eta = eta0 + _round24(np.broadcast_to(hump * np.exp(-30.0 * (x[None, :] + 0.4) ** 2), (ny, n)))
    q0 = np.zeros((3, ny, n))
    q0[0] = np.maximum(eta - B, 0.0)
    return Problem(2, (n, ny), (-1.0, -1.0), (1.0, 1.0), "shallow_water_dry", limiter, (bc,) * 4,
                   q0, B_cell=B.copy(), name=f"sw_beach_{n}x{ny}")


def acoustics_3d_layers(n: int = 512, width: float = 200.0, limiter: str = "mc",
                        bc: str = "wall", nsteps: int = 100,
                        centre=(0.5, 0.5, 0.25)) -> Problem:
    """3D variable-coefficient acoustics on [0,1]^3, m=4 (p,u,v,w): (rho,K)=(1,1)
    for cell-centre z < 0.5 and (4,4) above; Gaussian pulse at (0.5,0.5,0.25);
    reflecting walls (512^3, 100 steps)."""
    x = centres(n, 0.0, 1.0)
    z3 = x[:, None, None]
    y3 = x[None, :, None]
    x3 = x[None, None, :]
    r2 = (x3 - centre[0]) ** 2 + (y3 - centre[1]) ** 2 + (z3 - centre[2]) ** 2
    q0 = np.zeros((4, n, n, n))
    q0[0] = np.exp(-width * r2)
    upper = np.broadcast_to(z3 >= 0.5, (n, n, n))
    rho_cell = np.where(upper, 4.0, 1.0).astype(np.float64)
    K_cell = rho_cell.copy()
    return Problem(3, (n, n, n), (0.0,) * 3, (1.0,) * 3, "acoustics_var", limiter,
                   (bc,) * 6, q0, nsteps=nsteps, rho_cell=rho_cell, K_cell=K_cell,
                   name=f"acoustics3d_layers_{n}^3")


# --------------------------------------------------------------------------
# Ensembles
# --------------------------------------------------------------------------

def _min_image(d: np.ndarray) -> np.ndarray:
    """Minimum-image distance component on the unit period."""
    return d - np.round(d)


def sw_ensemble(B: int = 256, nmin: int = 64, nmax: int = 1024, seed: int = SEED,
                limiter: str = "minmod", nsteps: int = 50) -> List[Problem]:
    """Shallow-water ensemble on [0,1]^2, periodic: per instance, in draw order,
    side n ~ U{nmin..nmax}, hump count ~ U{1,2,3}, then per hump A ~ U(0.1,0.5),
    w ~ U(0.05,0.2), centre (cx, cy) ~ U[0,1]^2.  h = 1 + sum A exp(-(r/w)^2)
    with r the minimum-image periodic distance, zero momentum."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(B):
        n = int(rng.integers(nmin, nmax + 1))
        nh = int(rng.integers(1, 4))
        humps = [(rng.uniform(0.1, 0.5), rng.uniform(0.05, 0.2),
                  rng.uniform(0.0, 1.0), rng.uniform(0.0, 1.0)) for _ in range(nh)]
        c = centres(n, 0.0, 1.0)
        Y, X = np.meshgrid(c, c, indexing="ij")
        h = np.ones((n, n))
        for (A, w, cx, cy) in humps:
            rx = _min_image(X - cx)
            ry = _min_image(Y - cy)
            h += A * np.exp(-(rx * rx + ry * ry) / (w * w))
        q0 = np.zeros((3, n, n))
        q0[0] = h
        out.append(Problem(2, (n, n), (0.0, 0.0), (1.0, 1.0), "shallow_water", limiter,
                           ("periodic",) * 4, q0, nsteps=nsteps, name=f"sw_ens{i}_{n}"))
    return out


def box_filter5(a: np.ndarray) -> np.ndarray:
    """Separable 5-tap mean along every axis, clamp-to-edge, float64."""
    out = np.asarray(a, dtype=np.float64)
    for ax in range(out.ndim):
        pad = [(0, 0)] * out.ndim
        pad[ax] = (2, 2)
        p = np.pad(out, pad, mode="edge")
        n = out.shape[ax]
        acc = np.zeros_like(out)
        for k in range(5):
            sl = [slice(None)] * out.ndim
            sl[ax] = slice(k, k + n)
            acc += p[tuple(sl)]
        out = acc / 5.0
    return out


def acoustics3d_ensemble(B: int = 64, nmin: int = 128, nmax: int = 256, seed: int = SEED,
                         limiter: str = "mc", nsteps: int = 100, width: float = 200.0,
                         instances: Optional[Sequence[int]] = None) -> List[Problem]:
    """3D variable-coefficient acoustics ensemble on [0,1]^3 with walls: per
    instance, in draw order, side n ~ U{nmin..nmax}, pulse centre ~ U[0.25,0.75]^3,
    then rho and K per cell log-uniform in [0.5, 4] (each an n^3 draw in z,y,x
    order), each smoothed by a 5-tap box filter.  ``instances`` restricts which
    instances are materialised (the draws of the others are still consumed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lo, hi = np.log(0.5), np.log(4.0)
    keep = None if instances is None else set(int(i) for i in instances)
    out = []
    for i in range(B):
        n = int(rng.integers(nmin, nmax + 1))
        cen = rng.uniform(0.25, 0.75, size=3)
        if keep is not None and i not in keep:
            rng.uniform(lo, hi, size=2 * n ** 3)   # consume the same draws
            continue
        rho = box_filter5(np.exp(rng.uniform(lo, hi, size=(n, n, n))))
        K = box_filter5(np.exp(rng.uniform(lo, hi, size=(n, n, n))))
        c = centres(n, 0.0, 1.0)
        r2 = ((c[None, None, :] - cen[0]) ** 2 + (c[None, :, None] - cen[1]) ** 2
              + (c[:, None, None] - cen[2]) ** 2)
        q0 = np.zeros((4, n, n, n))
        q0[0] = np.exp(-width * r2)
        out.append(Problem(3, (n, n, n), (0.0,) * 3, (1.0,) * 3, "acoustics_var", limiter,
                           ("wall",) * 6, q0, nsteps=nsteps, rho_cell=rho, K_cell=K,
                           name=f"ac3_ens{i}_{n}"))
    return out


# --------------------------------------------------------------------------
# Small generic cases for tests (odd sizes, every system / limiter / BC)
# --------------------------------------------------------------------------

def random_smooth_state(problem_system: str, shape: Sequence[int], seed: int = SEED,
                        amplitude: float = 0.3) -> np.ndarray:
    """A smooth random state: a few random Fourier modes per field on the unit
    box. Shallow water gets h = 1 + perturbation (> 0.4 everywhere)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ndim = len(shape)
    sw = problem_system.startswith("shallow_water")
    m = 3 if sw else (ndim + 1)
    coords = np.meshgrid(*[centres(s, 0.0, 1.0) for s in shape], indexing="ij")
    q = np.zeros((m,) + tuple(shape))
    for f in range(m):
        for _ in range(3):
            k = rng.integers(1, 4, size=ndim)
            ph = rng.uniform(0, 2 * np.pi, size=ndim)
            a = rng.uniform(-amplitude, amplitude)
            mode = np.ones(tuple(shape))
            for d in range(ndim):
                mode = mode * np.cos(2 * np.pi * k[d] * coords[d] + ph[d])
            q[f] += a * mode
    if sw:
        q[0] += 1.0
    return q


def random_problem(system: str, shape_xyz: Sequence[int], limiter: str, bc,
                   seed: int = SEED, discontinuous: bool = False) -> Problem:
    """A small problem for parity tests. ``shape_xyz`` is (nx, ny[, nz]); the
    state is smooth random, plus a step discontinuity when ``discontinuous``.
    Variable acoustics get smooth random rho, K in [0.5, 4]."""
    ndim = len(shape_xyz)
    arr_shape = tuple(reversed(shape_xyz))
    q0 = random_smooth_state(system, arr_shape, seed=seed)
    if discontinuous:
        sl = [slice(None)] * ndim
        sl[-1] = slice(arr_shape[-1] // 3, 2 * arr_shape[-1] // 3)
        q0[(0,) + tuple(sl)] += 0.5
    if isinstance(bc, str):
        bc = (bc,) * (2 * ndim)
    rho_cell = K_cell = B_cell = None
    if system == "acoustics_var":
        rng = np.random.Generator(np.random.PCG64(seed + 7))
        rho_cell = box_filter5(np.exp(rng.uniform(np.log(0.5), np.log(4.0), size=arr_shape)))
        K_cell = box_filter5(np.exp(rng.uniform(np.log(0.5), np.log(4.0), size=arr_shape)))
    if system == "shallow_water_bathy":
        # smooth random bottom within [-0.2, 0.2] (the depth stays > 0.2)
        B_cell = 0.6 * random_smooth_state("acoustics", arr_shape, seed=seed + 11, amplitude=0.1)[0]
    if system == "shallow_water_dry":
        # the same random bottom plus a ridge that rises above the surface:
        # q0[0] is read as the surface eta, the depth is max(eta - B, 0) (dry
        # cells on and around the ridge), velocities q0[1], q0[2] where wet
        rng = np.random.Generator(np.random.PCG64(seed + 13))
        cx, cy = rng.uniform(0.3, 0.7, size=2)
        coords = np.meshgrid(*[centres(s_, 0.0, 1.0) for s_ in arr_shape], indexing="ij")
        r2 = (coords[-1] - cx) ** 2 + (coords[-2] - cy) ** 2
        B_cell = _round24(0.6 * random_smooth_state("acoustics", arr_shape, seed=seed + 11,
                                                   amplitude=0.1)[0] + 2.5 * np.exp(-30.0 * r2))
        eta = _round24(q0[0])
        h = np.maximum(eta - B_cell, 0.0)
        q0[1] = q0[1] * h
        q0[2] = q0[2] * h
        q0[0] = h
    return Problem(ndim, tuple(shape_xyz), (0.0,) * ndim, (1.0,) * ndim, system, limiter,
                   tuple(bc), q0, rho=1.0, K=4.0, rho_cell=rho_cell, K_cell=K_cell, B_cell=B_cell,
                   name=f"{system}_{'x'.join(map(str, shape_xyz))}_{limiter}")
