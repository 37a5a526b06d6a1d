"""Slab decomposition of one 2D grid across ranks, with wide halos.

This is the paper's idea for several GPUs (Sec. 8): independent subproblems
advanced for several local steps, then the overlap refreshed.  Rank r owns
rows [lo_r, hi_r) of the grid and holds a local grid of rows
[lo_r - H, hi_r + H).  On a side where the grid ends without periodic wrap
there is no halo, and the real boundary rule applies.  A step changes a cell
only from cells at most two rows away along y: the x sweep reads its own row,
the y sweep and the unsplit update read rows j-2 .. j+2.  So after k steps
only the 2k rows nearest each cut edge of a local grid are stale, and with
H >= 2k every owned row is exact.

One period of k steps:
  1. Halo refresh: every rank contributes its first H and last H owned rows
     to an all-gather, and writes its neighbours' rows into its halos.  An
     all-gather cannot deadlock and works the same over gloo and NCCL.  Two
     ranks that are each other's lower and upper neighbour (periodic wrap)
     need no tags.
  2. Speed agreement: the first period takes M = all-reduce max of
     max_d(max|s| / dx_d) over every local grid (a speeds-only pass; after
     step 1 all rows of every local grid are current, so this is the largest
     speed of the whole grid, or slightly more: an outer edge sees its
     boundary rule's ghost).  Every later period takes M = C / dt of the
     period before, C its all-reduced peak Courant number: the largest speed
     any rank met in any step of that period, which needs no extra pass.
  3. dt = cfl_desired / M (capped by dt_max), the same on every rank.
  4. k steps of that dt on every rank, with no communication.
  5. The largest Courant number any rank saw is all-reduced.  Above cfl_max,
     the period is redone from its start with dt scaled to cfl_desired.

The compute of a rank is a `stepper`, which holds the rank's local state.
With `solver_stepper`, a rank's GPU runs the CUDA path through the C ABI,
and only the 4H boundary and halo rows cross it per period.  Tests can plug
in other steppers.  A stepper has get_rows(y0, n) -> rows, set_rows(y0,
rows), max_speed() -> M, snapshot(), restore(), run_fixed(n, dt) -> largest
Courant number of the n steps, and get_q() -> local state.  Rows are torch
tensors of shape (m, n, nx), with y0 a row of the local grid.  The
communicator moves torch tensors.  `DistComm` uses torch.distributed, with
one rank per process (CPU tensors over gloo, device tensors over NCCL).
`LocalComm` runs every rank in one process, for emulating a decomposition
on one device.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Dict, List


@dataclass(frozen=True)
class SlabLayout:
    """Rows of each rank and the window of its local grid.

    ny: rows of the grid; P: ranks; H: halo rows per cut edge;
    periodic: the y boundary wraps (every edge is then a cut edge when P > 1).
    """

    ny: int
    P: int
    H: int
    periodic: bool

    def __post_init__(self):
        if self.P < 1 or self.H < 0:
            raise ValueError("need P >= 1 and H >= 0")
        # a neighbour's halo comes from one rank's owned rows (one rank: no halo)
        need = max(self.H, 2) if self.P > 1 else 2
        if any(self.rows(r)[1] - self.rows(r)[0] < need for r in range(self.P)):
            raise ValueError(f"{self.ny} rows over {self.P} ranks leave a slab thinner than "
                             f"{need} rows")

    def rows(self, r: int):
        """Owned rows [lo, hi) of rank r (balanced, the first ny % P ranks one more)."""
        base, extra = divmod(self.ny, self.P)
        lo = r * base + min(r, extra)
        return lo, lo + base + (1 if r < extra else 0)

    def lower(self, r: int):
        """Rank below r, or None at a non-periodic grid edge (or P == 1)."""
        if self.P == 1:
            return None
        if r > 0:
            return r - 1
        return self.P - 1 if self.periodic else None

    def upper(self, r: int):
        if self.P == 1:
            return None
        if r < self.P - 1:
            return r + 1
        return 0 if self.periodic else None

    def halos(self, r: int):
        """Halo rows below and above the owned rows of rank r."""
        return (self.H if self.lower(r) is not None else 0,
                self.H if self.upper(r) is not None else 0)

    def local_rows(self, r: int) -> int:
        lo, hi = self.rows(r)
        hl, hu = self.halos(r)
        return hl + (hi - lo) + hu

    def global_rows(self, r: int) -> List[int]:
        """Global row of every local row of rank r (wrapped when periodic)."""
        lo, hi = self.rows(r)
        hl, hu = self.halos(r)
        return [(g % self.ny) for g in range(lo - hl, hi + hu)]

    def owned_slice(self, r: int) -> slice:
        hl, _ = self.halos(r)
        lo, hi = self.rows(r)
        return slice(hl, hl + hi - lo)

    def y_bc(self, r: int, bc_lo: str, bc_hi: str):
        """Boundary kinds of rank r's local grid along y: the real ones at a
        grid edge without wrap, otherwise zeroth-order extrapolation (any
        kind would do: the rows it affects are stale by design)."""
        if self.P == 1:
            return bc_lo, bc_hi
        return (bc_lo if self.lower(r) is None else "extrap",
                bc_hi if self.upper(r) is None else "extrap")


class LocalComm:
    """All ranks in one process (emulation on one device)."""

    def allgather(self, parts: Dict[int, "object"], P: int) -> List["object"]:
        return [parts[r] for r in range(P)]

    def allreduce_max(self, values: Dict[int, float]) -> float:
        return max(values.values())


class DistComm:
    """One rank per process over torch.distributed (gloo or NCCL)."""

    def __init__(self, group=None):
        self.group = group

    def allgather(self, parts, P):
        import torch
        import torch.distributed as dist
        (mine,) = parts.values()
        out = [torch.empty_like(mine) for _ in range(P)]
        dist.all_gather(out, mine.contiguous(), group=self.group)
        return out

    def allreduce_max(self, values):
        import torch
        import torch.distributed as dist
        (v,) = values.values()
        dev = "cuda" if dist.get_backend(self.group) == "nccl" else "cpu"
        t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=self.group)
        return float(t.item())


def local_window(q, layout: SlabLayout, r: int):
    """Rank r's local grid (owned rows and halos) cut from a whole-grid state
    q of shape (m, ny, nx) (numpy array or torch tensor)."""
    idx = layout.global_rows(r)
    return q[:, idx, :]


def refresh_halos(steppers: Dict[int, "object"], layout: SlabLayout, comm) -> None:
    """Step 1 of a period: every rank's first and last H owned rows go into
    an all-gather; each rank writes its neighbours' rows into its halos."""
    H = layout.H
    if layout.P == 1 or H == 0:
        return
    import torch
    parts = {}
    for r, st in steppers.items():
        own = layout.owned_slice(r)
        parts[r] = torch.cat([st.get_rows(own.start, H), st.get_rows(own.stop - H, H)], dim=1)
    gathered = comm.allgather(parts, layout.P)
    for r, st in steppers.items():
        hl, hu = layout.halos(r)
        if hl:
            st.set_rows(0, gathered[layout.lower(r)][:, H:, :].contiguous())     # its top rows
        if hu:
            st.set_rows(layout.local_rows(r) - H, gathered[layout.upper(r)][:, :H, :].contiguous())


@dataclass
class SlabRunInfo:
    dts: List[float]          # the step sizes taken, in order (one per step)
    t: float                  # simulated time reached
    periods: int              # periods taken (each after a halo refresh)
    redone: int               # periods redone because a Courant number exceeded cfl_max
    cfl_max_seen: float       # largest Courant number of the kept periods


def run_steps(steppers: Dict[int, "object"], layout: SlabLayout, comm, nsteps: int, k: int,
              cfl_desired: float = 0.9, cfl_max: float = 1.0, dt_max: float = 1e9,
              t: float = 0.0, max_redo: int = 8) -> SlabRunInfo:
    """Advance every rank's local grid by `nsteps` steps in periods of at
    most k steps (see the module docstring).  `steppers` maps each rank this
    process runs to its stepper, which holds the local state.  Needs H >= 2k
    when there is more than one rank."""
    if k < 1 or (layout.P > 1 and layout.H < 2 * k):
        raise ValueError(f"a halo of {layout.H} rows covers at most {layout.H // 2} steps per period")
    dts: List[float] = []
    periods = redone = 0
    seen = 0.0
    done = 0
    M = None
    while done < nsteps:
        refresh_halos(steppers, layout, comm)
        if M is None:
            M = comm.allreduce_max({r: st.max_speed() for r, st in steppers.items()})
        dt = min(cfl_desired / M, dt_max) if M > 0 else dt_max
        n = min(k, nsteps - done)
        for st in steppers.values():
            st.snapshot()
        for attempt in range(max_redo + 1):
            c = comm.allreduce_max({r: st.run_fixed(n, dt) for r, st in steppers.items()})
            if c <= cfl_max:
                break
            if attempt == max_redo:
                raise RuntimeError(f"Courant number {c} above {cfl_max} after {max_redo} redos")
            redone += 1
            dt = dt * cfl_desired / c
            for st in steppers.values():
                st.restore()
        dts += [dt] * n
        t += n * dt
        done += n
        periods += 1
        seen = max(seen, c)
        M = c / dt          # the largest speed the period met, for the next one
    return SlabRunInfo(dts, t, periods, redone, seen)


def gather_grid(steppers: Dict[int, "object"], layout: SlabLayout, comm):
    """The whole grid (m, ny, nx) assembled from every rank's owned rows, on
    every rank (slabs are padded to equal size for the all-gather)."""
    import torch
    rmax = max(layout.rows(r)[1] - layout.rows(r)[0] for r in range(layout.P))
    parts = {}
    for r, st in steppers.items():
        own = layout.owned_slice(r)
        q = st.get_rows(own.start, own.stop - own.start)
        pad = torch.zeros(q.shape[0], rmax, q.shape[2], dtype=q.dtype, device=q.device)
        pad[:, :q.shape[1], :] = q
        parts[r] = pad
    got = comm.allgather(parts, layout.P)
    return torch.cat([got[r][:, :layout.rows(r)[1] - layout.rows(r)[0], :] for r in range(layout.P)],
                     dim=1)


class solver_stepper:
    """A rank's compute on its GPU: a `Solver` over the local grid.  Steps
    are fixed (claw_run_fixed_steps; run_steps takes the CFL decision on the
    speeds of all ranks), rows cross through claw_get_rows /
    claw_set_rows as float64 torch tensors on `device` ("cpu" for gloo:
    host tensors, copied), and the period's start is kept for a redo by
    claw_checkpoint / claw_rollback."""

    def __init__(self, solver, device="cuda"):
        self.s = solver
        self.device = device
        self._pending = []     # device rows whose copy may still be queued on the solver's stream

    def _sync(self, t):
        if t.is_cuda:
            import torch
            # written by torch on its stream; the solver reads on its own
            torch.cuda.current_stream().synchronize()

    def get_rows(self, y0, n):
        import torch
        out = torch.empty((self.s.shape[0], n, self.s.shape[2]), dtype=torch.float64, device=self.device)
        return self.s.get_rows(y0, out)

    def set_rows(self, y0, rows):
        self._sync(rows)
        self.s.set_rows(y0, rows)
        if rows.is_cuda:
            # the solver's copy runs on its stream: keep `rows` alive until a
            # synchronising call
            self._pending.append(rows)

    def max_speed(self) -> float:
        M = float(self.s.max_speed())          # synchronises the solver's stream
        self._pending.clear()
        return M

    def snapshot(self):
        self.s.checkpoint()          # a device copy in the state's own precision; synchronises
        self._pending.clear()

    def restore(self):
        self.s.rollback()

    def run_fixed(self, n, dt) -> float:
        return float(self.s.run_fixed_steps(n, dt))

    def get_q(self):
        import torch
        out = torch.empty(self.s.shape, dtype=torch.float64, device=self.device)
        return self.s.get_q(out)


def local_problem(prob, layout: SlabLayout, r: int):
    """Rank r's local problem: the rows of its window, its y boundary kinds,
    its rows of the per-cell material and bottom arrays.  2D only."""
    if prob.ndim != 2:
        raise ValueError("the slab decomposition splits 2D grids along y")
    idx = layout.global_rows(r)
    ny_loc = len(idx)
    dy = prob.dx[1]
    lo = prob.lower[1] + (layout.rows(r)[0] - layout.halos(r)[0]) * dy
    bc = list(prob.bc)
    bc[2], bc[3] = layout.y_bc(r, prob.bc[2], prob.bc[3])
    kw = dict(n=(prob.n[0], ny_loc), lower=(prob.lower[0], lo), upper=(prob.upper[0], lo + ny_loc * dy),
              bc=tuple(bc), q0=prob.q0[:, idx, :].copy(), cell_width=tuple(prob.dx))
    if prob.rho_cell is not None:
        kw["rho_cell"] = prob.rho_cell[idx, :].copy()
        kw["K_cell"] = prob.K_cell[idx, :].copy()
    if prob.B_cell is not None:
        kw["B_cell"] = prob.B_cell[idx, :].copy()
    return prob.with_(**kw)
