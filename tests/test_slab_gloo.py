"""Slab decomposition of one grid across ranks (host logic), on CPU.

The compute of each rank here is the oracle (it stands in for a rank's GPU);
the decomposition is what is tested: the layout, the halo refresh through an
all-gather, the agreement on the step size, the redo of a period.  A
decomposed run must equal the single grid advanced with the same step sizes,
bitwise, in every owned row (each line's arithmetic is the same; only the
halos differ, and they are refreshed before they could matter).
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1805_08846_gb300 import inputs
from paper_1805_08846_gb300 import slab as S


class OracleStepper:
    """A rank's compute done by the oracle (the state lives in numpy)."""

    def __init__(self, prob):
        import oracle
        self.o = oracle.Oracle(prob)
        self.q = prob.q0.copy()
        self.snap = None

    def get_rows(self, y0, n):
        return torch.from_numpy(self.q[:, y0:y0 + n, :].copy())

    def set_rows(self, y0, rows):
        self.q[:, y0:y0 + rows.shape[1], :] = rows.numpy()

    def max_speed(self):
        return self.o.max_speed_over_dx(self.q)

    def snapshot(self):
        self.snap = self.q.copy()

    def restore(self):
        self.q = self.snap.copy()

    def run_fixed(self, n, dt):
        peak = 0.0
        for _ in range(n):
            r = self.o.run_steps(self.q, 1, fixed_dt=dt)
            self.q = r["q"]
            peak = max(peak, r["cfl"])
        return peak

    def get_q(self):
        return torch.from_numpy(self.q.copy())


def single_grid(prob, dts):
    import oracle
    o = oracle.Oracle(prob)
    q = prob.q0
    for dt in dts:
        q = o.run_steps(q, 1, fixed_dt=dt)["q"]
    return q


def problem(split, ybc, shape=(30, 37), seed=3, system="shallow_water"):
    p = inputs.random_problem(system, shape, "mc", ("extrap", "wall", ybc, ybc),
                              seed=seed, discontinuous=True)
    q0 = p.q0.copy()
    q0[0, shape[1] // 3: shape[1] // 2, :] += 0.4           # a jump across the cuts' rows
    return p.with_(q0=q0, splitting=split)


def run_local(prob, P, k, nsteps, H=None):
    layout = S.SlabLayout(prob.n[1], P, 2 * k if H is None else H, prob.bc[2] == "periodic")
    steppers = {r: OracleStepper(S.local_problem(prob, layout, r)) for r in range(P)}
    info = S.run_steps(steppers, layout, S.LocalComm(), nsteps, k)
    return S.gather_grid(steppers, layout, S.LocalComm()).numpy(), info


def test_layout_covers_rows_and_windows_wrap():
    L = S.SlabLayout(20, 3, 4, True)
    assert [L.rows(r) for r in range(3)] == [(0, 7), (7, 14), (14, 20)]
    assert L.global_rows(0)[:4] == [16, 17, 18, 19] and L.global_rows(2)[-4:] == [0, 1, 2, 3]
    assert all(L.halos(r) == (4, 4) for r in range(3))
    W = S.SlabLayout(20, 3, 4, False)
    assert W.halos(0) == (0, 4) and W.halos(2) == (4, 0)
    assert W.y_bc(0, "wall", "wall") == ("wall", "extrap") and W.y_bc(1, "wall", "wall") == ("extrap", "extrap")
    one = S.SlabLayout(20, 1, 4, True)
    assert one.halos(0) == (0, 0) and one.y_bc(0, "periodic", "periodic") == ("periodic", "periodic")
    with pytest.raises(ValueError):
        S.SlabLayout(10, 4, 3, False)      # slabs of 2-3 rows cannot feed a 3-row halo
    assert S.SlabLayout(10, 1, 16, False).halos(0) == (0, 0)   # one rank: the halo is unused


class TensorStepper:
    """Holds a local state; steps change nothing (a Courant number of
    `speed` dt)."""

    def __init__(self, q, speed=0.0, max_speed=1.0):
        self.q, self.speed, self.M = q.clone(), speed, max_speed
        self.snap = None

    def get_rows(self, y0, n):
        return self.q[:, y0:y0 + n, :].clone()

    def set_rows(self, y0, rows):
        self.q[:, y0:y0 + rows.shape[1], :] = rows

    def max_speed(self):
        return self.M

    def snapshot(self):
        self.snap = self.q.clone()

    def restore(self):
        self.q = self.snap.clone()

    def run_fixed(self, n, dt):
        return self.speed * dt

    def get_q(self):
        return self.q.clone()


@pytest.mark.parametrize("periodic", [True, False])
def test_refresh_writes_the_neighbours_rows(periodic):
    rng = np.random.default_rng(5)
    q = torch.from_numpy(rng.normal(size=(3, 23, 6)))
    L = S.SlabLayout(23, 3, 3, periodic)
    steppers = {r: TensorStepper(S.local_window(q, L, r)) for r in range(3)}
    for r, st in steppers.items():           # stale halos
        hl, hu = L.halos(r)
        st.q[:, :hl, :] = -1.0
        st.q[:, st.q.shape[1] - hu:, :] = -1.0
    S.refresh_halos(steppers, L, S.LocalComm())
    for r in range(3):
        np.testing.assert_array_equal(steppers[r].q.numpy(), S.local_window(q, L, r).numpy())
    np.testing.assert_array_equal(S.gather_grid(steppers, L, S.LocalComm()).numpy(), q.numpy())


def test_a_period_above_cfl_max_is_redone_with_a_smaller_step():
    """max_speed 1 gives dt = 0.9; inside the period the speed is 1.5, so the
    first try has Courant number 1.35 > 1 and is redone at 0.9 * 0.9 / 1.35.
    The later periods take their speed from the period before (Courant
    number 0.9 at dt 0.6: speed 1.5), so they start at that step and keep it."""
    L = S.SlabLayout(12, 2, 2, False)
    steppers = {r: TensorStepper(torch.zeros(3, L.local_rows(r), 4, dtype=torch.float64), speed=1.5)
                for r in range(2)}
    info = S.run_steps(steppers, L, S.LocalComm(), nsteps=3, k=1)
    assert info.redone == 1 and info.periods == 3
    assert info.dts == pytest.approx([0.9 * 0.9 / 1.35] * 3)
    assert info.cfl_max_seen == pytest.approx(0.9)


def test_halo_too_narrow_for_the_period_is_rejected():
    L = S.SlabLayout(20, 2, 3, False)
    steppers = {r: TensorStepper(torch.zeros(3, L.local_rows(r), 4, dtype=torch.float64)) for r in range(2)}
    with pytest.raises(ValueError):
        S.run_steps(steppers, L, S.LocalComm(), nsteps=2, k=2)


@pytest.mark.parametrize("split", ["godunov", "unsplit", "strang"])
@pytest.mark.parametrize("ybc", ["periodic", "wall"])
def test_three_slabs_in_one_process_equal_the_single_grid(split, ybc):
    prob = problem(split, ybc)
    q, info = run_local(prob, 3, k=2, nsteps=5)
    assert info.periods == 3 and len(info.dts) == 5
    np.testing.assert_array_equal(q, single_grid(prob, info.dts))


@pytest.mark.parametrize("system,split", [("acoustics_var", "godunov"), ("acoustics_var", "unsplit"),
                                          ("shallow_water_bathy", "strang")])
def test_slabs_carry_their_rows_of_the_material_arrays(system, split):
    """Per-cell rho, K and the bottom elevation are cut into the slabs with
    their halos: the decomposed run still equals the single grid."""
    prob = problem(split, "periodic", system=system)
    q, info = run_local(prob, 3, k=2, nsteps=4)
    np.testing.assert_array_equal(q, single_grid(prob, info.dts))


def test_a_halo_narrower_than_two_rows_per_step_differs():
    """The exactness needs H >= 2k: one step with a one-row halo already
    changes owned rows next to the cuts (the stencil reaches two rows)."""
    prob = problem("godunov", "wall")
    layout = S.SlabLayout(prob.n[1], 2, 1, False)
    steppers = {r: OracleStepper(S.local_problem(prob, layout, r)) for r in range(2)}
    S.refresh_halos(steppers, layout, S.LocalComm())
    for st in steppers.values():
        st.run_fixed(1, 0.002)
    q = S.gather_grid(steppers, layout, S.LocalComm()).numpy()
    assert np.abs(q - single_grid(prob, [0.002])).max() > 1e-8


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir, split, ybc):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        prob = problem(split, ybc)
        layout = S.SlabLayout(prob.n[1], world, 4, ybc == "periodic")
        steppers = {rank: OracleStepper(S.local_problem(prob, layout, rank))}
        info = S.run_steps(steppers, layout, S.DistComm(), nsteps=7, k=2)
        q = S.gather_grid(steppers, layout, S.DistComm())
        if rank == 0:
            np.savez(os.path.join(out_dir, "slab.npz"), q=q.numpy(),
                     dts=np.array(info.dts), t=np.array(info.t))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("split,ybc", [("godunov", "periodic"), ("unsplit", "wall")])
def test_two_gloo_ranks_equal_the_single_grid(tmp_path, split, ybc):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path), split, ybc),
                       nprocs=world, join=True, start_method="spawn")
    out = np.load(os.path.join(tmp_path, "slab.npz"))
    prob = problem(split, ybc)
    assert len(out["dts"]) == 7
    np.testing.assert_array_equal(out["q"], single_grid(prob, list(out["dts"])))
    assert float(out["t"]) == pytest.approx(sum(out["dts"]), rel=1e-15)
