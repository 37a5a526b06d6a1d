"""Slab decomposition with the CUDA path as each rank's compute: the ranks
run in one process on one GPU (LocalComm), each slab a `Solver` over its
local grid.  The result must equal one `Solver` over the whole grid taking
the same step sizes (FP64: 1e-12 relative L-inf per field; FP32: the same
kernels on the same data, 1e-6).  Multi-rank transport is covered on CPU
ranks (tests/test_slab_gloo.py)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1805_08846_gb300 import Solver, inputs
from paper_1805_08846_gb300 import slab as S

pytestmark = pytest.mark.gpu


def problem(system, split, ybc, shape=(70, 61), seed=9):
    p = inputs.random_problem(system, shape, "mc", ("extrap", "wall", ybc, ybc), seed=seed,
                              discontinuous=True)
    q0 = p.q0.copy()
    q0[0, shape[1] // 3: shape[1] // 2, :] += 0.4
    return p.with_(q0=q0, splitting=split)


def decomposed(prob, P, k, nsteps, precision):
    layout = S.SlabLayout(prob.n[1], P, 2 * k, prob.bc[2] == "periodic")
    solvers = [Solver.from_problem(S.local_problem(prob, layout, r), precision=precision) for r in range(P)]
    steppers = {r: S.solver_stepper(solvers[r]) for r in range(P)}
    info = S.run_steps(steppers, layout, S.LocalComm(), nsteps, k,
                       cfl_desired=prob.cfl_desired, cfl_max=prob.cfl_max)
    q = S.gather_grid(steppers, layout, S.LocalComm()).cpu().numpy()
    for s in solvers:
        s.close()
    return q, info


def whole(prob, dts, precision):
    with Solver.from_problem(prob, precision=precision) as s:
        for dt in dts:
            s.step(dt)
        return s.get_q()


@pytest.mark.parametrize("system", ["shallow_water", "acoustics_var"])
@pytest.mark.parametrize("split", ["godunov", "strang", "unsplit"])
@pytest.mark.parametrize("ybc", ["periodic", "wall"])
def test_slabs_on_the_gpu_equal_the_whole_grid(system, split, ybc):
    prob = problem(system, split, ybc)
    q, info = decomposed(prob, 3, k=3, nsteps=8, precision=64)
    assert len(info.dts) == 8 and info.periods == 3
    ref = whole(prob, info.dts, 64)
    assert max(oracle.rel_linf(q[f], ref[f]) for f in range(3)) <= 1e-12


def test_slabs_fp32_equal_the_whole_grid():
    prob = problem("shallow_water", "godunov", "periodic", shape=(300, 257))
    q, info = decomposed(prob, 4, k=4, nsteps=10, precision=32)
    ref = whole(prob, info.dts, 32)
    assert max(oracle.rel_linf(q[f], ref[f]) for f in range(3)) <= 1e-6


def test_slabs_match_the_oracle():
    """The decomposed GPU run against the oracle taking the same step sizes."""
    prob = problem("shallow_water", "unsplit", "wall")
    q, info = decomposed(prob, 2, k=2, nsteps=6, precision=64)
    o = oracle.Oracle(prob)
    ref = prob.q0
    for dt in info.dts:
        ref = o.run_steps(ref, 1, fixed_dt=dt)["q"]
    assert max(oracle.rel_linf(q[f], ref[f]) for f in range(3)) <= 1e-12


def test_rows_round_trip_and_fixed_steps_report_their_peak():
    """claw_get_rows / claw_set_rows move exactly the rows asked for (device
    and host buffers); claw_run_fixed_steps keeps every step and reports the
    largest Courant number, as the oracle computes it."""
    prob = problem("shallow_water", "godunov", "wall", shape=(45, 33))
    with Solver.from_problem(prob, precision=64) as s:
        rows = s.get_rows(5, torch.empty(3, 7, 45, dtype=torch.float64, device="cuda")).cpu().numpy()
        np.testing.assert_array_equal(rows, prob.q0[:, 5:12, :])
        new = prob.q0[:, 30:33, :] * 1.01
        dev = torch.from_numpy(new.copy()).cuda()
        torch.cuda.synchronize()            # the solver reads on its own stream
        s.set_rows(30, dev)
        s.set_rows(0, prob.q0[:, 0:2, :] * 0.99)                     # host buffer
        q = s.get_q()
        np.testing.assert_array_equal(q[:, 30:, :], new)
        np.testing.assert_array_equal(q[:, :2, :], prob.q0[:, 0:2, :] * 0.99)
        np.testing.assert_array_equal(q[:, 2:30, :], prob.q0[:, 2:30, :])
        q1 = q.copy()
        peak = s.run_fixed_steps(3, 0.004)
        t, _, n = s.time()
        got = s.get_q()
    assert n == 3 and t == pytest.approx(0.012, rel=1e-15)
    o = oracle.Oracle(prob)
    ref, cfls = q1, []
    for _ in range(3):
        r = o.run_steps(ref, 1, fixed_dt=0.004)
        ref, cfls = r["q"], cfls + [r["cfl"]]
    assert max(oracle.rel_linf(got[f], ref[f]) for f in range(3)) <= 1e-12
    assert peak == pytest.approx(max(cfls), rel=1e-12)


@pytest.mark.parametrize("precision", [64, 32])
def test_checkpoint_and_rollback_are_bitwise(precision):
    """claw_rollback returns to the checkpoint's state and clock exactly, and
    the same steps taken again give the same result bit for bit."""
    from paper_1805_08846_gb300 import ClawError
    prob = problem("shallow_water", "unsplit", "periodic", shape=(64, 50))
    with Solver.from_problem(prob, precision=precision) as s:
        with pytest.raises(ClawError):
            s.rollback()                         # nothing to roll back to yet
        s.run_steps(2)
        q0, t0 = s.get_q(), s.time()
        s.checkpoint()
        s.run_fixed_steps(3, 0.003)
        q1, t1 = s.get_q(), s.time()
        s.rollback()
        np.testing.assert_array_equal(s.get_q(), q0)
        assert s.time() == t0
        s.run_fixed_steps(3, 0.003)
        np.testing.assert_array_equal(s.get_q(), q1)
        assert s.time() == t1
        s.rollback()                             # the same checkpoint again
        np.testing.assert_array_equal(s.get_q(), q0)



@pytest.mark.parametrize("precision", [64, 32])
def test_a_period_whose_courant_number_exceeds_cfl_max_is_redone_on_the_gpu(precision):
    """A radial dam break speeds up as its shock forms: a period of four steps
    at dt = 0.9 / M(start) reaches a Courant number above 1, so the slab loop
    rolls every slab back to its checkpoint (claw_rollback, halo rows
    included) and redoes the period with a smaller step.  The result equals
    one Solver over the whole grid taking the same steps (FP64 to 1e-12, FP32
    bit for bit: the same kernels on the same data)."""
    prob = inputs.sw_radial_dam_break(64, ny=60)
    q, info = decomposed(prob, 2, k=4, nsteps=8, precision=precision)
    assert info.redone > 0, info
    ref = whole(prob, info.dts, precision)
    if precision == 64:
        assert max(oracle.rel_linf(q[f], ref[f]) for f in range(3)) <= 1e-12
    else:
        np.testing.assert_array_equal(q, ref)
