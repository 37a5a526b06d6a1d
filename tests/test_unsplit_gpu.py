"""Parity of the unsplit update with transverse waves (CUDA path through the
C ABI) with the FP64 CPU oracle.

Tolerances as for the split step: the FP64 path to 1e-12 relative L-inf per
field; the FP32 form to 1e-5 relative L2 (acoustics) and 1e-4 relative L1 on
h (shallow water).  Grids are chosen so that the 28-column strips of the
kernel end ragged (x extents not multiples of 28, some below one strip) and
the row segments end ragged; the initial data carry a jump along x and one
along y so both limiters and both transverse splits see discontinuities.
"""
import numpy as np
import pytest

import oracle
from oracle import Oracle
from paper_1805_08846_gb300 import ClawError, Ensemble, Solver, inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def fieldwise(a, b):
    """Largest relative L-inf error over the fields, and where it sits."""
    worst = (0.0, None)
    for f in range(a.shape[0]):
        e = oracle.rel_linf(a[f], b[f])
        if e > worst[0]:
            worst = (e, (f,) + np.unravel_index(np.argmax(np.abs(a[f] - b[f])), a[f].shape))
    return worst


def unsplit_problem(system, shape, limiter, bc, seed=inputs.SEED):
    p = inputs.random_problem(system, shape, limiter, bc, seed=seed, discontinuous=True)
    q0 = p.q0.copy()
    ny = q0.shape[1]
    q0[0, ny // 4: (3 * ny) // 4, :] += 0.3          # a jump along y as well
    return p.with_(q0=q0, splitting="unsplit")


def check(prob, q, ref, precision):
    if precision == 64:
        err, where = fieldwise(q, ref)
        assert err <= TOL64, (err, where)
    elif prob.system == "shallow_water":
        err = oracle.rel_l1(q[0], ref[0])
        assert err <= 1e-4, err
    else:
        err = max(oracle.rel_l2(q[f], ref[f]) for f in range(q.shape[0]) if np.abs(ref[f]).max() > 0)
        assert err <= 1e-5, err


def run_both(prob, nsteps, precision, seg=None):
    ref = Oracle(prob).run_steps(prob.q0, nsteps)
    with Solver.from_problem(prob, precision=precision) as s:
        if seg is not None:
            s.set_segment(1, seg)
        s.run_steps(nsteps)
        q = s.get_q()
        t, dt, n = s.time()
    return q, (t, dt, n), ref


CASES = []
for system in ("acoustics", "acoustics_var", "shallow_water"):
    for limiter in ("none", "minmod", "mc", "first_order"):
        CASES.append((system, (61, 45), limiter, "periodic"))
    CASES += [(system, (37, 29), "mc", "wall"),
              (system, (131, 67), "minmod", "extrap"),
              (system, (57, 83), "mc", ("wall", "extrap", "periodic", "wall")),
              (system, (2, 5), "minmod", "wall"),
              (system, (29, 2), "mc", "periodic"),
              (system, (5, 40), "none", ("extrap", "periodic", "wall", "wall"))]


@pytest.mark.parametrize("system,shape,limiter,bc", CASES)
@pytest.mark.parametrize("precision", [64, 32])
def test_unsplit_matches_oracle(system, shape, limiter, bc, precision):
    prob = unsplit_problem(system, shape, limiter, bc)
    q, (t, dt, n), ref = run_both(prob, 10, precision)
    assert n == 10
    check(prob, q, ref["q"], precision)
    assert t == pytest.approx(ref["t"], rel=1e-13 if precision == 64 else 1e-5)


@pytest.mark.parametrize("seg", [8, 16, 24, 1000])
def test_unsplit_row_segments_do_not_change_the_result(seg):
    prob = unsplit_problem("shallow_water", (70, 53), "mc", ("periodic", "wall", "extrap", "wall"))
    q, _, ref = run_both(prob, 6, 64, seg=seg)
    err, where = fieldwise(q, ref["q"])
    assert err <= TOL64, (err, where)


def test_unsplit_advance_and_cfl_redo_match_oracle():
    """Advance to t_final under the CFL rule, with a first step at Courant
    number 1.5 that the step control must redo."""
    prob = unsplit_problem("acoustics", (45, 38), "mc", "wall")
    dt0 = 1.5 / Oracle(prob).max_speed_over_dx(prob.q0)
    ref = Oracle(prob).advance(prob.q0, 0.07, dt=dt0)
    with Solver.from_problem(prob, precision=64) as s:
        s.set_time(0.0, dt0, 0)
        s.advance(0.07)
        q = s.get_q()
        t, _, n = s.time()
        assert s.rejections() == ref["nrej"] >= 1
    assert n == ref["nacc"] and t == 0.07
    err, where = fieldwise(q, ref["q"])
    assert err <= TOL64, (err, where)


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("bc", ["periodic", "extrap", "wall"])
def test_unsplit_lake_at_rest_bitwise(precision, bc):
    prob = unsplit_problem("shallow_water", (61, 47), "mc", bc)
    q0 = np.zeros_like(prob.q0)
    q0[0] = 1.25
    prob = prob.with_(q0=q0)
    with Solver.from_problem(prob, precision=precision) as s:
        s.run_steps(10)
        q = s.get_q()
    np.testing.assert_array_equal(q, q0)


@pytest.mark.parametrize("bc", ["periodic", "wall"])
def test_unsplit_conserves_mass(bc):
    prob = unsplit_problem("shallow_water", (90, 64), "minmod", bc)
    with Solver.from_problem(prob, precision=64) as s:
        m0 = s.sums()[0]
        s.run_steps(20)
        m1 = s.sums()[0]
    assert abs(m1 - m0) <= 1e-13 * m0


def test_unsplit_ensemble_matches_oracle_per_instance():
    probs = [p.with_(splitting="unsplit") for p in inputs.sw_ensemble(B=5, nmin=16, nmax=90, nsteps=8)]
    for precision in (64, 32):
        e = Ensemble.from_problems(probs, precision=precision)
        e.run_steps(8)
        for i, p in enumerate(probs):
            ref = Oracle(p).run_steps(p.q0, 8)
            check(p, e.get_q(i), ref["q"], precision)
            assert e.time(i)[0] == pytest.approx(ref["t"], rel=1e-13 if precision == 64 else 1e-5)
        e.close()


def test_unsplit_autotune_keeps_state_and_result():
    prob = unsplit_problem("shallow_water", (200, 150), "minmod", "extrap")
    ref = Oracle(prob).run_steps(prob.q0, 4)
    with Solver.from_problem(prob, 64) as s:
        before = s.time()
        seg = s.autotune(2)
        assert s.time() == before
        s.run_steps(4)
        q = s.get_q()
    assert seg[1] >= 8
    err, where = fieldwise(q, ref["q"])
    assert err <= TOL64, (err, where)


def test_unsplit_rejects_3d_and_bathymetry():
    p3 = inputs.random_problem("acoustics", (9, 8, 7), "mc", "wall").with_(splitting="unsplit")
    with pytest.raises(ClawError):
        Solver.from_problem(p3)
    pb = inputs.random_problem("shallow_water_bathy", (9, 8), "mc", "wall").with_(splitting="unsplit")
    with pytest.raises(ClawError):
        Solver.from_problem(pb)


@pytest.fixture(scope="module")
def dam_break_4096():
    prob = inputs.sw_radial_dam_break(4096).with_(splitting="unsplit")
    return prob, Oracle(prob).run_steps(prob.q0, 3)


@pytest.mark.parametrize("precision", [64, 32])
def test_unsplit_radial_dam_break_4096(precision, dam_break_4096):
    """The 4096^2 radial dam break (minmod, outflow) for 3 unsplit steps in
    the benchmark's launch configuration (autotuned row segments)."""
    prob, ref = dam_break_4096
    with Solver.from_problem(prob, precision=precision) as s:
        s.autotune(2)
        s.run_steps(3)
        q = s.get_q()
        t, _, n = s.time()
    assert n == 3 and t == pytest.approx(ref["t"], rel=1e-13 if precision == 64 else 1e-5)
    if precision == 64:
        err, where = fieldwise(q, ref["q"])
        assert err <= TOL64, (err, where)
    else:
        assert oracle.rel_l1(q[0], ref["q"][0]) <= 1e-4
        assert oracle.rel_l1(q[0] - 1.0, ref["q"][0] - 1.0) <= 1e-3
