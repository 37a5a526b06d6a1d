"""Parity of the CUDA path with the oracle for shallow water with wetting and
drying (CLAW_SHALLOW_WATER_DRY: hydrostatic reconstruction around HLLE, dry
cells h <= dry_tol), through the C ABI.

FP64 to 1e-12 relative L-inf per field; FP32 to 1e-4 relative L1 on h (and
on hu, hv).  Cases: Ritter's dam break onto a dry bed along x and along y,
every limiter; random bottoms with an emerged ridge on odd grids spanning
several tiles with ragged tails, every boundary kind; a wave running up an
island and a beach; Strang splitting; an ensemble.  Invariants on the GPU: a
lake at rest around an emerged island stays bitwise at rest in both
precisions, the depth never goes negative, mass is conserved with walls.
"""
import numpy as np
import pytest

import oracle
from oracle import Oracle
from paper_1805_08846_gb300 import Ensemble, Solver, inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-4


def check(q, ref, precision):
    if precision == 64:
        err = max(oracle.rel_linf(q[f], ref[f]) for f in range(3))
        assert err <= TOL64, err
    else:
        errs = [oracle.rel_l1(q[f], ref[f]) for f in range(3)]
        assert max(errs) <= TOL32, errs
    assert q[0].min() >= 0.0


def run_both(prob, nsteps, precision):
    ref = Oracle(prob).run_steps(prob.q0, nsteps)
    with Solver.from_problem(prob, precision=precision) as s:
        s.run_steps(nsteps)
        q = s.get_q()
        t, dt, n = s.time()
    assert n == nsteps
    assert t == pytest.approx(ref["t"], rel=1e-13 if precision == 64 else 1e-5)
    return q, ref["q"]


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("limiter", ["none", "minmod", "mc", "first_order"])
@pytest.mark.parametrize("axis", [0, 1])
def test_ritter_dam_break(axis, limiter, precision):
    prob = inputs.sw_dry_dam_break(150, 5, axis=axis, limiter=limiter)
    q, ref = run_both(prob, 30, precision)
    check(q, ref, precision)


CASES = [((37, 29), "mc", "wall"), ((37, 29), "minmod", "periodic"), ((37, 29), "none", "extrap"),
         ((131, 70), "mc", ("extrap", "wall", "periodic", "periodic")),
         ((73, 20), "first_order", ("periodic", "periodic", "wall", "extrap")),
         ((150, 131), "minmod", "wall")]


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("shape,limiter,bc", CASES)
def test_random_bottom_with_an_emerged_ridge(shape, limiter, bc, precision):
    prob = inputs.random_problem("shallow_water_dry", shape, limiter, bc, discontinuous=True)
    assert (prob.q0[0] == 0.0).sum() > 0
    q, ref = run_both(prob, 12, precision)
    check(q, ref, precision)


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("bc", ["periodic", "extrap", "wall"])
@pytest.mark.parametrize("limiter", ["minmod", "mc"])
def test_lake_at_rest_around_an_island_bitwise(limiter, bc, precision):
    """B and h are multiples of 2^-24 below 1, exact in FP32 too."""
    prob = inputs.sw_island(96, 80, limiter=limiter, bc=bc, hump=0.0)
    with Solver.from_problem(prob, precision=precision) as s:
        s.run_steps(10)
        q = s.get_q()
    np.testing.assert_array_equal(q, prob.q0)


@pytest.mark.parametrize("precision", [64, 32])
def test_island_run_up(precision):
    prob = inputs.sw_island(120, 100, limiter="mc", bc="wall", hump=0.3)
    q, ref = run_both(prob, 40, precision)
    check(q, ref, precision)
    # mass conserved with walls, through the device's FP64 sums
    with Solver.from_problem(prob, precision=64) as s:
        m0 = s.sums()[0]
        s.run_steps(40)
        m1 = s.sums()[0]
    assert abs(m1 - m0) <= 1e-13 * m0


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("limiter", ["minmod", "mc"])
def test_beach_run_up_floods_and_drains(limiter, precision):
    prob = inputs.sw_beach(200, 12, limiter=limiter)
    q, ref = run_both(prob, 160, precision)
    check(q, ref, precision)
    flooded = (prob.q0[0] == 0.0) & (ref[0] > prob.dry_tol)
    assert flooded.sum() > 0


@pytest.mark.parametrize("precision", [64, 32])
def test_strang_splitting_with_dry_cells(precision):
    prob = inputs.random_problem("shallow_water_dry", (64, 45), "mc", "wall", discontinuous=True)
    q, ref = run_both(prob.with_(splitting="strang"), 10, precision)
    check(q, ref, precision)


@pytest.mark.parametrize("precision", [64, 32])
def test_ensemble_with_dry_cells(precision):
    probs = [inputs.random_problem("shallow_water_dry", (n, n + 7), "minmod", "wall", seed=s,
                                   discontinuous=True)
             for s, n in ((3, 30), (4, 77), (5, 51))]
    e = Ensemble.from_problems(probs, precision=precision)
    try:
        e.run_steps(10)
        for i, p in enumerate(probs):
            ref = Oracle(p).run_steps(p.q0, 10)
            check(e.get_q(i), ref["q"], precision)
    finally:
        e.close()


def test_unsplit_update_rejects_dry_states():
    from paper_1805_08846_gb300 import ClawError
    prob = inputs.sw_island(32, 32, hump=0.0).with_(splitting="unsplit")
    with pytest.raises(ClawError):
        Solver.from_problem(prob, precision=64)
