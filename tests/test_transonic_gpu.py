"""Parity of the CUDA path with the oracle where the Harten-Hyman entropy fix
acts: shallow-water dam breaks with a depth ratio of 10, whose rarefaction
fans span the initial jump (transonic 1-waves, and 3-waves in the mirrored
cases), along x, along y, and radially (both waves in both directions).

Every case first counts, on the oracle's states along the run, the
interfaces with a transonic 1- or 3-wave (lam_l < 0 < lam_m, or
lam_m < 0 < lam_r, at the Roe middle state), so a case cannot silently go
subsonic.  Then the CUDA path, through the C ABI, must match the oracle:
FP64 to 1e-12 relative L-inf per field, FP32 to 1e-4 relative L1 on h (and
on hu, hv) -- in the split sweeps (Godunov and Strang), the unsplit update
and an ensemble instance, with every limiter.
"""
import numpy as np
import pytest

import oracle
from paper_1805_08846_gb300 import Ensemble, Solver, inputs
from tests.transonic import oracle_run_counting

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-4
NSTEPS = 15

# name -> (problem factory, (direction, wave) pairs that must be transonic)
CASES = {
    "x": (lambda lim: inputs.sw_transonic_dam_break(120, 4, axis=0, limiter=lim), [(0, 1)]),
    "x_mirror": (lambda lim: inputs.sw_transonic_dam_break(120, 4, axis=0, mirror=True, limiter=lim),
                 [(0, 3)]),
    "y": (lambda lim: inputs.sw_transonic_dam_break(120, 4, axis=1, limiter=lim), [(1, 1)]),
    "y_mirror": (lambda lim: inputs.sw_transonic_dam_break(120, 4, axis=1, mirror=True, limiter=lim),
                 [(1, 3)]),
    "radial": (lambda lim: inputs.sw_radial_dam_break(48, ny=40, limiter=lim, h_in=1.0, h_out=0.1),
               [(0, 1), (0, 3), (1, 1), (1, 3)]),
}

_ORACLE = {}


def reference(name, limiter, splitting):
    """Oracle run of a case (cached) after checking that it is transonic."""
    key = (name, limiter, splitting)
    if key not in _ORACLE:
        make, must = CASES[name]
        prob = make(limiter).with_(splitting=splitting)
        ref, counts = oracle_run_counting(prob, NSTEPS)
        for dw in must:
            assert counts[dw] > 0, (key, counts)
        _ORACLE[key] = (prob, ref)
    return _ORACLE[key]


def check(prob, q, ref, precision):
    if precision == 64:
        err = max(oracle.rel_linf(q[f], ref["q"][f]) for f in range(3))
        assert err <= TOL64, err
    else:
        errs = [oracle.rel_l1(q[f], ref["q"][f]) for f in range(3)]
        assert max(errs) <= TOL32, errs


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("limiter", ["none", "minmod", "mc", "first_order"])
@pytest.mark.parametrize("name", list(CASES))
def test_transonic_godunov(name, limiter, precision):
    prob, ref = reference(name, limiter, "godunov")
    with Solver.from_problem(prob, precision=precision) as s:
        s.run_steps(NSTEPS)
        q = s.get_q()
        t, dt, n = s.time()
    assert n == NSTEPS
    check(prob, q, ref, precision)
    assert t == pytest.approx(ref["t"], rel=1e-13 if precision == 64 else 1e-5)


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("limiter", ["minmod", "mc"])
@pytest.mark.parametrize("splitting", ["strang", "unsplit"])
@pytest.mark.parametrize("name", list(CASES))
def test_transonic_strang_and_unsplit(name, splitting, limiter, precision):
    prob, ref = reference(name, limiter, splitting)
    with Solver.from_problem(prob, precision=precision) as s:
        s.run_steps(NSTEPS)
        q = s.get_q()
    check(prob, q, ref, precision)


@pytest.mark.parametrize("precision", [64, 32])
def test_transonic_radial_several_tiles(precision):
    """A radial case large enough for several tiles and ragged tails."""
    prob = inputs.sw_radial_dam_break(150, ny=130, limiter="mc", h_in=1.0, h_out=0.1)
    ref, counts = oracle_run_counting(prob, 10, chunks=2)
    assert min(counts.values()) > 0, counts
    with Solver.from_problem(prob, precision=precision) as s:
        s.run_steps(10)
        q = s.get_q()
    check(prob, q, ref, precision)


@pytest.mark.parametrize("precision", [64, 32])
def test_transonic_ensemble_instance(precision):
    """Ensemble of a transonic radial dam break beside subsonic and mirrored
    instances of other sizes; every instance against its own oracle run."""
    probs = [inputs.sw_radial_dam_break(48, ny=40, limiter="minmod", h_in=1.0, h_out=0.1),
             inputs.random_problem("shallow_water", (70, 40), "minmod", "extrap", discontinuous=True),
             inputs.sw_radial_dam_break(40, ny=48, limiter="minmod", h_in=0.1, h_out=1.0)]
    refs = []
    for k, p in enumerate(probs):
        ref, counts = oracle_run_counting(p, NSTEPS)
        if k != 1:
            assert min(counts.values()) > 0, (p.name, counts)
        refs.append(ref)
    e = Ensemble.from_problems(probs, precision=precision)
    try:
        e.run_steps(NSTEPS)
        for i, p in enumerate(probs):
            check(p, e.get_q(i), refs[i], precision)
    finally:
        e.close()
