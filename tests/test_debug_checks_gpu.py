"""The checked library (CLAW_DEBUG=1: every direct global access and bulk-copy
coordinate of the kernels is bounds-checked on the device, a failure reported
as CLAW_EBOUNDS) runs a matrix of small cases -- every system, splitting and
limiter family, both precisions, grids with ragged tiles, strips and
segments, both tile widths, tiny grids, ensembles, row access -- and must
report no failed check and still match the oracle.  It stands in for a
memory checker, which this pool does not offer.  The cases run in a child process, which loads
the checked library instead of the release one."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [
    # system, shape (x, y[, z]), limiter, bc, splitting
    ("shallow_water", (37, 29), "minmod", "extrap", "godunov"),
    ("shallow_water", (73, 20), "mc", ("periodic", "periodic", "wall", "extrap"), "strang"),
    ("shallow_water", (2, 5), "minmod", "wall", "godunov"),
    ("shallow_water", (61, 45), "mc", "wall", "unsplit"),
    ("shallow_water", (29, 2), "none", "periodic", "unsplit"),
    ("acoustics", (130, 67), "mc", ("wall", "extrap", "periodic", "wall"), "godunov"),
    ("acoustics", (129, 11), "first_order", "wall", "unsplit"),
    ("acoustics_var", (23, 19, 21), "mc", "wall", "godunov"),
    ("acoustics_var", (3, 2, 2), "mc", "periodic", "strang"),
    ("acoustics_var", (57, 83), "minmod", "periodic", "unsplit"),
    ("shallow_water_bathy", (44, 31), "mc", ("periodic", "periodic", "wall", "extrap"), "godunov"),
    ("shallow_water_dry", (45, 38), "mc", "wall", "godunov"),
    ("shallow_water_dry", (70, 20), "minmod", ("periodic", "periodic", "wall", "extrap"), "strang"),
]
# cases also run with narrow tiles (64 lines where offered), 8-cell segments
# and the list order
NARROW = {("acoustics_var", (23, 19, 21)), ("shallow_water", (37, 29)), ("shallow_water_dry", (45, 38))}


def run_cases():
    import oracle
    from oracle import Oracle
    from paper_1805_08846_gb300 import Ensemble, Solver, inputs
    from paper_1805_08846_gb300 import _lib as L
    assert L.debug_build() and L.library_path().endswith(os.path.join("_build_debug", "libclaw.so"))
    n = 0
    for system, shape, lim, bc, split in CASES:
        prob = inputs.random_problem(system, shape, lim, bc, discontinuous=True).with_(splitting=split)
        ref = Oracle(prob).run_steps(prob.q0, 6)["q"]
        shapes = [(0, 8, 0)] + ([(64, 8, 1)] if (system, shape) in NARROW else [])
        for precision in (64, 32):
            for lines, seg, order in shapes:
                with Solver.from_problem(prob, precision=precision) as s:
                    for d in range(prob.ndim):
                        if split != "unsplit":
                            s.set_tile_shape(d, lines, seg, order)   # many tiles and segment ends
                        else:
                            s.set_segment(d, seg)
                    s.run_steps(6)
                    q = s.get_q()
                if precision == 32 and system == "shallow_water_dry":
                    # wet / dry decisions taken in FP32: an L1 bound
                    err = max(oracle.rel_l1(q[f], ref[f]) for f in range(q.shape[0]))
                    assert err <= 1e-4, (system, shape, split, precision, err)
                else:
                    err = max(oracle.rel_linf(q[f], ref[f]) for f in range(q.shape[0]))
                    assert err <= (1e-12 if precision == 64 else 2e-3), (system, shape, split, precision, err)
                n += 1
    for probs in (inputs.sw_ensemble(B=4, nmin=9, nmax=70, nsteps=4),
                  inputs.acoustics3d_ensemble(B=3, nmin=6, nmax=20, nsteps=4)):
        e = Ensemble.from_problems(probs, precision=32)
        e.run_steps(4)
        for i, p in enumerate(probs):
            ref = Oracle(p).run_steps(p.q0, 4)["q"]
            q = e.get_q(i)
            assert max(oracle.rel_linf(q[f], ref[f]) for f in range(q.shape[0])) <= 2e-3
            n += 1
        e.close()
    prob = inputs.random_problem("shallow_water", (45, 33), "mc", "wall")
    with Solver.from_problem(prob, precision=32) as s:
        rows = s.get_rows(31, np.empty((3, 2, 45)))
        s.set_rows(0, rows)
        s.run_fixed_steps(3, 0.002)
        s.get_q()
        n += 1
    print(f"checked library: {n} cases, no failed check", flush=True)


def test_checked_library_reports_no_failed_check():
    env = dict(os.environ, CLAW_DEBUG="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__)], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "no failed check" in r.stdout


if __name__ == "__main__":
    sys.path.insert(0, ROOT)
    run_cases()
