"""The CFL speed pass that allocates nothing, checked against the oracle and claw_max_speed.

claw_max_speed_noalloc serves callers that cannot allocate device memory --
a framework that owns every byte of device memory through its own pool, or
a loop where an allocation could synchronise the device -- but hold their
state on the GPU already.  It keeps its scratch in a fixed array inside the
library, shared by all calls on a device.  Its result must equal the
oracle's CFL speed max_d(max|s| / dx_d) of the same state and the
solver-based claw_max_speed (same tolerance as the other FP64 parity tests),
on calls in a row: each call runs on the scratch the one before left behind.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_1805_08846_gb300 import Solver, inputs
from paper_1805_08846_gb300 import _lib as L

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def _solver_value(prob):
    with Solver.from_problem(prob, precision=64) as s:
        return s.max_speed()


def _noalloc_value(torch, prob, stream):
    q = torch.from_numpy(np.ascontiguousarray(prob.q0)).cuda()
    rho = K = None
    if prob.system == "acoustics_var":
        rho = torch.from_numpy(np.ascontiguousarray(prob.rho_cell)).cuda()
        K = torch.from_numpy(np.ascontiguousarray(prob.K_cell)).cuda()
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    params = L.make_params(rho=prob.rho, K=prob.K, g=prob.g, precision=64)
    L.claw_max_speed_noalloc(prob.n, prob.dx, prob.system, prob.bc, params, q, out, rho, K,
                             stream=stream)
    torch.cuda.synchronize()
    return float(out.item())


def test_noalloc_speed_pass_matches_the_oracle_and_claw_max_speed_on_calls_in_a_row():
    torch = pytest.importorskip("torch")
    stream = torch.cuda.Stream()
    # shallow water, variable-coefficient 3D acoustics, constant-coefficient
    # acoustics (2D and 3D): every solver branch of the speed pass, each call
    # on the scratch the previous one left behind
    probs = [inputs.sw_radial_dam_break(300, ny=211),
             inputs.random_problem("acoustics_var", (37, 29, 23), "mc",
                                   ("wall", "periodic", "extrap", "wall", "periodic", "wall")),
             inputs.acoustics_2d_pulse(130, ny=70, K=4.0),
             inputs.random_problem("acoustics", (21, 19, 33), "mc", "periodic")]
    for prob in probs:
        want = Oracle(prob).max_speed_over_dx(prob.q0)
        with torch.cuda.stream(stream):
            got = _noalloc_value(torch, prob, stream)
        assert abs(got - want) <= TOL64 * abs(want), (prob.name, got, want)
        assert abs(got - _solver_value(prob)) <= TOL64 * abs(want), prob.name


def test_noalloc_rejects_grids_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    q = torch.zeros(3 * 16, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(L.ClawError) as ei:
        # 2 x 2,100,000 cells: 2.1 M lines along x, more than the scratch holds
        L.claw_max_speed_noalloc((2, 2_100_000), (0.5, 1e-6), "shallow_water", "extrap",
                                 L.make_params(), q, out)
    assert ei.value.status == L.CLAW_EBOUNDS
