"""The CFL speed pass that allocates nothing, checked against claw_max_speed.

claw_max_speed_noalloc serves callers that cannot allocate device memory --
a framework that owns every byte of device memory through its own pool, or
a loop where an allocation could synchronise the device -- but hold their
state on the GPU already.  It keeps its scratch in a fixed array inside the
library, shared by all calls.  Its result must equal the solver-based
claw_max_speed (same tolerance as the other FP64 parity tests), on two calls
in a row: the second call runs on the scratch the first one left behind.
"""
import numpy as np
import pytest

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


def test_noalloc_speed_pass_matches_claw_max_speed_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    stream = torch.cuda.Stream()
    first = inputs.sw_radial_dam_break(300, ny=211)
    second = inputs.random_problem("acoustics_var", (37, 29, 23), "mc",
                                   ("wall", "periodic", "extrap", "wall", "periodic", "wall"))
    for prob in (first, second):
        want = _solver_value(prob)
        with torch.cuda.stream(stream):
            got = _noalloc_value(torch, prob, stream)
        assert abs(got - want) <= TOL64 * abs(want), (prob.name, got, want)


def test_noalloc_rejects_grids_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    q = torch.zeros(3 * 16, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(L.ClawError) as ei:
        # 2 x 2,100,000 cells: 2.1 M lines along x, more than the scratch holds
        L.claw_max_speed_noalloc((2, 2_100_000), (0.5, 1e-6), "shallow_water", "extrap",
                                 L.make_params(), q, out)
    assert ei.value.status == L.CLAW_EBOUNDS
