"""The transonic parity inputs really reach the entropy fix (CPU only).

The GPU parity cases of tests/test_transonic_gpu.py are only worth having if
their states contain transonic rarefactions; this checks, on the oracle's
own run, that each case has the transonic 1- or 3-wave interfaces it is
meant to have, and that the subsonic workloads of the other parity tests
have none (which is why these cases exist).
"""
import pytest

from paper_1805_08846_gb300 import inputs
from tests.transonic import oracle_run_counting, transonic_counts


@pytest.mark.parametrize("axis,mirror,wave", [(0, False, 1), (0, True, 3), (1, False, 1), (1, True, 3)])
def test_planar_transonic_dam_breaks(axis, mirror, wave):
    prob = inputs.sw_transonic_dam_break(120, 4, axis=axis, mirror=mirror, limiter="minmod")
    _, counts = oracle_run_counting(prob, 15)
    assert counts[(axis, wave)] > 0, counts
    # the other wave family and the direction across the jump stay subsonic
    assert counts[(axis, 4 - wave)] == 0 and counts[(1 - axis, 1)] == counts[(1 - axis, 3)] == 0, counts


def test_radial_transonic_dam_break_in_both_directions():
    prob = inputs.sw_radial_dam_break(48, ny=40, limiter="mc", h_in=1.0, h_out=0.1)
    _, counts = oracle_run_counting(prob, 15)
    assert min(counts.values()) > 0, counts


def test_the_other_parity_workloads_are_subsonic():
    for prob in (inputs.random_problem("shallow_water", (37, 29), "mc", "periodic", discontinuous=True),
                 inputs.sw_radial_dam_break(64)):
        assert sum(transonic_counts(prob, prob.q0).values()) == 0
