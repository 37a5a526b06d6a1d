"""Pins for the oracle's shallow water with wetting and drying
(shallow_water_dry: the bathymetry source of Sec. 3's Clawpack base, Eq. SW,
with dry cells, h <= dry_tol).  The paper is silent on dry states; the
reading is the HLLE solver with Einfeldt's speeds, the dry-bed front speed
u -/+ 2c, a wall where a dry bed rises above the neighbouring surface, and no
second-order correction at the shoreline.  Each pin is fixed by the
mathematics, not by the oracle's code: flux and jump identities, positivity
of the HLLE middle state, the exact dry-bed front speed, zero mass flux
through a wall, Ritter's exact solution, a lake at rest around an island,
mass conservation and non-negative depth on a beach.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import Oracle
from paper_1805_08846_gb300 import inputs
from tests.exact_sw import ritter_profile

G = 9.81
TOL = 1e-3


def sw_flux(q, g=G):
    h, hu, hv = q
    if h <= TOL:
        return np.array([0.0, 0.5 * g * h * h, 0.0])
    return np.array([hu, hu * hu / h + 0.5 * g * h * h, hu * hv / h])


def delta_of(ql, qr, B_l, B_r, g=G):
    """f(Q_r) - f(Q_l) - psi, psi = (0, -g h_bar (B_r - B_l), 0)."""
    hbar = 0.5 * (ql[0] + qr[0])
    return sw_flux(qr) - sw_flux(ql) - np.array([0.0, -g * hbar * (B_r - B_l), 0.0])


def rp(ql, qr, B_l=0.0, B_r=0.0):
    return oracle.riemann("shallow_water_dry", np.asarray(ql, float), np.asarray(qr, float),
                          B_l=B_l, B_r=B_r, dry_tol=TOL)


def random_wet_pair(rng):
    hl, hr = rng.uniform(0.05, 3.0, size=2)
    ul, ur, vl, vr = rng.uniform(-3.0, 3.0, size=4)
    return np.array([hl, hl * ul, hl * vl]), np.array([hr, hr * ur, hr * vr])


# ---------------------------------------------------------------- Riemann solver

def test_flat_bottom_wet_pairs_are_hlle():
    """On a flat bottom (no reconstruction) between wet cells the waves sum to
    the jump dQ, the speeds times the waves to the flux jump f(Q_r) - f(Q_l)
    (HLL consistency), the fluctuations add up to the flux jump, and the
    outer speeds bound the characteristic speeds of both cells (Einfeldt)."""
    rng = np.random.default_rng(71)
    for _ in range(300):
        ql, qr = random_wet_pair(rng)
        B = rng.uniform(-0.5, 0.5)
        W, s, am, ap = rp(ql, qr, B, B)
        df = sw_flux(qr) - sw_flux(ql)
        scale = np.abs(df).max() + np.abs(qr).max() + 1.0
        np.testing.assert_allclose(W.sum(0), qr - ql, atol=1e-13 * scale)
        np.testing.assert_allclose((s[:, None] * W).sum(0), df, atol=1e-13 * scale)
        np.testing.assert_allclose(am + ap, df, atol=1e-13 * scale)
        assert s[0] <= ql[1] / ql[0] - math.sqrt(G * ql[0]) + 1e-14
        assert s[2] >= qr[1] / qr[0] + math.sqrt(G * qr[0]) - 1e-14
        np.testing.assert_allclose(am, sum(s[p] * W[p] for p in range(3) if s[p] < 0) + 0 * am,
                                   atol=1e-13 * scale)


def test_bed_steps_add_the_hydrostatic_reconstruction_source():
    """Over a bed step the fluctuations add up to the flux jump less the
    source of the hydrostatic reconstruction,
      A-dQ + A+dQ = f(Q_r) - f(Q_l) + (0, g/2 (h_l^2 - h_l*^2) - g/2 (h_r^2 - h_r*^2), 0),
    h* = max(0, h + B - max(B_l, B_r)): a mass flux that telescopes (mass is
    conserved) and a momentum source that vanishes for a flat bed."""
    rng = np.random.default_rng(73)
    for _ in range(300):
        ql, qr = random_wet_pair(rng)
        B_l, B_r = rng.uniform(-0.5, 0.5, size=2)
        W, s, am, ap = rp(ql, qr, B_l, B_r)
        Bs = max(B_l, B_r)
        hls, hrs = max(0.0, ql[0] + B_l - Bs), max(0.0, qr[0] + B_r - Bs)
        hls, hrs = (hls if hls > TOL else 0.0), (hrs if hrs > TOL else 0.0)
        src = 0.5 * G * ((ql[0] ** 2 - hls ** 2) - (qr[0] ** 2 - hrs ** 2))
        expect = sw_flux(qr) - sw_flux(ql) + np.array([0.0, src, 0.0])
        scale = np.abs(expect).max() + 1.0
        np.testing.assert_allclose(am + ap, expect, atol=1e-13 * scale)
        assert am[0] + ap[0] == pytest.approx(qr[1] - ql[1], abs=1e-13 * scale)


def test_middle_state_depth_stays_positive_in_strong_rarefactions():
    """Einfeldt's speeds keep the HLLE middle depth h_l + W1[0] non-negative
    (flat bottom) even for two cells running apart near vacuum, where the
    Roe speeds alone would not."""
    rng = np.random.default_rng(72)
    for _ in range(1000):
        hl, hr = rng.uniform(0.01, 3.0, size=2)
        ul, ur = rng.uniform(-8.0, 0.0), rng.uniform(0.0, 8.0)
        W, s, am, ap = rp([hl, hl * ul, 0.0], [hr, hr * ur, 0.0])
        assert hl + W[0][0] >= 0.0


@pytest.mark.parametrize("h_l,u_l", [(1.0, 0.0), (0.5, 0.7), (2.0, -0.4)])
def test_dry_bed_front_speed(h_l, u_l):
    """A wet cell beside a dry bed at the same level: the fastest speed is the
    front of a rarefaction into a dry bed, u + 2 sqrt(g h) (closed form); the
    mirrored pair has u - 2 sqrt(g h); the fluctuations add up to the flux
    jump and no wave is kept for the correction (first order at the shore)."""
    c = math.sqrt(G * h_l)
    ql, qr = np.array([h_l, h_l * u_l, 0.1 * h_l]), np.array([0.0, 0.0, 0.0])
    W, s, am, ap = rp(ql, qr)
    assert s[2] == pytest.approx(u_l + 2.0 * c, rel=1e-15)
    assert s[0] <= u_l - c + 1e-15
    np.testing.assert_allclose(am + ap, delta_of(ql, qr, 0.0, 0.0), atol=1e-13)
    assert not W.any()
    flip = np.array([1.0, -1.0, 1.0])
    W, s, am, ap = rp(qr, ql * flip)
    assert s[0] == pytest.approx(-u_l - 2.0 * c, rel=1e-15)
    np.testing.assert_allclose(am + ap, delta_of(qr, ql * flip, 0.0, 0.0), atol=1e-13)


@pytest.mark.parametrize("u_l", [-0.8, 0.0, 0.5])
def test_wall_at_an_emerged_dry_bed(u_l):
    """A dry cell whose bed rises above the wet neighbour's surface is a wall:
    nothing enters the dry cell and the mass flux through the interface is
    zero, so the wet cell's mass fluctuation is exactly 0 - hu_l (A-dQ on the
    left, A+dQ = hu_r - 0 on the right when mirrored); water at rest stays at
    rest."""
    h_l, B_l, B_r = 0.6, 0.1, 0.9
    ql, qr = np.array([h_l, h_l * u_l, 0.2]), np.array([0.0, 0.0, 0.0])
    W, s, am, ap = rp(ql, qr, B_l, B_r)
    assert not ap.any()
    assert am[0] == pytest.approx(-ql[1], abs=1e-15)
    if u_l == 0.0:
        assert not am.any() and not W.any()
    flip = np.array([1.0, -1.0, 1.0])
    W, s, am, ap = rp(qr, ql * flip, B_r, B_l)
    assert not am.any()
    assert ap[0] == pytest.approx((ql * flip)[1], abs=1e-15)   # f_r[0] - 0


def test_two_dry_cells_exchange_nothing():
    W, s, am, ap = rp([0.0, 0.0, 0.0], [0.5 * TOL, 0.0, 0.0], 0.3, -0.2)
    assert not (W.any() or s.any() or am.any() or ap.any())


# ---------------------------------------------------------------- scheme

@pytest.mark.parametrize("limiter", ["minmod", "mc", "first_order"])
def test_ritter_dam_break_converges_without_negative_depth(limiter):
    """Dam break onto a dry bed: the depth converges to Ritter's exact
    solution in L1 (about first order: a fan ending at a front), it is never
    negative, no water runs ahead of the exact front, and the mass is kept."""
    errs = []
    front = 2.0 * math.sqrt(G) * 0.1
    for N in (200, 400, 800):
        p = inputs.sw_dry_dam_break(N, 2, limiter=limiter)
        r = Oracle(p).advance(p.q0, 0.1)
        x = inputs.centres(N, -1.0, 1.0)
        h = r["q"][0][0]
        h_ex, _ = ritter_profile(x, 0.1, 1.0)
        errs.append(np.abs(h - h_ex).mean() * 2.0)
        assert h.min() >= 0.0
        assert x[h > 0.0].max() <= front + 1.0 / N
        assert abs(h.sum() * 2.0 / N - 1.0) <= 1e-14
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[-1] < 5e-3 and min(rates) > 0.6, (errs, rates)


@pytest.mark.parametrize("bc", ["periodic", "extrap", "wall"])
@pytest.mark.parametrize("limiter", ["none", "minmod", "mc", "first_order"])
def test_lake_at_rest_around_an_emerged_island_bitwise(bc, limiter):
    """A lake at rest whose island top is dry stays exactly at rest: no wave
    between wet cells (flat surface, zero momentum), walls at the shore, and
    nothing between dry cells."""
    p = inputs.sw_island(48, 40, limiter=limiter, bc=bc, hump=0.0)
    assert (p.q0[0] == 0.0).sum() > 20
    r = Oracle(p).run_steps(p.q0, 8)["q"]
    np.testing.assert_array_equal(r, p.q0)


@pytest.mark.parametrize("limiter", ["minmod", "mc"])
def test_beach_run_up_keeps_mass_and_non_negative_depth(limiter):
    """A hump runs up a plane beach and falls back (cells flood and dry):
    with walls the total mass is kept to roundoff and the depth never goes
    negative."""
    p = inputs.sw_beach(200, 6, limiter=limiter)
    o = Oracle(p)
    q, t, dt = p.q0, 0.0, 0.0
    m0 = p.q0[0].sum()
    flooded = (p.q0[0] == 0.0)
    wetted = np.zeros_like(flooded)
    for _ in range(12):
        r = o.run_steps(q, 20, t=t, dt=dt)
        q, t, dt = r["q"], r["t"], r["dt"]
        assert q[0].min() >= 0.0
        assert abs(q[0].sum() - m0) <= 1e-13 * m0
        wetted |= q[0] > TOL
    assert (wetted & flooded).sum() > 0           # the run-up floods dry cells


def test_island_run_up_conserves_mass_with_walls():
    p = inputs.sw_island(64, 56, limiter="mc", bc="wall", hump=0.3)
    r = Oracle(p).run_steps(p.q0, 40)
    assert r["q"][0].min() >= 0.0
    assert abs(r["q"][0].sum() - p.q0[0].sum()) <= 1e-13 * p.q0[0].sum()
