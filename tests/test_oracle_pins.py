"""Pins for the CPU oracle: closed forms, invariants and special cases that the
paper's method (CUDACLAW Sec. 3: Eq. LW-update, Eq. CFL-condition, Eq.
acoustics, Eq. SW) and the mathematics fix, independent of the oracle's own
code.  Each pin is chosen so that a plausible slip in the oracle (a dropped
term, a wrong sign or index, a transposed operand) fails at least one.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import Oracle
from paper_1805_08846_gb300 import inputs
from tests.exact_sw import dam_break_profile, dam_break_state

G = 9.81


def line_problem(system, N, ny=2, limiter="mc", bc_x="periodic", bc_y="periodic",
                 lower=0.0, upper=1.0, q0=None, **kw):
    """A y-uniform 2D problem (ny rows), i.e. the 1D scheme along x."""
    m = 3
    q = np.zeros((m, ny, N)) if q0 is None else q0
    return inputs.Problem(2, (N, ny), (lower, 0.0), (upper, 1.0), system, limiter,
                          (bc_x, bc_x, bc_y, bc_y), q, **kw)


def sw_flux(q, g=G):
    h, hu, hv = q
    u = hu / h
    return np.array([hu, hu * u + 0.5 * g * h * h, hu * hv / h])


# ---------------------------------------------------------------- Riemann solvers

def test_acoustics_riemann_identities():
    """Sum of waves = jump; each wave is an eigenvector of its side's
    A = [[0, K], [1/rho, 0]] with eigenvalue s; a purely right-going jump
    (dp = Z du) has no left-going wave; A-dQ = s1 W1, A+dQ = s2 W2."""
    rng = np.random.default_rng(11)
    for _ in range(200):
        ql, qr = rng.normal(size=2), rng.normal(size=2)
        rl, kl, rr, kr = np.exp(rng.uniform(np.log(0.5), np.log(4.0), size=4))
        W, s, am, ap = oracle.riemann("acoustics", ql, qr, rl, kl, rr, kr)
        np.testing.assert_allclose(W.sum(0), qr - ql, rtol=1e-13, atol=1e-13)
        Al = np.array([[0.0, kl], [1.0 / rl, 0.0]])
        Ar = np.array([[0.0, kr], [1.0 / rr, 0.0]])
        np.testing.assert_allclose(Al @ W[0], s[0] * W[0], rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(Ar @ W[1], s[1] * W[1], rtol=1e-12, atol=1e-13)
        assert s[0] == pytest.approx(-math.sqrt(kl / rl), rel=1e-15)
        assert s[1] == pytest.approx(math.sqrt(kr / rr), rel=1e-15)
        np.testing.assert_allclose(am, s[0] * W[0], rtol=1e-14, atol=1e-15)
        np.testing.assert_allclose(ap, s[1] * W[1], rtol=1e-14, atol=1e-15)
    # purely right-going jump, constant medium rho = 1, K = 4 (Z = 2)
    du = 0.37
    W, s, am, ap = oracle.riemann("acoustics", [0.0, 0.0], [2.0 * du, du], 1, 4, 1, 4)
    assert abs(W[0]).max() < 1e-16
    np.testing.assert_allclose(W[1], [2.0 * du, du], rtol=1e-15)


def roe_matrix(ql, qr, g=G):
    """Flux Jacobian at the Roe-averaged state, written from the flux."""
    hl, hr = ql[0], qr[0]
    ul, ur, vl, vr = ql[1] / hl, qr[1] / hr, ql[2] / hl, qr[2] / hr
    w = np.sqrt(hl) / (np.sqrt(hl) + np.sqrt(hr))
    u = w * ul + (1 - w) * ur
    v = w * vl + (1 - w) * vr
    c2 = g * 0.5 * (hl + hr)
    return np.array([[0.0, 1.0, 0.0], [c2 - u * u, 2 * u, 0.0], [-u * v, v, u]])


def random_sw_pair(rng):
    hl, hr = rng.uniform(0.1, 5.0, size=2)
    ul, ur, vl, vr = rng.uniform(-3.0, 3.0, size=4)
    return np.array([hl, hl * ul, hl * vl]), np.array([hr, hr * ur, hr * vr])


def test_sw_roe_identities():
    """Roe property sum_p s_p W_p = f(Q_r) - f(Q_l); sum W = dQ; each wave an
    eigenvector of the Roe matrix; with the entropy fix still
    A-dQ + A+dQ = f(Q_r) - f(Q_l)."""
    rng = np.random.default_rng(5)
    for _ in range(500):
        ql, qr = random_sw_pair(rng)
        W, s, am, ap = oracle.riemann("shallow_water", ql, qr)
        df = sw_flux(qr) - sw_flux(ql)
        scale = np.abs(df).max() + np.abs(sw_flux(ql)).max()
        np.testing.assert_allclose(W.sum(0), qr - ql, rtol=0, atol=1e-13 * (1 + np.abs(qr).max()))
        assert np.abs((s[:, None] * W).sum(0) - df).max() <= 1e-13 * scale
        assert np.abs(am + ap - df).max() <= 1e-13 * scale
        sq = lambda v: math.sqrt(v) if v > 0 else float("nan")
        lam_l = ql[1] / ql[0] - sq(G * ql[0])
        hm1 = ql[0] + W[0][0]
        lam_m1 = (ql[1] + W[0][1]) / hm1 - sq(G * hm1)
        lam_r = qr[1] / qr[0] + sq(G * qr[0])
        hm3 = qr[0] - W[2][0]
        lam_m3 = (qr[1] - W[2][1]) / hm3 + sq(G * hm3)
        if not (lam_l < 0 < lam_m1) and not (lam_m3 < 0 < lam_r):
            plain = sum(min(s[p], 0.0) * W[p] for p in range(3))
            np.testing.assert_allclose(am, plain, rtol=1e-13, atol=1e-13 * scale)
        A = roe_matrix(ql, qr)
        for p in range(3):
            np.testing.assert_allclose(A @ W[p], s[p] * W[p], rtol=0,
                                       atol=1e-12 * (1 + np.abs(W[p]).max() * (1 + abs(s[p]) + 10)))


def test_sw_entropy_fix_splits_transonic_waves():
    """Harten-Hyman: for a transonic 1-rarefaction (lam_l < 0 < lam_m at the
    Roe middle state) the split uses beta = (lam_m - s1)/(lam_m - lam_l);
    fluctuations still sum to the flux difference and differ from the plain
    min(s,0) W split.  The mirrored pair exercises the 3-wave."""
    ql = np.array([1.0, 2.9, 0.3])
    qr = np.array([0.8, 0.8 * 3.2, -0.16])
    W, s, am, ap = oracle.riemann("shallow_water", ql, qr)
    df = sw_flux(qr) - sw_flux(ql)
    np.testing.assert_allclose(am + ap, df, rtol=1e-14, atol=1e-14)
    lam_l = 2.9 - math.sqrt(G * 1.0)
    hm = 1.0 + W[0][0]
    lam_m = (2.9 + W[0][1]) / hm - math.sqrt(G * hm)
    assert lam_l < 0 < lam_m                     # transonic 1-wave
    beta = (lam_m - s[0]) / (lam_m - lam_l)
    plain_am = sum(min(s[p], 0.0) * W[p] for p in range(3))
    expect_am = beta * lam_l * W[0] + sum(min(s[p], 0.0) * W[p] for p in (1, 2))
    np.testing.assert_allclose(am, expect_am, rtol=1e-13, atol=1e-15)
    assert np.abs(am - plain_am).max() > 1e-3
    # mirrored pair (swap sides, negate normal momentum): transonic 3-wave
    flip = np.array([1.0, -1.0, 1.0])
    ql2, qr2 = qr * flip, ql * flip
    W, s, am, ap = oracle.riemann("shallow_water", ql2, qr2)
    np.testing.assert_allclose(am + ap, sw_flux(qr2) - sw_flux(ql2), rtol=1e-14, atol=1e-14)
    lam_r = qr2[1] / qr2[0] + math.sqrt(G * qr2[0])
    hm = qr2[0] - W[2][0]
    lam_m = (qr2[1] - W[2][1]) / hm + math.sqrt(G * hm)
    assert lam_m < 0 < lam_r
    beta = (lam_r - s[2]) / (lam_r - lam_m)
    expect_ap = (1 - beta) * lam_r * W[2] + sum(max(s[p], 0.0) * W[p] for p in (0, 1))
    np.testing.assert_allclose(ap, expect_ap, rtol=1e-13, atol=1e-15)


def test_sw_mirror_symmetry_of_solver():
    """Swapping left/right and negating the normal momentum mirrors the
    problem (f(flip q) = -flip f(q)): A-dQ of the mirrored problem is the
    original A+dQ with the normal component negated, and vice versa."""
    rng = np.random.default_rng(7)
    flip = np.array([1.0, -1.0, 1.0])
    for _ in range(200):
        ql, qr = random_sw_pair(rng)
        _, _, am, ap = oracle.riemann("shallow_water", ql, qr)
        _, _, am2, ap2 = oracle.riemann("shallow_water", qr * flip, ql * flip)
        np.testing.assert_allclose(am2, ap * flip, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(ap2, am * flip, rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- limiter

@pytest.mark.parametrize("theta,minmod,mc", [
    (-1.0, 0.0, 0.0), (0.0, 0.0, 0.0), (0.25, 0.25, 0.5), (0.5, 0.5, 0.75),
    (1.0, 1.0, 1.0), (2.0, 1.0, 1.5), (3.0, 1.0, 2.0), (10.0, 1.0, 2.0)])
def test_limiter_table(theta, minmod, mc):
    """minmod phi = max(0, min(1, theta)); MC phi = max(0, min((1+theta)/2, 2, 2 theta))."""
    assert oracle.phi("minmod", theta) == minmod
    assert oracle.phi("mc", theta) == mc
    assert oracle.phi("none", theta) == 1.0
    assert oracle.phi("first_order", theta) == 0.0


# ---------------------------------------------------------------- whole scheme

def right_going_acoustic(N, f, ny=2, rho=1.0, K=4.0, limiter="mc"):
    Z = math.sqrt(rho * K)
    x = inputs.centres(N, 0.0, 1.0)
    q0 = np.zeros((3, ny, N))
    q0[0] = f(x)[None, :]
    q0[1] = q0[0] / Z
    return line_problem("acoustics", N, ny=ny, limiter=limiter, q0=q0, rho=rho, K=K)


@pytest.mark.parametrize("limiter", ["none", "minmod", "mc", "first_order"])
def test_exact_translation_at_courant_one(limiter):
    """At nu*c = 1 the correction vanishes and upwinding is an exact shift:
    a right-going wave moves one cell per step (any limiter)."""
    N = 64
    rng = np.random.default_rng(3)
    prof = rng.normal(size=N)
    p = right_going_acoustic(N, lambda x: prof, limiter=limiter)
    o = Oracle(p)
    dt = p.dx[0] / 2.0                    # c = 2
    r = o.run_steps(p.q0, 5, fixed_dt=dt)
    np.testing.assert_allclose(r["q"][0], np.roll(p.q0[0], 5, axis=1), rtol=0, atol=1e-14)
    np.testing.assert_allclose(r["q"][1], np.roll(p.q0[1], 5, axis=1), rtol=0, atol=1e-14)


def test_extrapolation_boundaries_at_courant_one():
    """Zeroth-order extrapolation ghosts copy the edge cell, so the edge
    interfaces see no jump: at nu*c = 1 a right-going wave shifts out through
    the right edge and the left edge cell keeps its value,
    Q_i <- Q_{i-1} (i >= 1), Q_0 <- Q_0."""
    N = 40
    rng = np.random.default_rng(8)
    prof = rng.normal(size=N)
    p = right_going_acoustic(N, lambda x: prof)
    p = p.with_(bc=("extrap", "extrap", "periodic", "periodic"))
    r = Oracle(p).run_steps(p.q0, 3, fixed_dt=p.dx[0] / 2.0)["q"]
    expect = np.concatenate([np.full(3, prof[0]), prof[:-3]])
    np.testing.assert_allclose(r[0][0], expect, rtol=0, atol=1e-14)


def test_x_and_y_sweeps_agree_by_transposition():
    """A wave along y on an x-uniform grid equals, transposed, the same wave
    along x: the y sweep acts on (p, v) exactly as the x sweep on (p, u)."""
    N, ny = 48, 4
    x = inputs.centres(N, 0.0, 1.0)
    f = np.exp(-80 * (x - 0.4) ** 2)
    qx = np.zeros((3, ny, N)); qx[0] = f; qx[1] = f / 2.0
    qy = np.zeros((3, N, ny)); qy[0] = f[:, None]; qy[2] = f[:, None] / 2.0
    px = line_problem("acoustics", N, ny=ny, q0=qx, K=4.0)
    py = inputs.Problem(2, (ny, N), (0, 0), (1, 1), "acoustics", "mc", ("periodic",) * 4, qy, K=4.0)
    dt = 0.9 * px.dx[0] / 2.0
    rx = Oracle(px).run_steps(qx, 7, fixed_dt=dt)["q"]
    ry = Oracle(py).run_steps(qy, 7, fixed_dt=dt)["q"]
    np.testing.assert_array_equal(rx[0], ry[0].T)
    np.testing.assert_array_equal(rx[1], ry[2].T)
    np.testing.assert_array_equal(rx[2], ry[1].T)


def acoustic_sweep_exact(q, d, Z):
    """One sweep of constant acoustics along d at Courant number 1: the
    right-going characteristic variable (u_d + p/Z)/2 moves one cell forward,
    the left-going one (u_d - p/Z)/2 one cell back; other velocities stay."""
    pr, un = q[0], q[1 + d]
    w_right = 0.5 * (un + pr / Z)
    w_left = 0.5 * (un - pr / Z)
    axis = q.ndim - 2 - d                 # x is the last array axis
    w_right = np.roll(w_right, 1, axis=axis)
    w_left = np.roll(w_left, -1, axis=axis)
    out = q.copy()
    out[0] = Z * (w_right - w_left)
    out[1 + d] = w_right + w_left
    return out


def test_strang_step_is_symmetric_composition_of_shifts():
    """Strang splitting x(dt/2) y(dt) x(dt/2): with dy = 2 dx and c dt = 2 dx
    every sweep runs at Courant number 1 and is an exact characteristic
    shift, so one step is shift_x . shift_y . shift_x (Godunov's x, y order
    would give shift_y . shift_x over a full dt in x instead)."""
    N, Z = 32, 2.0
    rng = np.random.default_rng(41)
    q0 = rng.normal(size=(3, N // 2, N))
    p = inputs.Problem(2, (N, N // 2), (0, 0), (1, 1), "acoustics", "mc", ("periodic",) * 4, q0,
                       K=4.0, splitting="strang")
    assert p.dx[1] == 2 * p.dx[0]
    r = Oracle(p).run_steps(q0, 1, fixed_dt=p.dx[0])["q"]        # c = 2
    expect = acoustic_sweep_exact(acoustic_sweep_exact(acoustic_sweep_exact(q0, 0, Z), 1, Z), 0, Z)
    np.testing.assert_allclose(r, expect, rtol=0, atol=1e-13)


def test_strang_3d_step_is_symmetric_composition_of_shifts():
    """3D Strang x(dt/2) y(dt/2) z(dt) y(dt/2) x(dt/2) with dz = 2 dx = 2 dy,
    c dt = 2 dx: five exact shifts in that order."""
    N, Z = 16, 2.0
    rng = np.random.default_rng(43)
    q0 = rng.normal(size=(4, N // 2, N, N))
    p = inputs.Problem(3, (N, N, N // 2), (0, 0, 0), (1, 1, 1), "acoustics", "minmod", ("periodic",) * 6,
                       q0, K=4.0, splitting="strang")
    r = Oracle(p).run_steps(q0, 1, fixed_dt=p.dx[0])["q"]
    e = q0
    for d in (0, 1, 2, 1, 0):
        e = acoustic_sweep_exact(e, d, Z)
    np.testing.assert_allclose(r, e, rtol=0, atol=1e-13)


def test_strang_on_y_uniform_data_is_two_half_steps():
    """On y-uniform data the y sweep changes nothing, so a Strang step of dt
    is x(dt/2) twice: bitwise the same as two Godunov steps of dt/2."""
    N = 40
    rng = np.random.default_rng(47)
    row = np.stack([1.0 + 0.3 * rng.random(N), 0.2 * rng.normal(size=N), 0.1 * rng.normal(size=N)])
    q0 = np.repeat(row[:, None, :], 3, axis=1)
    pg = line_problem("shallow_water", N, ny=3, limiter="mc", q0=q0)
    ps = pg.with_(splitting="strang")
    dt = 0.4 * pg.dx[0] / 4.0
    rs = Oracle(ps).run_steps(q0, 3, fixed_dt=dt)["q"]
    rg = Oracle(pg).run_steps(q0, 6, fixed_dt=dt / 2)["q"]
    np.testing.assert_array_equal(rs, rg)


def test_split_step_at_courant_one_is_composed_shifts():
    """Constant acoustics with c dt = dx = dy: each sweep moves the
    right-going characteristic variable (u_d + p/Z)/2 one cell forward and
    the left-going one (u_d - p/Z)/2 one cell back, and leaves the other
    velocity alone.  One step of Eq. LW-update is the x map followed by the
    y map (it does not commute with the reverse order)."""
    N, Z = 24, 2.0
    rng = np.random.default_rng(21)
    q0 = rng.normal(size=(3, N, N))
    p = inputs.Problem(2, (N, N), (0, 0), (1, 1), "acoustics", "mc", ("periodic",) * 4, q0, K=4.0)

    def sweep_exact(q, d):
        pr, un = q[0], q[1 + d]
        w_right = 0.5 * (un + pr / Z)
        w_left = 0.5 * (un - pr / Z)
        axis = 1 if d == 0 else 0            # x is the last array axis
        w_right = np.roll(w_right, 1, axis=axis)
        w_left = np.roll(w_left, -1, axis=axis)
        out = q.copy()
        out[0] = Z * (w_right - w_left)
        out[1 + d] = w_right + w_left
        return out

    r = Oracle(p).run_steps(q0, 1, fixed_dt=p.dx[0] / 2.0)["q"]
    xy = sweep_exact(sweep_exact(q0, 0), 1)
    yx = sweep_exact(sweep_exact(q0, 1), 0)
    np.testing.assert_allclose(r, xy, rtol=0, atol=1e-13)
    assert np.abs(xy - yx).max() > 0.1


def test_first_order_step_is_characteristic_upwinding():
    """Without the correction term a step of constant-coefficient acoustics
    is upwinding of the two characteristic variables: w+ = (u + p/Z)/2 moves
    right at c, w- = (u - p/Z)/2 left, so in one x sweep
        w+_i <- w+_i - nu c (w+_i - w+_{i-1}),  w-_i <- w-_i + nu c (w-_{i+1} - w-_i),
    and p = Z (w+ - w-), u = w+ + w-; v is untouched.  Random periodic data
    on a y-uniform grid (the y sweep is then a no-op)."""
    N, ny, rho, K = 50, 2, 1.0, 4.0
    c, Z = math.sqrt(K / rho), math.sqrt(K * rho)
    rng = np.random.default_rng(31)
    row = rng.normal(size=(3, N))
    q0 = np.repeat(row[:, None, :], ny, axis=1)
    p = line_problem("acoustics", N, ny=ny, limiter="first_order", q0=q0, rho=rho, K=K)
    nu_c = 0.6
    r = Oracle(p).run_steps(q0, 1, fixed_dt=nu_c * p.dx[0] / c)["q"]
    pr, u = row[0], row[1]
    wp, wm = 0.5 * (u + pr / Z), 0.5 * (u - pr / Z)
    wp1 = wp - nu_c * (wp - np.roll(wp, 1))
    wm1 = wm + nu_c * (np.roll(wm, -1) - wm)
    np.testing.assert_allclose(r[0][0], Z * (wp1 - wm1), rtol=0, atol=1e-13)
    np.testing.assert_allclose(r[1][0], wp1 + wm1, rtol=0, atol=1e-13)
    np.testing.assert_array_equal(r[2][0], row[2])


def plane_wave_error(N, limiter):
    f = lambda x: np.sin(2 * np.pi * x)
    p = right_going_acoustic(N, f, limiter=limiter)
    r = Oracle(p).advance(p.q0, 0.25)      # c = 2: half a period
    x = inputs.centres(N, 0.0, 1.0)
    exact = f(x - 2.0 * 0.25)
    return np.abs(r["q"][0][0] - exact).mean()


@pytest.mark.parametrize("limiter,order", [("none", 1.9), ("mc", 1.5)])
def test_plane_wave_convergence(limiter, order):
    """Smooth periodic acoustic wave at CFL 0.9: observed order ~2 without a
    limiter (Lax-Wendroff), >= 1.5 with MC."""
    e = [plane_wave_error(N, limiter) for N in (64, 128, 256)]
    rates = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert min(rates) >= order, (e, rates)


def test_plane_wave_first_order_convergence():
    """Without the correction term the method is first order: the error of
    the smooth wave halves with the cell width (rate in [0.85, 1.2])."""
    e = [plane_wave_error(N, "first_order") for N in (128, 256, 512)]
    rates = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert 0.85 <= min(rates) and max(rates) <= 1.2, (e, rates)


def test_diagonal_plane_wave_converges():
    """A plane wave along the diagonal (both sweeps active) converges to the
    exact translate (Godunov splitting: at least first order)."""
    def err(N):
        c, Z = 2.0, 2.0
        xs = inputs.centres(N, 0.0, 1.0)
        Y, X = np.meshgrid(xs, xs, indexing="ij")
        f = lambda X, Y: np.sin(2 * np.pi * (X + Y))
        q0 = np.zeros((3, N, N))
        q0[0] = f(X, Y)
        q0[1] = q0[0] / (Z * math.sqrt(2))
        q0[2] = q0[0] / (Z * math.sqrt(2))
        p = inputs.Problem(2, (N, N), (0, 0), (1, 1), "acoustics", "none", ("periodic",) * 4, q0, K=4.0)
        t = 0.125
        r = Oracle(p).advance(q0, t)
        s = c * t / math.sqrt(2)
        return np.abs(r["q"][0] - f(X - s, Y - s)).mean()
    e = [err(N) for N in (32, 64, 128)]
    rates = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert min(rates) >= 0.9, (e, rates)
    assert e[-1] < 0.02


@pytest.mark.parametrize("limiter", ["minmod", "mc"])
def test_tvd_single_family(limiter):
    """A purely right-going acoustic step is scalar advection of one wave
    family; with a TVD limiter its total variation never grows, and the
    profile stays within its initial bounds (no new extrema)."""
    N = 100
    p = right_going_acoustic(N, lambda x: np.where((x > 0.2) & (x < 0.5), 1.0, 0.0),
                             limiter=limiter)
    o = Oracle(p)
    q = p.q0
    tv = np.abs(np.diff(q[0][0], append=q[0][0][:1])).sum()
    dt = 0.8 * p.dx[0] / 2.0
    for _ in range(40):
        q = o.run_steps(q, 1, fixed_dt=dt)["q"]
        tv_new = np.abs(np.diff(q[0][0], append=q[0][0][:1])).sum()
        assert tv_new <= tv + 1e-12
        assert q[0].min() >= -1e-12 and q[0].max() <= 1 + 1e-12
        tv = tv_new


def test_impedance_jump_reflection_and_transmission():
    """A right-going pulse meeting an impedance jump Z 1 -> 4 (c = 1 both
    sides) reflects with amplitude (Z2-Z1)/(Z1+Z2) = 0.6 and transmits with
    2 Z2/(Z1+Z2) = 1.6 (normal incidence)."""
    N = 800
    x = inputs.centres(N, 0.0, 1.0)
    q0 = np.zeros((3, 2, N))
    q0[0] = np.exp(-((x - 0.25) / 0.04) ** 2)
    q0[1] = q0[0]                                   # Z1 = 1: right-going
    def run(jump):
        rho = np.where(x >= 0.5, 4.0 if jump else 1.0, 1.0) * np.ones((2, N))
        p = line_problem("acoustics_var", N, q0=q0, bc_x="extrap", rho_cell=rho, K_cell=rho.copy())
        return Oracle(p).advance(q0, 0.5)["q"][0][0]
    with_jump, without = run(True), run(False)
    peak = without[x >= 0.5].max()                  # same travel, no interface
    T = with_jump[x >= 0.5].max() / peak
    R = with_jump[x < 0.5].max() / peak
    assert T == pytest.approx(1.6, rel=0.01)
    assert R == pytest.approx(0.6, rel=0.01)


def sw_line_run(h_l, h_r, N, t, limiter="minmod"):
    x = inputs.centres(N, -1.0, 1.0)
    q0 = np.zeros((3, 2, N))
    q0[0] = np.where(x < 0.0, h_l, h_r)
    p = line_problem("shallow_water", N, limiter=limiter, bc_x="extrap", lower=-1.0,
                     upper=1.0, q0=q0)
    r = Oracle(p).advance(q0, t)
    return x, r["q"][:, 0, :]


def test_stoker_dam_break_converges():
    """1D dam break h_l = 2, h_r = 1 (Stoker): the L1 error in h against the
    exact solution drops at about first order (a shock is present)."""
    st = dam_break_state(2.0, 1.0)
    assert st["h_m"] == pytest.approx(1.45384089, abs=1e-8)
    assert st["u_m"] == pytest.approx(1.30583375, abs=1e-8)
    assert st["shock"] == pytest.approx(4.18312792, abs=1e-8)
    errs = []
    for N in (200, 400, 800):
        x, q = sw_line_run(2.0, 1.0, N, 0.1)
        h_ex, hu_ex = dam_break_profile(x, 0.1, 2.0, 1.0)
        errs.append(np.abs(q[0] - h_ex).mean() * 2.0)
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[-1] < 2e-3, errs
    assert min(rates) > 0.7, (errs, rates)


def test_transonic_dam_break_entropy_fix():
    """Dam break h_l = 1, h_r = 0.1: the rarefaction fan spans xi = 0, the case
    the entropy fix exists for.  The scheme converges to the exact (entropy)
    solution, including near x = 0, where an unfixed Roe scheme keeps a
    stationary expansion shock."""
    st = dam_break_state(1.0, 0.1)
    assert st["h_m"] == pytest.approx(0.39617482, abs=1e-8)
    assert st["head"] < 0.0 < st["tail"]
    errs, near0 = [], []
    for N in (200, 400, 800):
        x, q = sw_line_run(1.0, 0.1, N, 0.1)
        h_ex, _ = dam_break_profile(x, 0.1, 1.0, 0.1)
        errs.append(np.abs(q[0] - h_ex).mean() * 2.0)
        w = np.abs(x) < 0.05
        near0.append(np.abs(q[0][w] - h_ex[w]).max())
    assert errs[-1] < 3e-3 and errs[2] < errs[1] < errs[0], errs
    assert near0[-1] < 0.01 and near0[-1] < near0[0], near0


# ---------------------------------------------------------------- invariants

@pytest.mark.parametrize("bc", ["periodic", "extrap", "wall"])
@pytest.mark.parametrize("limiter", ["none", "minmod", "mc", "first_order"])
def test_lake_at_rest_bitwise(bc, limiter):
    """Constant depth and zero momentum stay exactly as they are."""
    q0 = np.zeros((3, 13, 17))
    q0[0] = 1.7
    p = inputs.Problem(2, (17, 13), (0, 0), (1, 1), "shallow_water", limiter, (bc,) * 4, q0)
    r = Oracle(p).run_steps(q0, 10)
    np.testing.assert_array_equal(r["q"], q0)


@pytest.mark.parametrize("bc", ["periodic", "wall"])
def test_sw_conservation(bc):
    """Total mass is conserved to roundoff with periodic or wall boundaries;
    both momenta too with periodic boundaries."""
    p = inputs.random_problem("shallow_water", (37, 29), "minmod", bc, discontinuous=True)
    r = Oracle(p).run_steps(p.q0, 30)
    s0 = [math.fsum(p.q0[f].ravel()) for f in range(3)]
    s1 = [math.fsum(r["q"][f].ravel()) for f in range(3)]
    assert abs(s1[0] - s0[0]) <= 1e-13 * abs(s0[0])
    if bc == "periodic":
        scale = math.fsum(np.abs(p.q0[0]).ravel())
        assert abs(s1[1] - s0[1]) <= 1e-13 * scale
        assert abs(s1[2] - s0[2]) <= 1e-13 * scale


@pytest.mark.parametrize("bc", ["periodic", "wall"])
def test_acoustics_conservation(bc):
    """Constant coefficients: sum p is conserved with periodic or wall
    boundaries; sum rho u and sum rho v with periodic ones."""
    p = inputs.random_problem("acoustics", (31, 23), "mc", bc, discontinuous=True)
    r = Oracle(p).run_steps(p.q0, 30)
    scale = math.fsum(np.abs(p.q0[0]).ravel())
    assert abs(math.fsum(r["q"][0].ravel()) - math.fsum(p.q0[0].ravel())) <= 1e-13 * scale
    if bc == "periodic":
        for f in (1, 2):
            assert abs(math.fsum(r["q"][f].ravel()) - math.fsum(p.q0[f].ravel())) <= 1e-13 * scale


def test_acoustics_3d_conservation_and_axes():
    """3D: sum p conserved with walls; a pulse symmetric under x <-> z stays
    symmetric up to the splitting order, and a z-directed wave on an
    x,y-uniform grid is the transposed x-directed one."""
    N = 24
    x = inputs.centres(N, 0.0, 1.0)
    f = np.exp(-60 * (x - 0.45) ** 2)
    qz = np.zeros((4, N, 2, 2)); qz[0] = f[:, None, None]; qz[3] = f[:, None, None] / 2.0
    qx = np.zeros((4, 2, 2, N)); qx[0] = f; qx[1] = f / 2.0
    pz = inputs.Problem(3, (2, 2, N), (0,) * 3, (1,) * 3, "acoustics", "mc", ("periodic",) * 6, qz, K=4.0)
    px = inputs.Problem(3, (N, 2, 2), (0,) * 3, (1,) * 3, "acoustics", "mc", ("periodic",) * 6, qx, K=4.0)
    dt = 0.9 / N / 2.0
    rz = Oracle(pz).run_steps(qz, 6, fixed_dt=dt)["q"]
    rx = Oracle(px).run_steps(qx, 6, fixed_dt=dt)["q"]
    np.testing.assert_array_equal(rz[0][:, 0, 0], rx[0][0, 0, :])
    np.testing.assert_array_equal(rz[3][:, 0, 0], rx[1][0, 0, :])
    p3 = inputs.random_problem("acoustics", (11, 9, 10), "mc", "wall", discontinuous=True)
    r3 = Oracle(p3).run_steps(p3.q0, 12)["q"]
    scale = math.fsum(np.abs(p3.q0[0]).ravel())
    assert abs(math.fsum(r3[0].ravel()) - math.fsum(p3.q0[0].ravel())) <= 1e-13 * scale


@pytest.mark.parametrize("system", ["acoustics", "shallow_water"])
def test_wall_equals_mirror_extended_periodic(system):
    """Reflecting walls on [0,1] equal the periodic problem on the
    mirror-doubled domain (normal component odd), restricted to [0,1]."""
    N, ny = 20, 6
    p = inputs.random_problem(system, (N, ny), "mc", ("wall", "wall", "periodic", "periodic"),
                              discontinuous=True)
    q = p.q0
    mirror = q[:, :, ::-1].copy()
    mirror[1] *= -1.0
    qe = np.concatenate([mirror, q], axis=2)
    pe = inputs.Problem(2, (2 * N, ny), (-1.0, 0.0), (1.0, 1.0), system, "mc",
                        ("periodic",) * 4, qe, rho=p.rho, K=p.K)
    dt = 0.4 * p.dx[0] / (5.0 if system == "shallow_water" else 2.0)
    r = Oracle(p).run_steps(q, 8, fixed_dt=dt)["q"]
    re = Oracle(pe).run_steps(qe, 8, fixed_dt=dt)["q"]
    np.testing.assert_allclose(r, re[:, :, N:], rtol=0, atol=1e-13)


def test_y_uniform_problem_has_no_y_update():
    """On a y-uniform state every y Riemann problem has zero jump: the y sweep
    changes nothing, bit for bit, and all rows stay identical."""
    N, ny = 40, 5
    x = inputs.centres(N, -1.0, 1.0)
    q0 = np.zeros((3, ny, N))
    q0[0] = np.where(x < 0.1, 2.0, 1.0)
    q0[1] = 0.3 * np.sin(3 * x)
    p = line_problem("shallow_water", N, ny=ny, limiter="minmod", bc_x="extrap",
                     lower=-1.0, upper=1.0, q0=q0)
    o = Oracle(p)
    dt = 0.002
    qs, _ = o.sweep(0, q0, dt)
    qy, _ = o.sweep(1, qs, dt)
    np.testing.assert_array_equal(qy, qs)
    for j in range(1, ny):
        np.testing.assert_array_equal(qy[:, j], qy[:, 0])


def test_radial_dam_break_mirror_symmetry():
    """The radial dam break on [-1,1]^2 is symmetric under x -> -x and under
    y -> -y separately (momentum component odd)."""
    p = inputs.sw_radial_dam_break(48, nsteps=20)
    q = Oracle(p).run_steps(p.q0, 20)["q"]
    scale = np.abs(q).max()
    assert np.abs(q[0] - q[0][:, ::-1]).max() <= 1e-13 * scale
    assert np.abs(q[1] + q[1][:, ::-1]).max() <= 1e-13 * scale
    assert np.abs(q[2] - q[2][:, ::-1]).max() <= 1e-13 * scale
    assert np.abs(q[0] - q[0][::-1, :]).max() <= 1e-13 * scale
    assert np.abs(q[2] + q[2][::-1, :]).max() <= 1e-13 * scale


def test_outflow_conserves_mass_before_fronts_reach_boundary():
    """Outflow (extrapolation) boundaries do not change the mass while the
    waves stay inside the domain."""
    p = inputs.sw_radial_dam_break(64)
    r = Oracle(p).advance(p.q0, 0.03)          # fronts move ~0.14 from r = 0.5
    q = r["q"]
    assert r["nacc"] >= 4
    assert np.abs(q[0][0, :] - 1.0).max() == 0.0 and np.abs(q[0][:, 0] - 1.0).max() == 0.0
    s0 = math.fsum(p.q0[0].ravel())
    assert abs(math.fsum(q[0].ravel()) - s0) <= 1e-13 * s0


# ---------------------------------------------------------------- time step

def test_dt_rule_constant_acoustics():
    """128^2 acoustics with c = 2 on [0,1]^2: every step is 0.9 / (2 * 128),
    so 100 steps reach t = 100 * 0.9/256 = 0.3515625 (up to summation)."""
    p = inputs.acoustics_2d_pulse(128)
    r = Oracle(p).run_steps(p.q0, 100)
    assert r["dt"] == 0.9 / 256
    assert r["nacc"] == 100 and r["nrej"] == 0
    assert r["t"] == pytest.approx(0.3515625, rel=1e-14)


def test_cfl_violation_is_redone():
    """A first step that is too large (Courant number 1.5 > 1) is rejected
    and redone at cfl_desired: the accepted step has Courant number 0.9."""
    p = inputs.acoustics_2d_pulse(32)
    o = Oracle(p)
    dt_bad = 1.5 / (2.0 * 32)
    r = o.run_steps(p.q0, 1, dt=dt_bad)
    assert r["nrej"] == 1 and r["nacc"] == 1
    assert r["cfl"] == pytest.approx(0.9, rel=1e-14)
    assert r["t"] == pytest.approx(0.9 / 64, rel=1e-14)


def test_advance_lands_on_t_final():
    p = inputs.sw_radial_dam_break(32)
    r = Oracle(p).advance(p.q0, 0.01)
    assert r["t"] == 0.01
    assert r["nacc"] >= 1


# ---------------------------------------------------------------- bathymetry

def sw_flux_with_source_jump(ql, qr, B_l, B_r, g=G):
    """f(Q_r) - f(Q_l) - psi with psi = (0, -g h_bar (B_r - B_l), 0)."""
    fl, fr = sw_flux(np.asarray(ql, float)), sw_flux(np.asarray(qr, float))
    hbar = 0.5 * (ql[0] + qr[0])
    return fr - fl - np.array([0.0, -g * hbar * (B_r - B_l), 0.0])


def test_bathymetry_fwaves_decompose_flux_jump_minus_source():
    """The f-waves sum to f(Q_r) - f(Q_l) - psi, each lies on its Roe
    eigenvector (Z_p = beta_p (1, s_p, v_hat) for p = 1, 3; Z_2 = (0, 0, .)),
    and the fluctuations split the same sum by the sign of s_p."""
    rng = np.random.default_rng(51)
    for _ in range(200):
        ql = np.array([rng.uniform(0.2, 3.0), rng.uniform(-2, 2), rng.uniform(-2, 2)])
        qr = np.array([rng.uniform(0.2, 3.0), rng.uniform(-2, 2), rng.uniform(-2, 2)])
        B_l, B_r = rng.uniform(-0.5, 0.5, size=2)
        Z, s, am, ap = oracle.riemann("shallow_water_bathy", ql, qr, B_l=B_l, B_r=B_r)
        delta = sw_flux_with_source_jump(ql, qr, B_l, B_r)
        scale = np.abs(delta).max() + 1.0
        assert np.abs(Z.sum(axis=0) - delta).max() <= 1e-13 * scale
        assert np.abs(am + ap - delta).max() <= 1e-13 * scale
        for p in (0, 2):
            assert abs(Z[p][1] - s[p] * Z[p][0]) <= 1e-13 * scale
        assert Z[1][0] == 0.0 and Z[1][1] == 0.0
        np.testing.assert_allclose(am, sum(Z[p] for p in range(3) if s[p] < 0) + 0 * am, atol=1e-14 * scale)


@pytest.mark.parametrize("bc", ["periodic", "extrap", "wall"])
@pytest.mark.parametrize("limiter", ["none", "minmod", "mc", "first_order"])
def test_bathymetry_lake_at_rest_bitwise(bc, limiter):
    """Well-balanced: a flat surface at rest over a seamount stays exactly at
    rest (the flux jump and the source cancel at every interface)."""
    p = inputs.sw_bathymetry(48, limiter=limiter, bc=bc, hump=0.0)
    r = Oracle(p).run_steps(p.q0, 8)["q"]
    np.testing.assert_array_equal(r, p.q0)


def test_bathymetry_momentum_changes_by_the_source_only():
    """Periodic, y-uniform data: one step keeps sum h and sum hv, and sum hu
    changes by exactly -nu g sum_I h_bar_I (B_I - B_{I-1}) over the N
    interfaces (the fluctuations telescope except for the source; the
    correction fluxes telescope)."""
    N, ny = 64, 2
    rng = np.random.default_rng(57)
    x = inputs.centres(N, 0.0, 1.0)
    B = 0.2 * np.sin(2 * np.pi * x) + 0.05 * np.cos(6 * np.pi * x)
    h = 1.0 + 0.1 * np.cos(2 * np.pi * x + 0.3)
    hu = 0.2 * np.sin(4 * np.pi * x)
    hv = 0.1 * np.cos(2 * np.pi * x)
    q0 = np.repeat(np.stack([h, hu, hv])[:, None, :], ny, axis=1)
    p = line_problem("shallow_water_bathy", N, ny=ny, limiter="mc", q0=q0,
                     B_cell=np.repeat(B[None, :], ny, axis=0))
    dt = 0.3 * p.dx[0] / 4.0
    r = Oracle(p).run_steps(q0, 1, fixed_dt=dt)["q"]
    nu = dt / p.dx[0]
    hbar = 0.5 * (h + np.roll(h, 1))
    dB = B - np.roll(B, 1)
    expect = hu.sum() - nu * G * np.sum(hbar * dB)
    assert abs(r[0][0].sum() - h.sum()) <= 1e-13 * h.sum()
    assert abs(r[1][0].sum() - expect) <= 1e-13 * np.abs(hu).sum()
    assert abs(r[2][0].sum() - hv.sum()) <= 1e-13 * np.abs(hv).sum()


@pytest.mark.parametrize("limiter", ["none", "first_order"])
def test_bathymetry_flat_bottom_matches_shallow_water(limiter):
    """With a flat bottom psi = 0 and, by the Roe property, Z_p = s_p W_p; the
    f-wave correction 1/2 sign(s)(1 - nu|s|) Z then equals 1/2 |s|(1 - nu|s|) W,
    so without a limiter (and in first order) the scheme is the shallow-water
    scheme (subsonic data: no entropy fix)."""
    pb = inputs.random_problem("shallow_water_bathy", (41, 33), limiter, "periodic")
    pb = pb.with_(B_cell=np.full_like(pb.B_cell, 0.25))
    ps = pb.with_(system="shallow_water", B_cell=None)
    rb = Oracle(pb).run_steps(pb.q0, 6)
    rs = Oracle(ps).run_steps(ps.q0, 6)
    for f in range(3):
        assert oracle.rel_linf(rb["q"][f], rs["q"][f]) <= 1e-12
    assert rb["t"] == pytest.approx(rs["t"], rel=1e-14)


def test_bathymetry_mass_conservation_periodic():
    p = inputs.random_problem("shallow_water_bathy", (45, 38), "minmod", "periodic", discontinuous=True)
    r = Oracle(p).run_steps(p.q0, 10)["q"]
    assert abs(r[0].sum() - p.q0[0].sum()) <= 1e-13 * p.q0[0].sum()


# ---------------------------------------------------------------- unsplit update

def test_transverse_acoustics_sums_to_B_times_fluctuation():
    """Constant coefficients: the down- and up-going parts add up to B a with
    B = [[0, 0, K], [0, 0, 0], [1/rho, 0, 0]] on (p, u_n, u_t); the down part
    moves at -c, the up part at +c along eigenvectors (-+Z, 0, 1)."""
    rng = np.random.default_rng(61)
    for rho, K in ((1.0, 4.0), (2.5, 0.7)):
        B = np.array([[0, 0, K], [0, 0, 0], [1 / rho, 0, 0]])
        Z = math.sqrt(rho * K)
        for _ in range(20):
            a = rng.normal(size=3)
            bm, bp = oracle.transverse("acoustics", a, rho=(rho,) * 3, K=(K,) * 3)
            np.testing.assert_allclose(bm + bp, B @ a, rtol=0, atol=1e-14 * (1 + np.abs(B @ a).max()))
            assert bm[1] == 0.0 and bp[1] == 0.0
            assert abs(bm[0] + Z * bm[2]) <= 1e-14 * (1 + abs(bm[0]))
            assert abs(bp[0] - Z * bp[2]) <= 1e-14 * (1 + abs(bp[0]))


def test_transverse_shallow_water_sums_to_jacobian_for_equal_states():
    """With equal states around the cell the Roe averages are that state and
    the two parts add up to the transverse flux Jacobian (along u_t) applied
    to a: for g(q) = (h v, h u v, h v^2 + g h^2/2) in (h, h u, h v)."""
    rng = np.random.default_rng(67)
    for _ in range(50):
        h, u, v = rng.uniform(0.3, 3.0), rng.uniform(-1, 1), rng.uniform(-1, 1)
        q = np.array([h, h * u, h * v])
        J = np.array([[0.0, 0.0, 1.0],
                      [-u * v, v, u],
                      [G * h - v * v, 0.0, 2 * v]])
        a = rng.normal(size=3)
        bm, bp = oracle.transverse("shallow_water", a, q, q, q)
        np.testing.assert_allclose(bm + bp, J @ a, rtol=0, atol=1e-12 * (1 + np.abs(J @ a).max()))


@pytest.mark.parametrize("system", ["acoustics", "shallow_water"])
def test_unsplit_on_y_uniform_data_is_the_1d_scheme(system):
    """y-uniform periodic data: the y Riemann problems vanish and the
    transverse fluxes are equal on every row, so the unsplit step equals the
    split step (whose y sweep does nothing) bitwise."""
    N, ny = 40, 4
    rng = np.random.default_rng(71)
    row = rng.normal(size=(3, N))
    if system == "shallow_water":
        row[0] = 1.0 + 0.2 * np.abs(row[0])
    q0 = np.repeat(row[:, None, :], ny, axis=1)
    pg = line_problem(system, N, ny=ny, limiter="mc", q0=q0, K=4.0)
    pu = pg.with_(splitting="unsplit")
    dt = 0.3 * pg.dx[0] / 4.0
    np.testing.assert_array_equal(Oracle(pu).run_steps(q0, 3, fixed_dt=dt)["q"],
                                  Oracle(pg).run_steps(q0, 3, fixed_dt=dt)["q"])


@pytest.mark.parametrize("system", ["acoustics", "acoustics_var", "shallow_water"])
def test_unsplit_commutes_with_transposition(system):
    """The unsplit update treats x and y alike: transposing the data (and
    swapping u, v) transposes the result, to rounding -- dimensional
    splitting does not (its x-then-y order shows at O(dt^2))."""
    p = inputs.random_problem(system, (24, 24), "mc", "periodic", discontinuous=True)
    qT = np.stack([p.q0[0].T, p.q0[2].T, p.q0[1].T])
    pT = p.with_(q0=qT)
    if system == "acoustics_var":
        pT = pT.with_(rho_cell=p.rho_cell.T.copy(), K_cell=p.K_cell.T.copy())
    out = {}
    for split in ("unsplit", "godunov"):
        r = Oracle(p.with_(splitting=split)).run_steps(p.q0, 5, fixed_dt=0.002)["q"]
        rT = Oracle(pT.with_(splitting=split)).run_steps(qT, 5, fixed_dt=0.002)["q"]
        out[split] = np.abs(r - np.stack([rT[0].T, rT[2].T, rT[1].T])).max()
    assert out["unsplit"] <= 1e-14
    assert out["godunov"] >= 1e-4


def test_unsplit_diagonal_plane_wave_second_order():
    """A plane wave along the diagonal (both directions and the transverse
    terms active): second order without a limiter."""
    def err(N):
        c, Z = 2.0, 2.0
        xs = inputs.centres(N, 0.0, 1.0)
        Y, X = np.meshgrid(xs, xs, indexing="ij")
        f = lambda X, Y: np.sin(2 * np.pi * (X + Y))
        q0 = np.zeros((3, N, N))
        q0[0] = f(X, Y)
        q0[1] = q0[0] / (Z * math.sqrt(2))
        q0[2] = q0[0] / (Z * math.sqrt(2))
        p = inputs.Problem(2, (N, N), (0, 0), (1, 1), "acoustics", "none", ("periodic",) * 4, q0, K=4.0,
                           splitting="unsplit")
        t = 0.125
        r = Oracle(p).advance(q0, t)
        s = c * t / math.sqrt(2)
        return np.abs(r["q"][0] - f(X - s, Y - s)).mean()
    e = [err(N) for N in (32, 64, 128)]
    rates = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert min(rates) >= 1.9, (e, rates)


@pytest.mark.parametrize("bc", ["periodic", "wall"])
def test_unsplit_conserves_and_keeps_lake_at_rest(bc):
    p = inputs.random_problem("shallow_water", (33, 27), "minmod", bc, discontinuous=True).with_(splitting="unsplit")
    r = Oracle(p).run_steps(p.q0, 8)["q"]
    assert abs(r[0].sum() - p.q0[0].sum()) <= 1e-13 * p.q0[0].sum()
    q = np.zeros((3, 27, 33))
    q[0] = 1.7
    lake = p.with_(q0=q)
    np.testing.assert_array_equal(Oracle(lake).run_steps(q, 5)["q"], q)


def test_transverse_acoustics_with_different_cells_is_the_normal_solver():
    """Per-cell coefficients: the down-going part of a fluctuation a is the
    left-going flux (A-dQ) of the normal Riemann problem between the cell
    below and the cell for the jump a in (p, u_t), the up-going part the
    right-going flux (A+dQ) of the problem between the cell and the cell
    above."""
    rng = np.random.default_rng(73)
    for _ in range(30):
        rho = rng.uniform(0.5, 4.0, size=3)
        K = rng.uniform(0.5, 4.0, size=3)
        a = rng.normal(size=3)
        bm, bp = oracle.transverse("acoustics", a, rho=rho, K=K)
        jump = [a[0], a[2]]
        _, _, am_lo, _ = oracle.riemann("acoustics", [0.0, 0.0], jump, rho[0], K[0], rho[1], K[1])
        _, _, _, ap_hi = oracle.riemann("acoustics", [0.0, 0.0], jump, rho[1], K[1], rho[2], K[2])
        np.testing.assert_allclose([bm[0], bm[2]], am_lo, rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose([bp[0], bp[2]], ap_hi, rtol=1e-13, atol=1e-15)
        assert bm[1] == 0.0 and bp[1] == 0.0


def test_transverse_shallow_water_uses_each_neighbour_for_its_half():
    """The down-going part depends on the cell below (not above) and the
    up-going part on the cell above (not below)."""
    rng = np.random.default_rng(79)
    def state():
        h = rng.uniform(0.5, 2.0)
        return np.array([h, h * rng.uniform(-0.5, 0.5), h * rng.uniform(-0.5, 0.5)])
    qc, qd, qu, other = state(), state(), state(), state()
    a = rng.normal(size=3)
    bm, bp = oracle.transverse("shallow_water", a, qd, qc, qu)
    bm2, bp2 = oracle.transverse("shallow_water", a, qd, qc, other)
    bm3, bp3 = oracle.transverse("shallow_water", a, other, qc, qu)
    np.testing.assert_array_equal(bm, bm2)
    np.testing.assert_array_equal(bp, bp3)
    assert np.abs(bp - bp2).max() > 1e-6 and np.abs(bm - bm3).max() > 1e-6


def test_unsplit_is_exact_for_quadratic_data():
    """Constant-coefficient acoustics without a limiter: one unsplit step of
    cell averages of quadratic data equals the cell averages of the exact
    solution q0 - t L q0 + t^2/2 L^2 q0 (L = A d/dx + B d/dy; every higher
    derivative vanishes) away from the boundary -- the transverse waves give
    the cross term t^2/2 (AB + BA) q_xy.  Dimensional splitting misses it."""
    rho, K = 1.0, 4.0
    A = np.array([[0, K, 0], [1 / rho, 0, 0], [0, 0, 0]])
    B = np.array([[0, 0, K], [0, 0, 0], [1 / rho, 0, 0]])
    coef = np.random.default_rng(83).normal(size=(3, 6))   # a + b x + c y + d x^2 + e xy + f y^2
    N = 24
    dx = 1.0 / N
    xs = inputs.centres(N, 0.0, 1.0)
    Y, X = np.meshgrid(xs, xs, indexing="ij")
    a_, b_, c_, d_, e_, f_ = (coef[:, k][:, None, None] for k in range(6))
    q0 = a_ + b_ * X + c_ * Y + d_ * X ** 2 + e_ * X * Y + f_ * Y ** 2 + (d_ + f_) * dx ** 2 / 12
    Px = b_ + 2 * d_ * X + e_ * Y
    Py = c_ + e_ * X + 2 * f_ * Y
    Lq = np.einsum("ij,jyx->iyx", A, Px) + np.einsum("ij,jyx->iyx", B, Py)
    L2q = A @ A @ (2 * coef[:, 3]) + (A @ B + B @ A) @ coef[:, 4] + B @ B @ (2 * coef[:, 5])
    dt = 0.7 * dx / 2.0
    exact = q0 - dt * Lq + 0.5 * dt ** 2 * L2q[:, None, None]
    p = inputs.Problem(2, (N, N), (0, 0), (1, 1), "acoustics", "none", ("extrap",) * 4, q0, K=K,
                       splitting="unsplit")
    r = Oracle(p).run_steps(q0, 1, fixed_dt=dt)["q"]
    assert np.abs(r - exact)[:, 4:-4, 4:-4].max() <= 1e-13 * np.abs(exact).max()
    rg = Oracle(p.with_(splitting="godunov")).run_steps(q0, 1, fixed_dt=dt)["q"]
    assert np.abs(rg - exact)[:, 4:-4, 4:-4].max() >= 1e-5
