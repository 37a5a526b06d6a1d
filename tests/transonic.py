"""Where the Harten-Hyman entropy fix acts in a shallow-water state.

The fix (the fluctuation split of a transonic rarefaction, used by the
shallow-water Riemann solver of Sec. 3 / Eq. LW-update) only runs at an
interface whose 1-wave has lam_l < 0 < lam_m at the Roe middle state
q_m = Q_l + W1, or whose 3-wave has lam_m < 0 < lam_r at q_m = Q_r - W3.
This module counts such interfaces in a state, from the oracle's Riemann
solver, so that a parity case can show it really reaches the fix rather
than silently staying subsonic.
"""
import math

import numpy as np

import oracle


def transonic_counts(prob, q):
    """{(d, wave): number of interfaces along direction d whose wave 1 or 3
    is a transonic rarefaction} for a 2D shallow-water state q[f, y, x]."""
    g = prob.g
    out = {}
    for d in range(prob.ndim):
        # reduced state along d: (h, normal momentum, transverse momentum)
        h, qn, qt = q[0], q[1 + d], q[2 - d]
        if d == 1:
            h, qn, qt = h.T, qn.T, qt.T
        n1 = n3 = 0
        for row in range(h.shape[0]):
            for i in range(h.shape[1] - 1):
                ql = np.array([h[row, i], qn[row, i], qt[row, i]])
                qr = np.array([h[row, i + 1], qn[row, i + 1], qt[row, i + 1]])
                W, s, am, ap = oracle.riemann("shallow_water", ql, qr, g=g)
                lam_l = ql[1] / ql[0] - math.sqrt(g * ql[0])
                hm = ql[0] + W[0][0]
                if hm > 0.0 and lam_l < 0.0 < (ql[1] + W[0][1]) / hm - math.sqrt(g * hm):
                    n1 += 1
                lam_r = qr[1] / qr[0] + math.sqrt(g * qr[0])
                hm = qr[0] - W[2][0]
                if hm > 0.0 and (qr[1] - W[2][1]) / hm + math.sqrt(g * hm) < 0.0 < lam_r:
                    n3 += 1
        out[(d, 1)] = n1
        out[(d, 3)] = n3
    return out


def oracle_run_counting(prob, nsteps, chunks=3):
    """Run the oracle for nsteps accepted steps in `chunks` pieces (bitwise
    the same as one run: the step size carries over) and add up the
    transonic interfaces of the state at the start of every piece and at
    the end.  Returns (oracle result of the whole run, counts)."""
    o = oracle.Oracle(prob)
    q, t, dt = prob.q0, 0.0, 0.0
    total = {}
    sizes = [nsteps // chunks + (1 if k < nsteps % chunks else 0) for k in range(chunks)]
    res = None
    for k, n in enumerate(sizes):
        for key, v in transonic_counts(prob, q).items():
            total[key] = total.get(key, 0) + v
        res = o.run_steps(q, n, t=t, dt=dt)
        q, t, dt = res["q"], res["t"], res["dt"]
        res["nacc"] = sum(sizes[:k + 1])
    for key, v in transonic_counts(prob, q).items():
        total[key] = total.get(key, 0) + v
    return res, total
