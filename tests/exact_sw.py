"""Exact solution of the 1D shallow-water dam-break Riemann problem.

Written independently of the oracle (closed forms plus a scalar root find),
so it can pin the oracle's shallow-water scheme.  Left state (h_l, 0), right
state (h_r, 0), h_l > h_r > 0: a left rarefaction and a right shock.

  rarefaction:  u_m = 2 (sqrt(g h_l) - sqrt(g h_m)),
  shock:        u_m = (h_m - h_r) sqrt(g/2 (1/h_m + 1/h_r)),
  shock speed:  S = h_m u_m / (h_m - h_r),
  fan (xi between -sqrt(g h_l) and u_m - sqrt(g h_m)):
                h = (2 sqrt(g h_l) - xi)^2 / (9 g),  u = 2 (sqrt(g h_l) + xi) / 3.
"""
import numpy as np
from scipy.optimize import brentq


def dam_break_state(h_l, h_r, g=9.81):
    def mismatch(hm):
        u_rare = 2.0 * (np.sqrt(g * h_l) - np.sqrt(g * hm))
        u_shock = (hm - h_r) * np.sqrt(0.5 * g * (1.0 / hm + 1.0 / h_r))
        return u_rare - u_shock

    hm = brentq(mismatch, h_r, h_l, xtol=1e-15, rtol=1e-15, maxiter=500)
    um = 2.0 * (np.sqrt(g * h_l) - np.sqrt(g * hm))
    S = hm * um / (hm - h_r)
    head = -np.sqrt(g * h_l)
    tail = um - np.sqrt(g * hm)
    return dict(h_m=hm, u_m=um, shock=S, head=head, tail=tail)


def dam_break_profile(x, t, h_l, h_r, x0=0.0, g=9.81):
    """(h, hu) at positions x and time t > 0."""
    st = dam_break_state(h_l, h_r, g)
    xi = (np.asarray(x, dtype=np.float64) - x0) / t
    h = np.empty_like(xi)
    u = np.empty_like(xi)
    left = xi <= st["head"]
    fan = (xi > st["head"]) & (xi <= st["tail"])
    mid = (xi > st["tail"]) & (xi <= st["shock"])
    right = xi > st["shock"]
    h[left], u[left] = h_l, 0.0
    c_l = np.sqrt(g * h_l)
    h[fan] = (2.0 * c_l - xi[fan]) ** 2 / (9.0 * g)
    u[fan] = 2.0 * (c_l + xi[fan]) / 3.0
    h[mid], u[mid] = st["h_m"], st["u_m"]
    h[right], u[right] = h_r, 0.0
    return h, h * u


def ritter_profile(x, t, h_l, x0=0.0, g=9.81):
    """Ritter's dam break onto a dry bed (h_l, 0) | (0, 0), flat bottom, t > 0:
    still water left of xi = -c_l, the fan h = (2 c_l - xi)^2 / (9 g),
    u = 2 (c_l + xi) / 3 for -c_l < xi < 2 c_l (c_l = sqrt(g h_l)), dry beyond
    the front xi = 2 c_l.  Returns (h, hu)."""
    c_l = np.sqrt(g * h_l)
    xi = (np.asarray(x, dtype=np.float64) - x0) / t
    fan = (xi > -c_l) & (xi < 2.0 * c_l)
    h = np.where(xi <= -c_l, h_l, 0.0)
    u = np.zeros_like(xi)
    h[fan] = (2.0 * c_l - xi[fan]) ** 2 / (9.0 * g)
    u[fan] = 2.0 * (c_l + xi[fan]) / 3.0
    return h, h * u
