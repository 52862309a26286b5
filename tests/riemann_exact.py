"""Exact solution of the 1D shallow-water Riemann problem on a flat bed.

Textbook construction (Toro 2001, ch. 5 "exact Riemann solver" for the SWE):
the star depth h* solves f_L(h*) + f_R(h*) + u_R - u_L = 0 with
f_K(h) = 2 (sqrt(g h) - sqrt(g h_K)) for a rarefaction (h <= h_K) and
f_K(h) = (h - h_K) sqrt(g (h + h_K) / (2 h h_K)) for a shock (h > h_K).
Dry-bed (Ritter) and two-rarefaction cases use their closed forms.
Independent of the oracle: a pin, not a re-typing of it.
"""
import math

import numpy as np


def _fK(h, hK, g):
    if h <= hK:
        return 2.0 * (math.sqrt(g * h) - math.sqrt(g * hK))
    return (h - hK) * math.sqrt(0.5 * g * (h + hK) / (h * hK))


def star_state(hL, uL, hR, uR, g=9.81):
    """(h*, u*) for two wet states; bisection on the monotone f."""
    f = lambda h: _fK(h, hL, g) + _fK(h, hR, g) + uR - uL  # noqa: E731
    lo, hi = 1e-14, 10.0 * max(hL, hR) + (uL - uR) ** 2 / g + 1.0
    if f(lo) > 0:  # dry middle (vacuum): not used by these tests
        raise ValueError("vacuum generated")
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) > 0:
            hi = mid
        else:
            lo = mid
    hs = 0.5 * (lo + hi)
    us = 0.5 * (uL + uR) + 0.5 * (_fK(hs, hR, g) - _fK(hs, hL, g))
    return hs, us


def sample(xi, hL, uL, hR, uR, g=9.81):
    """Depth and velocity at similarity coordinate xi = (x - x0)/t (array)."""
    xi = np.asarray(xi, dtype=np.float64)
    h = np.empty_like(xi)
    u = np.empty_like(xi)
    cL, cR = math.sqrt(g * hL), math.sqrt(g * hR)
    if hR == 0.0:  # dry bed on the right (Ritter-type)
        head, front = uL - cL, uL + 2 * cL
        for i, s in enumerate(xi):
            if s <= head:
                h[i], u[i] = hL, uL
            elif s >= front:
                h[i], u[i] = 0.0, 0.0
            else:
                c = (uL + 2 * cL - s) / 3.0
                h[i], u[i] = c * c / g, (uL + 2 * cL + 2 * s) / 3.0
        return h, u
    hs, us = star_state(hL, uL, hR, uR, g)
    cs = math.sqrt(g * hs)
    for i, s in enumerate(xi):
        if s <= us:  # left of the contact
            if hs > hL:  # left shock
                SL = uL - cL * math.sqrt(0.5 * (hs + hL) * hs / (hL * hL))
                h[i], u[i] = (hL, uL) if s <= SL else (hs, us)
            else:
                if s <= uL - cL:
                    h[i], u[i] = hL, uL
                elif s >= us - cs:
                    h[i], u[i] = hs, us
                else:
                    c = (uL + 2 * cL - s) / 3.0
                    h[i], u[i] = c * c / g, (uL + 2 * cL + 2 * s) / 3.0
        else:
            if hs > hR:  # right shock
                SR = uR + cR * math.sqrt(0.5 * (hs + hR) * hs / (hR * hR))
                h[i], u[i] = (hR, uR) if s >= SR else (hs, us)
            else:
                if s >= uR + cR:
                    h[i], u[i] = hR, uR
                elif s <= us + cs:
                    h[i], u[i] = hs, us
                else:
                    c = (-uR + 2 * cR + s) / 3.0
                    h[i], u[i] = c * c / g, (uR - 2 * cR + 2 * s) / 3.0
    return h, u


def shock_speed_right(hL, uL, hR, uR, g=9.81):
    hs, us = star_state(hL, uL, hR, uR, g)
    cR = math.sqrt(g * hR)
    return uR + cR * math.sqrt(0.5 * (hs + hR) * hs / (hR * hR))
