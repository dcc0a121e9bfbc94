"""Exact solution of the 1D Euler Riemann problem for an ideal gas.

Textbook construction (Godunov's exact solver): the star-region pressure solves
f_L(p) + f_R(p) + (u_R - u_L) = 0 with the shock / rarefaction branches of f_K,
found by Newton iteration; the solution is then sampled along x/t.  Used only as
an independent reference for shock-tube tests.
"""
import math

import numpy as np


def _fk(p, rho, pk, g):
    a = math.sqrt(g * pk / rho)
    if p > pk:                                   # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        s = math.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (p + B))
    e = (g - 1.0) / (2.0 * g)                    # rarefaction
    return 2.0 * a / (g - 1.0) * ((p / pk) ** e - 1.0), (p / pk) ** (-(g + 1.0) / (2.0 * g)) / (rho * a)


def star_state(left, right, g):
    rl, ul, pl = left
    rr, ur, pr = right
    p = max(1e-12, 0.5 * (pl + pr))
    for _ in range(200):
        fl, dl = _fk(p, rl, pl, g)
        fr, dr = _fk(p, rr, pr, g)
        f = fl + fr + (ur - ul)
        pn = max(1e-14, p - f / (dl + dr))
        if abs(pn - p) <= 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _fk(p, rl, pl, g)
    fr, _ = _fk(p, rr, pr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def _sample_vacuum(left, right, g, xi):
    """Two rarefactions separated by vacuum (u_R - u_L >= 2(a_L + a_R)/(g-1))."""
    rl, ul, pl = left
    rr, ur, pr = right
    al, ar = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    sl_vac = ul + 2 * al / (g - 1)
    sr_vac = ur - 2 * ar / (g - 1)
    out = np.zeros((3, len(xi)))
    for n, s in enumerate(xi):
        if s <= ul - al:
            st = (rl, ul, pl)
        elif s < sl_vac:
            u = 2 / (g + 1) * (al + (g - 1) / 2 * ul + s)
            c = 2 / (g + 1) * (al + (g - 1) / 2 * (ul - s))
            st = (rl * (c / al) ** (2 / (g - 1)), u, pl * (c / al) ** (2 * g / (g - 1)))
        elif s <= sr_vac:
            st = (0.0, 0.5 * (sl_vac + sr_vac), 0.0)
        elif s < ur + ar:
            u = 2 / (g + 1) * (-ar + (g - 1) / 2 * ur + s)
            c = 2 / (g + 1) * (ar - (g - 1) / 2 * (ur - s))
            st = (rr * (c / ar) ** (2 / (g - 1)), u, pr * (c / ar) ** (2 * g / (g - 1)))
        else:
            st = (rr, ur, pr)
        out[:, n] = st
    return out


def sample(left, right, g, xi):
    """(rho, u, p) at similarity coordinates xi = (x - x0) / t."""
    rl, ul, pl = left
    rr, ur, pr = right
    if ur - ul >= 2 * (math.sqrt(g * pl / rl) + math.sqrt(g * pr / rr)) / (g - 1):
        return _sample_vacuum(left, right, g, xi)
    ps, us = star_state(left, right, g)
    out = np.zeros((3, len(xi)))
    for n, s in enumerate(xi):
        if s <= us:                              # left of contact
            al = math.sqrt(g * pl / rl)
            if ps > pl:
                sl = ul - al * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                if s <= sl:
                    st = (rl, ul, pl)
                else:
                    r = rl * ((ps / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pl + 1))
                    st = (r, us, ps)
            else:
                ast = al * (ps / pl) ** ((g - 1) / (2 * g))
                if s <= ul - al:
                    st = (rl, ul, pl)
                elif s >= us - ast:
                    st = (rl * (ps / pl) ** (1 / g), us, ps)
                else:
                    u = 2 / (g + 1) * (al + (g - 1) / 2 * ul + s)
                    c = 2 / (g + 1) * (al + (g - 1) / 2 * (ul - s))
                    r = rl * (c / al) ** (2 / (g - 1))
                    st = (r, u, pl * (c / al) ** (2 * g / (g - 1)))
        else:                                    # right of contact
            ar = math.sqrt(g * pr / rr)
            if ps > pr:
                sr = ur + ar * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                if s >= sr:
                    st = (rr, ur, pr)
                else:
                    r = rr * ((ps / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pr + 1))
                    st = (r, us, ps)
            else:
                ast = ar * (ps / pr) ** ((g - 1) / (2 * g))
                if s >= ur + ar:
                    st = (rr, ur, pr)
                elif s <= us + ast:
                    st = (rr * (ps / pr) ** (1 / g), us, ps)
                else:
                    u = 2 / (g + 1) * (-ar + (g - 1) / 2 * ur + s)
                    c = 2 / (g + 1) * (ar - (g - 1) / 2 * (ur - s))
                    r = rr * (c / ar) ** (2 / (g - 1))
                    st = (r, u, pr * (c / ar) ** (2 * g / (g - 1)))
        out[:, n] = st
    return out
