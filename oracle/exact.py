"""Exact solutions used to pin the oracle (test infrastructure only).

* The advected density wave: with u = 1 in every direction and p = 1, the
  Euler equations transport rho unchanged, rho(x, t) = rho0(x - t (1,..,1)).
* The exact solution of the one-dimensional Riemann problem for an ideal gas
  (the Sod shock tube of Sec. 5.5 is one): the star pressure solves
  f_L(p) + f_R(p) + (u_R - u_L) = 0, where f_K is the shock (Rankine-Hugoniot)
  branch for p > p_K and the isentropic rarefaction branch otherwise; the
  solution is then sampled on x / t.  Written from the standard pressure-
  function formulation of the exact Riemann solver (e.g. Toro, "Riemann
  Solvers and Numerical Methods for Fluid Dynamics", ch. 4).
"""
import math

import numpy as np


def density_wave_rho(x_sum, t, dim, amp=0.2):
    """rho at points whose coordinate sum is x_sum, at time t, domain [0, 2)^dim."""
    return 1.0 + amp * np.sin(np.pi * (x_sum - dim * t))


def _fK(p, rho, pK, gamma):
    """Pressure function of one side and its derivative."""
    a = math.sqrt(gamma * pK / rho)
    if p > pK:  # shock
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pK
        q = math.sqrt(A / (p + B))
        return (p - pK) * q, q * (1.0 - 0.5 * (p - pK) / (p + B))
    # rarefaction
    e = (gamma - 1.0) / (2.0 * gamma)
    f = 2.0 * a / (gamma - 1.0) * ((p / pK) ** e - 1.0)
    df = 1.0 / (rho * a) * (p / pK) ** (-(gamma + 1.0) / (2.0 * gamma))
    return f, df


def star_state(left, right, gamma=1.4, tol=1e-14):
    """(p*, u*) for left/right primitive states (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    p = max(1e-12, 0.5 * (pl + pr))
    for _ in range(200):
        fl, dfl = _fK(p, rl, pl, gamma)
        fr, dfr = _fK(p, rr, pr, gamma)
        g = fl + fr + (ur - ul)
        pn = max(1e-14, p - g / (dfl + dfr))
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _fK(p, rl, pl, gamma)
    fr, _ = _fK(p, rr, pr, gamma)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def riemann_sample(left, right, xi, gamma=1.4):
    """Primitive state (rho, u, p) at similarity coordinates xi = (x - x0) / t."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(left, right, gamma)
    al = math.sqrt(gamma * pl / rl)
    ar = math.sqrt(gamma * pr / rr)
    g1 = (gamma - 1.0) / (gamma + 1.0)
    xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
    out = np.zeros((3, xi.size))
    for k, s in enumerate(xi):
        if s <= us:  # left of the contact
            if ps > pl:  # left shock
                rs = rl * (ps / pl + g1) / (g1 * ps / pl + 1.0)
                sl = ul - al * math.sqrt((gamma + 1.0) / (2 * gamma) * ps / pl + (gamma - 1.0) / (2 * gamma))
                out[:, k] = (rl, ul, pl) if s < sl else (rs, us, ps)
            else:  # left rarefaction
                rs = rl * (ps / pl) ** (1.0 / gamma)
                asl = al * (ps / pl) ** ((gamma - 1.0) / (2 * gamma))
                head, tail = ul - al, us - asl
                if s < head:
                    out[:, k] = (rl, ul, pl)
                elif s > tail:
                    out[:, k] = (rs, us, ps)
                else:
                    u = 2.0 / (gamma + 1.0) * (al + (gamma - 1.0) / 2.0 * ul + s)
                    c = 2.0 / (gamma + 1.0) * (al + (gamma - 1.0) / 2.0 * (ul - s))
                    rho = rl * (c / al) ** (2.0 / (gamma - 1.0))
                    out[:, k] = (rho, u, pl * (c / al) ** (2.0 * gamma / (gamma - 1.0)))
        else:  # right of the contact
            if ps > pr:  # right shock
                rs = rr * (ps / pr + g1) / (g1 * ps / pr + 1.0)
                sr = ur + ar * math.sqrt((gamma + 1.0) / (2 * gamma) * ps / pr + (gamma - 1.0) / (2 * gamma))
                out[:, k] = (rr, ur, pr) if s > sr else (rs, us, ps)
            else:  # right rarefaction
                rs = rr * (ps / pr) ** (1.0 / gamma)
                asr = ar * (ps / pr) ** ((gamma - 1.0) / (2 * gamma))
                head, tail = ur + ar, us + asr
                if s > head:
                    out[:, k] = (rr, ur, pr)
                elif s < tail:
                    out[:, k] = (rs, us, ps)
                else:
                    u = 2.0 / (gamma + 1.0) * (-ar + (gamma - 1.0) / 2.0 * ur + s)
                    c = 2.0 / (gamma + 1.0) * (ar - (gamma - 1.0) / 2.0 * (ur - s))
                    rho = rr * (c / ar) ** (2.0 / (gamma - 1.0))
                    out[:, k] = (rho, u, pr * (c / ar) ** (2.0 * gamma / (gamma - 1.0)))
    return out
