"""Exact solution of the 1-D Riemann problem for an ideal gas (textbook
construction: the star-region pressure solves f_L(p) + f_R(p) + u_R - u_L = 0
with shock (Rankine--Hugoniot) or rarefaction (isentropic) branches; the
solution is then sampled along x/t).  Used as the inviscid reference of the
Sod shock tube (Sec. III.B)."""
import math

import numpy as np


def _branch(p, rho_k, p_k, gamma):
    """f_k(p) and its derivative for side k (shock if p > p_k, else rarefaction)."""
    c_k = math.sqrt(gamma * p_k / rho_k)
    if p > p_k:
        A = 2.0 / ((gamma + 1.0) * rho_k)
        B = (gamma - 1.0) / (gamma + 1.0) * p_k
        s = math.sqrt(A / (p + B))
        return (p - p_k) * s, s * (1.0 - 0.5 * (p - p_k) / (p + B))
    r = (p / p_k) ** ((gamma - 1.0) / (2.0 * gamma))
    return 2.0 * c_k / (gamma - 1.0) * (r - 1.0), (p / p_k) ** (-(gamma + 1.0) / (2.0 * gamma)) / (rho_k * c_k)


def star_state(rhoL, uL, pL, rhoR, uR, pR, gamma):
    p = 0.5 * (pL + pR)
    for _ in range(100):
        fL, dL = _branch(p, rhoL, pL, gamma)
        fR, dR = _branch(p, rhoR, pR, gamma)
        f = fL + fR + uR - uL
        dp = f / (dL + dR)
        p = max(p - dp, 1e-12)
        if abs(dp) < 1e-14 * p:
            break
    fL, _ = _branch(p, rhoL, pL, gamma)
    fR, _ = _branch(p, rhoR, pR, gamma)
    u = 0.5 * (uL + uR) + 0.5 * (fR - fL)
    return p, u


def sample(x, t, x0, left, right, gamma):
    """rho, u, p at positions x and time t > 0 for a discontinuity at x0."""
    rhoL, uL, pL = left
    rhoR, uR, pR = right
    ps, us = star_state(rhoL, uL, pL, rhoR, uR, pR, gamma)
    cL = math.sqrt(gamma * pL / rhoL)
    cR = math.sqrt(gamma * pR / rhoR)
    g1 = (gamma - 1.0) / (gamma + 1.0)
    out = np.zeros((3, len(x)))
    for k, xx in enumerate(x):
        S = (xx - x0) / t
        if S <= us:  # left of the contact
            if ps > pL:  # left shock
                rs = rhoL * (ps / pL + g1) / (g1 * ps / pL + 1.0)
                SL = uL - cL * math.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pL + (gamma - 1.0) / (2.0 * gamma))
                out[:, k] = (rhoL, uL, pL) if S < SL else (rs, us, ps)
            else:  # left rarefaction
                rs = rhoL * (ps / pL) ** (1.0 / gamma)
                cs = cL * (ps / pL) ** ((gamma - 1.0) / (2.0 * gamma))
                SH, ST = uL - cL, us - cs
                if S < SH:
                    out[:, k] = (rhoL, uL, pL)
                elif S > ST:
                    out[:, k] = (rs, us, ps)
                else:
                    u = 2.0 / (gamma + 1.0) * (cL + (gamma - 1.0) / 2.0 * uL + S)
                    c = 2.0 / (gamma + 1.0) * (cL + (gamma - 1.0) / 2.0 * (uL - S))
                    rho = rhoL * (c / cL) ** (2.0 / (gamma - 1.0))
                    out[:, k] = (rho, u, pL * (c / cL) ** (2.0 * gamma / (gamma - 1.0)))
        else:  # right of the contact
            if ps > pR:  # right shock
                rs = rhoR * (ps / pR + g1) / (g1 * ps / pR + 1.0)
                SR = uR + cR * math.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pR + (gamma - 1.0) / (2.0 * gamma))
                out[:, k] = (rhoR, uR, pR) if S > SR else (rs, us, ps)
            else:  # right rarefaction
                rs = rhoR * (ps / pR) ** (1.0 / gamma)
                cs = cR * (ps / pR) ** ((gamma - 1.0) / (2.0 * gamma))
                SH, ST = uR + cR, us + cs
                if S > SH:
                    out[:, k] = (rhoR, uR, pR)
                elif S < ST:
                    out[:, k] = (rs, us, ps)
                else:
                    u = 2.0 / (gamma + 1.0) * (-cR + (gamma - 1.0) / 2.0 * uR + S)
                    c = 2.0 / (gamma + 1.0) * (cR - (gamma - 1.0) / 2.0 * (uR - S))
                    rho = rhoR * (c / cR) ** (2.0 / (gamma - 1.0))
                    out[:, k] = (rho, u, pR * (c / cR) ** (2.0 * gamma / (gamma - 1.0)))
    return out
