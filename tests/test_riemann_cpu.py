"""Checks of the exact Riemann helper by invariants (no tabulated values):
Rankine--Hugoniot fluxes are continuous across its shock, entropy p/rho^gamma
and the Riemann invariant u + 2c/(gamma-1) are constant through its left
rarefaction, and p, u are continuous at the contact."""
import math

import numpy as np

from riemann import sample


def test_sod_solution_satisfies_jump_and_isentropic_relations():
    g = 1.4
    L, R = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    t = 0.2
    x = np.linspace(-0.5, 1.5, 40001)
    rho, u, p = sample(x, t, 0.5, L, R, g)
    # locate the shock: the largest density jump right of the contact
    j = np.argmax(np.abs(np.diff(rho)) * (x[:-1] > 0.8))
    a, b = j - 2, j + 3
    s = (x[j] - 0.5) / t  # shock speed
    m = lambda r, v: r * (v - s)
    E = lambda r, v, pp: pp / (g - 1) + 0.5 * r * v * v
    assert math.isclose(m(rho[a], u[a]), m(rho[b], u[b]), rel_tol=2e-3)
    assert math.isclose(m(rho[a], u[a]) * (u[a] - s) + p[a], m(rho[b], u[b]) * (u[b] - s) + p[b], rel_tol=2e-3)
    # isentropic left rarefaction (between the head x = 0.5 - c_L t and the contact)
    cL = math.sqrt(g)
    sel = (x > 0.5 - cL * t + 0.01) & (x < 0.5 + 0.1 * t)
    ent = p[sel] / rho[sel] ** g
    inv = u[sel] + 2 * np.sqrt(g * p[sel] / rho[sel]) / (g - 1)
    assert np.allclose(ent, 1.0, rtol=1e-10) and np.allclose(inv, 2 * cL / (g - 1), rtol=1e-10)
    # contact: pressure and velocity continuous, density jumps
    k = np.argmin(np.abs(x - (0.5 + u[np.argmax(x > 0.7)] * t)))
    assert abs(p[k - 5] - p[k + 5]) < 1e-10 and abs(u[k - 5] - u[k + 5]) < 1e-10
    assert rho[k - 5] - rho[k + 5] > 0.1
