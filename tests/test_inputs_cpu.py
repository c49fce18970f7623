"""Checks of the seeded input generators that fix a physical property by
construction (Sec. III.E, III.F): the shock--vortex states satisfy the
Rankine--Hugoniot jump conditions (mass, momentum and energy fluxes equal
across the stationary shock, and the normal-shock Mach relation), the vortex
reaches its tangential Mach number at r = r_v, and the Couette set-up has the
requested Mach, Reynolds and Eckert numbers."""
import math

import numpy as np
import pytest

from paper_2510_04197_gb300 import inputs as I


def far_states(sv, gamma):
    """Unperturbed left and right states on a row far from the vortex."""
    F = sv.fields
    j = 0  # bottom row: the vortex (exp(-r^2/2) factor) is negligible there
    rho, ux, T = F.rho[j], F.ux[j], F.T[j]
    p = rho * T  # R = 1
    return (rho[0], ux[0], p[0]), (rho[-1], ux[-1], p[-1])


@pytest.mark.parametrize("make", [lambda: I.shock_vortex(N=256),
                                  lambda: I.shock_vortex_case("C", 280, 240),
                                  lambda: I.shock_vortex_case("G", 280, 240)])
def test_shock_states_satisfy_rankine_hugoniot(make):
    gamma = 1.4
    sv = make()
    (rl, ul, pl), (rr, ur, pr) = far_states(sv, gamma)
    El = pl / (gamma - 1) + 0.5 * rl * ul * ul
    Er = pr / (gamma - 1) + 0.5 * rr * ur * ur
    assert math.isclose(rl * ul, rr * ur, rel_tol=1e-9)
    assert math.isclose(rl * ul * ul + pl, rr * ur * ur + pr, rel_tol=1e-9)
    assert math.isclose((El + pl) * ul, (Er + pr) * ur, rel_tol=1e-9)
    Ml = ul / math.sqrt(gamma * pl / rl)
    Mr = ur / math.sqrt(gamma * pr / rr)
    assert math.isclose(Mr * Mr, ((gamma - 1) * Ml * Ml + 2) / (2 * gamma * Ml * Ml - (gamma - 1)), rel_tol=1e-9)
    assert Ml > 1.0 > Mr


def test_vortex_tangential_mach_number():
    """Case G geometry: along the vertical line through the vortex centre the
    velocity perturbation peaks at r = r_v with magnitude Ma_v c_s,l."""
    Nx, Ny = 2800, 2400  # dx = 0.01: the peak is resolved to 1e-4
    sv = I.shock_vortex_case("G", Nx, Ny)
    F = sv.fields
    x = (np.arange(Nx) + 0.5) * 28.0 / Nx
    y = (np.arange(Ny) + 0.5) * 24.0 / Ny
    i = int(np.argmin(np.abs(x - 6.0)))
    du = F.ux[:, i] - F.ux[0, i]  # subtract the (left) base flow
    k = int(np.argmax(np.abs(du)))
    assert abs(abs(y[k] - 12.0) - 1.0) < 0.011
    assert math.isclose(np.abs(du).max(), 0.39 * sv.cs_l, rel_tol=1e-4)


@pytest.mark.parametrize("Ma,Ec", [(0.5, 4.0), (1.2, 40.0)])
def test_couette_numbers(Ma, Ec):
    gamma = 1.4
    cs = I.couette(Nx=4, Ny=128, Ma=Ma, Ec=Ec, gamma=gamma)
    assert math.isclose(cs.u0 / math.sqrt(gamma * cs.T_C), Ma, rel_tol=1e-12)
    assert math.isclose(cs.u0 * 1.0 / cs.mu, 100.0, rel_tol=1e-12)  # Re = rho u0 L / mu, rho = 1
    Cp = gamma / (gamma - 1)
    assert math.isclose(cs.u0 ** 2 / (Cp * (cs.T_H - cs.T_C)), Ec, rel_tol=1e-9)
