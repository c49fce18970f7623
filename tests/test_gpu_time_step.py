"""The fixed time step of the explicit scheme (Sec. III.A.3 rule, held fixed
from the initial field) and the limits dvbm_init enforces on it: the fastest
population crosses at most one cell per step (max_i |v_i| dt / min(dx, dy) <= 1,
the upwind stencil's domain of dependence), and dt <= min(tau1, tau2) =
mu / p_max * min(1, 1/Pr) (forward-Euler relaxation, tau from Sec. II.C with
p = rho R T).  The paper states neither limit; each is checked just inside
and just outside, and a refused dvbm_init leaves the context as it was."""
import math

import numpy as np
import pytest
import torch

from paper_2510_04197_gb300 import inputs as I

pytestmark = pytest.mark.gpu

XI_MAX = {0: math.sqrt(5 + math.sqrt(10)), 1: math.sqrt(3 + math.sqrt(6))}  # D2Q25, D2Q16


@pytest.fixture(scope="module")
def D():
    from paper_2510_04197_gb300 import build, dvbm
    import os
    if not os.path.exists(dvbm.LIBPATH):
        build.build()
    return dvbm


def fields(Nx, Ny, T_max=1.0):
    """rho = 1, u = 0, T from 1 up to T_max (p = rho T peaks at T_max)."""
    F = I.uniform(Nx, Ny)
    T = np.ones((Ny, Nx))
    T[Ny // 2, Nx // 3] = T_max
    return [torch.tensor(a) for a in (F.rho, F.ux, F.uy, T)]


def status_of(D, fn):
    try:
        fn()
    except D.DVBMError as e:
        return e.status, str(e)
    return D.OK, ""


@pytest.mark.parametrize("lattice", [0, 1])
def test_one_cell_per_step_limit(D, lattice):
    """dx = 1/8, dy = 1/16: the limit is min(dx, dy) / (xi_max sqrt(R T_ref))."""
    Nx = Ny = 8
    limit = (0.5 / Ny) / XI_MAX[lattice]
    for dt, ok in ((0.995 * limit, True), (1.005 * limit, False)):
        sim = D.Simulation(Nx, Ny, 0.71, 1.4, 1.0, lattice=lattice, Lx=1.0, Ly=0.5, dt=dt)
        st, msg = status_of(D, lambda: sim.init(*fields(Nx, Ny)))
        if ok:
            assert st == D.OK, msg
            sim.step(1)
        else:
            assert st == D.EINVAL and "cells per step" in msg, (st, msg)


def test_cfl_rule_can_exceed_the_lattice_limit(D):
    """The paper's CFL rule measures |u| + c_s, slower than the fastest
    population (xi_max = 2.86 against c_s = 1.18 at rest): CFL 0.4 is inside,
    CFL 0.5 moves the fastest population 1.21 cells per step."""
    for cfl, ok in ((0.4, True), (0.5, False)):
        sim = D.Simulation(8, 8, 0.71, 1.4, 1.0, cfl=cfl)
        st, msg = status_of(D, lambda: sim.init(*fields(8, 8)))
        assert (st == D.OK) == ok, (cfl, st, msg)


@pytest.mark.parametrize("lattice", [0, 1])
@pytest.mark.parametrize("Pr", [0.71, 2.0])
def test_relaxation_time_limit(D, lattice, Pr):
    """tau_min = mu / p_max * min(1, 1/Pr), set by the largest pressure of the
    initial field (here one cell at p = 1.5), not by its mean."""
    mu, T_max = 2e-3, 1.5
    tau_min = mu / T_max * min(1.0, 1.0 / Pr)
    for dt, ok in ((0.995 * tau_min, True), (1.005 * tau_min, False)):
        sim = D.Simulation(8, 8, Pr, 1.4, mu, lattice=lattice, dt=dt)
        st, msg = status_of(D, lambda: sim.init(*fields(8, 8, T_max)))
        if ok:
            assert st == D.OK, msg
        else:
            assert st == D.EINVAL and "relaxation time" in msg, (st, msg)


def test_refused_init_leaves_the_context_as_it_was(D):
    mu, dt = 2e-3, 1.5e-3  # inside the limit at p = 1, outside at p = 2
    sim = D.Simulation(8, 8, 0.71, 1.4, mu, dt=dt)
    sim.init(*fields(8, 8))
    sim.step(3)
    before = sim.populations().clone()
    st, msg = status_of(D, lambda: sim.init(*fields(8, 8, T_max=2.0)))
    assert st == D.EINVAL, msg
    assert sim.steps == 3 and sim.dt == dt
    assert torch.equal(sim.populations(), before)
    sim.step(1)  # still a working context


def test_set_state_without_init_checks_opts_dt(D):
    good = D.Simulation(8, 8, 0.71, 1.4, 1.0, dt=1e-3)
    good.init(*fields(8, 8))
    st = good.get_state()
    limit = (1.0 / 8) / XI_MAX[0]
    bad = D.Simulation(8, 8, 0.71, 1.4, 1.0, dt=1.01 * limit)
    s, msg = status_of(D, lambda: bad.set_state(st))
    assert s == D.EINVAL and "cells per step" in msg, (s, msg)
    ok = D.Simulation(8, 8, 0.71, 1.4, 1.0, dt=0.99 * limit)
    ok.set_state(st)
    assert ok.steps == 0
