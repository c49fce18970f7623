"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle on the
same seeded inputs.  FP64 storage: per-field relative max-norm error 1e-12;
FP32-deviation storage: 1e-5 on smooth flows."""
import math

import numpy as np
import pytest
import torch

from oracle import dvbm_oracle as O
from paper_2510_04197_gb300 import inputs as I
from helpers import field_errors, oracle_run, abi_to_oracle_perm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    from paper_2510_04197_gb300 import build, dvbm
    import os
    if not os.path.exists(dvbm.LIBPATH):
        build.build()
    assert torch.cuda.is_available()
    return dvbm


def gpu_run(D, F, Pr, gamma, mu, nsteps, storage=0, bcs=None, dt=None, cfl=0.01, **kw):
    Ny, Nx = F.rho.shape
    opts = dict(Lx=F.Lx, Ly=F.Ly, cfl=cfl, **kw)
    if dt:
        opts["dt"] = dt
    sim = D.Simulation(Nx, Ny, Pr, gamma, mu, bcs=bcs, storage=storage, **opts)
    sim.init(*(torch.tensor(a) for a in (F.rho, F.ux, F.uy, F.T)))
    sim.step(nsteps)
    m = {k: v.cpu().numpy() for k, v in sim.moments().items()}
    return sim, m


def test_config1_wave_decay_fp64_1000_steps(D):
    """64 x 64 shear + entropy waves over a Ma = 0.1 mean flow, Pr = 0.71,
    gamma = 1.4, 1000 steps at CFL 0.01: FP64 fields within 1e-12 of the oracle."""
    F = I.wave_decay(64, 64, Ma=0.1, amp=1e-3)
    sim, g = gpu_run(D, F, 0.71, 1.4, 0.01, 1000)
    _, o = oracle_run(F, 0.71, 1.4, 0.01, sim.dt, 1000)
    e = field_errors(g, o)
    assert max(e.values()) < 1e-12, e


def deviation_errors(gpu, ora):
    """Max-norm errors per field relative to the field's largest deviation
    from its own mean (rho, each velocity component, T): the dynamic part of
    the flow, not its mean state, sets the scale."""
    e = {}
    for k in ("rho", "ux", "uy", "T"):
        o = np.asarray(ora[k])
        e[k] = np.abs(np.asarray(gpu[k]) - o).max() / np.abs(o - o.mean()).max()
    return e


@pytest.mark.parametrize("Pr", [0.71, 2.0])
def test_large_amplitude_64_squared_1000_steps(D, Pr):
    """O(0.1) density and temperature perturbations over a Ma 0.5 flow, 64^2,
    1000 steps (t = 0.2, about a quarter of a viscous time of the largest
    mode): errors relative to each field's largest deviation from its mean
    at most 1e-10.  The bound: a step rounds each population at about 1e-16
    of its value; over 1000 steps that grows to ~1e-13 of the mean state,
    i.e. ~1e-12 of a deviation of 0.1, with two orders of margin."""
    F = I.random_smooth(64, 64, seed=21, amp=0.1, Ma=0.5)
    sim, g = gpu_run(D, F, Pr, 1.4, 2e-3, 1000, dt=2e-4)
    _, o = oracle_run(F, Pr, 1.4, 2e-3, sim.dt, 1000)
    e = deviation_errors(g, o)
    assert max(e.values()) < 1e-10, e
    # the run is far from the linear regime: the fields changed by O(amp)
    assert np.abs(o["rho"] - F.rho).max() > 1e-2


@pytest.mark.parametrize("Pr", [0.5, 1.0, 2.0])
@pytest.mark.parametrize("shape", [(40, 24), (37, 13)])
def test_ragged_grids_all_prandtl_cases(D, Pr, shape):
    """Ragged tiles (Nx, Ny not multiples of the 32 x 8 CTA tile), every
    Prandtl branch, O(1) non-equilibrium: 100 steps within 1e-12."""
    Nx, Ny = shape
    F = I.random_smooth(Nx, Ny, seed=11, amp=0.1, Ma=0.5)
    sim, g = gpu_run(D, F, Pr, 1.4, 2e-3, 100, dt=2e-4)
    _, o = oracle_run(F, Pr, 1.4, 2e-3, sim.dt, 100)
    e = field_errors(g, o)
    assert max(e.values()) < 1e-12, e


def test_populations_match_oracle_after_one_step(D):
    """Element-wise population parity (ABI order mapped onto the oracle's)."""
    F = I.random_smooth(33, 18, seed=3, amp=0.1, Ma=0.6)
    sim, _ = gpu_run(D, F, 0.71, 1.67, 2e-3, 1, dt=2e-4)
    s, _ = oracle_run(F, 0.71, 1.67, 2e-3, sim.dt, 1)
    pops = sim.populations().cpu().numpy()
    perm = abi_to_oracle_perm(s.lat)
    f = pops[:25][perm]
    g = pops[25:][perm]
    assert np.abs(f - s.f.numpy()).max() < 1e-14 * np.abs(s.f.numpy()).max() * 10
    assert np.abs(g - s.g.numpy()).max() < 1e-14 * np.abs(s.g.numpy()).max() * 10


def test_fp32_deviation_storage_smooth_flow(D):
    """FP32-deviation storage on the config-1 flow: relative L-inf error against
    the FP64 oracle at most 1e-5 after 1000 steps."""
    F = I.wave_decay(64, 64, Ma=0.1, amp=1e-3)
    sim, g = gpu_run(D, F, 0.71, 1.4, 0.01, 1000, storage=1)
    _, o = oracle_run(F, 0.71, 1.4, 0.01, sim.dt, 1000)
    e = field_errors(g, o)
    assert max(e.values()) < 1e-5, e


def test_uniform_state_fixed_point_and_conservation(D):
    F = I.random_smooth(48, 40, seed=5, amp=0.1, Ma=0.5)
    sim, _ = gpu_run(D, F, 0.71, 1.4, 2e-3, 0, dt=2e-4)
    t0 = sim.totals()
    sim.step(200)
    t1 = sim.totals()
    for a, b in zip(t0, t1):
        assert abs(a - b) < 1e-13 * max(1.0, abs(a)), (t0, t1)


def test_checkpoint_resume_is_bitwise(D):
    F = I.random_smooth(40, 24, seed=7, amp=0.1, Ma=0.5)
    a, _ = gpu_run(D, F, 2.0, 1.4, 2e-3, 20, dt=2e-4)
    ref = a.populations().clone()
    b, _ = gpu_run(D, F, 2.0, 1.4, 2e-3, 10, dt=2e-4)
    st = b.get_state()
    c, _ = gpu_run(D, F, 2.0, 1.4, 2e-3, 0, dt=2e-4)
    c.set_state(st)
    assert c.steps == 10
    c.step(10)
    assert torch.equal(c.populations(), ref)


@pytest.mark.parametrize("beta", [1.0, 1.5, 2.0, math.sqrt(2.0)])
def test_limiter_parameter_range(D, beta):
    """The generalized limiter over its range (Sec. III.A.2: beta = 1 is
    minmod, beta = 2 the MC limiter).  Rational beta run the small-integer
    limiter, irrational beta (sqrt 2) the 64-bit fixed-point one; O(1)
    gradients on a ragged grid, 100 steps, fields within 1e-12."""
    F = I.random_smooth(40, 24, seed=5, amp=0.15, Ma=0.6)
    sim, g = gpu_run(D, F, 0.71, 1.4, 2e-3, 100, dt=2e-4, beta=beta)
    _, o = oracle_run(F, 0.71, 1.4, 2e-3, sim.dt, 100, beta=beta)
    e = field_errors(g, o)
    assert max(e.values()) < 1e-12, (beta, e)


@pytest.mark.parametrize("R,T_ref", [(0.5, 2.0), (287.0, 300.0)])
def test_gas_constant_and_reference_temperature(D, R, T_ref):
    """Lattice velocities scale with c = sqrt(R T_ref) (App. G): the same
    dimensionless flow in physical units (u c, T T_ref, mu c) stays within
    1e-12 of the oracle for air-like R and T_ref too."""
    F0 = I.random_smooth(40, 24, seed=7, amp=0.1, Ma=0.5)
    c = math.sqrt(R * T_ref)
    F = I.Fields(F0.rho, F0.ux * c, F0.uy * c, F0.T * T_ref, F0.Lx, F0.Ly)
    mu = 2e-3 * c
    sim, g = gpu_run(D, F, 0.71, 1.4, mu, 100, dt=2e-4 / c, R=R, T_ref=T_ref)
    _, o = oracle_run(F, 0.71, 1.4, mu, sim.dt, 100, R=R, T_ref=T_ref)
    e = field_errors(g, o)
    assert max(e.values()) < 1e-12, (R, T_ref, e)


@pytest.mark.parametrize("Pr", [1.0, 2.0])
def test_fp32_deviation_storage_other_prandtl_branches(D, Pr):
    """FP32-deviation storage in the Pr = 1 and Pr > 1 branches of Table I
    (smooth O(0.1) flow on a ragged grid, 300 steps): relative L-inf error
    against the FP64 oracle at most 1e-5."""
    F = I.random_smooth(40, 24, seed=3, amp=0.05, Ma=0.3)
    sim, g = gpu_run(D, F, Pr, 1.4, 2e-3, 300, storage=1, dt=2e-4)
    _, o = oracle_run(F, Pr, 1.4, 2e-3, sim.dt, 300)
    e = field_errors(g, o)
    assert max(e.values()) < 1e-5, (Pr, e)


def test_fp32_deviation_storage_with_walls(D):
    """FP32-deviation storage with the no-slip isothermal walls (ghost node +
    non-equilibrium extrapolation, Sec. III.E): thermal Couette start-up,
    4 x 24 cells, 200 steps, relative L-inf error against the FP64 oracle
    at most 1e-5."""
    cs = I.couette(Nx=4, Ny=24, Ma=0.5, gamma=1.4)
    F = cs.fields
    dt = min(0.4 * (F.Ly / 24) / math.sqrt(5 + math.sqrt(10)), 0.25 * cs.mu / 2.0)
    bcs = [D.PERIODIC, D.PERIODIC, (D.WALL, (0.0, 0.0), cs.T_C), (D.WALL, (cs.u0, 0.0), cs.T_H)]
    sim, g = gpu_run(D, F, 2.0, 1.4, cs.mu, 200, storage=1, bcs=bcs, dt=dt)
    ob = (O.BC(), O.BC(), O.BC(O.WALL, (0.0, 0.0), cs.T_C), O.BC(O.WALL, (cs.u0, 0.0), cs.T_H))
    _, o = oracle_run(F, 2.0, 1.4, cs.mu, dt, 200, bcs=ob)
    e = field_errors(g, o)
    assert max(e.values()) < 1e-5, e
