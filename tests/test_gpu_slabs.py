"""Slab decomposition along y on one GPU: a grid split into bands, one libdvbm
context per band, halo rows moved with dvbm_halo_pack / dvbm_halo_unpack and
device-to-device copies (paper_2510_04197_gb300.slab.LocalSlabs).

* Bands whose heights are multiples of the step kernel's 8-row tile tile the
  grid exactly as the undecomposed run does, so the run is bitwise equal to
  the single-context run: periodic 64^2 for 1000 steps (and within 1e-12 of
  the oracle), zero-gradient x, walls in y, FP32-deviation storage, D2Q16.
* Ragged bands (heights not multiples of 8) change the step kernel's tiles,
  hence its block exponents: within 1e-12 of the oracle.
* The halo contract: a stale halo, several steps per call, a missing or an
  unexpected halo buffer and a time step beyond the limits are refused.
"""
import math
import os

import numpy as np
import pytest
import torch

from oracle import dvbm_oracle as O
from paper_2510_04197_gb300 import inputs as I
from helpers import field_errors, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    from paper_2510_04197_gb300 import build, dvbm
    if not os.path.exists(dvbm.LIBPATH):
        build.build()
    assert torch.cuda.is_available()
    return dvbm


def _fields(F):
    return [torch.tensor(a) for a in (F.rho, F.ux, F.uy, F.T)]


def _single(D, F, nsteps, **kw):
    Ny, Nx = F.rho.shape
    sim = D.Simulation(Nx, Ny, kw.pop("Pr", 0.71), 1.4, kw.pop("mu", 2e-3), Lx=F.Lx, Ly=F.Ly, check_every=-1, **kw)
    sim.init(*_fields(F))
    sim.step(nsteps)
    return sim


def _slabs(D, F, nsteps, parts=2, heights=None, **kw):
    from paper_2510_04197_gb300 import slab
    Ny, Nx = F.rho.shape
    sl = slab.LocalSlabs(Nx, Ny, parts, kw.pop("Pr", 0.71), 1.4, kw.pop("mu", 2e-3), heights=heights, Lx=F.Lx,
                         Ly=F.Ly, check_every=-1, **kw)
    sl.init(*_fields(F))
    sl.step(nsteps)
    return sl


def test_two_bands_periodic_1000_steps_bitwise_and_oracle(D):
    F = I.random_smooth(64, 64, seed=21, amp=0.1, Ma=0.5)
    a = _single(D, F, 1000, dt=2e-4)
    b = _slabs(D, F, 1000, parts=2, dt=2e-4)
    assert b.heights == [32, 32]
    assert torch.equal(a.populations(), b.populations())
    g = {k: v.cpu().numpy() for k, v in b.moments().items()}
    _, o = oracle_run(F, 0.71, 1.4, 2e-3, b.dt, 1000)
    e = field_errors(g, o)
    assert max(e.values()) < 1e-12, e
    a.close()
    b.close()


def test_cfl_time_step_is_the_smallest_band_step(D):
    """Without a fixed dt every band takes the smallest of the bands' CFL
    steps, which is the undecomposed grid's CFL step."""
    F = I.random_smooth(64, 48, seed=4, amp=0.2, Ma=0.8)
    a = _single(D, F, 0, cfl=0.05)
    b = _slabs(D, F, 0, parts=3, cfl=0.05)
    assert all(s.dt == a.dt for s in b.sims), (a.dt, [s.dt for s in b.sims])


def test_zero_gradient_x_three_bands_bitwise(D):
    F = I.random_smooth(48, 48, seed=8, amp=0.1, Ma=0.5)
    bcs = [D.ZEROGRAD, D.ZEROGRAD, D.PERIODIC, D.PERIODIC]
    a = _single(D, F, 200, dt=2e-4, bcs=bcs)
    b = _slabs(D, F, 200, parts=3, dt=2e-4, bcs=bcs)
    assert b.heights == [16, 16, 16]
    assert torch.equal(a.populations(), b.populations())


def test_walls_in_y_three_bands_bitwise(D):
    """Thermal Couette start-up: walls at the bottom of the first band and
    the top of the last one, EXTERNAL halos between the bands."""
    cs = I.couette(Nx=4, Ny=24, Ma=0.5, gamma=1.4)
    F = cs.fields
    dt = min(0.4 * (F.Ly / 24) / math.sqrt(5 + math.sqrt(10)), 0.25 * cs.mu / 2.0)
    bcs = [D.PERIODIC, D.PERIODIC, (D.WALL, (0.0, 0.0), cs.T_C), (D.WALL, (cs.u0, 0.0), cs.T_H)]
    a = _single(D, F, 300, dt=dt, bcs=bcs, Pr=2.0, mu=cs.mu)
    b = _slabs(D, F, 300, parts=3, dt=dt, bcs=bcs, Pr=2.0, mu=cs.mu)
    assert b.heights == [8, 8, 8]
    assert torch.equal(a.populations(), b.populations())


@pytest.mark.parametrize("lattice,storage", [(0, 1), (1, 0)])
def test_other_storage_and_lattice_bitwise(D, lattice, storage):
    F = I.random_smooth(40, 32, seed=9, amp=0.1, Ma=0.5)
    a = _single(D, F, 100, dt=2e-4, lattice=lattice, storage=storage)
    b = _slabs(D, F, 100, parts=2, dt=2e-4, lattice=lattice, storage=storage)
    assert b.heights == [16, 16]
    assert torch.equal(a.populations(), b.populations())


def test_ragged_bands_match_oracle(D):
    F = I.random_smooth(48, 64, seed=17, amp=0.1, Ma=0.5)
    bcs = [D.ZEROGRAD, D.ZEROGRAD, D.PERIODIC, D.PERIODIC]
    b = _slabs(D, F, 200, heights=[24, 17, 23], dt=2e-4, bcs=bcs)
    g = {k: v.cpu().numpy() for k, v in b.moments().items()}
    ob = (O.BC(O.ZEROGRAD), O.BC(O.ZEROGRAD), O.BC(), O.BC())
    _, o = oracle_run(F, 0.71, 1.4, 2e-3, b.dt, 200, bcs=ob)
    e = field_errors(g, o)
    assert max(e.values()) < 1e-12, e
    t = b.totals()
    assert all(np.isfinite(t))


def test_halo_contract(D):
    F = I.random_smooth(32, 16, seed=2, amp=0.1, Ma=0.5)
    bcs = [D.PERIODIC, D.PERIODIC, D.EXTERNAL, D.EXTERNAL]
    sim = D.Simulation(32, 16, 0.71, 1.4, 2e-3, bcs=bcs, dt=2e-4, Lx=F.Lx, Ly=F.Ly)
    sim.init(*_fields(F))
    lo, hi = sim.halo_buffer(), sim.halo_buffer()
    assert sim.halo_bytes == lo.numel() * lo.element_size() == 2 * 32 * 50 * 8
    with pytest.raises(D.DVBMError) as ei:  # no halo supplied since dvbm_init
        sim.step(1)
    assert ei.value.status == D.ESTATE
    sim.halo_pack(lo, hi)
    with pytest.raises(D.DVBMError) as ei:  # both sides are external: both buffers needed
        sim.halo_unpack(hi, None)
    assert ei.value.status == D.EINVAL
    sim.halo_unpack(hi, lo)  # the band is its own periodic neighbour
    with pytest.raises(D.DVBMError) as ei:
        sim.step(2)
    assert ei.value.status == D.EINVAL
    sim.step(1)
    with pytest.raises(D.DVBMError) as ei:  # stale again after the step
        sim.step(1)
    assert ei.value.status == D.ESTATE
    with pytest.raises(D.DVBMError) as ei:  # one cell per step at most
        sim.set_dt(1.0)
    assert ei.value.status == D.EINVAL
    assert sim.dt == 2e-4
    # the periodic self-exchange equals the ordinary periodic context
    ref = D.Simulation(32, 16, 0.71, 1.4, 2e-3, dt=2e-4, Lx=F.Lx, Ly=F.Ly)
    ref.init(*_fields(F))
    ref.step(1)
    assert torch.equal(ref.populations(), sim.populations())
    plain = D.Simulation(32, 16, 0.71, 1.4, 2e-3, dt=2e-4, Lx=F.Lx, Ly=F.Ly)
    plain.init(*_fields(F))
    with pytest.raises(D.DVBMError) as ei:  # no external side: nothing to unpack
        plain.halo_unpack(lo, hi)
    assert ei.value.status == D.EINVAL
