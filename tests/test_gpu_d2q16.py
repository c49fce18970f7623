"""Total-energy split (I) on the D2Q16 lattice (the paper's first model):
CUDA path vs the FP64 oracle, per-field relative 1e-12 (FP64 storage)."""
import math

import numpy as np
import pytest
import torch

from oracle import dvbm_oracle as O
from paper_2510_04197_gb300 import inputs as I
from helpers import abi_to_oracle_perm, field_errors, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    from paper_2510_04197_gb300 import build, dvbm
    import os
    if not os.path.exists(dvbm.LIBPATH):
        build.build()
    return dvbm


def run16(D, F, Pr, gamma, mu, n, bcs=None, dt=None, cfl=0.01):
    Ny, Nx = F.rho.shape
    kw = dict(Lx=F.Lx, Ly=F.Ly, cfl=cfl)
    if dt:
        kw["dt"] = dt
    sim = D.Simulation(Nx, Ny, Pr, gamma, mu, bcs=bcs, lattice=D.D2Q16_SPLIT_I, **kw)
    sim.init(*(torch.tensor(a) for a in (F.rho, F.ux, F.uy, F.T)))
    sim.step(n)
    return sim, {k: v.cpu().numpy() for k, v in sim.moments().items()}


def test_d2q16_wave_decay_1000_steps(D):
    F = I.wave_decay(64, 64, Ma=0.1, amp=1e-3)
    sim, g = run16(D, F, 0.71, 1.4, 0.01, 1000)
    _, o = oracle_run(F, 0.71, 1.4, 0.01, sim.dt, 1000, split="I")
    e = field_errors(g, o)
    assert max(e.values()) < 1e-12, e


@pytest.mark.parametrize("Pr", [0.5, 1.0, 2.0])
def test_d2q16_ragged_all_prandtl(D, Pr):
    F = I.random_smooth(37, 13, seed=31, amp=0.1, Ma=0.4)
    sim, g = run16(D, F, Pr, 1.4, 2e-3, 100, dt=2e-4)
    _, o = oracle_run(F, Pr, 1.4, 2e-3, sim.dt, 100, split="I")
    e = field_errors(g, o)
    assert max(e.values()) < 1e-12, e


def test_d2q16_populations_one_step(D):
    F = I.random_smooth(33, 18, seed=4, amp=0.1, Ma=0.5)
    sim, _ = run16(D, F, 2.0, 1.67, 2e-3, 1, dt=2e-4)
    s, _ = oracle_run(F, 2.0, 1.67, 2e-3, sim.dt, 1, split="I")
    pops = sim.populations().cpu().numpy()
    perm = abi_to_oracle_perm(s.lat)
    for a, b in ((pops[:16][perm], s.f.numpy()), (pops[16:][perm], s.g.numpy())):
        assert np.abs(a - b).max() < 1e-13 * np.abs(b).max()


def test_d2q16_wall_and_zero_gradient_parity(D):
    cs = I.couette(Nx=4, Ny=24, Ma=0.5, gamma=1.4)
    F = cs.fields
    dt = min(0.4 * (F.Ly / 24) / math.sqrt(3 + math.sqrt(6)), 0.25 * cs.mu)
    bcs = [D.ZEROGRAD, D.ZEROGRAD, (D.WALL, (0.0, 0.0), cs.T_C), (D.WALL, (cs.u0, 0.0), cs.T_H)]
    sim, g = run16(D, F, 0.71, 1.4, cs.mu, 150, bcs=bcs, dt=dt)
    ob = (O.BC(O.ZEROGRAD), O.BC(O.ZEROGRAD), O.BC(O.WALL, (0.0, 0.0), cs.T_C), O.BC(O.WALL, (cs.u0, 0.0), cs.T_H))
    _, o = oracle_run(F, 0.71, 1.4, cs.mu, dt, 150, bcs=ob, split="I")
    e = field_errors(g, o)
    assert max(e.values()) < 1e-12, e


def test_d2q16_conserves_totals(D):
    F = I.random_smooth(48, 40, seed=6, amp=0.1, Ma=0.5)
    sim, _ = run16(D, F, 0.71, 1.4, 2e-3, 0, dt=2e-4)
    t0 = sim.totals()
    sim.step(200)
    t1 = sim.totals()
    for a, b in zip(t0, t1):
        assert abs(a - b) < 1e-13 * max(1.0, abs(a)), (t0, t1)
