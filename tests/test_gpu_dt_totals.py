"""The CUDA path's time step and domain totals against the oracle.

* dt: dvbm_init fixes dt = CFL min(dx, dy) / max(|u| + sqrt(gamma R T)) over
  the initial field (Sec. III.A.3, reading R10) in its own reduction kernel;
  the oracle's cfl_dt (pinned by hand-worked examples in
  tests/test_oracle_cfl.py) must give the same dt to 1e-15 relative, for both
  lattices, on non-square cells and for non-unit R, and on the hand-worked
  example fields themselves (tiled onto a grid the ABI accepts).
* totals: dvbm_totals (mass, momentum, total energy of the current state,
  Sec. III.B conservation) against the oracle's totals of the same
  populations, read back through dvbm_get_state: 1e-13 relative (momentum
  relative to total mass times c, since periodic flows carry almost none).
"""
import math
import os

import numpy as np
import pytest
import torch

from oracle import dvbm_oracle as O
from paper_2510_04197_gb300 import inputs as I
from helpers import abi_to_oracle_perm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    from paper_2510_04197_gb300 import build, dvbm
    if not os.path.exists(dvbm.LIBPATH):
        build.build()
    assert torch.cuda.is_available()
    return dvbm


def _t(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64)


@pytest.mark.parametrize("lattice", [0, 1])
@pytest.mark.parametrize("shape,L,R,cfl", [((64, 64), (1.0, 1.0), 1.0, 0.01),
                                           ((64, 48), (1.0, 0.5), 1.0, 0.3),
                                           ((37, 29), (2.0, 1.0), 287.0, 0.05)])
def test_init_dt_matches_oracle_cfl_dt(D, lattice, shape, L, R, cfl):
    Nx, Ny = shape
    T_ref = 300.0 if R != 1.0 else 1.0
    c = math.sqrt(R * T_ref)
    F = I.random_smooth(Nx, Ny, seed=Nx + Ny, amp=0.2, Ma=0.8)
    ux, uy, T = F.ux * c, F.uy * c, F.T * T_ref  # the same dimensionless flow in physical units
    sim = D.Simulation(Nx, Ny, 0.71, 1.4, 1e-2 * c, lattice=lattice, Lx=L[0], Ly=L[1], cfl=cfl, R=R, T_ref=T_ref)
    sim.init(*(torch.tensor(a) for a in (F.rho, ux, uy, T)))
    P = O.Params(Pr=0.71, gamma=1.4, mu=1e-2 * c, R=R, T_ref=T_ref, split="I" if lattice == 1 else "II")
    dt_o = O.cfl_dt(P, O.Grid(Nx, Ny, L[0], L[1]), _t(ux), _t(uy), _t(T), cfl)
    assert abs(sim.dt - dt_o) <= 1e-15 * dt_o, (sim.dt, dt_o)
    sim.close()


def test_init_dt_on_worked_examples(D):
    """The hand-worked examples of tests/golden/cfl_dt_worked_examples.txt,
    tiled 4x4 times so the grid meets the ABI's minimum size (tiling changes
    neither the largest speed nor, with the domain scaled along, the cell
    size): dvbm_init's dt equals the hand-computed fraction."""
    from test_oracle_cfl import read_cases
    for case in read_cases():
        cells = np.array(case["cells"]).reshape(case["Ny"], case["Nx"], 3)
        tiled = np.tile(cells, (4, 4, 1))
        Ny, Nx = tiled.shape[:2]
        sim = D.Simulation(Nx, Ny, 0.71, case["gamma"], 10.0, Lx=4 * case["Lx"], Ly=4 * case["Ly"],
                           cfl=case["cfl"], R=case["R"])
        sim.init(torch.ones(Ny, Nx, dtype=torch.float64), *(torch.tensor(tiled[..., k].copy()) for k in range(3)))
        assert abs(sim.dt - case["dt"]) <= 1e-15 * case["dt"], (case["name"], sim.dt, case["dt"])
        sim.close()


def _oracle_state(sim, lattice, storage, rho0=1.0, T0=1.0, gamma=1.4, R=1.0):
    """The context's populations in the oracle's order (FP32-deviation
    storage: the reference w rho0, w rho0 (C_v - R) T0 added back)."""
    kind = "D2Q16" if lattice == 1 else "D2Q25"
    lat = O.Lattice(R, 1.0, kind)
    perm = abi_to_oracle_perm(lat)
    pops = sim.populations().double().cpu()
    Q = lat.Q
    if storage == 1:
        w = torch.tensor([float(x) for x in lat.w], dtype=torch.float64)
        # ABI order c = 5 p + q; lat.w is in the oracle's order: map it back
        inv = np.argsort(perm)
        w_abi = w[inv]
        gref = rho0 * (R / (gamma - 1.0) - R) * T0
        pops = pops + torch.cat([w_abi * rho0, w_abi * gref])[:, None, None]
    return lat, pops[:Q][perm], pops[Q:][perm]


@pytest.mark.parametrize("lattice,storage", [(0, 0), (0, 1), (1, 0)])
@pytest.mark.parametrize("nsteps", [0, 50])
def test_totals_match_oracle_totals(D, lattice, storage, nsteps):
    Nx, Ny = 48, 40
    F = I.random_smooth(Nx, Ny, seed=13, amp=0.15, Ma=0.6)
    sim = D.Simulation(Nx, Ny, 0.71, 1.4, 2e-3, lattice=lattice, storage=storage, Lx=1.0, Ly=40 / 48, dt=2e-4)
    sim.init(*(torch.tensor(a) for a in (F.rho, F.ux, F.uy, F.T)))
    sim.step(nsteps)
    got = sim.totals()
    lat, f, g = _oracle_state(sim, lattice, storage)
    P = O.Params(Pr=0.71, gamma=1.4, mu=2e-3, split="I" if lattice == 1 else "II")
    ref = O.totals(lat, P, O.Grid(Nx, Ny, 1.0, 40 / 48), f, g)
    mass = abs(ref[0])
    assert abs(got[0] - ref[0]) <= 1e-13 * mass, (got, ref)
    for k in (1, 2):
        assert abs(got[k] - ref[k]) <= 1e-13 * mass, (k, got, ref)
    assert abs(got[3] - ref[3]) <= 1e-13 * abs(ref[3]), (got, ref)
    sim.close()
