"""Parity at the extreme grid shapes the ABI accepts: the widest grid
(Nx = 2^20 cells, Ny = 4: 32 768 CTAs along x) and the tallest (Nx = 4,
Ny = 65 535: 8 192 CTAs along y, a ragged last tile).  Periodic on both axes,
so the ghost exchange wraps over 4 cells on the short axis.  One CUDA step is
checked against the oracle's update of sampled cells (corners, edges, random
cells) from the same pre-step populations, for D2Q25 split II in both storage
forms and D2Q16 split I.  dt = 0.25 min(dx, dy) (the fastest D2Q25 population
moves 0.71 cells) and mu = 4 dt (dt / tau about 1/4), so that advection and
relaxation both change every population by a visible amount."""
import numpy as np
import pytest
import torch

from oracle import dvbm_oracle as O
from paper_2510_04197_gb300 import inputs as I
from helpers import abi_to_oracle_perm

pytestmark = pytest.mark.gpu

SHAPES = [(1 << 20, 4), (4, 65535)]
CASES = [("d2q25-fp64", 0, 0), ("d2q25-fp32dev", 0, 1), ("d2q16-fp64", 1, 0)]


@pytest.fixture(scope="module")
def D():
    from paper_2510_04197_gb300 import build, dvbm
    import os
    if not os.path.exists(dvbm.LIBPATH):
        build.build()
    return dvbm


def sample_cells(Nx, Ny, n_random=40, seed=5):
    rng = np.random.default_rng(seed)
    cells = [(0, 0), (0, Nx - 1), (Ny - 1, 0), (Ny - 1, Nx - 1), (Ny // 2, Nx // 2), (1, Nx - 2), (Ny - 2, 1),
             (Ny - 1, Nx // 3)]
    cells += [(int(rng.integers(0, Ny)), int(rng.integers(0, Nx))) for _ in range(n_random)]
    return cells


def patches(pops, cells, Nx, Ny):
    """[npop, B, 5, 5] cross neighbourhoods (periodic wrap) of sampled cells."""
    ys = torch.tensor([[(y + d) % Ny for d in range(-2, 3)] for (y, x) in cells], device=pops.device)
    xs = torch.tensor([[(x + d) % Nx for d in range(-2, 3)] for (y, x) in cells], device=pops.device)
    return pops[:, ys[:, :, None], xs[:, None, :]].double().cpu()


@pytest.mark.parametrize("name,lattice,storage", CASES)
@pytest.mark.parametrize("shape", SHAPES)
def test_extreme_grid_step_matches_oracle_at_sampled_cells(D, shape, name, lattice, storage):
    Nx, Ny = shape
    F = I.random_smooth(Nx, Ny, seed=9, amp=0.05, Ma=0.3)  # Lx = 1, Ly = Ny / Nx: dx = dy
    h = 1.0 / Nx
    dt, mu, Pr, gamma = 0.25 * h, h, 0.71, 1.4
    sim = D.Simulation(Nx, Ny, Pr, gamma, mu, lattice=lattice, storage=storage, Lx=F.Lx, Ly=F.Ly, dt=dt,
                       check_every=-1)
    sim.init(*(torch.tensor(a) for a in (F.rho, F.ux, F.uy, F.T)))
    sim.step(2)  # leave the equilibrium initial state
    cells = sample_cells(Nx, Ny)
    before = patches(sim.populations(), cells, Nx, Ny)
    sim.step(1)
    after = sim.populations()
    ys = torch.tensor([c[0] for c in cells], device=after.device)
    xs = torch.tensor([c[1] for c in cells], device=after.device)
    got = after[:, ys, xs].double().cpu()
    lat = O.Lattice(kind="D2Q16") if lattice == 1 else O.Lattice()
    Q = lat.Q
    if storage == 1:  # deviations -> populations: reference w rho0 (f), w rho0 (C_v - R) T0 (g)
        wa, wb = (7 + 2 * np.sqrt(10)) / 60, (7 - 2 * np.sqrt(10)) / 60
        wnode = np.array([8 / 15, wa, wa, wb, wb])
        wabi = torch.tensor(np.outer(wnode, wnode).reshape(25), dtype=torch.float64)
        ref = torch.cat([wabi, wabi * (1.0 / (gamma - 1.0) - 1.0)])
        before = before + ref[:, None, None, None]
        got = got + ref[:, None]
    perm = abi_to_oracle_perm(lat)
    P = O.Params(Pr=Pr, gamma=gamma, mu=mu, split="I" if lattice == 1 else "II")
    grid = O.Grid(Nx, Ny, F.Lx, F.Ly)
    fo, go = O.step_patch(lat, P, grid, before[:Q][perm], before[Q:][perm], sim.dt)
    fg, gg = got[:Q][perm], got[Q:][perm]
    # the step changes the populations by a visible fraction of themselves
    moved = (fo - before[:Q][perm][:, :, 2, 2]).abs().max() / fo.abs().max()
    assert moved > 1e-3, float(moved)
    tol = 1e-13 if storage == 0 else 2e-7
    ef = (fg - fo).abs().max() / fo.abs().max()
    eg = (gg - go).abs().max() / go.abs().max()
    assert ef < tol and eg < tol, (name, shape, float(ef), float(eg))
