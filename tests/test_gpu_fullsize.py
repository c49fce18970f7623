"""Parity at the benchmark's full size (4096^2 periodic multimode flow, the
launch configuration bench.py times): one CUDA step is checked against the
oracle's update of sampled single cells (random cells plus domain corners and
edges), computed from the same pre-step populations.  FP64 storage: every
population within 1e-13 of the largest population; FP32-deviation storage:
within 2e-7 (float storage of the new deviation)."""
import numpy as np
import pytest
import torch

from oracle import dvbm_oracle as O
from paper_2510_04197_gb300 import inputs as I
from helpers import abi_to_oracle_perm

pytestmark = pytest.mark.gpu
N = 4096


@pytest.fixture(scope="module")
def D():
    from paper_2510_04197_gb300 import build, dvbm
    import os
    if not os.path.exists(dvbm.LIBPATH):
        build.build()
    return dvbm


def sample_cells(n_random=48, seed=7):
    rng = np.random.default_rng(seed)
    cells = [(0, 0), (0, N - 1), (N - 1, 0), (N - 1, N - 1), (0, N // 2), (N - 1, 17), (N // 3, 0), (5, N - 2),
             (1, 1), (N - 2, N - 2)]
    cells += [tuple(int(v) for v in rng.integers(0, N, 2)) for _ in range(n_random)]
    return cells


def patches(pops, cells):
    """[50, B, 5, 5] cross neighbourhoods (periodic wrap) of sampled cells."""
    ys = torch.tensor([[(y + d) % N for d in range(-2, 3)] for (y, x) in cells], device=pops.device)
    xs = torch.tensor([[(x + d) % N for d in range(-2, 3)] for (y, x) in cells], device=pops.device)
    out = pops[:, ys[:, :, None], xs[:, None, :]]  # [50, B, 5, 5]
    return out.double().cpu()


@pytest.mark.parametrize("storage", [0, 1])
def test_fullsize_step_matches_oracle_at_sampled_cells(D, storage):
    F = I.multimode(N, seed=0, rms_Ma=0.3)
    sim = D.Simulation(N, N, 0.71, 1.4, 5e-5, storage=storage, check_every=-1)
    sim.init(*(torch.tensor(a) for a in (F.rho, F.ux, F.uy, F.T)))
    sim.step(3)  # leave the equilibrium initial state
    cells = sample_cells()
    before = patches(sim.populations(), cells)
    sim.step(1)
    after = sim.populations()
    ys = torch.tensor([c[0] for c in cells], device=after.device)
    xs = torch.tensor([c[1] for c in cells], device=after.device)
    got = after[:, ys, xs].double().cpu()  # [50, B]
    lat = O.Lattice()
    perm = abi_to_oracle_perm(lat)
    if storage == 1:  # deviations -> populations: reference w rho0 (f), w rho0 (C_v - R) T0 (g)
        wa, wb = (7 + 2 * np.sqrt(10)) / 60, (7 - 2 * np.sqrt(10)) / 60
        wnode = np.array([8 / 15, wa, wa, wb, wb])
        wabi = torch.tensor(np.outer(wnode, wnode).reshape(25), dtype=torch.float64)
        gref = 1.0 * (1.0 / 0.4 - 1.0) * 1.0
        ref = torch.cat([wabi, wabi * gref])
        before = before + ref[:, None, None, None]
        got = got + ref[:, None]
    fb = before[:25][perm]
    gb = before[25:][perm]
    P = O.Params(Pr=0.71, gamma=1.4, mu=5e-5)
    grid = O.Grid(N, N)
    fo, go = O.step_patch(lat, P, grid, fb, gb, sim.dt)
    fg, gg = got[:25][perm], got[25:][perm]
    tol = 1e-13 if storage == 0 else 2e-7
    ef = (fg - fo).abs().max() / fo.abs().max()
    eg = (gg - go).abs().max() / go.abs().max()
    assert ef < tol and eg < tol, (float(ef), float(eg))


def test_fullsize_d2q16_step_matches_oracle_at_sampled_cells(D):
    """The same check for the total-energy split (I) on D2Q16, the bench's
    third leg: one CUDA step at 4096^2 against the oracle's update of sampled
    cells, every population within 1e-13 of the largest."""
    F = I.multimode(N, seed=0, rms_Ma=0.3)
    sim = D.Simulation(N, N, 0.71, 1.4, 5e-5, lattice=D.D2Q16_SPLIT_I, check_every=-1)
    sim.init(*(torch.tensor(a) for a in (F.rho, F.ux, F.uy, F.T)))
    sim.step(3)
    cells = sample_cells()
    before = patches(sim.populations(), cells)  # [32, B, 5, 5]
    sim.step(1)
    after = sim.populations()
    ys = torch.tensor([c[0] for c in cells], device=after.device)
    xs = torch.tensor([c[1] for c in cells], device=after.device)
    got = after[:, ys, xs].double().cpu()
    lat = O.Lattice(kind="D2Q16")
    perm = abi_to_oracle_perm(lat)
    P = O.Params(Pr=0.71, gamma=1.4, mu=5e-5, split="I")
    fo, go = O.step_patch(lat, P, O.Grid(N, N), before[:16][perm], before[16:][perm], sim.dt)
    fg, gg = got[:16][perm], got[16:][perm]
    ef = (fg - fo).abs().max() / fo.abs().max()
    eg = (gg - go).abs().max() / go.abs().max()
    assert ef < 1e-13 and eg < 1e-13, (float(ef), float(eg))
