"""Shared test helpers: run the oracle on the same seeded inputs as the CUDA
path, map the ABI population order onto the oracle's, and compare fields."""
import numpy as np
import torch

from oracle import dvbm_oracle as O

DT = torch.float64


def oracle_run(F, Pr, gamma, mu, dt, nsteps, bcs=None, R=1.0, T_ref=1.0, beta=1.2, split="II"):
    t = lambda a: torch.tensor(np.asarray(a), dtype=DT)
    Ny, Nx = F.rho.shape
    grid = O.Grid(Nx, Ny, F.Lx, F.Ly, bcs) if bcs else O.Grid(Nx, Ny, F.Lx, F.Ly)
    P = O.Params(Pr=Pr, gamma=gamma, mu=mu, R=R, T_ref=T_ref, beta=beta, split=split)
    s = O.Simulation(grid, P, t(F.rho), t(F.ux), t(F.uy), t(F.T), dt=dt)
    s.run(nsteps)
    rho, ux, uy, T = s.fields()
    return s, {"rho": rho.numpy(), "ux": ux.numpy(), "uy": uy.numpy(), "T": T.numpy()}


def abi_to_oracle_perm(lat):
    """perm[i] = ABI population index of the oracle's population i (matched by velocity)."""
    from paper_2510_04197_gb300.dvbm import abi_velocities, D2Q16_SPLIT_I, D2Q25_SPLIT_II
    vx, vy = abi_velocities(lat.R, lat.T_ref, D2Q16_SPLIT_I if lat.Q == 16 else D2Q25_SPLIT_II)
    perm = []
    for i in range(lat.Q):
        d = np.abs(vx - float(lat.vx[i])) + np.abs(vy - float(lat.vy[i]))
        j = int(np.argmin(d))
        assert d[j] < 1e-12
        perm.append(j)
    assert sorted(perm) == list(range(lat.Q))
    return perm


def field_errors(gpu, ora):
    """Relative max-norm errors per field: rho, velocity vector, T."""
    g = {k: np.asarray(v) for k, v in gpu.items()}
    e = {}
    e["rho"] = np.abs(g["rho"] - ora["rho"]).max() / np.abs(ora["rho"]).max()
    du = np.sqrt((g["ux"] - ora["ux"]) ** 2 + (g["uy"] - ora["uy"]) ** 2).max()
    e["u"] = du / np.sqrt(ora["ux"] ** 2 + ora["uy"] ** 2).max()
    e["T"] = np.abs(g["T"] - ora["T"]).max() / np.abs(ora["T"]).max()
    return e
