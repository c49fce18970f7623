"""Slab decomposition of the step along y on CPU ranks (gloo, world size 2).

Each rank owns a band of rows, exchanges two halo rows with each neighbour
per step (point-to-point send/recv, periodic ring), and steps its band with
the oracle.  The gathered result must be bitwise equal to the undecomposed
run: the decomposition changes no arithmetic.  This is the exchange step a
multi-GPU run of one grid would need; every GPU run here uses one GPU, so it
is validated on CPU ranks."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import dvbm_oracle as O
from paper_2510_04197_gb300 import inputs as I

DT = torch.float64


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _setup(Nx, Ny):
    F = I.random_smooth(Nx, Ny, seed=12, amp=0.1, Ma=0.5)
    P = O.Params(Pr=0.71, gamma=1.4, mu=2e-3)
    lat = O.Lattice()
    grid = O.Grid(Nx, Ny, F.Lx, F.Ly)
    t = lambda a: torch.tensor(a, dtype=DT)
    f, g = O.init_populations(lat, P, t(F.rho), t(F.ux), t(F.uy), t(F.T))
    return lat, P, grid, f, g


class _SlabGrid(O.Grid):
    """A band of rows of a larger grid: same dx and dy as the full grid."""

    def __init__(self, full: O.Grid, rows: int):
        super().__init__(full.Nx, rows, full.Lx, full.Ly, full.bcs)
        self._dx, self._dy = full.dx, full.dy

    @property
    def dx(self):
        return self._dx

    @property
    def dy(self):
        return self._dy


def _worker(rank, world, port, Nx, Ny, nsteps, dt, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lat, P, grid, f, g = _setup(Nx, Ny)
        rows = Ny // world
        y0 = rank * rows
        slab = _SlabGrid(grid, rows)
        fl, gl = f[:, y0:y0 + rows].clone(), g[:, y0:y0 + rows].clone()
        up, down = (rank + 1) % world, (rank - 1) % world
        for _ in range(nsteps):
            # send my two bottom rows down and two top rows up; receive halos
            bot = torch.cat([fl[:, :2], gl[:, :2]]).contiguous()
            top = torch.cat([fl[:, -2:], gl[:, -2:]]).contiguous()
            from_down = torch.empty_like(top)
            from_up = torch.empty_like(bot)
            # tag 1: rows travelling down the ring, tag 2: rows travelling up
            reqs = [dist.isend(bot, down, tag=1), dist.isend(top, up, tag=2),
                    dist.irecv(from_down, down, tag=2), dist.irecv(from_up, up, tag=1)]
            for r in reqs:
                r.wait()
            Q = lat.Q
            fpy = torch.cat([from_down[:Q], fl, from_up[:Q]], dim=1)
            gpy = torch.cat([from_down[Q:], gl, from_up[Q:]], dim=1)
            fl, gl = O.step_with_y_halos(lat, P, slab, fl, gl, fpy, gpy, dt)
        parts = [torch.empty_like(fl) for _ in range(world)] if rank == 0 else None
        gparts = [torch.empty_like(gl) for _ in range(world)] if rank == 0 else None
        dist.gather(fl, parts, dst=0)
        dist.gather(gl, gparts, dst=0)
        if rank == 0:
            torch.save((torch.cat(parts, dim=1), torch.cat(gparts, dim=1)), out_path)
    finally:
        dist.destroy_process_group()


def test_slab_decomposition_is_bitwise_equal(tmp_path):
    Nx, Ny, nsteps, dt = 12, 16, 5, 2e-4
    out = str(tmp_path / "slabs.pt")
    mp.start_processes(_worker, args=(2, _free_port(), Nx, Ny, nsteps, dt, out), nprocs=2, join=True,
                       start_method="spawn")
    fd, gd = torch.load(out)
    lat, P, grid, f, g = _setup(Nx, Ny)
    for _ in range(nsteps):
        f, g = O.step(lat, P, grid, f, g, dt)
    assert torch.equal(fd, f) and torch.equal(gd, g)
