"""Slab decomposition of the step along y on CPU ranks (gloo).

Each rank owns a band of rows and exchanges two halo rows with each
neighbour per step through ``paper_2510_04197_gb300.slab.exchange`` -- the
same point-to-point exchange a multi-GPU run uses with NCCL -- with its halo
buffers in the library's [npop][2][Nx] layout (f planes then g planes).  Each
band is stepped with the oracle.  The decomposition changes no arithmetic, but
torch's CPU kernels may round a band-shaped array differently from the full
one, so the gathered result must equal the undecomposed run to rounding
(1e-14 of the largest population), while halos delivered to the wrong side
(a planted mistake) miss it by orders of magnitude.  World sizes 2 (both
neighbours of a band are the same rank) and 3, y-periodic and zero-gradient
in y."""
import os
import socket

import pytest
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


def _setup(Nx, Ny, periodic):
    F = I.random_smooth(Nx, Ny, seed=12, amp=0.1, Ma=0.5)
    P = O.Params(Pr=0.71, gamma=1.4, mu=2e-3)
    lat = O.Lattice()
    ybc = O.BC() if periodic else O.BC(O.ZEROGRAD)
    grid = O.Grid(Nx, Ny, F.Lx, F.Ly, (O.BC(), O.BC(), ybc, ybc))
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


def _worker(rank, world, port, Nx, Ny, nsteps, dt, periodic, out_path, swap=False):
    from paper_2510_04197_gb300 import slab
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lat, P, grid, f, g = _setup(Nx, Ny, periodic)
        Q = lat.Q
        rows = Ny // world
        y0 = rank * rows
        band = _SlabGrid(grid, rows)
        fl, gl = f[:, y0:y0 + rows].clone(), g[:, y0:y0 + rows].clone()
        lower, upper = slab.neighbours(rank, world, periodic)
        recv_lo = torch.empty(2 * Q, 2, Nx, dtype=DT) if lower is not None else None
        recv_hi = torch.empty(2 * Q, 2, Nx, dtype=DT) if upper is not None else None
        for _ in range(nsteps):
            send_lo = torch.cat([fl[:, :2], gl[:, :2]]).contiguous()    # rows y = 0, 1
            send_hi = torch.cat([fl[:, -2:], gl[:, -2:]]).contiguous()  # rows y = rows - 2, rows - 1
            if swap:  # planted mistake: each band's halos land on the wrong side
                slab.exchange(dist, rank, world, periodic, send_lo, send_hi, recv_hi, recv_lo)
            else:
                slab.exchange(dist, rank, world, periodic, send_lo, send_hi, recv_lo, recv_hi)
            # ghost rows at a non-periodic domain edge come from the boundary condition
            fb, gb = O.pad_axis(lat, P, fl, gl, 1, grid.bcs[2], grid.bcs[3])
            below = recv_lo if recv_lo is not None else torch.cat([fb[:, :2], gb[:, :2]])
            above = recv_hi if recv_hi is not None else torch.cat([fb[:, -2:], gb[:, -2:]])
            fpy = torch.cat([below[:Q], fl, above[:Q]], dim=1)
            gpy = torch.cat([below[Q:], gl, above[Q:]], dim=1)
            fl, gl = O.step_with_y_halos(lat, P, band, fl, gl, fpy, gpy, dt)
        parts = [torch.empty_like(fl) for _ in range(world)] if rank == 0 else None
        gparts = [torch.empty_like(gl) for _ in range(world)] if rank == 0 else None
        dist.gather(fl, parts, dst=0)
        dist.gather(gl, gparts, dst=0)
        if rank == 0:
            torch.save((torch.cat(parts, dim=1), torch.cat(gparts, dim=1)), out_path)
    finally:
        dist.destroy_process_group()


def _run(tmp_path, world, periodic, swap=False):
    Nx, Ny, nsteps, dt = 12, 6 * world, 5, 2e-4
    out = str(tmp_path / f"slabs{int(swap)}.pt")
    mp.start_processes(_worker, args=(world, _free_port(), Nx, Ny, nsteps, dt, periodic, out, swap), nprocs=world,
                       join=True, start_method="spawn")
    fd, gd = torch.load(out)
    lat, P, grid, f, g = _setup(Nx, Ny, periodic)
    for _ in range(nsteps):
        f, g = O.step(lat, P, grid, f, g, dt)
    return float((fd - f).abs().max() / f.abs().max()), float((gd - g).abs().max() / g.abs().max())


@pytest.mark.parametrize("world,periodic", [(2, True), (3, True), (3, False)])
def test_slab_decomposition_matches_undecomposed_run(tmp_path, world, periodic):
    ef, eg = _run(tmp_path, world, periodic)
    assert ef < 1e-14 and eg < 1e-14, (ef, eg)


def test_halos_on_the_wrong_side_are_caught(tmp_path):
    ef, eg = _run(tmp_path, 3, True, swap=True)
    assert ef > 1e-8 and eg > 1e-8, (ef, eg)
