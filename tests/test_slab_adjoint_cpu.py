"""Host logic of the slab-decomposed backward pass on CPU ranks (gloo): the
drivers ``slab.RankSlab.adjoint`` and ``slab.LocalSlabs.adjoint`` around a
stand-in band that scripts the stepwise pass (the GPU tests run the library's
own).  Checked: every rank takes the same actions; after each action the
ghost rows a band unpacks are the rows its lower and upper neighbours packed
for that same action (lower ghosts = the lower band's highest rows, upper
ghosts = the upper band's lowest rows); the parameter gradients are the sum
of the bands' shares; field gradients stay per band (LocalSlabs concatenates
them in band order).  World sizes 2 (both neighbours the same rank) and 3;
ghost rows planted on the wrong side are caught."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

NPOP, NX, ROWS = 3, 4, 5
ACTIONS = [1, 1, 3, 1, 3, 2, 2, 1, 1, 3, 2, 0]  # restore, recompute + code rows ..., adjoint steps ..., done


class FakeBand:
    """Scripted stepwise pass: pack writes (band, action, side) codes, unpack
    records what arrived."""

    def __init__(self, band, swap=False):
        self.band, self.action, self.swap = band, 0, swap
        self.received = []

    def halo_buffer(self):
        return torch.zeros((NPOP, 2, NX), dtype=torch.float64)

    def adjoint_begin(self, dL_drho, dL_dT):
        self.action = 0

    def adjoint_advance(self):
        a = ACTIONS[self.action]
        self.action += 1
        return a

    def adjoint_halo_pack(self, lo=None, hi=None):
        for buf, side in ((lo, 0), (hi, 1)):
            if buf is not None:
                buf.fill_(1000 * self.band + 10 * self.action + side)

    def adjoint_halo_unpack(self, lo=None, hi=None):
        if self.swap:  # planted mistake: each side's rows land in the other side's ghost rows
            lo, hi = hi, lo
        self.received.append((self.action, None if lo is None else float(lo[0, 0, 0]),
                              None if hi is None else float(hi[0, 0, 0])))

    def adjoint_finish(self):
        g = {k: torch.full((ROWS, NX), float(self.band)) for k in ("rho0", "ux0", "uy0", "T0")}
        g.update(mu=1.0 + self.band, Pr=0.5 * self.band, gamma=-1.0)
        return g


def _expected(band, world, periodic=True):
    """(action, lower ghost code, upper ghost code) per exchange of band."""
    from paper_2510_04197_gb300 import slab
    lower, upper = slab.neighbours(band, world, periodic)
    out = []
    for action in range(len(ACTIONS)):  # exchanges after begin (action 0) and after each nonzero advance
        if action > 0 and ACTIONS[action - 1] == 0:
            break
        lo = None if lower is None else 1000 * lower + 10 * action + 1  # the lower band's highest rows
        hi = None if upper is None else 1000 * upper + 10 * action + 0  # the upper band's lowest rows
        out.append((action, lo, hi))
    return out


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_path, swap=False):
    from paper_2510_04197_gb300 import slab
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rs = object.__new__(slab.RankSlab)  # a band without the library: the stand-in pass
        rs.dist, rs.rank, rs.world, rs.periodic = dist, rank, world, True
        rs.sim = FakeBand(rank, swap)
        rs.sim.device = "cpu"
        lower, upper = slab.neighbours(rank, world, True)
        rs.send_lo = rs.sim.halo_buffer() if lower is not None else None
        rs.send_hi = rs.sim.halo_buffer() if upper is not None else None
        rs.recv_lo = rs.sim.halo_buffer() if lower is not None else None
        rs.recv_hi = rs.sim.halo_buffer() if upper is not None else None
        g = rs.adjoint(None, None)
        torch.save({"received": rs.sim.received, "params": (g["mu"], g["Pr"], g["gamma"]),
                    "rho0": g["rho0"]}, f"{out_path}.{rank}")
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_rank_slab_adjoint_exchanges(tmp_path, world):
    out = str(tmp_path / "adj")
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    for r in range(world):
        res = torch.load(f"{out}.{r}")
        assert res["received"] == _expected(r, world), (r, res["received"])
        assert res["params"] == (sum(1.0 + b for b in range(world)), sum(0.5 * b for b in range(world)),
                                 -1.0 * world)
        assert torch.equal(res["rho0"], torch.full((ROWS, NX), float(r)))  # the band's own gradients


def test_rank_slab_adjoint_swapped_halos_are_caught(tmp_path):
    out = str(tmp_path / "adj")
    mp.start_processes(_worker, args=(3, _free_port(), out, True), nprocs=3, join=True, start_method="spawn")
    for r in range(3):
        assert torch.load(f"{out}.{r}")["received"] != _expected(r, 3)


@pytest.mark.parametrize("parts,periodic", [(3, True), (2, True), (3, False)])
def test_local_slabs_adjoint_exchanges(parts, periodic):
    from paper_2510_04197_gb300 import slab
    ls = object.__new__(slab.LocalSlabs)
    ls.heights = [ROWS] * parts
    ls.sims = [FakeBand(b) for b in range(parts)]
    ls.periodic = periodic
    ls.nb = [slab.neighbours(b, parts, periodic) for b in range(parts)]
    ls.out_lo = [s.halo_buffer() for s in ls.sims]
    ls.out_hi = [s.halo_buffer() for s in ls.sims]
    dr = torch.zeros((ROWS * parts, NX))
    g = ls.adjoint(dr, dr)
    for b, s in enumerate(ls.sims):
        assert s.received == _expected(b, parts, periodic), (b, s.received)
    assert g["mu"] == sum(1.0 + b for b in range(parts))
    assert torch.equal(g["rho0"], torch.cat([torch.full((ROWS, NX), float(b)) for b in range(parts)]))
