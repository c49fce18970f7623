"""The multi-GPU slab driver (paper_2510_04197_gb300.slab.RankSlab) on one GPU
with a one-rank NCCL process group: the band is the whole grid, its halo rows
go out through dvbm_halo_pack and come back through dvbm_halo_unpack (the
periodic self-exchange), and the time step and the totals go through NCCL
all-reduces.  Ranks that wait on one another are not run on one GPU; the
exchange between several ranks is covered by the gloo tests on CPU.

* y-periodic grid (both y sides EXTERNAL): 200 steps bitwise equal to the
  plain periodic context, for FP64 and FP32-deviation storage and for D2Q16;
  the CFL time step (all-reduce MIN) and the totals (all-reduce SUM) equal
  the plain context's.
* walls in y (no EXTERNAL side on a one-band grid): the same.
"""
import math
import os
import socket

import pytest
import torch

from paper_2510_04197_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    from paper_2510_04197_gb300 import build, dvbm
    if not os.path.exists(dvbm.LIBPATH):
        build.build()
    assert torch.cuda.is_available()
    return dvbm


@pytest.fixture(scope="module")
def dist():
    import torch.distributed as td
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    td.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1,
                          device_id=torch.device("cuda", torch.cuda.current_device()))
    yield td
    td.destroy_process_group()


def _fields(F):
    return [torch.tensor(a) for a in (F.rho, F.ux, F.uy, F.T)]


@pytest.mark.parametrize("lattice,storage", [(0, 0), (0, 1), (1, 0)])
def test_one_rank_periodic_band_equals_plain_context(D, dist, lattice, storage):
    from paper_2510_04197_gb300 import slab
    F = I.random_smooth(64, 48, seed=13, amp=0.1, Ma=0.5)
    kw = dict(Lx=F.Lx, Ly=F.Ly, check_every=-1, lattice=lattice, storage=storage, cfl=0.2)
    a = D.Simulation(64, 48, 0.71, 1.4, 2e-3, **kw)
    a.init(*_fields(F))
    b = slab.RankSlab(dist, 64, 48, 0.71, 1.4, 2e-3, **kw)
    assert b.sim.halo_bytes > 0  # both y sides are EXTERNAL
    b.init(*_fields(F))
    assert b.sim.dt == a.dt
    a.step(200)
    b.step(200)
    assert torch.equal(a.populations(), b.sim.populations())
    ta, tb = a.totals(), b.totals()
    assert all(x == y for x, y in zip(ta, tb)), (ta, tb)
    a.close()
    b.close()


def test_one_rank_band_with_walls_equals_plain_context(D, dist):
    from paper_2510_04197_gb300 import slab
    cs = I.couette(Nx=4, Ny=24, Ma=0.5, gamma=1.4)
    F = cs.fields
    dt = min(0.4 * (F.Ly / 24) / math.sqrt(5 + math.sqrt(10)), 0.25 * cs.mu / 2.0)
    bcs = [D.PERIODIC, D.PERIODIC, (D.WALL, (0.0, 0.0), cs.T_C), (D.WALL, (cs.u0, 0.0), cs.T_H)]
    kw = dict(Lx=F.Lx, Ly=F.Ly, dt=dt, bcs=bcs)
    a = D.Simulation(4, 24, 2.0, 1.4, cs.mu, **kw)
    a.init(*_fields(F))
    b = slab.RankSlab(dist, 4, 24, 2.0, 1.4, cs.mu, **kw)
    assert b.send_lo is None and b.send_hi is None  # no neighbour band: nothing to exchange
    b.init(*_fields(F))
    a.step(300)
    b.step(300)
    assert torch.equal(a.populations(), b.sim.populations())
    a.close()
    b.close()
