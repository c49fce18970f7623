"""The stepwise adjoint (dvbm_adjoint_begin / _advance / _halo_pack /
_halo_unpack / _finish) and the slab-decomposed backward pass built on it.

* On a whole periodic grid the stepwise pass is dvbm_adjoint's arithmetic
  (rational limiter: recorded branch codes and moments; general beta: the
  branches derived from the recomputed states, in both): bitwise the same
  gradients, for Pr < 1 and Pr > 1, beta = 1.2 and sqrt(2), and checkpoint
  intervals that do and do not divide the step count.
* A grid split into bands along y (LocalSlabs, one context per band, the
  halo rows of every restored, recomputed and adjoint state and the code
  rows of every recomputed step exchanged after the action that produced
  them): the gradients of the initial fields equal dvbm_adjoint on the
  undecomposed grid bitwise for bands of whole 8-row tiles, and to 1e-12 for
  ragged bands; dL/d(mu, Pr, gamma), sums over every cell and step of terms
  of both signs taken band by band in another order, to 1e-10 relative
  (measured: 1.6e-12 for gamma).
* RankSlab over a one-rank NCCL group (the band is the whole grid, its halos
  its own rows): bitwise equal to the undecomposed stepwise pass.
* The contract: dvbm_adjoint refuses a band, finish refuses an unfinished
  pass, advance and the halo calls refuse a pass never begun, a new step
  ends a pass in progress, and a recorded run that has stepped keeps its dt.
"""
import os
import socket

import pytest
import torch

from paper_2510_04197_gb300 import inputs as I

pytestmark = pytest.mark.gpu
FIELDS = ("rho0", "ux0", "uy0", "T0")


@pytest.fixture(scope="module")
def D():
    from paper_2510_04197_gb300 import build, dvbm
    if not os.path.exists(dvbm.LIBPATH):
        build.build()
    assert torch.cuda.is_available()
    return dvbm


def _problem(Nx, Ny, seed=3):
    F = I.random_smooth(Nx, Ny, seed=seed, amp=0.1, Ma=0.5)
    G = I.random_smooth(Nx, Ny, seed=seed + 50, amp=0.1, Ma=0.5)
    return F, G


def _fields(F):
    return [torch.tensor(a, device="cuda") for a in (F.rho, F.ux, F.uy, F.T)]


def _loss_grads(m, target):
    N = m["rho"].numel()
    return (m["rho"] - target["rho"]) / N, (m["T"] - target["T"]) / N


def _single(D, F, Pr, nsteps, every, dt, **kw):
    sim = D.Simulation(F.rho.shape[1], F.rho.shape[0], Pr, 1.4, 2e-3, Lx=F.Lx, Ly=F.Ly, dt=dt, check_every=-1,
                       **kw)
    sim.record(every)
    sim.init(*_fields(F))
    sim.step(nsteps)
    return sim


def _target(D, G, Pr, nsteps, dt, **kw):
    sim = D.Simulation(G.rho.shape[1], G.rho.shape[0], Pr, 1.4, 2e-3, Lx=G.Lx, Ly=G.Ly, dt=dt, check_every=-1,
                       **kw)
    sim.init(*_fields(G))
    sim.step(nsteps)
    m = sim.moments()
    sim.close()
    return m


def _close(a, b, tol_field=1e-12, tol_param=1e-10):
    for k in FIELDS:
        e = float((a[k] - b[k]).abs().max() / b[k].abs().max())
        assert e < tol_field, (k, e)
    for k in ("mu", "Pr", "gamma"):
        assert abs(a[k] - b[k]) <= tol_param * abs(b[k]), (k, a[k], b[k])


def _equal(a, b):
    assert all(torch.equal(a[k], b[k]) for k in FIELDS), [float((a[k] - b[k]).abs().max()) for k in FIELDS]
    assert all(a[k] == b[k] for k in ("mu", "Pr", "gamma")), [(a[k], b[k]) for k in ("mu", "Pr", "gamma")]


@pytest.mark.parametrize("Pr,nsteps,every,beta", [(0.71, 40, 7, 1.2), (2.0, 24, 6, 1.2), (0.71, 1, 1, 1.2),
                                                  (0.71, 30, 7, 2 ** 0.5)])
def test_stepwise_equals_monolithic_on_a_periodic_grid(D, Pr, nsteps, every, beta):
    F, G = _problem(48, 40)
    dt = 2e-4
    tgt = _target(D, G, Pr, nsteps, dt, beta=beta)
    sim = _single(D, F, Pr, nsteps, every, dt, beta=beta)
    dr, dT = _loss_grads(sim.moments(), tgt)
    a = sim.adjoint(dr, dT)
    b = sim.adjoint_stepwise(dr, dT)
    # rational limiter: both run the coded arithmetic; general beta: both
    # derive the branches from the states
    _equal(b, a)
    # a second pass on the same recording gives the same result
    c = sim.adjoint_stepwise(dr, dT)
    assert all(torch.equal(b[k], c[k]) for k in FIELDS)
    sim.close()


def _slab_adjoint(D, F, Pr, nsteps, every, dt, parts=None, heights=None):
    from paper_2510_04197_gb300 import slab
    Ny, Nx = F.rho.shape
    sl = slab.LocalSlabs(Nx, Ny, parts or 2, Pr, 1.4, 2e-3, heights=heights, Lx=F.Lx, Ly=F.Ly, dt=dt,
                         check_every=-1)
    sl.record(every)
    sl.init(*_fields(F))
    sl.step(nsteps)
    return sl


@pytest.mark.parametrize("parts,heights,Pr", [(2, None, 0.71), (3, None, 2.0), (3, [16, 9, 15], 0.71)])
def test_bands_equal_the_undecomposed_pass(D, parts, heights, Pr):
    F, G = _problem(40, 40 if heights else 48)
    nsteps, every, dt = 30, 7, 2e-4
    tgt = _target(D, G, Pr, nsteps, dt)
    sim = _single(D, F, Pr, nsteps, every, dt)
    dr, dT = _loss_grads(sim.moments(), tgt)
    ref = sim.adjoint_stepwise(dr, dT)
    sl = _slab_adjoint(D, F, Pr, nsteps, every, dt, parts=parts, heights=heights)
    if heights is None:  # whole tiles: the decomposed forward run is bitwise the same
        assert torch.equal(sl.populations(), sim.populations())
    got = sl.adjoint(dr, dT)
    mono = sim.adjoint(dr, dT)
    _equal(ref, mono)
    if heights is None:  # whole tiles: bitwise the undecomposed dvbm_adjoint
        assert all(torch.equal(got[k], mono[k]) for k in FIELDS)
    _close(got, mono)
    sl.close()
    sim.close()


def test_rank_slab_one_rank_nccl(D):
    import torch.distributed as td
    from paper_2510_04197_gb300 import slab
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    own = not td.is_initialized()
    if own:
        td.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1,
                              device_id=torch.device("cuda", torch.cuda.current_device()))
    try:
        F, G = _problem(40, 32)
        nsteps, every, dt = 20, 5, 2e-4
        tgt = _target(D, G, 0.71, nsteps, dt)
        sim = _single(D, F, 0.71, nsteps, every, dt)
        dr, dT = _loss_grads(sim.moments(), tgt)
        ref = sim.adjoint_stepwise(dr, dT)
        band = slab.RankSlab(td, 40, 32, 0.71, 1.4, 2e-3, Lx=F.Lx, Ly=F.Ly, dt=dt, check_every=-1)
        band.record(every)
        band.init(*_fields(F))
        band.step(nsteps)
        got = band.adjoint(dr, dT)
        assert all(torch.equal(got[k], ref[k]) for k in FIELDS)
        for k in ("mu", "Pr", "gamma"):
            assert got[k] == ref[k], (k, got[k], ref[k])
        band.close()
        sim.close()
    finally:
        if own:
            td.destroy_process_group()


def test_stepwise_contract(D):
    from paper_2510_04197_gb300 import slab
    F, G = _problem(32, 32)
    sl = _slab_adjoint(D, F, 0.71, 6, 3, 2e-4, parts=2)
    band = sl.sims[0]
    with pytest.raises(D.DVBMError) as ei:  # the recompute needs the dt the run stepped with
        band.set_dt(1e-4)
    assert ei.value.status == D.ESTATE
    band.set_dt(2e-4)  # the same dt is accepted
    z = torch.zeros((16, 32), dtype=torch.float64, device="cuda")
    with pytest.raises(D.DVBMError) as ei:  # a band needs its neighbours at every step
        band.adjoint(z, z)
    assert ei.value.status == D.EINVAL
    with pytest.raises(D.DVBMError) as ei:  # no pass begun
        band.adjoint_advance()
    assert ei.value.status == D.ESTATE
    with pytest.raises(D.DVBMError) as ei:
        band.adjoint_halo_pack(sl.out_lo[0], sl.out_hi[0])
    assert ei.value.status == D.ESTATE
    band.adjoint_begin(z, z)
    with pytest.raises(D.DVBMError) as ei:  # not complete
        band.adjoint_finish()
    assert ei.value.status == D.ESTATE
    with pytest.raises(D.DVBMError) as ei:  # both sides of a band are external
        band.adjoint_halo_unpack(sl.out_lo[1], None)
    assert ei.value.status == D.EINVAL
    sl.exchange()
    band.step(1)  # a new step ends the pass in progress
    with pytest.raises(D.DVBMError) as ei:
        band.adjoint_advance()
    assert ei.value.status == D.ESTATE
    sl.close()
    plain = D.Simulation(32, 32, 0.71, 1.4, 2e-3, Lx=F.Lx, Ly=F.Ly, dt=2e-4)
    plain.init(*_fields(F))
    with pytest.raises(D.DVBMError) as ei:  # nothing recorded
        plain.adjoint_begin(z.new_zeros((32, 32)), None)
    assert ei.value.status == D.ESTATE
    plain.close()
