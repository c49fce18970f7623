"""Failure detection on the CUDA path: the instability flag that the step
kernels raise for a cell with rho <= 0, T <= 0 or a non-finite value (the
positivity the moments of Sec. II.D.1 and the temperature of
Eq. Total_energy_MB need), and the host-side time limit on every wait for the
stream.

Every failure is made on the host: an unphysical or non-finite state written
through dvbm_set_state, or a time limit shorter than the work queued on the
stream.  No kernel waits on anything: the step kernels OR a flag word that the
host reads, and the host polls an event under its own limit."""
import numpy as np
import pytest
import torch

from paper_2510_04197_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    from paper_2510_04197_gb300 import build, dvbm
    import os
    if not os.path.exists(dvbm.LIBPATH):
        build.build()
    return dvbm


# (lattice, storage): D2Q25 split II in both storage forms and D2Q16 split I
CASES = [("d2q25-fp64", 0, 0), ("d2q25-fp32dev", 0, 1), ("d2q16-fp64", 1, 0)]


def make(D, lattice, storage, F, **opts):
    Ny, Nx = F.rho.shape
    sim = D.Simulation(Nx, Ny, 0.71, 1.4, 2e-3, storage=storage, lattice=lattice, Lx=F.Lx, Ly=F.Ly, **opts)
    sim.init(*(torch.tensor(a) for a in (F.rho, F.ux, F.uy, F.T)))
    return sim


def planted(sim, what, x=13, y=7):
    """A packed copy of the current state with one cell (x, y) made bad."""
    st = sim.get_state().clone()
    pops = sim.populations(st)  # view [npop, Ny, Nx] into st
    half = sim.npop // 2         # f planes first, then g
    if what == "nan":
        pops[half + 3, y, x] = float("nan")
    elif what == "rho":
        # f = -2 (FP64) or deviation -2 from w_i rho0 <= 1 (FP32DEV): rho < 0
        pops[:half, y, x] = -2.0
    elif what == "T":
        # g = -10 (FP64) or deviation -10 from w_i rho0 (C_v - R) T0 <= 1.5
        # (FP32DEV): E below the kinetic energy, T < 0, rho unchanged
        pops[half:, y, x] = -10.0
    return st


@pytest.mark.parametrize("name,lattice,storage", CASES)
@pytest.mark.parametrize("what", ["nan", "rho", "T"])
def test_bad_cell_raises_unstable(D, name, lattice, storage, what):
    F = I.random_smooth(40, 24, seed=3, amp=0.05, Ma=0.3)
    sim = make(D, lattice, storage, F, dt=2e-4, check_every=1)
    sim.step(2)
    sim.set_state(planted(sim, what))
    with pytest.raises(D.DVBMError) as ei:
        sim.step(5)
    assert ei.value.status == D.EUNSTABLE, (name, what, str(ei.value))
    # checked after every step: the first step from the planted state reports it
    assert sim.steps == 3, sim.steps
    assert "after 3 steps" in str(ei.value)
    # the totals pass counts bad cells of the current state independently of the flag
    with pytest.raises(D.DVBMError) as et:
        sim.totals()
    assert et.value.status == D.EUNSTABLE


@pytest.mark.parametrize("name,lattice,storage", CASES)
def test_resume_after_unstable_from_restored_state(D, name, lattice, storage):
    """set_state clears the flag: a run that reported EUNSTABLE continues from
    a restored checkpoint exactly like a fresh context from that checkpoint."""
    F = I.random_smooth(40, 24, seed=4, amp=0.05, Ma=0.3)
    sim = make(D, lattice, storage, F, dt=2e-4)
    sim.step(4)
    good = sim.get_state().clone()
    sim.set_state(planted(sim, "nan"))
    with pytest.raises(D.DVBMError) as ei:
        sim.step(1)
    assert ei.value.status == D.EUNSTABLE
    sim.set_state(good)
    sim.step(6)
    fresh = make(D, lattice, storage, F, dt=2e-4)
    fresh.set_state(good)
    fresh.step(6)
    assert sim.steps == fresh.steps == 10
    assert torch.equal(sim.populations(), fresh.populations())


def test_unchecked_run_reports_at_the_next_check(D):
    """check_every < 0 never checks inside dvbm_step; the bad cell is still
    reported by the next totals pass."""
    F = I.random_smooth(40, 24, seed=5, amp=0.05, Ma=0.3)
    sim = make(D, 0, 0, F, dt=2e-4, check_every=-1)
    sim.step(1)
    sim.set_state(planted(sim, "rho"))
    sim.step(3)
    with pytest.raises(D.DVBMError) as ei:
        sim.totals()
    assert ei.value.status == D.EUNSTABLE


@pytest.fixture(scope="module")
def long_run(D):
    """1024^2 FP64 periodic flow: 300 steps take several hundred ms on one GPU,
    far beyond the 20 ms limit given to the contexts below."""
    F = I.wave_decay(1024, 1024, Ma=0.1, amp=1e-3)
    ref = make(D, 0, 0, F, dt=1e-4)
    ref.step(300)
    pops = ref.populations().clone()
    mom = {k: v.cpu().numpy() for k, v in ref.moments().items()}
    ref.close()
    return F, pops, mom


@pytest.mark.parametrize("where", ["step", "totals", "moments_host"])
def test_time_limit_returns_etimeout_and_the_work_runs_on(D, long_run, where):
    """A wait that outlasts opts.timeout_s returns ETIMEOUT instead of
    blocking, also where the result is copied into pageable host memory (such
    a copy would otherwise block until the stream is done); the queued steps
    still run, and once the stream is idle the context is intact."""
    F, pops, mom = long_run
    sim = make(D, 0, 0, F, dt=1e-4, timeout_s=0.02, check_every=0 if where == "step" else -1)
    torch.cuda.synchronize()
    with pytest.raises(D.DVBMError) as ei:
        sim.step(300)
        if where == "totals":
            sim.totals()
        elif where == "moments_host":
            sim.moments_host()
    assert ei.value.status == D.ETIMEOUT, str(ei.value)
    torch.cuda.synchronize()
    assert sim.steps == 300
    assert torch.equal(sim.populations(), pops)
    got = sim.moments_host()
    for k in ("rho", "ux", "uy", "T"):
        assert np.array_equal(got[k], mom[k]), k
