"""Parity with the oracle on the shock--vortex workload (Sec. III.F), where the
limiter is active across the shock and in the vortex.

* 256^2, 400 steps (the FP32-deviation shock test's size): the FP64 CUDA
  fields within 1e-12 of the oracle's (max norm, relative to the field's
  largest value); the FP32-deviation fields within relative L1 1e-4 of the
  *oracle* for rho and T across the shock (the storage form's stated error),
  and within 1e-5 in max norm.
* 1024^2 (the square shock--vortex configuration), after 1000 CUDA steps in
  each storage form: one more step checked cell by cell against the oracle's
  update of the same pre-step populations, at 64 cells chosen on the shock
  and 64 in the vortex core (limiter-active stencils): FP64 within 1e-13 of
  the largest population, FP32 deviations within 2e-7.
"""
import math
import os

import numpy as np
import pytest
import torch

from oracle import dvbm_oracle as O
from paper_2510_04197_gb300 import inputs as I
from helpers import abi_to_oracle_perm, field_errors, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    from paper_2510_04197_gb300 import build, dvbm
    if not os.path.exists(dvbm.LIBPATH):
        build.build()
    assert torch.cuda.is_available()
    return dvbm


SV_BCS_ORACLE = (O.BC(O.ZEROGRAD), O.BC(O.ZEROGRAD), O.BC(), O.BC())


def _gpu_shock_vortex(D, sv, N, nsteps, storage):
    F = sv.fields
    bcs = [D.ZEROGRAD, D.ZEROGRAD, D.PERIODIC, D.PERIODIC]
    sim = D.Simulation(N, N, 0.75, 1.4, sv.mu, bcs=bcs, storage=storage, cfl=0.01, check_every=-1)
    sim.init(*(torch.tensor(a) for a in (F.rho, F.ux, F.uy, F.T)))
    sim.step(nsteps)
    return sim


@pytest.fixture(scope="module")
def oracle_256():
    sv = I.shock_vortex(N=256)
    return sv


def test_shock_vortex_256_fp64_and_fp32_deviation_against_oracle(D, oracle_256):
    sv = oracle_256
    N, n = 256, 400
    out, dt = {}, None
    for st in (0, 1):
        sim = _gpu_shock_vortex(D, sv, N, n, st)
        out[st] = {k: v.cpu().numpy() for k, v in sim.moments().items()}
        dt = sim.dt
        sim.close()
    _, o = oracle_run(sv.fields, 0.75, 1.4, sv.mu, dt, n, bcs=SV_BCS_ORACLE)
    e64 = field_errors(out[0], o)
    assert max(e64.values()) < 1e-12, e64
    e32 = field_errors(out[1], o)
    assert max(e32.values()) < 1e-5, e32
    for k in ("rho", "T"):
        l1 = np.abs(out[1][k] - o[k]).sum() / np.abs(o[k]).sum()
        assert l1 < 1e-4, (k, l1)


def _cells_shock_and_core(N, dt, nsteps, sv, seed=5):
    """64 cells straddling the stationary shock (x = 0.5) and 64 in the core
    of the vortex, advected with the pre-shock flow for nsteps steps."""
    rng = np.random.default_rng(seed)
    dx = 1.0 / N
    xs = 0.5 / dx - 0.5  # shock between columns N/2 - 1 and N/2
    shock = [(int(rng.integers(2, N - 2)), int(round(xs)) + int(rng.integers(-3, 4))) for _ in range(64)]
    xv = 0.35 + sv.fields.ux[0, 0] * dt * nsteps  # vortex centre moves with the pre-shock flow
    core = []
    while len(core) < 64:
        r, a = 0.6 * 0.075 * math.sqrt(rng.random()), 2 * math.pi * rng.random()
        x, y = xv + r * math.cos(a), 0.5 + r * math.sin(a)
        core.append((int(y / dx), int(x / dx)))
    return shock + core


def _patches(pops, cells, N):
    ys = torch.tensor([[(y + d) % N for d in range(-2, 3)] for (y, x) in cells], device=pops.device)
    xs = torch.tensor([[x + d for d in range(-2, 3)] for (y, x) in cells], device=pops.device)
    return pops[:, ys[:, :, None], xs[:, None, :]].double().cpu()


@pytest.mark.parametrize("storage", [0, 1])
def test_shock_vortex_1024_sampled_step_after_1000_steps(D, storage):
    N, n = 1024, 1000
    sv = I.shock_vortex(N=N)
    sim = _gpu_shock_vortex(D, sv, N, n, storage)
    cells = _cells_shock_and_core(N, sim.dt, n, sv)
    assert all(2 <= x < N - 2 for (_, x) in cells)
    before = _patches(sim.populations(), cells, N)
    sim.step(1)
    after = sim.populations()
    ys = torch.tensor([c[0] for c in cells], device=after.device)
    xs = torch.tensor([c[1] for c in cells], device=after.device)
    got = after[:, ys, xs].double().cpu()
    lat = O.Lattice()
    perm = abi_to_oracle_perm(lat)
    if storage == 1:
        w = torch.tensor([float(v) for v in lat.w], dtype=torch.float64)[np.argsort(perm)]
        gref = 1.0 / 0.4 - 1.0
        ref = torch.cat([w, w * gref])
        before = before + ref[:, None, None, None]
        got = got + ref[:, None]
    P = O.Params(Pr=0.75, gamma=1.4, mu=sv.mu)
    fo, go = O.step_patch(lat, P, O.Grid(N, N, bcs=SV_BCS_ORACLE), before[:25][perm], before[25:][perm], sim.dt)
    fg, gg = got[:25][perm], got[25:][perm]
    tol = 1e-13 if storage == 0 else 2e-7
    ef = float((fg - fo).abs().max() / fo.abs().max())
    eg = float((gg - go).abs().max() / go.abs().max())
    # the sampled stencils do cross the shock: the density jumps there
    rho_b = before[:25].sum(0)  # [B, 5, 5]
    jump = (rho_b[:64, 2, :].max(1).values / rho_b[:64, 2, :].min(1).values).max()
    assert float(jump) > 1.2, float(jump)
    assert ef < tol and eg < tol, (ef, eg)
    sim.close()
