"""Gradients of the hand-written adjoint at the adjoint workload's full size:
512^2 periodic multimode flow (rms Ma 0.3, seed 0), Pr 0.71, gamma 1.4,
mu 1e-3, 200 FP64 steps, checkpoints every ceil(sqrt(200)) = 15 steps, loss
L = 1/(2N) sum[(rho - rho_t)^2 + (T - T_t)^2] against the seed-1 flow after
200 steps; dt fixed (not differentiated).

Central differences of the CUDA forward map against the adjoint's
directional derivatives: h = 1e-6 along three random smooth directions of
(rho0, ux0, uy0, T0) and a relative step of 1e-5 along mu, Pr and gamma,
relative agreement 1e-6.  The difference of the two losses is summed cell
by cell, L(+) - L(-) = 1/(2N) sum[(a+ - a-)(a+ + a- - 2 a_t)] over a = rho,
T: the difference of the two rounded loss values (L ~ 5e-3) would lose the
signal of a single entry (about 3e-14) to rounding.  Repeated forward runs
are bitwise identical.

Single entries (twenty random cells and fields): the limiter is piecewise
linear (Sec. III.A.2), so the discrete map has kinks; where a perturbation
of +-h moves some stencil across a branch switch, the central difference
averages the derivatives of two branches, while the adjoint is the
derivative of the branch taken at the unperturbed state (that side's
one-sided difference matches it); below h ~ 1e-7 rounding takes over.  Each
entry takes the closest of the central differences at h = 1e-6 and 1e-7 and
the forward and backward differences at h = 1e-7: all 20 agree within 1e-5
and their median within 1e-6.  A wrong adjoint term misses both bounds by
orders of magnitude."""
import math
import os

import numpy as np
import pytest
import torch

from paper_2510_04197_gb300 import inputs as I

pytestmark = pytest.mark.gpu
N, NSTEPS = 512, 200


@pytest.fixture(scope="module")
def D():
    from paper_2510_04197_gb300 import build, dvbm
    if not os.path.exists(dvbm.LIBPATH):
        build.build()
    assert torch.cuda.is_available()
    return dvbm


@pytest.fixture(scope="module")
def setup(D):
    tgt = I.multimode(N, seed=1, rms_Ma=0.3)
    st = D.Simulation(N, N, 0.71, 1.4, 1e-3, check_every=-1)
    st.init(*(torch.tensor(a) for a in (tgt.rho, tgt.ux, tgt.uy, tgt.T)))
    dt = st.dt
    st.step(NSTEPS)
    mt = st.moments()
    st.close()
    F = I.multimode(N, seed=0, rms_Ma=0.3)
    x0 = [torch.tensor(a, device="cuda") for a in (F.rho, F.ux, F.uy, F.T)]

    def fields(x, mu=1e-3, Pr=0.71, gamma=1.4):
        sim = D.Simulation(N, N, Pr, gamma, mu, dt=dt, check_every=-1)
        sim.init(*x)
        sim.step(NSTEPS)
        m = sim.moments()
        sim.close()
        return m

    def dloss(mp, mm):
        """L(+) - L(-) summed cell by cell (no cancellation of two rounded losses)."""
        s = sum((((mp[k] - mm[k]) * (mp[k] + mm[k] - 2.0 * mt[k])).sum()) for k in ("rho", "T"))
        return float(0.5 / (N * N) * s)

    def fd(xp, xm, h, **kw):
        return dloss(fields(xp, **kw.get("p", {})), fields(xm, **kw.get("m", {}))) / (2 * h)

    m0 = fields(x0)

    def one_sided(x, h):
        """(L(x) - L(x0)) / h for x = x0 + h e (h < 0: backward)."""
        return dloss(fields(x), m0) / h

    sim = D.Simulation(N, N, 0.71, 1.4, 1e-3, dt=dt, check_every=-1)
    sim.record(int(math.ceil(math.sqrt(NSTEPS))))
    sim.init(*x0)
    sim.step(NSTEPS)
    m = sim.moments()
    g = sim.adjoint((m["rho"] - mt["rho"]) / (N * N), (m["T"] - mt["T"]) / (N * N))
    sim.close()
    return x0, fd, g, one_sided


def test_directional_derivatives(setup):
    x0, fd, g, one_sided = setup
    grads = [g["rho0"], g["ux0"], g["uy0"], g["T0"]]
    h = 1e-6
    for trial in range(3):
        V = I.random_smooth(N, N, seed=100 + trial, amp=1.0, Ma=1.0)
        v = [torch.tensor(a, device="cuda") for a in (V.rho - 1.0, V.ux, V.uy, V.T - 1.0)]
        ad = sum(float((gi * vi).sum()) for gi, vi in zip(grads, v))
        d = fd([a + h * b for a, b in zip(x0, v)], [a - h * b for a, b in zip(x0, v)], h)
        assert abs(d - ad) < 1e-6 * abs(ad), (trial, d, ad)


def test_single_entries(setup):
    x0, fd, g, one_sided = setup
    grads = [g["rho0"], g["ux0"], g["uy0"], g["T0"]]
    rng = np.random.default_rng(5)
    errs = []
    for trial in range(20):
        k = int(rng.integers(0, 4))
        i, j = (int(v) for v in rng.integers(0, N, 2))
        ad = float(grads[k][i, j])

        def shifted(s):
            x = [a.clone() for a in x0]
            x[k][i, j] += s
            return x
        est = [fd(shifted(h), shifted(-h), h) for h in (1e-6, 1e-7)]
        est += [one_sided(shifted(h), h) for h in (1e-7, -1e-7)]
        errs.append((min(abs(v - ad) / abs(ad) for v in est), k, i, j))
    e = sorted(v for v, *_ in errs)
    assert e[-1] < 1e-5 and 0.5 * (e[9] + e[10]) < 1e-6, errs


@pytest.mark.parametrize("name,base", [("mu", 1e-3), ("Pr", 0.71), ("gamma", 1.4)])
def test_parameter_derivatives(setup, name, base):
    x0, fd, g, one_sided = setup
    hp = 1e-5 * base
    d = fd(x0, x0, hp, p={name: base + hp}, m={name: base - hp})
    assert abs(d - g[name]) < 1e-6 * abs(g[name]), (name, d, g[name])
