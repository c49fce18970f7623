"""The hand-written adjoint (dvbm_record / dvbm_adjoint, DVBMFunction) against
(1) the oracle's discrete adjoint -- torch.autograd applied to the FP64 CPU
oracle's forward map, element by element -- and (2) central finite
differences of the CUDA forward map itself.  Loss:
L = 1/(2N) sum[(rho_n - rho_t)^2 + (T_n - T_t)^2], dt held fixed."""

import numpy as np
import pytest
import torch

from oracle import dvbm_oracle as O
from paper_2510_04197_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DT = torch.float64


@pytest.fixture(scope="module")
def D():
    from paper_2510_04197_gb300 import build, dvbm
    import os
    if not os.path.exists(dvbm.LIBPATH):
        build.build()
    return dvbm


def targets(Nx, Ny):
    T = I.random_smooth(Nx, Ny, seed=99, amp=0.05, Ma=0.2)
    return T.rho, T.T


def gpu_grad(D, F, Pr, gamma, mu, dt, n, rho_t, T_t, every):
    Ny, Nx = F.rho.shape
    sim = D.Simulation(Nx, Ny, Pr, gamma, mu, Lx=F.Lx, Ly=F.Ly, dt=dt)
    sim.record(every)
    sim.init(*(torch.tensor(a) for a in (F.rho, F.ux, F.uy, F.T)))
    sim.step(n)
    m = sim.moments()
    N = Nx * Ny
    rt, Tt = torch.tensor(rho_t, device="cuda"), torch.tensor(T_t, device="cuda")
    L = 0.5 / N * (((m["rho"] - rt) ** 2).sum() + ((m["T"] - Tt) ** 2).sum())
    g = sim.adjoint((m["rho"] - rt) / N, (m["T"] - Tt) / N)
    sim.close()
    return float(L), g


def oracle_grad(F, Pr, gamma, mu, dt, n, rho_t, T_t):
    t = lambda a: torch.tensor(a, dtype=DT, requires_grad=True)
    rho0, ux0, uy0, T0 = t(F.rho), t(F.ux), t(F.uy), t(F.T)
    pm, pP, pg = [torch.tensor(v, dtype=DT, requires_grad=True) for v in (mu, Pr, gamma)]
    P = O.Params(Pr=pP, gamma=pg, mu=pm)
    lat = O.Lattice()
    Ny, Nx = F.rho.shape
    grid = O.Grid(Nx, Ny, F.Lx, F.Ly)
    f, g = O.init_populations(lat, P, rho0, ux0, uy0, T0)
    for _ in range(n):
        f, g = O.step(lat, P, grid, f, g, dt)
    rho, ux, uy, T, _ = O.macroscopic(lat, P, f, g)
    N = Nx * Ny
    L = 0.5 / N * (((rho - torch.tensor(rho_t)) ** 2).sum() + ((T - torch.tensor(T_t)) ** 2).sum())
    L.backward()
    return float(L.detach()), {"rho0": rho0.grad.numpy(), "ux0": ux0.grad.numpy(), "uy0": uy0.grad.numpy(),
                      "T0": T0.grad.numpy(), "mu": float(pm.grad), "Pr": float(pP.grad), "gamma": float(pg.grad)}


@pytest.mark.parametrize("Pr", [0.71, 2.0, 1.0])
def test_adjoint_matches_oracle_autograd(D, Pr):
    """Every gradient entry of the CUDA adjoint equals the oracle's discrete
    adjoint (reverse-mode AD of the oracle) to 1e-12 of its field maximum
    (measured: at most 4e-14), on a ragged 13 x 11 periodic grid over 6 steps
    with checkpoints every 2.  The parameter gradients are sums over every
    cell and step of terms of both signs, whose cancellation magnifies the
    rounding of the terms: 1e-10 relative (measured: at most 3e-11)."""
    F = I.random_smooth(13, 11, seed=21, amp=0.08, Ma=0.4)
    rho_t, T_t = targets(13, 11)
    dt, n = 2e-4, 6
    Lg, g = gpu_grad(D, F, Pr, 1.4, 2e-3, dt, n, rho_t, T_t, every=2)
    Lo, o = oracle_grad(F, Pr, 1.4, 2e-3, dt, n, rho_t, T_t)
    assert abs(Lg - Lo) < 1e-13 * max(1.0, abs(Lo))
    for k in ("rho0", "ux0", "uy0", "T0"):
        a = g[k].cpu().numpy()
        scale = np.abs(o[k]).max()
        assert np.abs(a - o[k]).max() < 1e-12 * scale, (k, np.abs(a - o[k]).max() / scale)
    for k in ("mu", "Pr", "gamma"):
        if Pr == 1.0 and k == "Pr":
            continue  # one-sided at Pr = 1 (the branch switches there)
        assert abs(g[k] - o[k]) < 1e-10 * max(abs(o[k]), 1e-30), (k, g[k], o[k])


def test_adjoint_matches_central_differences(D):
    """Directional derivatives along random smooth directions of the initial
    fields (h = 1e-6) and along each parameter (relative step 1e-4) vs central differences of the
    CUDA forward map: relative agreement 1e-6.  32 x 24 periodic, 40 steps,
    checkpoints every 7 (ceil(sqrt 40))."""
    F = I.random_smooth(32, 24, seed=5, amp=0.1, Ma=0.5)
    rho_t, T_t = targets(32, 24)
    Pr, gamma, mu, dt, n = 0.71, 1.4, 2e-3, 2e-4, 40
    L0, g = gpu_grad(D, F, Pr, gamma, mu, dt, n, rho_t, T_t, every=7)

    def loss(F2, Pr2=Pr, g2=gamma, mu2=mu):
        Ny, Nx = F2.rho.shape
        sim = D.Simulation(Nx, Ny, Pr2, g2, mu2, Lx=F2.Lx, Ly=F2.Ly, dt=dt)
        sim.init(*(torch.tensor(a) for a in (F2.rho, F2.ux, F2.uy, F2.T)))
        sim.step(n)
        m = {k: v.cpu().numpy() for k, v in sim.moments().items()}
        sim.close()
        return 0.5 / (Nx * Ny) * (((m["rho"] - rho_t) ** 2).sum() + ((m["T"] - T_t) ** 2).sum())

    h = 1e-6
    rng = np.random.default_rng(3)
    for trial in range(3):
        V = I.random_smooth(32, 24, seed=100 + trial)
        d = {k: getattr(V, k) - getattr(V, k).mean() for k in ("rho", "ux", "uy", "T")}
        keys = ("rho", "ux", "uy", "T")
        Fp = I.Fields(*[getattr(F, k) + h * d[k] for k in keys], F.Lx, F.Ly)
        Fm = I.Fields(*[getattr(F, k) - h * d[k] for k in keys], F.Lx, F.Ly)
        fd = (loss(Fp) - loss(Fm)) / (2 * h)
        ad = sum(float((g[k + "0"].cpu().numpy() * d[k]).sum()) for k in ("rho", "ux", "uy", "T"))
        assert abs(fd - ad) < 1e-6 * abs(ad), (trial, fd, ad)
    for k, base in (("mu", mu), ("Pr", Pr), ("gamma", gamma)):
        hp = 1e-4 * base  # parameter steps below ~1e-5 relative are roundoff-dominated
        kw = {"mu2": mu, "Pr2": Pr, "g2": gamma}
        key = {"mu": "mu2", "Pr": "Pr2", "gamma": "g2"}[k]
        kw[key] = base + hp
        lp = loss(F, **kw)
        kw[key] = base - hp
        lm = loss(F, **kw)
        fd = (lp - lm) / (2 * hp)
        assert abs(fd - g[k]) < 1e-6 * abs(g[k]), (k, fd, g[k])


def test_autograd_function_end_to_end(D):
    """DVBMFunction gives the same gradients through torch.autograd."""
    from paper_2510_04197_gb300.autograd import run
    F = I.random_smooth(16, 16, seed=8, amp=0.05, Ma=0.3)
    rho_t, T_t = targets(16, 16)
    fields = [torch.tensor(getattr(F, k), device="cuda", requires_grad=True) for k in ("rho", "ux", "uy", "T")]
    params = torch.tensor([2e-3, 0.71, 1.4], dtype=DT, requires_grad=True)
    rho, T = run(*fields, params, 9, dt=2e-4)
    L = 0.5 / 256 * (((rho - torch.tensor(rho_t, device="cuda")) ** 2).sum() +
                     ((T - torch.tensor(T_t, device="cuda")) ** 2).sum())
    L.backward()
    _, g = gpu_grad(D, F, 0.71, 1.4, 2e-3, 2e-4, 9, rho_t, T_t, every=3)
    assert torch.allclose(fields[0].grad, g["rho0"], rtol=1e-12, atol=1e-18)
    assert abs(float(params.grad[0]) - g["mu"]) < 1e-10 * abs(g["mu"])


def test_autograd_gradients_follow_input_devices(D):
    """Gradients come back on the devices of the inputs (fields on the host and
    parameters on the GPU, and the reverse), equal between the two placements;
    a second backward through the same forward is refused."""
    from paper_2510_04197_gb300.autograd import run
    F = I.random_smooth(16, 16, seed=8, amp=0.05, Ma=0.3)
    rho_t, T_t = targets(16, 16)

    def loss(dev_f, dev_p):
        fields = [torch.tensor(getattr(F, k), device=dev_f, requires_grad=True) for k in ("rho", "ux", "uy", "T")]
        params = torch.tensor([2e-3, 0.71, 1.4], dtype=DT, device=dev_p, requires_grad=True)
        rho, T = run(*fields, params, 9, dt=2e-4)
        L = 0.5 / 256 * (((rho - torch.tensor(rho_t, device=rho.device)) ** 2).sum() +
                         ((T - torch.tensor(T_t, device=T.device)) ** 2).sum())
        return L, fields, params

    L1, f1, p1 = loss("cuda", "cpu")
    L1.backward()
    L2, f2, p2 = loss("cpu", "cuda")
    L2.backward(retain_graph=True)
    assert all(t.grad.device.type == "cuda" for t in f1) and p1.grad.device.type == "cpu"
    assert all(t.grad.device.type == "cpu" for t in f2) and p2.grad.device.type == "cuda"
    for a, b in zip(f1, f2):
        assert torch.allclose(a.grad.cpu(), b.grad, rtol=1e-13, atol=0)
    assert torch.allclose(p1.grad, p2.grad.cpu(), rtol=1e-13, atol=0)
    with pytest.raises(RuntimeError, match="one backward pass"):
        L2.backward()


def test_adjoint_requires_recording(D):
    F = I.random_smooth(8, 8, seed=1)
    sim = D.Simulation(8, 8, 0.71, 1.4, 2e-3, dt=2e-4)
    sim.init(*(torch.tensor(a) for a in (F.rho, F.ux, F.uy, F.T)))
    sim.step(2)
    with pytest.raises(D.DVBMError) as e:
        sim.adjoint(torch.zeros(8, 8, dtype=DT), None)
    assert e.value.status == D.ESTATE
