"""Pin of the oracle's discrete adjoint (torch.autograd applied to the oracle
forward map): directional derivatives match central finite differences of
the same forward map, for the initial fields and for (mu, Pr, gamma)."""
import numpy as np
import pytest
import torch

from oracle import dvbm_oracle as O
from paper_2510_04197_gb300 import inputs as I

DT = torch.float64


def loss_and_grad(F, Pr, gamma, mu, dt, n, rho_t, T_t, grad=True):
    t = lambda a: torch.tensor(a, dtype=DT, requires_grad=grad)
    fields = [t(getattr(F, k)) for k in ("rho", "ux", "uy", "T")]
    pm, pP, pg = [torch.tensor(v, dtype=DT, requires_grad=grad) for v in (mu, Pr, gamma)]
    P = O.Params(Pr=pP, gamma=pg, mu=pm)
    lat = O.Lattice()
    Ny, Nx = F.rho.shape
    grid = O.Grid(Nx, Ny, F.Lx, F.Ly)
    f, g = O.init_populations(lat, P, *fields)
    for _ in range(n):
        f, g = O.step(lat, P, grid, f, g, dt)
    rho, ux, uy, T, _ = O.macroscopic(lat, P, f, g)
    L = 0.5 / (Nx * Ny) * (((rho - torch.tensor(rho_t)) ** 2).sum() + ((T - torch.tensor(T_t)) ** 2).sum())
    if not grad:
        return float(L), None
    L.backward()
    return float(L), [x.grad.numpy() for x in fields] + [float(pm.grad), float(pP.grad), float(pg.grad)]


@pytest.mark.parametrize("Pr", [0.71, 2.0])
def test_oracle_adjoint_matches_finite_differences(Pr):
    F = I.random_smooth(10, 8, seed=4, amp=0.08, Ma=0.4)
    Tg = I.random_smooth(10, 8, seed=9, amp=0.05, Ma=0.2)
    gamma, mu, dt, n = 1.4, 2e-3, 2e-4, 4
    _, g = loss_and_grad(F, Pr, gamma, mu, dt, n, Tg.rho, Tg.T)
    h = 1e-6
    for trial in range(2):
        V = I.random_smooth(10, 8, seed=50 + trial)
        d = [getattr(V, k) - getattr(V, k).mean() for k in ("rho", "ux", "uy", "T")]
        keys = ("rho", "ux", "uy", "T")
        Fp = I.Fields(*[getattr(F, k) + h * dk for k, dk in zip(keys, d)], F.Lx, F.Ly)
        Fm = I.Fields(*[getattr(F, k) - h * dk for k, dk in zip(keys, d)], F.Lx, F.Ly)
        fd = (loss_and_grad(Fp, Pr, gamma, mu, dt, n, Tg.rho, Tg.T, False)[0]
              - loss_and_grad(Fm, Pr, gamma, mu, dt, n, Tg.rho, Tg.T, False)[0]) / (2 * h)
        ad = sum(float((gk * dk).sum()) for gk, dk in zip(g[:4], d))
        assert abs(fd - ad) < 1e-6 * abs(ad), (fd, ad)
    for i, (name, base) in enumerate((("mu", mu), ("Pr", Pr), ("gamma", gamma))):
        hp = 1e-4 * base  # parameter steps below ~1e-5 relative are roundoff-dominated
        args = [Pr, gamma, mu]
        idx = {"mu": 2, "Pr": 0, "gamma": 1}[name]
        ap = list(args); ap[idx] = base + hp
        am = list(args); am[idx] = base - hp
        fd = (loss_and_grad(F, *ap, dt, n, Tg.rho, Tg.T, False)[0]
              - loss_and_grad(F, *am, dt, n, Tg.rho, Tg.T, False)[0]) / (2 * hp)
        assert abs(fd - g[4 + i]) < 1e-6 * abs(g[4 + i]), (name, fd, g[4 + i])


def test_oracle_adjoint_dot_product_against_forward_mode():
    """Dot-product test of the discrete adjoint: for the map (rho0, u0, T0) ->
    (rho_n, T_n) of the oracle, the forward-mode directional derivative J v
    (torch.func.jvp, dual numbers) and the reverse-mode product J^T w
    (torch.autograd) satisfy <w, J v> = <J^T w, v> to roundoff."""
    F = I.random_smooth(8, 6, seed=11, amp=0.08, Ma=0.4)
    gamma, mu, dt, n, Pr = 1.4, 2e-3, 2e-4, 3, 0.71
    lat = O.Lattice()
    Ny, Nx = F.rho.shape
    grid = O.Grid(Nx, Ny, F.Lx, F.Ly)
    P = O.Params(Pr=Pr, gamma=gamma, mu=mu)

    def forward(rho, ux, uy, T):
        f, g = O.init_populations(lat, P, rho, ux, uy, T)
        for _ in range(n):
            f, g = O.step(lat, P, grid, f, g, dt)
        r, _, _, t, _ = O.macroscopic(lat, P, f, g)
        return torch.stack([r, t])

    x = tuple(torch.tensor(getattr(F, k), dtype=DT) for k in ("rho", "ux", "uy", "T"))
    rng = np.random.default_rng(3)
    v = tuple(torch.tensor(rng.standard_normal(F.rho.shape), dtype=DT) for _ in range(4))
    w = torch.tensor(rng.standard_normal((2,) + F.rho.shape), dtype=DT)
    _, Jv = torch.func.jvp(forward, x, v)
    xr = tuple(a.clone().requires_grad_(True) for a in x)
    JTw = torch.autograd.grad(forward(*xr), xr, grad_outputs=w)
    lhs = float((w * Jv).sum())
    rhs = float(sum((a * b).sum() for a, b in zip(JTw, v)))
    assert abs(lhs - rhs) < 1e-12 * max(abs(lhs), 1.0), (lhs, rhs)
