"""Pins of the oracle's boundary conditions against what the scheme and the
paper fix, measured through plain lattice sums rather than the oracle's own
ghost code.

- Zero-gradient sides (Sec. III.A.3): both ghost layers repeat the boundary
  cell, so every boundary face carries v_i f_i of the boundary cell whatever
  the limiter (all slopes across the face vanish).  The update is in flux form
  (Eq. finalDiscretePDE) and the collision conserves mass, momentum and energy,
  so the one-step change of each domain total is the net flux through the two
  open sides, a closed form of the pre-step boundary populations.
- Wall ghosts (Sec. III.E): the ghost populations carry, in their own moments,
  the ghost state rho_G = rho_B, u_G = 2 u_W - u_B, T_G = 2 T_W - T_B and the
  non-equilibrium stress of the interior cell they mirror; ghost k mirrors
  interior cell k (reading R12).
- A uniform flow at the wall temperature between walls moving with it is a
  fixed point of the step; walls moving otherwise change it.
"""
import pytest
import torch

from oracle import dvbm_oracle as O
from paper_2510_04197_gb300 import inputs as I

MODELS = [("II", "D2Q25"), ("I", "D2Q16")]


def t(a):
    return torch.tensor(a, dtype=torch.float64)


def moments(lat, split, f, g):
    """rho, j_x, j_y, E and the second moment of f, by lattice sums (Sec. II.D.1)."""
    vx = lat.vx.view(-1, *([1] * (f.dim() - 1)))
    vy = lat.vy.view(-1, *([1] * (f.dim() - 1)))
    rho, jx, jy = f.sum(0), (vx * f).sum(0), (vy * f).sum(0)
    E = g.sum(0) if split == "I" else g.sum(0) + (0.5 * (vx * vx + vy * vy) * f).sum(0)
    M2 = ((vx * vx * f).sum(0), (vx * vy * f).sum(0), (vy * vy * f).sum(0))
    return rho, jx, jy, E, M2


def temperature(P, rho, jx, jy, E):
    """Eq. Total_energy_MB: E = rho C_v T + rho u^2 / 2."""
    return (E / rho - 0.5 * (jx * jx + jy * jy) / (rho * rho)) * (P.gamma - 1.0) / P.R


@pytest.mark.parametrize("split,kind", MODELS)
def test_zero_gradient_totals_change_by_the_boundary_flux(split, kind):
    P = O.Params(Pr=0.71, gamma=1.4, mu=0.02, split=split)
    lat = O.Lattice(kind=kind)
    zg = O.BC(O.ZEROGRAD)
    F = I.random_smooth(12, 8, seed=2, amp=0.05, Ma=0.4)
    grid = O.Grid(12, 8, 1.0, 1.0, (zg, zg, O.BC(), O.BC()))  # dx = 1/12, dy = 1/8
    f, g = O.init_populations(lat, P, t(F.rho), t(F.ux), t(F.uy), t(F.T))
    dt = 0.01  # largest node moves 0.34 cells; dt / tau about 1/2
    for _ in range(2):  # leave the equilibrium initial state
        f, g = O.step(lat, P, grid, f, g, dt)
    f1, g1 = O.step(lat, P, grid, f, g, dt)
    dV = grid.dx * grid.dy

    def totals(f, g):
        rho, jx, jy, E, _ = moments(lat, split, f, g)
        return torch.stack([rho.sum(), jx.sum(), jy.sum(), E.sum()]) * dV

    # conserved densities carried by each population: 1, v_x, v_y and its energy
    vx, vy = lat.vx.view(-1, 1), lat.vy.view(-1, 1)

    def densities(fc, gc):
        e = gc if split == "I" else gc + 0.5 * (vx * vx + vy * vy) * fc
        return torch.stack([fc, vx * fc, vy * fc, e])  # [4, Q, Ny]

    out = densities(f[:, :, -1], g[:, :, -1])  # boundary cells at x = Lx
    inn = densities(f[:, :, 0], g[:, :, 0])    # boundary cells at x = 0
    net = ((vx * (out - inn)).sum(1)).sum(-1) * grid.dy  # [4]
    expected = totals(f, g) - dt * net
    got = totals(f1, g1)
    rho, jx, jy, E, _ = moments(lat, split, f, g)
    scale = torch.stack([rho.abs().sum(), rho.abs().sum(), rho.abs().sum(), E.abs().sum()]) * dV
    assert ((dt * net).abs() / scale).max() > 1e-4  # the open sides do carry a flux
    err = ((got - expected).abs() / scale).max()
    assert err < 1e-14, float(err)


@pytest.mark.parametrize("split,kind", MODELS)
@pytest.mark.parametrize("lower", [True, False])
def test_wall_ghosts_carry_the_mirrored_state(split, kind, lower):
    P = O.Params(Pr=2.0, gamma=1.4, mu=0.02, split=split)
    lat = O.Lattice(kind=kind)
    F = I.random_smooth(6, 9, seed=4, amp=0.08, Ma=0.5)
    grid = O.Grid(6, 9, F.Lx, F.Ly)
    f, g = O.init_populations(lat, P, t(F.rho), t(F.ux), t(F.uy), t(F.T))
    for _ in range(2):  # non-equilibrium interior populations
        f, g = O.step(lat, P, grid, f, g, 0.01)
    uW, TW = (0.13, -0.05), 1.1
    wall = O.BC(O.WALL, uW, TW)
    fp, gp = O.pad_axis(lat, P, f, g, 1, wall, wall)  # rows: G2 G1 | 0 .. Ny-1 | G1 G2
    Ny = 9
    pairs = [(1, 2), (0, 3)] if lower else [(Ny + 2, Ny + 1), (Ny + 3, Ny)]  # (ghost k, interior k)
    for gi, bi in pairs:
        rG, jxG, jyG, EG, M2G = moments(lat, split, fp[:, gi], gp[:, gi])
        rB, jxB, jyB, EB, M2B = moments(lat, split, fp[:, bi], gp[:, bi])
        TB, TG = temperature(P, rB, jxB, jyB, EB), temperature(P, rG, jxG, jyG, EG)
        uxG, uyG = jxG / rG, jyG / rG
        uxB, uyB = jxB / rB, jyB / rB
        assert torch.allclose(rG, rB, rtol=1e-14, atol=0)
        assert torch.allclose(uxG, 2 * uW[0] - uxB, rtol=0, atol=1e-14)
        assert torch.allclose(uyG, 2 * uW[1] - uyB, rtol=0, atol=1e-14)
        assert torch.allclose(TG, 2 * TW - TB, rtol=1e-13, atol=0)
        # non-equilibrium stress: M2 minus its Maxwellian value rho (u u + R T I)
        neqG = (M2G[0] - rG * (uxG * uxG + P.R * TG), M2G[1] - rG * uxG * uyG, M2G[2] - rG * (uyG * uyG + P.R * TG))
        neqB = (M2B[0] - rB * (uxB * uxB + P.R * TB), M2B[1] - rB * uxB * uyB, M2B[2] - rB * (uyB * uyB + P.R * TB))
        for a, b in zip(neqG, neqB):
            assert torch.allclose(a, b, rtol=0, atol=1e-13)
        assert max(float(b.abs().max()) for b in neqB) > 1e-5  # the interior is off equilibrium


@pytest.mark.parametrize("split,kind", MODELS)
def test_uniform_flow_between_walls_moving_with_it_is_a_fixed_point(split, kind):
    P = O.Params(Pr=0.71, gamma=1.4, mu=0.02, split=split)
    lat = O.Lattice(kind=kind)
    U, TW = 0.3, 1.2
    one = torch.ones(10, 4, dtype=torch.float64)
    f, g = O.init_populations(lat, P, 0.9 * one, U * one, 0.0 * one, TW * one)
    for uw, fixed in ((U, True), (0.1, False)):
        wall = O.BC(O.WALL, (uw, 0.0), TW)
        grid = O.Grid(4, 10, 1.0, 2.5, (O.BC(), O.BC(), wall, wall))
        f1, g1 = O.step(lat, P, grid, f, g, 0.01)
        change = max(float((f1 - f).abs().max() / f.abs().max()), float((g1 - g).abs().max() / g.abs().max()))
        assert (change < 1e-14) if fixed else (change > 1e-5), (uw, change)
