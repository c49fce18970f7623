"""Seeded synthetic initial fields (rho, u_x, u_y, T) for the DVBM workloads.

This module only builds macroscopic input fields on the cell centres
x_j = (j + 1/2) dx, y_k = (k + 1/2) dy.  It holds none of the kinetic method's
arithmetic (no lattice, no equilibria, no update) and is shared by the CUDA
path's tests/benchmark and by the CPU oracle's tests as a common input source.

All fields are float64 numpy arrays of shape [Ny, Nx] (row-major, x fastest).
Workloads follow the paper's test problems (Sec. III.D wave decays, Sec. III.E
thermal Couette, Sec. III.F shock--vortex) and a random-phase multimode flow
used for throughput measurements.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Fields:
    rho: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    T: np.ndarray
    Lx: float = 1.0
    Ly: float = 1.0

    @property
    def shape(self):
        return self.rho.shape


def _centres(N: int, L: float):
    return (np.arange(N, dtype=np.float64) + 0.5) * (L / N)


def wave_decay(Nx=64, Ny=64, Ma=0.1, amp=1e-3, gamma=1.4, R=1.0, rho0=1.0, T0=1.0,
               shear=True, entropy=True, Lx=1.0, Ly=1.0) -> Fields:
    """Shear wave u_y = A sin(2 pi x/Lx) on x (Sec. III.D.1) and entropy wave
    rho = rho0 + A sin(2 pi y/Ly), T = rho0 T0/rho on y (Sec. III.D.3), over a
    mean flow u_x = Ma sqrt(gamma R T0).  The two modes sit on orthogonal axes."""
    x = _centres(Nx, Lx)[None, :]
    y = _centres(Ny, Ly)[:, None]
    u0 = Ma * math.sqrt(gamma * R * T0)
    rho = np.full((Ny, Nx), rho0)
    if entropy:
        rho = rho0 + amp * np.sin(2 * math.pi * y / Ly) + 0.0 * x
    T = rho0 * T0 / rho
    ux = np.full((Ny, Nx), u0)
    uy = (amp * np.sin(2 * math.pi * x / Lx) + 0.0 * y) if shear else np.zeros((Ny, Nx))
    return Fields(np.ascontiguousarray(rho), ux, np.ascontiguousarray(uy), np.ascontiguousarray(T), Lx, Ly)


def sound_wave(Nx=64, Ny=5, Ma=0.0, amp=1e-3, gamma=1.4, R=1.0, rho0=1.0, T0=1.0, Lx=1.0) -> Fields:
    """Density perturbation rho = rho0 + A sin(2 pi x/Lx) at uniform T
    (Sec. III.D.2)."""
    x = _centres(Nx, Lx)[None, :]
    u0 = Ma * math.sqrt(gamma * R * T0)
    rho = rho0 + amp * np.sin(2 * math.pi * x / Lx) + np.zeros((Ny, 1))
    return Fields(rho, np.full((Ny, Nx), u0), np.zeros((Ny, Nx)), np.full((Ny, Nx), T0), Lx, Ny * Lx / Nx)


@dataclass
class CouetteSetup:
    fields: Fields
    u0: float
    T_C: float
    T_H: float
    mu: float
    Ec: float


def couette(Nx=4, Ny=256, Ma=0.5, T_C=1.0, T_H=1.2, gamma=1.4, R=1.0, Re=100.0, Ly=1.0,
            profile="linear", Pr=None, Ec=None) -> CouetteSetup:
    """Thermal Couette flow (Sec. III.E): bottom wall at rest at T_C, top wall
    moving with u0 = Ma sqrt(gamma R T_C) at T_H; rho = 1/(R T_C);
    Re = rho u0 Ly / mu; Ec = u0^2 / (C_p (T_H - T_C)).  Given ``Ec``, T_H
    follows from it (the paper's cases: Ma 0.5 / Ec 4 and Ma 1.2 / Ec 40).
    ``profile="linear"``: linear u and T (the paper's initial condition);
    ``profile="analytic"``: the steady profiles (needs Pr), at uniform pressure."""
    y = _centres(Ny, Ly)[:, None] / Ly + np.zeros((1, Nx))
    u0 = Ma * math.sqrt(gamma * R * T_C)
    rho_c = 1.0 / (R * T_C)
    mu = rho_c * u0 * Ly / Re
    Cp = gamma * R / (gamma - 1.0)
    if Ec is not None:
        T_H = T_C + u0 * u0 / (Cp * Ec)
    Ec = u0 * u0 / (Cp * (T_H - T_C))
    ux = u0 * y
    if profile == "linear":
        T = T_C + (T_H - T_C) * y
        rho = np.full_like(y, rho_c)
    else:
        T = T_C + (T_H - T_C) * (y + 0.5 * Pr * Ec * y * (1.0 - y))
        rho = rho_c * T_C / T  # uniform pressure p = rho_c R T_C
    return CouetteSetup(Fields(rho, ux, np.zeros_like(y), T, Nx * Ly / Ny, Ly), u0, T_C, T_H, mu, Ec)


def couette_analytic_T(y_over_L, T_C, T_H, Pr, Ec):
    """(T - T_C)/(T_H - T_C) = eta + Pr Ec/2 eta (1 - eta), Sec. III.E."""
    eta = y_over_L
    return T_C + (T_H - T_C) * (eta + 0.5 * Pr * Ec * eta * (1.0 - eta))


@dataclass
class ShockVortexSetup:
    fields: Fields
    mu: float
    cs_l: float
    p_r: float


def shock_vortex(N=1024, Ma_s=1.2, Ma_v=0.25, r_v=0.075, Re_v=800.0, gamma=1.4, R=1.0,
                 x_s=0.5, x_v=0.35, y_v=0.5, L=1.0, Ny=None, Ly=None) -> ShockVortexSetup:
    """Stationary normal shock with Rankine--Hugoniot states and an isentropic
    vortex (Sec. III.F), on [0, L] x [0, Ly] with N x Ny cells (square by
    default).  Pre-shock (left) state rho_l = p_l = 1, u_l = Ma_s c_{s,l};
    post-shock state from the jump conditions; vortex of core radius r_v
    centred at (x_v, y_v) perturbs the local (left or right) state;
    mu = rho_l c_{s,l} r_v / Re_v."""
    Ny = N if Ny is None else Ny
    Ly = L if Ly is None else Ly
    rho_l, p_l = 1.0, 1.0
    cs_l = math.sqrt(gamma * p_l / rho_l)
    u_l = Ma_s * cs_l
    M2 = Ma_s * Ma_s
    rho_r = rho_l * (gamma + 1) * M2 / ((gamma - 1) * M2 + 2)
    p_r = p_l * (2 * gamma * M2 - (gamma - 1)) / (gamma + 1)
    u_r = u_l * ((gamma - 1) * M2 + 2) / ((gamma + 1) * M2)
    x = _centres(N, L)[None, :] + np.zeros((Ny, 1))
    y = _centres(Ny, Ly)[:, None] + np.zeros((1, N))
    left = x <= x_s
    rho_inf = np.where(left, rho_l, rho_r)
    p_inf = np.where(left, p_l, p_r)
    ux_inf = np.where(left, u_l, u_r)
    r2 = ((x - x_v) ** 2 + (y - y_v) ** 2) / (r_v * r_v)
    e = np.exp((1.0 - r2) / 2.0)
    ux = ux_inf + cs_l * Ma_v * (y - y_v) / r_v * e
    uy = -cs_l * Ma_v * (x - x_v) / r_v * e
    base = 1.0 - (gamma - 1) / 2.0 * Ma_v * Ma_v * np.exp(1.0 - r2)
    rho = rho_inf * base ** (1.0 / (gamma - 1))
    p = p_inf * base ** (gamma / (gamma - 1))
    T = p / (rho * R)
    mu = rho_l * cs_l * r_v / Re_v
    return ShockVortexSetup(Fields(rho, ux, uy, T, L, Ly), mu, cs_l, p_r)


# Sec. III.F cases of the shock--vortex interaction: (Ma_s, Ma_v)
SHOCK_VORTEX_CASES = {"C": (1.2, 0.25), "G": (1.29, 0.39)}


def shock_vortex_case(case="G", Nx=1680, Ny=1440, gamma=1.4, R=1.0) -> ShockVortexSetup:
    """The paper's shock--vortex geometry (Sec. III.F): domain [0, 28] x [0, 24],
    shock at x_s = 8, vortex of radius r_v = 1 centred at (6, 12),
    Re_v = 800, at the paper's resolution 1680 x 1440 by default (a smaller
    Nx x Ny keeps dx = dy when Nx/Ny = 28/24)."""
    Ma_s, Ma_v = SHOCK_VORTEX_CASES[case]
    return shock_vortex(N=Nx, Ny=Ny, Ma_s=Ma_s, Ma_v=Ma_v, r_v=1.0, Re_v=800.0, gamma=gamma, R=R,
                        x_s=8.0, x_v=6.0, y_v=12.0, L=28.0, Ly=24.0)


def _spectral_field(N: int, rng: np.random.Generator, k_peak=8.0, k_width=2.0, k_max=32):
    """Real random-phase Fourier sum over integer wavevectors |k| <= k_max with
    amplitude exp(-(|k| - k_peak)^2 / (2 k_width^2)), normalised to unit rms."""
    spec = np.zeros((N, N), dtype=np.complex128)
    kk = np.fft.fftfreq(N, d=1.0 / N)
    KX, KY = np.meshgrid(kk, kk)
    K = np.sqrt(KX * KX + KY * KY)
    mask = (K <= k_max) & (K > 0)
    amp = np.exp(-((K - k_peak) ** 2) / (2 * k_width * k_width)) * mask
    phase = rng.uniform(0.0, 2 * math.pi, size=(N, N))
    spec = amp * np.exp(1j * phase)
    fld = np.real(np.fft.ifft2(spec)) * N * N
    fld -= fld.mean()
    return fld / np.sqrt(np.mean(fld * fld))


def multimode(N=1024, seed=0, rms_Ma=0.3, rms_dT=0.05, gamma=1.4, R=1.0, T0=1.0) -> Fields:
    """Random-phase multimode flow for throughput runs: u_x, u_y independent
    spectral fields (Gaussian shell spectrum peaking at |k| = 8, width 2,
    |k| <= 32) scaled so the rms Mach number of |u| is ``rms_Ma``;
    T = T0 (1 + dT) with the same spectrum at rms ``rms_dT``; rho = 1/T
    (uniform pressure).  Seeded PCG64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ux = _spectral_field(N, rng)
    uy = _spectral_field(N, rng)
    dT = _spectral_field(N, rng)
    cs = math.sqrt(gamma * R * T0)
    scale = rms_Ma * cs / math.sqrt(np.mean(ux * ux + uy * uy))
    T = T0 * (1.0 + rms_dT * dT)
    rho = 1.0 / T
    return Fields(rho, ux * scale, uy * scale, T, 1.0, 1.0)


def uniform(Nx=8, Ny=8, rho=1.0, ux=0.0, uy=0.0, T=1.0) -> Fields:
    z = np.zeros((Ny, Nx))
    return Fields(z + rho, z + ux, z + uy, z + T, 1.0, Ny / Nx)


def random_smooth(Nx=16, Ny=12, seed=0, amp=0.05, Ma=0.2, gamma=1.4, R=1.0) -> Fields:
    """Small smooth random fields (few low Fourier modes) for parity and
    gradient checks on small grids."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = _centres(Nx, 1.0)[None, :]
    y = _centres(Ny, Ny / Nx)[:, None] * (Nx / Ny)

    def fld():
        out = np.zeros((Ny, Nx))
        for kx in range(0, 3):
            for ky in range(0, 3):
                if kx == 0 and ky == 0:
                    continue
                ph = rng.uniform(0, 2 * math.pi)
                out += rng.normal() * np.cos(2 * math.pi * (kx * x + ky * y) + ph)
        return out / np.sqrt(np.mean(out * out))

    cs = math.sqrt(gamma * R)
    return Fields(1.0 + amp * fld(), Ma * cs * (0.5 + 0.5 * fld()), Ma * cs * 0.5 * fld(),
                  1.0 + amp * fld(), 1.0, Ny / Nx)
