"""Test infrastructure: a pytest plugin that plants one plausible mistake in
the oracle (in memory, in the child process it is loaded into), chosen by the
environment variable DVBM_ORACLE_MUTATION.  tests/test_oracle_mutations.py
runs the oracle's pins under each mistake and requires every one to fail."""
import os

import torch

MUTATIONS = [
    "relaxation_times_swapped",   # tau1 <-> tau2 (Sec. II.C)
    "single_relaxation_time",     # tau2 = tau1: the two-rate relaxation lost
    "first_order_faces",          # NND face value without the limited slope
    "limiter_beta_ignored",       # beta fixed at 1 (minmod) whatever the parameter
    "feq_fourth_order_error",     # a spurious He_4(xi_x) term in f^eq
    "quasi_equilibrium_negated",  # f* - f^eq (and g* - g^eq) with the wrong sign
    "energy_without_kinetic_part",  # split II: E = sum g, the v^2/2 f part dropped
    "cv_over_gamma",              # C_v = R / gamma instead of R / (gamma - 1)
    "wall_velocity_unreflected",  # u_G = u_W - u_B instead of 2 u_W - u_B
    "wall_temperature_copied",    # T_G = T_W instead of 2 T_W - T_B
    "wall_neq_negated",           # f_G = f^eq_G - (f_B - f^eq_B)
    "wall_neq_dropped",           # f_G = f^eq_G
    "wall_ghosts_swapped",        # ghost 1 mirrors interior cell 2 and vice versa
    "zero_gradient_second_cell",  # zero-gradient ghosts copy the second cell
    "face_areas_swapped",         # dy on y-faces and dx on x-faces
    "split1_energy_with_kinetic_part",  # split I: E = sum g + v^2/2 f instead of sum g
    "downwind_faces",             # faces reconstructed from the downwind side
    "prandtl_branch_ignored",     # Pr > 1 relaxed with the Pr < 1 mapping of tau1, tau2
    "d2q16_weights_swapped",      # D2Q16 inner and outer 1-D weights exchanged
    "cfl_speed_at_reference_temperature",  # c_s = sqrt(gamma R T_ref) in the time-step rule
    "cfl_separate_maxima",        # max |u| + max c_s taken over different cells
]


def _apply(O, name):
    if name == "relaxation_times_swapped":
        f0 = O.relaxation_times
        O.relaxation_times = lambda P, rho, T: tuple(reversed(f0(P, rho, T)))
    elif name == "single_relaxation_time":
        f0 = O.relaxation_times
        O.relaxation_times = lambda P, rho, T: (f0(P, rho, T)[0],) * 2
    elif name == "first_order_faces":
        O.face_values = lambda Fm2, Fm1, F0, Fp1, vpos, beta: torch.where(
            vpos.view((-1,) + (1,) * (Fm1.dim() - 1)), Fm1, F0)
    elif name == "limiter_beta_ignored":
        f0 = O.face_values
        O.face_values = lambda Fm2, Fm1, F0, Fp1, vpos, beta: f0(Fm2, Fm1, F0, Fp1, vpos, 1.0)
    elif name == "feq_fourth_order_error":
        f0 = O.equilibria

        def eq(lat, P, rho, ux, uy, T):
            feq, geq = f0(lat, P, rho, ux, uy, T)
            xi = lat.vx / (P.R * P.T_ref) ** 0.5
            shape = (-1,) + (1,) * (feq.dim() - 1)
            return feq + 0.01 * (lat.w * (xi ** 4 - 6 * xi ** 2 + 3)).view(shape) * rho, geq
        O.equilibria = eq
    elif name == "quasi_equilibrium_negated":
        f0 = O.quasi_equilibria

        def qe(lat, P, f, g, rho, ux, uy, T, feq, geq):
            fs, gs = f0(lat, P, f, g, rho, ux, uy, T, feq, geq)
            return 2 * feq - fs, 2 * geq - gs
        O.quasi_equilibria = qe
    elif name == "energy_without_kinetic_part":
        f0 = O.macroscopic

        def mac(lat, P, f, g):
            rho, ux, uy, T, E = f0(lat, P, f, g)
            if P.split == "I":
                return rho, ux, uy, T, E
            E = g.sum(0)
            return rho, ux, uy, (E / rho - 0.5 * (ux * ux + uy * uy)) / P.Cv(), E
        O.macroscopic = mac
    elif name == "cv_over_gamma":
        O.Params.Cv = lambda self: self.R / self.gamma
    elif name.startswith("wall_") and name != "wall_ghosts_swapped":
        def ghost(lat, P, fB, gB, bc):
            rho, ux, uy, T, _ = O.macroscopic(lat, P, fB, gB)
            feqB, geqB = O.equilibria(lat, P, rho, ux, uy, T)
            k = 1.0 if name == "wall_velocity_unreflected" else 2.0
            TG = bc.T_wall + 0.0 * T if name == "wall_temperature_copied" else 2.0 * bc.T_wall - T
            feqG, geqG = O.equilibria(lat, P, rho, k * bc.u_wall[0] - ux, k * bc.u_wall[1] - uy, TG)
            s = {"wall_neq_negated": -1.0, "wall_neq_dropped": 0.0}.get(name, 1.0)
            return feqG + s * (fB - feqB), geqG + s * (gB - geqB)
        O._wall_ghost = ghost
    elif name in ("wall_ghosts_swapped", "zero_gradient_second_cell"):
        f0 = O.pad_axis

        def pad(lat, P, f, g, axis, lo, hi):
            fp, gp = f0(lat, P, f, g, axis, lo, hi)
            n = f.shape[axis]
            if name == "wall_ghosts_swapped" and lo.kind == O.WALL:
                for A in (fp, gp):
                    a = A.narrow(axis, 0, 1).clone()
                    A.narrow(axis, 0, 1).copy_(A.narrow(axis, 1, 1))
                    A.narrow(axis, 1, 1).copy_(a)
            if name == "zero_gradient_second_cell" and lo.kind == O.ZEROGRAD:
                for src, A in ((f, fp), (g, gp)):
                    for k in (0, 1):
                        A.narrow(axis, k, 1).copy_(src.narrow(axis, 1, 1))
                        A.narrow(axis, n + 2 + k, 1).copy_(src.narrow(axis, n - 2, 1))
            return fp, gp
        O.pad_axis = pad
    elif name == "face_areas_swapped":
        f0 = O.advective_term

        def adv(lat, P, grid, fpx, fpy):
            g2 = O.Grid(grid.Nx, grid.Ny, grid.Ly * grid.Nx / grid.Ny, grid.Lx * grid.Ny / grid.Nx, grid.bcs)
            return f0(lat, P, g2, fpx, fpy)
        O.advective_term = adv
    elif name == "split1_energy_with_kinetic_part":
        f0 = O.macroscopic

        def mac1(lat, P, f, g):
            rho, ux, uy, T, E = f0(lat, P, f, g)
            if P.split != "I":
                return rho, ux, uy, T, E
            v2 = (lat.vx * lat.vx + lat.vy * lat.vy).view((-1,) + (1,) * (f.dim() - 1))
            E = g.sum(0) + (0.5 * v2 * f).sum(0)
            return rho, ux, uy, (E / rho - 0.5 * (ux * ux + uy * uy)) / P.Cv(), E
        O.macroscopic = mac1
    elif name == "downwind_faces":
        f0 = O.face_values
        O.face_values = lambda Fm2, Fm1, F0, Fp1, vpos, beta: f0(Fm2, Fm1, F0, Fp1, ~vpos, beta)
    elif name == "prandtl_branch_ignored":
        def tau(P, rho, T):
            t1 = P.mu / (rho * P.R * T)
            return t1, t1 / P.Pr
        O.relaxation_times = tau
    elif name == "d2q16_weights_swapped":
        f0 = O.Lattice.__init__

        def init(self, *a, **k):
            f0(self, *a, **k)
            if self.Q == 16:
                w1 = [self.w1[1], self.w1[0], self.w1[3], self.w1[2]]
                self.w1 = w1
                self.w = torch.tensor([w1[p] * w1[q] for p in range(4) for q in range(4)], dtype=O.DT)
        O.Lattice.__init__ = init
    elif name == "cfl_speed_at_reference_temperature":
        def cfl_ref(P, grid, ux, uy, T, cfl):
            speed = torch.sqrt(ux * ux + uy * uy) + (float(P.gamma) * P.R * P.T_ref) ** 0.5
            return cfl * min(grid.dx, grid.dy) / float(speed.max())
        O.cfl_dt = cfl_ref
    elif name == "cfl_separate_maxima":
        def cfl_sep(P, grid, ux, uy, T, cfl):
            umax = float(torch.sqrt(ux * ux + uy * uy).max())
            cmax = float(torch.sqrt(float(P.gamma) * P.R * T).max())
            return cfl * min(grid.dx, grid.dy) / (umax + cmax)
        O.cfl_dt = cfl_sep
    else:
        raise ValueError(f"unknown mutation {name}")


def pytest_configure(config):
    name = os.environ.get("DVBM_ORACLE_MUTATION", "")
    if name:
        from oracle import dvbm_oracle as O
        _apply(O, name)
