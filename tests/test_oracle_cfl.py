"""Pin of the oracle's time-step rule (Sec. III.A.3; reading R10: the global
maximum of |u| + sqrt(gamma R T) over the initial field) against worked
examples computed by hand (tests/golden/cfl_dt_worked_examples.txt)."""
import os
from fractions import Fraction

import pytest
import torch

from oracle import dvbm_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cfl_dt_worked_examples.txt")


def read_cases():
    cases, cur = [], None
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if not line:
            continue
        tok = line.split()
        if tok[0] == "case":
            cur = {"name": tok[1], "gamma": float(tok[2]), "R": float(tok[3]), "Nx": int(tok[4]),
                   "Ny": int(tok[5]), "Lx": float(tok[6]), "Ly": float(tok[7]), "cfl": float(tok[8]),
                   "dt": float(Fraction(tok[9])), "cells": []}
            cases.append(cur)
        else:
            cur["cells"].append([float(v) for v in tok])
    return cases


CASES = read_cases()


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_cfl_dt_worked_examples(case):
    assert len(case["cells"]) == case["Nx"] * case["Ny"]
    c = torch.tensor(case["cells"], dtype=torch.float64).reshape(case["Ny"], case["Nx"], 3)
    P = O.Params(Pr=0.71, gamma=case["gamma"], mu=1e-3, R=case["R"])
    grid = O.Grid(case["Nx"], case["Ny"], case["Lx"], case["Ly"])
    dt = O.cfl_dt(P, grid, c[..., 0], c[..., 1], c[..., 2], case["cfl"])
    assert abs(dt - case["dt"]) <= 1e-15 * case["dt"], (dt, case["dt"])


def test_cfl_dt_scales_with_cfl_and_cell_size():
    """dt is linear in CFL and in the cell size, and invariant under a
    reflection of the velocity field."""
    case = CASES[0]
    c = torch.tensor(case["cells"], dtype=torch.float64).reshape(case["Ny"], case["Nx"], 3)
    P = O.Params(Pr=0.71, gamma=case["gamma"], mu=1e-3, R=case["R"])
    g1 = O.Grid(case["Nx"], case["Ny"], case["Lx"], case["Ly"])
    g2 = O.Grid(case["Nx"], case["Ny"], 2 * case["Lx"], 2 * case["Ly"])
    d1 = O.cfl_dt(P, g1, c[..., 0], c[..., 1], c[..., 2], 0.3)
    assert abs(O.cfl_dt(P, g1, c[..., 0], c[..., 1], c[..., 2], 0.6) - 2 * d1) < 1e-15 * d1
    assert abs(O.cfl_dt(P, g2, c[..., 0], c[..., 1], c[..., 2], 0.3) - 2 * d1) < 1e-15 * d1
    assert abs(O.cfl_dt(P, g1, -c[..., 1], -c[..., 0], c[..., 2], 0.3) - d1) < 1e-15 * d1
