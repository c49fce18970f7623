"""Pins of the FP64 CPU oracle against facts fixed outside the oracle itself.

Each test compares the oracle with a closed form, a textbook/library routine
(numpy's Hermite polynomials and Gauss--Hermite quadrature of the continuous
Maxwellian), a constraint equation printed in the paper, or an invariant that
a dropped term, a wrong sign or a transposed index would break.
"""
import math
import re

import numpy as np
import pytest
import torch
from numpy.polynomial import hermite_e as He

from oracle import dvbm_oracle as O

DT = torch.float64


@pytest.fixture(scope="module")
def lat():
    return O.Lattice()


def rand_state(lat, P, shape=(3, 4), seed=0, noise=1e-3):
    """Random macroscopic state and non-equilibrium populations around it."""
    g = torch.Generator().manual_seed(seed)
    rho = 0.8 + 0.4 * torch.rand(shape, generator=g, dtype=DT)
    ux = 0.6 * (torch.rand(shape, generator=g, dtype=DT) - 0.5)
    uy = 0.6 * (torch.rand(shape, generator=g, dtype=DT) - 0.5)
    T = 0.7 + 0.6 * torch.rand(shape, generator=g, dtype=DT)
    feq, geq = O.equilibria(lat, P, rho, ux, uy, T)
    f = feq * (1 + noise * torch.randn(feq.shape, generator=g, dtype=DT))
    gg = geq * (1 + noise * torch.randn(geq.shape, generator=g, dtype=DT))
    return f, gg


# ---------------------------------------------------------------- lattice ---

def test_lattice_matches_printed_table(lat):
    """App. G Table D2Q25 (with the /60 weight reading), parsed from the
    golden text fixture and evaluated independently of the oracle."""
    s = math.sqrt(10.0)
    rows = []
    with open(__file__.replace("test_oracle_pins.py", "golden/d2q25_table.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            rows.append(line.split()[1:])
    pts = []
    for vx, vy, wa, wb in rows:
        def vals(e):
            if e.startswith("+-"):
                x = eval(e[2:], {"sqrt": math.sqrt, "s": s})
                return [x, -x]
            return [eval(e, {"sqrt": math.sqrt, "s": s})]
        w = eval(wa, {"s": s}) * eval(wb, {"s": s})
        for a in vals(vx):
            for b in vals(vy):
                pts.append((a, b, w))
    assert len(pts) == 25
    table = sorted(pts)
    ours = sorted(zip(lat.vx.tolist(), lat.vy.tolist(), lat.w.tolist()))
    for (a, b, w), (c, d, x) in zip(table, ours):
        assert abs(a - c) < 1e-14 and abs(b - d) < 1e-14 and abs(w - x) < 1e-15


def test_lattice_gauss_hermite_exactness(lat):
    """sum_i w_i xi^k = (k-1)!! for even k <= 8 and 0 for odd k <= 9: the
    five-point rule is exact to degree 2Q - 1 = 9 (App. C)."""
    for k in range(10):
        s = sum(w * x ** k for w, x in zip(lat.w1, lat.xi1))
        exact = 0.0 if k % 2 else float(np.prod(np.arange(k - 1, 0, -2))) if k > 0 else 1.0
        assert abs(s - exact) < 1e-12 * max(1.0, exact)
    # 2-D: weights sum to one; compare with numpy's He_5 roots/weights
    x, w = He.hermegauss(5)
    w = w / math.sqrt(2 * math.pi)
    assert np.allclose(sorted(x), lat.xi1, atol=1e-14)
    assert np.allclose([w[np.argmin(abs(x - a))] for a in lat.xi1], lat.w1, atol=1e-15)
    assert abs(float(lat.w.sum()) - 1.0) < 1e-15


@pytest.mark.parametrize("RT", [1.0, 1.7])
def test_hermite_tensors_factorise_into_textbook_polynomials(RT):
    """H_tuple(v) = (R T_ref)^{n/2} He_a(v_x/c) He_b(v_y/c), a = #x indices
    (App. D Eq. Hermitepolynomials-0-4 vs numpy.polynomial.hermite_e)."""
    lt = O.Lattice(R=RT, T_ref=1.0)
    c = math.sqrt(lt.c2)
    for n in range(5):
        for t in O.tuples(n):
            a = t.count(0)
            b = n - a
            ref = c ** n * He.hermeval(lt.vx.numpy() / c, [0] * a + [1]) * He.hermeval(lt.vy.numpy() / c, [0] * b + [1])
            assert np.allclose(O.hermite(lt, t).numpy(), ref, atol=1e-12, rtol=1e-13)


def test_hermite_orthogonality_on_lattice(lat):
    """sum_i w_i H_s H_t = (R T_ref)^n a! b! if s, t are permutations of each
    other (a x-indices, b y-indices), else 0 -- exact on D2Q25 for n <= 4
    (degree 8 <= 9)."""
    for n in range(5):
        for s in O.tuples(n):
            for t in O.tuples(n):
                val = float((lat.w * O.hermite(lat, s) * O.hermite(lat, t)).sum())
                a = s.count(0)
                exp = math.factorial(a) * math.factorial(n - a) * lat.c2 ** n if sorted(s) == sorted(t) else 0.0
                assert abs(val - exp) < 1e-12 * max(1.0, exp)
    for m, n in [(0, 2), (1, 3), (2, 4), (0, 4)]:
        for s in O.tuples(m):
            for t in O.tuples(n):
                assert abs(float((lat.w * O.hermite(lat, s) * O.hermite(lat, t)).sum())) < 1e-12


# -------------------------------------------------------------- equilibria ---

def continuous_maxwell_moment(rho, ux, uy, T, R, tup, npts=12):
    """Moment of the continuous Maxwell--Boltzmann distribution (Eq.
    MB-equilibrium) by Gauss--Hermite quadrature in shifted, scaled
    coordinates (numpy.polynomial.hermite_e.hermegauss, exact here)."""
    x, w = He.hermegauss(npts)
    w = w / math.sqrt(2 * math.pi)
    s = math.sqrt(R * T)
    tot = 0.0
    for i in range(npts):
        for j in range(npts):
            v = (ux + s * x[i], uy + s * x[j])
            tot += w[i] * w[j] * np.prod([v[a] for a in tup])
    return rho * tot


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_feq_reproduces_maxwellian_moments_to_fourth_order(lat, seed):
    """sum_i v^n f_i^eq equals the continuous Maxwellian moment for n <= 4
    (Sec. II.D.3: N = 4 on a fifth-order quadrature, split II)."""
    rng = np.random.default_rng(seed)
    P = O.Params(gamma=1.4)
    rho, ux, uy, T = 0.5 + rng.random(), 1.5 * (rng.random() - 0.5), 1.5 * (rng.random() - 0.5), 0.5 + 1.5 * rng.random()
    t = lambda z: torch.tensor([z], dtype=DT)
    feq, geq = O.equilibria(lat, P, t(rho), t(ux), t(uy), t(T))
    eps = (P.Cv() - P.R) * T  # C_v T - R T D/2 with D = 2
    for n in range(5):
        for tup in O.tuples(n):
            ref = continuous_maxwell_moment(rho, ux, uy, T, P.R, tup)
            got = float(O.lattice_moment(lat, feq, tup))
            assert abs(got - ref) < 1e-12 * max(1.0, abs(ref)), (tup, got, ref)
            if n <= 2:  # g^eq moments are eps times the Maxwellian ones (App. A, split II)
                got_g = float(O.lattice_moment(lat, geq, tup))
                assert abs(got_g - eps * ref) < 1e-12 * max(1.0, abs(eps * ref))


def test_feq_fifth_moment_is_not_reproduced(lat):
    """Negative control: the fourth-order expansion does not carry fifth-order
    moments (shows the moment test above can fail)."""
    P = O.Params()
    t = lambda z: torch.tensor([z], dtype=DT)
    feq, _ = O.equilibria(lat, P, t(1.0), t(0.7), t(0.3), t(1.3))
    tup = (0, 0, 0, 0, 0)
    ref = continuous_maxwell_moment(1.0, 0.7, 0.3, 1.3, 1.0, tup)
    got = float(O.lattice_moment(lat, feq, tup))
    assert abs(got - ref) > 1e-6


def test_theta_form_equals_semi_recursive_and_lattice_projection(lat):
    """The explicit theta-form equilibrium coefficients (App. D) equal both the
    semi-recursive formulas applied to Maxwellian moments and the Hermite
    projection sum_i f_i^eq H_n(v_i) of the expanded populations."""
    P = O.Params()
    f, _ = rand_state(lat, P, noise=0.0)
    rho, ux, uy, T, _ = O.macroscopic(lat, P, f, torch.zeros_like(f))
    rho = torch.tensor([1.1], dtype=DT); ux = torch.tensor([0.4], dtype=DT)
    uy = torch.tensor([-0.2], dtype=DT); T = torch.tensor([1.3], dtype=DT)
    M = {t: O.maxwell_moment(lat, P.R, rho, (ux, uy), T, t) for n in range(5) for t in O.tuples(n)}
    a_sr = O.coefficients_from_moments(lat, M, 4)
    feq, _ = O.equilibria(lat, P, rho, ux, uy, T)
    for n in range(5):
        for t in O.tuples(n):
            a_th = O.a_eq_f(lat, rho, (ux, uy), T, t)
            proj = (O.hermite(lat, t).view(-1, 1) * feq).sum(0)
            assert torch.allclose(a_th, a_sr[t], atol=1e-13, rtol=1e-13)
            assert torch.allclose(a_th, proj, atol=1e-13, rtol=1e-13)


# ------------------------------------------------------- quasi-equilibria ---

def _lsum(lat, F, wgt):
    return torch.einsum("i,i...->...", wgt, F)


@pytest.mark.parametrize("Pr", [0.5, 0.71, 0.75, 2.0, 1.3])
def test_quasi_equilibria_satisfy_paper_constraints(lat, Pr):
    """f*, g* satisfy the conservation constraints (Eqs. eq_con_fstar1/2,
    eq_con_gstar_total (II)), the pressure-tensor constraint (Eq.
    QE_Pr<1_conserved, or the trace-fixed Eq.
    disc_QE_Pr>1_quasiconserved_conservationFix) and the heat-flux constraint
    (Eq. QE_Pr<1_quasiconserved (II) or QE_Pr>1_conserved (II)), each written
    here as the paper prints it, with lattice sums."""
    P = O.Params(Pr=Pr, gamma=1.4)
    f, g = rand_state(lat, P, noise=5e-2, seed=3)
    rho, ux, uy, T, _ = O.macroscopic(lat, P, f, g)
    feq, geq = O.equilibria(lat, P, rho, ux, uy, T)
    fs, gs = O.quasi_equilibria(lat, P, f, g, rho, ux, uy, T, feq, geq)
    vx, vy = lat.vx, lat.vy
    v2 = vx * vx + vy * vy
    one = torch.ones_like(vx)
    tol = 1e-13
    # mass, momentum
    for wgt in (one, vx, vy):
        assert torch.allclose(_lsum(lat, fs, wgt), _lsum(lat, f, wgt), atol=tol, rtol=tol)
    # total energy (II)
    E = _lsum(lat, g, one) + _lsum(lat, f, 0.5 * v2)
    Es = _lsum(lat, gs, one) + _lsum(lat, fs, 0.5 * v2)
    assert torch.allclose(Es, E, atol=tol, rtol=tol)
    u = (ux, uy)
    V = (vx, vy)

    def P2(F):
        return {(a, b): _lsum(lat, F, V[a] * V[b]) for a in (0, 1) for b in (0, 1)}

    def heat(Fg, Ff, P2F):  # int v_a g + v_a v^2/2 f - u_b int v_a v_b f
        return [(_lsum(lat, Fg, V[a]) + _lsum(lat, Ff, V[a] * 0.5 * v2)
                 - (u[0] * P2F[(a, 0)] + u[1] * P2F[(a, 1)])) for a in (0, 1)]

    P2s, P2f, P2e = P2(fs), P2(f), P2(feq)
    if Pr < 1:
        for k in P2s:
            assert torch.allclose(P2s[k], P2e[k], atol=tol, rtol=tol)
        lhs, rhs = heat(gs, fs, P2s), heat(g, f, P2f)
    else:
        tr = _lsum(lat, f - feq, v2)
        for (a, b) in P2s:
            assert torch.allclose(P2s[(a, b)], P2f[(a, b)] - (a == b) / 2.0 * tr, atol=tol, rtol=tol)
        lhs, rhs = heat(gs, fs, P2s), heat(geq, feq, P2e)
    for a in (0, 1):
        assert torch.allclose(lhs[a], rhs[a], atol=1e-12, rtol=1e-12)
    # Table I entries that stay at equilibrium: M_4(f*), M_0 and M_2 of g*
    for t in O.tuples(4):
        assert torch.allclose(O.lattice_moment(lat, fs, t), O.lattice_moment(lat, feq, t), atol=1e-12)
    for t in [()] + O.tuples(2):
        assert torch.allclose(O.lattice_moment(lat, gs, t), O.lattice_moment(lat, geq, t), atol=1e-12)
    if Pr > 1:
        assert torch.allclose(gs, geq, atol=1e-15)
    else:  # M_1(g*) = M_1(g)
        for t in O.tuples(1):
            assert torch.allclose(O.lattice_moment(lat, gs, t), O.lattice_moment(lat, g, t), atol=1e-13)


def test_quasi_equilibrium_is_not_equilibrium_off_pr1(lat):
    """Negative control for the test above: away from Pr = 1 and off
    equilibrium, f* differs from f^eq; at Pr = 1 they coincide."""
    f, g = rand_state(lat, O.Params(), noise=5e-2)
    for Pr, differs in [(0.71, True), (2.0, True), (1.0, False)]:
        P = O.Params(Pr=Pr)
        rho, ux, uy, T, _ = O.macroscopic(lat, P, f, g)
        feq, geq = O.equilibria(lat, P, rho, ux, uy, T)
        fs, gs = O.quasi_equilibria(lat, P, f, g, rho, ux, uy, T, feq, geq)
        assert (float((fs - feq).abs().max()) > 1e-6) == differs


def test_fstar_of_equilibrium_is_equilibrium(lat):
    """Eq. fstar(feq)=feq: the QE of an equilibrium state is that state."""
    for Pr in (0.5, 2.0):
        P = O.Params(Pr=Pr)
        feq, geq = rand_state(lat, P, noise=0.0)
        rho, ux, uy, T, _ = O.macroscopic(lat, P, feq, geq)
        fe2, ge2 = O.equilibria(lat, P, rho, ux, uy, T)
        fs, gs = O.quasi_equilibria(lat, P, feq, geq, rho, ux, uy, T, fe2, ge2)
        assert torch.allclose(fs, feq, atol=1e-13) and torch.allclose(gs, geq, atol=1e-13)


@pytest.mark.parametrize("Pr", [0.5, 1.0, 2.0])
def test_collision_conserves_mass_momentum_energy(lat, Pr):
    """The two-rate relaxation (Eq. Qstar) conserves rho, rho u and E (II)
    to roundoff (cf. the conservation claim of Sec. III.B)."""
    P = O.Params(Pr=Pr, mu=1e-3)
    f, g = rand_state(lat, P, noise=5e-2, seed=7)
    rho, ux, uy, T, _ = O.macroscopic(lat, P, f, g)
    t1, t2 = O.relaxation_times(P, rho, T)
    feq, geq = O.equilibria(lat, P, rho, ux, uy, T)
    fs, gs = O.quasi_equilibria(lat, P, f, g, rho, ux, uy, T, feq, geq)
    Cf = -(f - fs) / t1 - (fs - feq) / t2
    Cg = -(g - gs) / t1 - (gs - geq) / t2
    scale = float((f.abs() / t1).sum(0).max())
    v2 = lat.vx ** 2 + lat.vy ** 2
    for q in (Cf.sum(0), _lsum(lat, Cf, lat.vx), _lsum(lat, Cf, lat.vy), Cg.sum(0) + _lsum(lat, Cf, 0.5 * v2)):
        assert float(q.abs().max()) < 1e-14 * scale


def test_relaxation_time_mapping():
    """Pr <= 1: tau1 = mu/p, tau2 = tau1/Pr; Pr >= 1: tau2 = mu/p,
    tau1 = tau2/Pr (Sec. II.C); tau1 <= tau2 always (Eq. slowfast)."""
    rho = torch.tensor([2.0], dtype=DT); T = torch.tensor([1.5], dtype=DT)
    p = 2.0 * 1.5
    for Pr in (0.5, 1.0, 2.0):
        t1, t2 = O.relaxation_times(O.Params(Pr=Pr, mu=0.3), rho, T)
        nu_tau = float(t1 if Pr <= 1 else t2)
        assert abs(nu_tau - 0.3 / p) < 1e-15
        assert abs(float(t1 / t2) - (Pr if Pr <= 1 else 1 / Pr)) < 1e-15
        assert float(t1) <= float(t2)


# ------------------------------------------------------------------ limiter ---

def test_limiter_reduces_to_textbook_minmod_and_mc():
    """phi with beta = 1 is minmod(r) = max(0, min(1, r)); with beta = 2 it is
    the monotonized-central limiter max(0, min(2r, (1+r)/2, 2))."""
    r = torch.linspace(-3, 5, 801, dtype=DT)
    b = torch.ones_like(r)
    assert torch.allclose(O.limiter_phi(r, b, 1.0), torch.clamp(torch.minimum(r, torch.ones_like(r)), min=0))
    mc = torch.clamp(torch.minimum(torch.minimum(2 * r, 0.5 * (1 + r)), torch.full_like(r, 2.0)), min=0)
    assert torch.allclose(O.limiter_phi(r, b, 2.0), mc)


def test_limited_slope_division_free_identity():
    """(b/2) phi(a, b) = 1/2 minmod3(beta a, (a+b)/2, beta b) for b != 0 (the
    division-free form used by the CUDA kernels), and 0 at b = 0."""
    g = torch.Generator().manual_seed(1)
    a = torch.randn(20000, generator=g, dtype=DT)
    b = torch.randn(20000, generator=g, dtype=DT)
    b[:100] = 0.0
    a[100:200] = 0.0
    beta = 1.2
    x, y, z = beta * a, 0.5 * (a + b), beta * b
    same = (torch.sign(x) == torch.sign(z)) & (torch.sign(x) == torch.sign(y)) & (x != 0)
    mm = torch.where(same, torch.sign(y) * torch.minimum(torch.minimum(x.abs(), y.abs()), z.abs()), torch.zeros_like(x))
    assert torch.allclose(O.half_b_phi(a, b, beta), 0.5 * mm, atol=1e-15, rtol=1e-14)


# --------------------------------------------------------- step invariants ---

def _sim(fields, P, bcs=None, cfl=0.2, dt=None):
    """Oracle simulation; unless given, dt is the CFL rule capped at half the
    smallest relaxation time (explicit Euler relaxation needs dt < 2 tau)."""
    t = lambda z: torch.tensor(z, dtype=DT)
    Ny, Nx = fields.rho.shape
    grid = O.Grid(Nx, Ny, fields.Lx, fields.Ly, bcs) if bcs else O.Grid(Nx, Ny, fields.Lx, fields.Ly)
    if dt is None:
        rho, T = t(fields.rho), t(fields.T)
        t1, t2 = O.relaxation_times(P, rho, T)
        dt = min(O.cfl_dt(P, grid, t(fields.ux), t(fields.uy), T, cfl), 0.5 * float(torch.minimum(t1, t2).min()))
    return O.Simulation(grid, P, t(fields.rho), t(fields.ux), t(fields.uy), t(fields.T), cfl=cfl, dt=dt)


def test_uniform_state_is_fixed_point():
    from paper_2510_04197_gb300 import inputs as I
    for Pr in (0.5, 2.0):
        s = _sim(I.uniform(6, 5, rho=1.2, ux=0.3, uy=-0.1, T=0.9), O.Params(Pr=Pr, mu=1e-3))
        f0, g0 = s.f.clone(), s.g.clone()
        s.run(3)
        assert float((s.f - f0).abs().max()) < 1e-15 and float((s.g - g0).abs().max()) < 1e-15


def test_periodic_run_conserves_totals():
    """Flux form telescopes and the collision conserves: domain totals of
    mass, momentum and energy stay at roundoff level."""
    from paper_2510_04197_gb300 import inputs as I
    s = _sim(I.random_smooth(12, 10, seed=2, amp=0.1, Ma=0.4), O.Params(Pr=0.71, mu=2e-3))
    t0 = O.totals(s.lat, s.P, s.grid, s.f, s.g)
    s.run(30)
    t1 = O.totals(s.lat, s.P, s.grid, s.f, s.g)
    for a, b in zip(t0, t1):
        assert abs(a - b) < 2e-15 * 30 * max(1.0, abs(a))


def test_x_independent_field_reduces_to_1d():
    """A field that depends on y only stays x-independent and matches the run
    on a narrower grid (the x-fluxes cancel exactly)."""
    from paper_2510_04197_gb300 import inputs as I
    F = I.random_smooth(8, 10, seed=4)
    for a in ("rho", "ux", "uy", "T"):
        getattr(F, a)[:] = getattr(F, a)[:, :1]
    s = _sim(F, O.Params(mu=2e-3))
    s.run(5)
    assert float((s.f - s.f[:, :, :1]).abs().max()) == 0.0


def test_pr_one_is_continuous_limit():
    """At Pr -> 1 both QE branches reduce to BGK because tau1 -> tau2 (Sec. II.B
    'in the limit Pr = 1 ... QEDFs equivalent to EDFs')."""
    from paper_2510_04197_gb300 import inputs as I
    F = I.random_smooth(8, 8, seed=5, amp=0.1, Ma=0.3)
    res = {}
    for Pr in (1.0 - 1e-7, 1.0, 1.0 + 1e-7):
        s = _sim(F, O.Params(Pr=Pr, mu=2e-3), dt=1e-4)
        s.run(2)
        res[Pr] = s.f
    assert float((res[1.0 - 1e-7] - res[1.0]).abs().max()) < 1e-9
    assert float((res[1.0 + 1e-7] - res[1.0]).abs().max()) < 1e-9
    # and the two branches are really different away from 1
    s1 = _sim(F, O.Params(Pr=0.9, mu=2e-3), dt=1e-4).run(2)
    s2 = _sim(F, O.Params(Pr=1.0 / 0.9, mu=2e-3 / 0.9), dt=1e-4).run(2)
    assert float((s1.f - s2.f).abs().max()) > 1e-9


def test_step_patch_matches_full_step():
    """The single-cell patch update equals the full-grid update at that cell."""
    from paper_2510_04197_gb300 import inputs as I
    s = _sim(I.random_smooth(9, 7, seed=6, amp=0.1, Ma=0.4), O.Params(Pr=2.0, mu=2e-3))
    s.run(1)
    f0, g0 = s.f, s.g
    f1, g1 = O.step(s.lat, s.P, s.grid, f0, g0, s.dt)
    Ny, Nx = f0.shape[1:]
    cells = [(0, 0), (3, 4), (6, 8), (2, 7)]
    fp, gp = [], []
    for (y, x) in cells:
        ys = [(y + d) % Ny for d in range(-2, 3)]
        xs = [(x + d) % Nx for d in range(-2, 3)]
        fp.append(f0[:, ys][:, :, xs]); gp.append(g0[:, ys][:, :, xs])
    fn, gn = O.step_patch(s.lat, s.P, s.grid, torch.stack(fp, 1), torch.stack(gp, 1), s.dt)
    for k, (y, x) in enumerate(cells):
        assert torch.allclose(fn[:, k], f1[:, y, x], atol=1e-15, rtol=1e-14)
        assert torch.allclose(gn[:, k], g1[:, y, x], atol=1e-15, rtol=1e-14)


def test_similarity_under_gas_constant_and_reference_temperature():
    """Dimensional analysis: with velocities scaled by c = sqrt(R T_ref),
    temperatures by T_ref, mu by c and dt by 1/c, the lattice (App. G,
    v_i = c xi_i) and every relaxation rate scale consistently, so the density
    field is the same function of the dimensionless inputs, and u / c, T / T_ref
    too; a wrong power of c or T_ref anywhere breaks it."""
    from helpers import oracle_run
    from paper_2510_04197_gb300 import inputs as I
    F0 = I.random_smooth(20, 12, seed=7, amp=0.1, Ma=0.5)
    out = {}
    for R, T_ref in ((1.0, 1.0), (287.0, 300.0)):
        c = math.sqrt(R * T_ref)
        F = I.Fields(F0.rho, F0.ux * c, F0.uy * c, F0.T * T_ref, F0.Lx, F0.Ly)
        _, o = oracle_run(F, 0.71, 1.4, 2e-3 * c, 2e-4 / c, 30, R=R, T_ref=T_ref)
        out[(R, T_ref)] = (o["rho"], o["ux"] / c, o["T"] / T_ref)
    for a, b in zip(out[(1.0, 1.0)], out[(287.0, 300.0)]):
        assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()
