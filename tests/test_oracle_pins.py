"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: the references are brute-force
determinant-space evaluation of the defining matrix elements, exact FCI for
two electrons, exact rational order conditions, printed values from the paper,
closed forms and textbook routines.
"""
import json
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import brute, closed, fci, rk, spectrum, spinorb
from paper_2205_05175_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _system(o, v, seed=7, offdiag=0.1):
    f, B, mu = synth.make_system(o, v, seed=seed)
    f = f + synth.random_symmetric(synth.rng_for(seed + 1), o + v, offdiag)  # f_ov != 0 as under a field
    return f, B, mu


# --- residual equations ------------------------------------------------------------

def test_brute_force_reduces_to_slater_condon_rules_at_zero_amplitudes():
    """With T = Lambda = 0 the determinant-space definitions reduce to textbook matrix elements
    between determinants (Slater-Condon rules), independent of the bit-string machinery:
    <Phi_i^a|H|Phi_0> = f_ia, <Phi_ij^ab|H|Phi_0> = <ab||ij>, R_mu = <Phi_0|H|Phi_mu>, the
    reference energy sum_i f_ii - 1/2 sum_ij <ij||ij>, and the reference density."""
    o, v = 2, 3
    f, B, _ = _system(o, v)
    fso, w = spinorb.spin_orbital_operators(f, spinorb.eri_chemist(B))
    N, nv = 2 * o, 2 * v
    bc = brute.BruteCC(fso, w, N)
    z1, z2 = np.zeros((N, nv), complex), np.zeros((N, N, nv, nv), complex)
    o1, o2, e = bc.omega(z1, z2)
    occ, vir = np.arange(N), N + np.arange(nv)
    assert np.abs(o1 - fso[np.ix_(occ, vir)]).max() < 1e-13
    assert np.abs(o2 - w[np.ix_(vir, vir, occ, occ)].transpose(2, 3, 0, 1)).max() < 1e-13
    assert abs(e) < 1e-13
    eref = np.trace(fso[:N, :N]) - 0.5 * np.einsum("ijij->", w[:N, :N, :N, :N])
    assert abs(bc.Eref - eref) < 1e-12
    r1, r2 = bc.lambda_residual(z1, z2, z1, z2)
    assert np.abs(r1 - fso[np.ix_(occ, vir)]).max() < 1e-13
    assert np.abs(r2 - w[np.ix_(occ, occ, vir, vir)]).max() < 1e-13
    rho = bc.density(z1, z2, z1, z2)
    assert np.abs(rho - np.diag([1.0] * N + [0.0] * nv)).max() < 1e-14
    assert np.abs(o2).max() > 1e-3 and np.abs(o1).max() > 1e-3     # non-trivial values


@pytest.mark.parametrize("o,v", [(1, 3), (2, 2), (2, 3)])
def test_spin_orbital_residual_matches_brute_force(o, v):
    """Eq. derivT: Omega_mu = <mu|e^-T H e^T|0> for general complex spin-orbital amplitudes."""
    f, B, _ = _system(o, v)
    fso, w = spinorb.spin_orbital_operators(f, spinorb.eri_chemist(B))
    t1, t2 = synth.random_general_so_amplitudes(2 * o, 2 * v, seed=11, s1=0.1, s2=0.1)
    bc = brute.BruteCC(fso, w, 2 * o)
    b1, b2, be = bc.omega(t1, t2)
    s1, s2, se = spinorb.omega(fso, w, 2 * o, t1, t2)
    assert np.abs(b1 - s1).max() < 1e-13
    assert np.abs(b2 - s2).max() < 1e-13
    assert abs(be - se) < 1e-13
    assert np.abs(b2).max() > 0.1  # non-trivial values


@pytest.mark.parametrize("o,v", [(1, 3), (2, 3), (3, 4)])
def test_closed_shell_residual_matches_spin_orbital(o, v):
    """The closed-shell residual is the (a a) / (a b a b) spin block of the spin-orbital one,
    and the spin-orbital residual of embedded amplitudes is the embedding of it."""
    f, B, _ = _system(o, v)
    fso, w = spinorb.spin_orbital_operators(f, spinorb.eri_chemist(B))
    t1, t2 = synth.random_amplitudes(o, v, seed=11, s1=0.1, s2=0.1)
    c1, c2, ce = closed.omega(t1, t2, f, closed.Integrals(B, o))
    s1, s2, se = spinorb.omega(fso, w, 2 * o, *spinorb.embed_amplitudes(t1, t2))
    e1, e2 = spinorb.embed_amplitudes(c1, c2)
    assert np.abs(e1 - s1).max() < 1e-13
    assert np.abs(e2 - s2).max() < 1e-13
    assert abs(ce - se) < 1e-13


@pytest.mark.parametrize("o,v", [(1, 3), (2, 2)])
def test_lambda_residual_matches_brute_force(o, v):
    """Eq. derivL: <0|(1+Lambda)[Hbar, tau_mu]|0> by explicit matrices equals the
    closed-shell R mapped through the multiplier embedding (so the closed-shell
    Lambda dynamics is the restriction of the spin-orbital one)."""
    f, B, _ = _system(o, v)
    fso, w = spinorb.spin_orbital_operators(f, spinorb.eri_chemist(B))
    t1, t2 = synth.random_amplitudes(o, v, seed=11, s1=0.1, s2=0.1)
    l1, l2 = synth.random_amplitudes(o, v, seed=12, s1=0.1, s2=0.1)
    bc = brute.BruteCC(fso, w, 2 * o)
    R1s, R2s = bc.lambda_residual(*spinorb.embed_amplitudes(t1, t2), *spinorb.embed_multipliers(l1, l2))
    R1, R2 = closed.lambda_residual(t1, t2, l1, l2, f, closed.Integrals(B, o))
    Q1, Q2 = spinorb.embed_multipliers(R1, R2)
    assert np.abs(R1s - Q1).max() < 1e-13
    assert np.abs(R2s - Q2).max() < 1e-13
    assert np.abs(R2s).max() > 0.1


@pytest.mark.parametrize("o,v", [(1, 3), (2, 2)])
def test_dipole_matches_brute_force_density(o, v):
    """Eq. dipole: mu_x = <0|(1+Lambda)e^-T mu_x e^T|0> = Tr(rho mu_x)."""
    f, B, mu = _system(o, v)
    fso, w = spinorb.spin_orbital_operators(f, spinorb.eri_chemist(B))
    t1, t2 = synth.random_amplitudes(o, v, seed=11, s1=0.1, s2=0.1)
    l1, l2 = synth.random_amplitudes(o, v, seed=12, s1=0.1, s2=0.1)
    bc = brute.BruteCC(fso, w, 2 * o)
    ts, ls = spinorb.embed_amplitudes(t1, t2), spinorb.embed_multipliers(l1, l2)
    rho = bc.density(*ts, *ls)
    d_b = np.array([np.sum(rho * spinorb.spin_orbital_one_body(mu[x])) for x in range(3)])
    d_c = closed.dipole(t1, t2, l1, l2, mu, o)
    assert np.abs(d_b - d_c).max() < 1e-13


def test_lambda_is_exact_gradient_five_point():
    """R(t,l).u equals dL/ds along a pair-symmetric direction u; the five-point
    stencil is exact for the (at most quartic) Lagrangian."""
    o, v = 3, 5
    f, B, _ = _system(o, v)
    V = closed.Integrals(B, o)
    t1, t2 = synth.random_amplitudes(o, v, seed=21, s1=0.1, s2=0.1)
    l1, l2 = synth.random_amplitudes(o, v, seed=22, s1=0.1, s2=0.1)
    u1, u2 = synth.random_amplitudes(o, v, seed=23, s1=1.0, s2=1.0)
    R1, R2 = closed.lambda_residual(t1, t2, l1, l2, f, V)
    L = lambda s: closed.lagrangian(t1 + s * u1, t2 + s * u2, l1, l2, f, V)
    h = 0.3
    d = (L(-2 * h) - 8 * L(-h) + 8 * L(h) - L(2 * h)) / (12 * h)
    assert abs(d - (np.sum(R1 * u1) + np.sum(R2 * u2))) < 1e-12 * max(1.0, abs(d))


# --- two-electron exactness, Jacobian, stationarity ---------------------------------

@pytest.fixture(scope="module")
def two_electron():
    o, v = 1, 4
    f, B, mu = synth.make_system(o, v, seed=5)
    s = rk.RTCC(f, B, mu, o)
    y0, ec, _ = s.ground_state()
    F = fci.FCI(f, B, mu, o)
    e0, psi0, w, _ = F.ground()
    return s, y0, ec, F, e0, psi0, w


def test_two_electron_ground_state_is_fci(two_electron):
    s, y0, ec, F, e0, psi0, _ = two_electron
    assert abs(ec - (e0 - F.bc.Eref)) < 1e-11
    assert np.abs(s.dipole(y0) - F.dipole(psi0)).max() < 1e-11


def test_two_electron_dipole_follows_fci_with_h4_error(two_electron):
    """CCSD is exact for two electrons: RT-CC mu(t) -> FCI mu(t), error ~ h^4 (RK4), Im mu -> 0."""
    s, y0, _, F, _, psi0, _ = two_electron
    fld = rk.Field(E0=0.05, omega=0.5, sigma=0.5, t0=1.0)
    T = 2.0
    _, mf = F.propagate(psi0, fld, T, 1e-4, 1000)
    errs = []
    for h in (0.1, 0.05):
        _, mm, _, _ = rk.propagate(s, y0, fld, rk.Integrator(method="rk4", h=h, nsteps=int(round(T / h))))
        errs.append(np.abs(mm[-1] - mf[-1]).max())
        assert np.abs(mm[-1].imag).max() < 1e-8
    assert errs[1] < 1e-6
    assert 10.0 < errs[0] / errs[1] < 25.0


def test_jacobian_eigenvalues_are_fci_singlet_excitations(two_electron):
    s, y0, _, F, e0, _, w = two_electron
    t1, t2, _, _ = rk.unpack(y0, s.o, s.v)
    J = fci.jacobian(t1, t2, s.f, s.V)
    ev = np.sort(np.linalg.eigvals(J).real)
    exc = np.sort(w - e0)
    for e in ev:
        assert np.min(np.abs(exc - e)) < 1e-9


def test_zero_field_stationarity_monomer_shape():
    """At zero field the converged ground state is a fixed point: y(t) = y0, mu(t) = mu0."""
    o, v = 5, 19
    f, B, mu = synth.make_system(o, v, seed=synth.SEED_BASE + 0)
    s = rk.RTCC(f, B, mu, o)
    y0, _, _ = s.ground_state(tol=1e-12)
    fld = rk.Field(E0=0.0)
    _, mm, y, _ = rk.propagate(s, y0, fld, rk.Integrator(method="rk4", h=0.05, nsteps=6))
    assert np.abs(y - y0).max() < 1e-10
    assert np.abs(mm - mm[0]).max() < 1e-10


# --- integrators -------------------------------------------------------------------

def _fr(s):
    return Fr(s)


def test_cash_karp_printed_coefficients_need_two_sign_fixes():
    g = json.load(open(os.path.join(GOLDEN, "cash_karp_printed.json")))
    a = [[_fr(x) for x in row] for row in g["a_printed"]]
    sums = [sum(row, Fr(0)) for row in a]
    # printed rows 4 and 6 do not sum to any consistent node; the corrected ones do
    assert sums[3] == Fr(12, 5) and sums[5] != Fr(7, 8)
    tab = rk.CK_TABLE
    for i, row in enumerate(tab["a"]):
        assert sum(row, Fr(0)) == tab["c"][i]
    assert [_fr(x) for x in g["b_37_378"]] == tab["b5"]
    assert [_fr(x) for x in g["b_2825_27648"]] == tab["b4"]


def _order_conditions(tab, bkey):
    """Highest order p such that the quadrature conditions sum b_i c_i^k = 1/(k+1), k < p hold,
    together with the order-3/4 tree conditions."""
    b, c, a = tab[bkey], tab["c"], tab["a"]
    s = len(b)
    A = [[(a[i][j] if j < len(a[i]) else Fr(0)) for j in range(s)] for i in range(s)]
    conds = {1: [sum(b, Fr(0)) - 1],
             2: [sum(b[i] * c[i] for i in range(s)) - Fr(1, 2)],
             3: [sum(b[i] * c[i] ** 2 for i in range(s)) - Fr(1, 3),
                 sum(b[i] * A[i][j] * c[j] for i in range(s) for j in range(s)) - Fr(1, 6)],
             4: [sum(b[i] * c[i] ** 3 for i in range(s)) - Fr(1, 4),
                 sum(b[i] * c[i] * A[i][j] * c[j] for i in range(s) for j in range(s)) - Fr(1, 8),
                 sum(b[i] * A[i][j] * c[j] ** 2 for i in range(s) for j in range(s)) - Fr(1, 12),
                 sum(b[i] * A[i][j] * A[j][k] * c[k] for i in range(s) for j in range(s) for k in range(s)) - Fr(1, 24)],
             5: [sum(b[i] * c[i] ** 4 for i in range(s)) - Fr(1, 5)]}
    p = 0
    for k in range(1, 6):
        if all(x == 0 for x in conds[k]):
            p = k
        else:
            break
    return p


def test_butcher_orders():
    assert _order_conditions(rk.RK4_TABLE, "b") == 4
    assert _order_conditions(rk.CK_TABLE, "b5") == 5   # 37/378: fifth order (paper calls it fourth)
    assert _order_conditions(rk.CK_TABLE, "b4") == 4


def test_rk4_global_error_scales_as_h4_on_linear_ode():
    lam = -0.3 + 1.7j
    class Lin(rk.RTCC):
        def __init__(self):
            pass
        def rhs(self, tt, y, fld):
            return lam * y
    s = Lin()
    errs = []
    for h in (0.1, 0.05):
        y = np.array([1.0 + 0j])
        for n in range(int(round(2.0 / h))):
            y = s.rk4_step(n * h, y, h, None)
        errs.append(abs(y[0] - np.exp(lam * 2.0)))
    assert 14.0 < errs[0] / errs[1] < 17.0


def test_mixed_step_sequence_on_linear_ode_is_the_product_of_rk4_factors():
    """Sec. 4.2 mixed-step RK4 as read here: h1 while t < t_switch with the crossing step cut to
    land on t_switch, then h2, the last step cut to land on t_end.  On y' = lam y every RK4 step of
    size h multiplies y by R(lam h), R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24, so the samples are the
    running products of R over that exact step sequence."""
    lam = -0.4 + 2.1j

    class Lin(rk.RTCC):
        def __init__(self):
            pass

        def rhs(self, tt, y, fld):
            return lam * y

        def dipole(self, y):
            return y.copy()

    integ = rk.Integrator(method="mixed", h1=0.1, h2=0.25, t_switch=0.33, t_end=1.5)
    tt, mm, _, st = rk.propagate(Lin(), np.array([1.0 + 0j]), None, integ)
    steps = [0.1, 0.1, 0.1, 0.03, 0.25, 0.25, 0.25, 0.25, 0.17]
    assert np.allclose(np.diff(tt), steps, rtol=0, atol=1e-12) and st["accepted"] == len(steps)
    R = lambda z: 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
    want = np.cumprod([1.0 + 0j] + [R(lam * h) for h in np.diff(tt)])
    assert np.abs(mm[:, 0] - want).max() < 1e-14


def test_ck_local_error_orders_on_linear_ode():
    lam = -0.3 + 1.7j
    class Lin(rk.RTCC):
        def __init__(self):
            pass
        def rhs(self, tt, y, fld):
            return lam * y
    s = Lin()
    e5, e4 = [], []
    tab = rk.as_float(rk.CK_TABLE)
    for h in (0.2, 0.1):
        ks = s.stages(tab, 0.0, np.array([1.0 + 0j]), h, None)
        y5 = 1 + h * sum(b * k for b, k in zip(tab["b5"], ks))
        y4 = 1 + h * sum(b * k for b, k in zip(tab["b4"], ks))
        ex = np.exp(lam * h)
        e5.append(abs(y5[0] - ex))
        e4.append(abs(y4[0] - ex))
        # the attempt propagates the fifth-order solution and estimates with |y5 - y4|, which is
        # the fourth-order solution's own error up to the much smaller fifth-order one
        ya, delta = s.ck_attempt(0.0, np.array([1.0 + 0j]), h, None)
        assert abs(ya[0] - ex) == pytest.approx(e5[-1], rel=1e-6)
        assert abs(delta / e4[-1] - 1) < 2 * e5[-1] / e4[-1] + 1e-12
    assert 50 < e5[0] / e5[1] < 80     # h^6 local error
    assert 25 < e4[0] / e4[1] < 40     # h^5 local error


def _embedded_attempt(tab, y, h, lam):
    """One Cash-Karp attempt on y' = lam y: (fifth-order solution, |y5 - y4|)."""
    ks = []
    for i in range(len(tab["c"])):
        ks.append(lam * (y + h * sum(tab["a"][i][j] * ks[j] for j in range(i))))
    y5 = y + h * sum(b * k for b, k in zip(tab["b5"], ks))
    y4 = y + h * sum(b * k for b, k in zip(tab["b4"], ks))
    return y5, abs(y5 - y4)


def test_ck_controller_drives_the_error_estimate_to_its_target():
    """Eq. ck-h-final on an undamped oscillator y' = i y, where the estimate grows as h^5 and |y|
    stays 1: from a tiny first step h grows by the 5x clamp, then settles where the estimate is
    safety^5 tol (an exponent other than 1/5 settles at safety^(1/p) tol instead, a wrong safety
    elsewhere); a step far too long is rejected and the 1/4-exponent retry lands at
    safety^5 tol (tol/Delta)^(1/4) and is accepted."""
    tab = rk.as_float(rk.CK_TABLE)
    tol, safety = 1e-10, 0.84
    y, h, hs, ratios = 1.0 + 0j, 1e-4, [], []
    for _ in range(30):
        y5, d = _embedded_attempt(tab, y, h, 1j)
        acc, hn = rk.ck_controller(h, d, tol, safety)
        assert acc
        hs.append(h)
        ratios.append(d / tol)
        y, h = y5, hn
    grow = [b / a for a, b in zip(hs, hs[1:])]
    assert grow[0] == pytest.approx(5.0, rel=1e-14) and grow[1] == pytest.approx(5.0, rel=1e-14)
    assert max(abs(r / safety ** 5 - 1) for r in ratios[12:]) < 1e-4
    h_eq = hs[-1]
    _, d = _embedded_attempt(tab, 1.0 + 0j, 2.0 * h_eq, 1j)
    acc, hn = rk.ck_controller(2.0 * h_eq, d, tol, safety)
    assert not acc and 0.2 * 2.0 * h_eq < hn < 2.0 * h_eq
    _, d2 = _embedded_attempt(tab, 1.0 + 0j, hn, 1j)
    assert rk.ck_controller(hn, d2, tol, safety)[0]
    assert d2 / tol == pytest.approx(safety ** 5 * (tol / d) ** 0.25, rel=0.05)
    # the clamps of the reading: [0.2 h, 5 h] and [h_min, h_max]
    assert rk.ck_controller(0.01, 1.0, tol)[1] == pytest.approx(0.002)
    assert rk.ck_controller(0.5, 0.0, tol, h_max=1.0)[1] == 1.0


def test_field_matches_printed_values():
    g = json.load(open(os.path.join(GOLDEN, "field_envelope.json")))
    fld = rk.Field(E0=g["E0"], omega=0.0, sigma=g["sigma"], t0=g["t0"], carrier="cos", sign=-1.0)
    for p in g["points"]:
        val = abs(fld.amplitude(p["t"]))
        if p.get("order_of_magnitude"):
            assert 1e-11 < val < 1e-9
        else:
            assert abs(val - p["abs_E"]) / p["abs_E"] < p["rel_tol"]
    assert fld.amplitude(g["t0"]) == -g["E0"]


# --- spectrum post-processing ------------------------------------------------------

def test_spline_reproduces_cubic_with_natural_ends_and_line():
    x = np.sort(np.random.default_rng(0).uniform(0, 3, 12))
    x[0], x[-1] = 0.0, 3.0
    xn = np.linspace(0, 3, 50)
    lin = 0.3 - 1.2 * x
    assert np.abs(spectrum.natural_cubic_spline(x, lin, xn) - (0.3 - 1.2 * xn)).max() < 1e-12
    yv = np.sin(x)
    assert np.abs(spectrum.natural_cubic_spline(x, yv, x) - yv).max() < 1e-14


def test_spline_reproduces_a_natural_spline_in_the_truncated_power_basis():
    """Sec. 4.2 interpolation: a C2 piecewise cubic with knots at the samples and zero second
    derivative at both ends is the unique natural cubic spline through its own values, so the
    interpolant must reproduce it between the knots.  Built independently of the tridiagonal
    solve: s(x) = a + b x + sum_j c_j (x - x_j)_+^3 over the interior knots, with
    sum_j c_j (x_end - x_j) = 0 so that s''(x_end) = 0 (s'' vanishes left of the first knot)."""
    rng = np.random.default_rng(3)
    x = np.sort(rng.uniform(0.0, 5.0, 15))
    x[0], x[-1] = 0.0, 5.0
    c = rng.standard_normal(13)
    c[-1] = -np.sum(c[:-1] * (x[-1] - x[1:-2])) / (x[-1] - x[-2])

    def s_true(z):
        z = np.asarray(z, float)
        return 0.4 - 0.7 * z + np.sum(c[:, None] * np.maximum(z[None, :] - x[1:-1, None], 0.0) ** 3, axis=0)

    xn = np.linspace(0.0, 5.0, 997)
    got = spectrum.natural_cubic_spline(x, s_true(x), xn)
    assert np.abs(got - s_true(xn)).max() < 1e-10 * max(1.0, np.abs(s_true(xn)).max())
    # the same data with one interior value moved is not reproduced (the test can fail)
    y = s_true(x)
    y[7] += 1e-3
    assert np.abs(spectrum.natural_cubic_spline(x, y, xn) - s_true(xn)).max() > 1e-4


def test_delta_pulse_spectrum_peaks_at_oscillation_frequencies():
    dt = 0.05
    t = dt * np.arange(4000)
    w1, w2 = 0.7, 1.3
    mu = np.zeros((len(t), 3))
    mu[:, 2] = 0.4 * np.sin(w1 * t) + 0.2 * np.sin(w2 * t)
    om = np.linspace(0.2, 2.0, 3601)
    I = spectrum.spectrum(t, mu, om, (0, 0, 1), kappa=1.0, gamma=0.01)
    peaks = [om[k] for k in range(1, len(om) - 1) if I[k] > I[k - 1] and I[k] > I[k + 1] and I[k] > 0.2 * I.max()]
    assert len(peaks) == 2
    assert abs(peaks[0] - w1) < 2e-3 and abs(peaks[1] - w2) < 2e-3


def test_matrix_pencil_recovers_frequencies():
    dt = 0.1
    k = np.arange(400)
    y = 0.3 * np.exp(-1j * 0.81 * k * dt) + 0.1 * np.exp(-1j * 1.37 * k * dt) + 0.05 * np.exp(1j * 0.81 * k * dt)
    w = np.sort(spectrum.matrix_pencil(y, dt, 3).real)
    assert np.allclose(w, [-0.81, 0.81, 1.37], atol=1e-9)


def _fci_kick_dipole(o, v, kappa, dt, T):
    """Exact mu_z(t) after a delta kick E(t) = kappa delta(t) z: psi(0+) = exp(i kappa M_z) psi_0,
    then free evolution in the eigenbasis of the field-free Hamiltonian (two electrons, FCI)."""
    f, B, mu = synth.make_system(o, v)
    F = fci.FCI(f, B, mu, o)
    e0, psi0, w, U = F.ground()
    lam, Q = np.linalg.eigh(F.M[2])
    c = U.conj().T @ (Q @ (np.exp(1j * kappa * lam) * (Q.conj().T @ psi0)))
    Mp = U.conj().T @ F.M[2] @ U
    t = dt * np.arange(int(round(T / dt)) + 1)
    A = np.exp(-1j * np.outer(t, w)) * c[None, :]
    mus = np.zeros((len(t), 3))
    mus[:, 2] = np.real(np.einsum("ti,ij,tj->t", A.conj(), Mp, A))
    k0 = int(np.argmin(np.abs(w - e0)))
    strength = np.abs(Mp[k0, :]) ** 2
    strength[k0] = 0.0
    return t, mus, w - e0, strength


def test_kick_spectrum_line_strength_and_noise_floor():
    """Sec. 2.2 (polarisability from the induced dipole) and the noise study of Sec. 4.1
    (Fig. sp-noise).  After a weak delta kick of area kappa the induced dipole is, to first order,
    2 kappa sum_k |<0|mu_z|k>|^2 sin(w_k t), so the damped transform gives a line at each
    excitation energy w_k of height |<0|mu_z|k>|^2 (1 - exp(-gamma T)) / gamma.  Uniform noise of
    amplitude eps on the samples after t = 0 adds Im[dt sum_n eta_n exp((i w - gamma) t_n)] / kappa,
    whose root-mean-square over w is dt eps sqrt(sum_n exp(-2 gamma t_n) / 6) / kappa.  A dropped dt,
    a missing factor of the damping or a kappa in the wrong place fails one of these."""
    kappa = 0.01 * 0.01 * np.sqrt(2 * np.pi)    # area of the Sec. 4.1 noise-study pulse (E0 = 0.01, sigma = 0.01)
    dt, T, gamma = 0.05, 300.0, 0.01
    t, mus, exc, strength = _fci_kick_dipole(1, 4, kappa, dt, T)
    om = np.linspace(0.5, 3.0, 2501)
    I0 = spectrum.spectrum(t, mus, om, (0, 0, 1), kappa=kappa, gamma=gamma)
    k = int(np.argmax(strength))
    j = int(np.argmax(I0))
    assert abs(om[j] - exc[k]) < 1e-3
    assert abs(I0[j] / (strength[k] * (1 - np.exp(-gamma * T)) / gamma) - 1) < 2e-3
    rng = np.random.Generator(np.random.PCG64(2205_05175))
    floor = dt * np.sqrt(np.sum(np.exp(-2 * gamma * t[1:])) / 6) / kappa
    for eps in (1e-6, 1e-5, 1e-4):
        noisy = mus.copy()
        noisy[1:, 2] += rng.uniform(-eps, eps, len(t) - 1)
        dI = spectrum.spectrum(t, noisy, om, (0, 0, 1), kappa=kappa, gamma=gamma) - I0
        assert 0.75 < np.sqrt(np.mean(dI ** 2)) / (eps * floor) < 1.25
        assert abs(om[int(np.argmax(I0 + dI))] - exc[k]) < 1e-3


# --- real-time spectrum peaks = EOM-CCSD excitation energies (Sec. 3: EOM-CCSD stick spectra) ----

def _rt_modes(o, v, h, T):
    """Strongest response frequencies of Re mu_z(t) after a weak kick, by matrix pencil, and the
    eigenvalues of the CC Jacobian dOmega/dt (EOM-CCSD excitation energies) carried through the
    RK4 map: a mode exp(-i w t) advances by R(-i w h) per step, R the RK4 stability polynomial."""
    f, B, mu = synth.make_system(o, v, seed=7)
    s = rk.RTCC(f, B, mu, o)
    y0, _, _ = s.ground_state(tol=1e-12)
    t1, t2, _, _ = rk.unpack(y0, o, v)
    ev = np.linalg.eigvals(fci.jacobian(t1, t2, s.f, s.V)).real
    z = -1j * ev * h
    w_rk = 1j * np.log(1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24) / h
    kick = rk.Field(E0=1e-4, omega=0.0, sigma=0.02, t0=0.1, carrier="cos")
    tt, mm, _, _ = rk.propagate(s, y0, kick, rk.Integrator(method="rk4", h=h, nsteps=int(round(T / h))))
    tt, mm = np.asarray(tt), np.asarray(mm)
    y = mm[tt > 0.4, 2].real - mm[0, 2].real
    N, L = len(y), len(y) // 2
    sv = np.linalg.svd(np.array([y[i:i + L + 1] for i in range(N - L)]), compute_uv=False)
    w = spectrum.matrix_pencil(y, h, int(np.sum(sv > 1e-6 * sv[0])))
    c, *_ = np.linalg.lstsq(np.exp(-1j * np.outer(h * np.arange(N), w)), y.astype(complex), rcond=None)
    strongest = [w[k] for k in np.argsort(-np.abs(c)) if w[k].real > 0]
    return strongest, w_rk


def test_rt_peaks_are_eom_ccsd_energies_two_electrons():
    """Linear response of RT-CCSD oscillates at the Jacobian eigenvalues (for two electrons
    these are the FCI excitation energies, pinned above)."""
    strongest, w_rk = _rt_modes(1, 3, 0.05, 20.0)
    for w in strongest[:4]:
        assert np.min(np.abs(w_rk - w)) < 1e-6, w


def test_rt_peaks_are_eom_ccsd_energies_four_electrons():
    """Four electrons, where CCSD is not FCI: the strongest RT modes sit at EOM-CCSD energies."""
    strongest, w_rk = _rt_modes(2, 3, 0.05, 40.0)
    for w in strongest[:3]:
        assert np.min(np.abs(w_rk - w)) < 2e-5, w


# --- adjoint reference: forward-mode tangent of the RK4 propagation -------------------------

def test_tangent_gradient_matches_central_differences():
    """The oracle's forward tangent (exact five-point JVPs, analytic dA/dtheta) against central
    differences (delta 1e-5) of its own RK4 propagation; J itself must coincide."""
    from oracle import tangent
    o, v = 2, 5
    f, B, mu = synth.make_system(o, v)
    h, nsteps = 0.05, 20
    t = h * np.arange(nsteps + 1)
    w = np.zeros((nsteps + 1, 3))
    w[:, 0] = np.exp(-0.5 * (t - 0.6) ** 2 / 0.3 ** 2)
    theta = np.array([0.08, 0.7, 0.4])
    s = rk.RTCC(f, B, mu, o)
    y0, _, _ = s.ground_state(tol=1e-12)

    def J(th):
        fld = rk.Field(E0=th[0], omega=th[1], sigma=th[2], t0=1.0)
        _, m, _, _ = rk.propagate(s, y0, fld, rk.Integrator(method="rk4", h=h, nsteps=nsteps))
        return float(np.sum(w * m.real))

    fd = np.array([(J(theta + d) - J(theta - d)) / 2e-5 for d in 1e-5 * np.eye(3)])
    Jt, g = tangent.tangent_gradient(s, y0, rk.Field(E0=theta[0], omega=theta[1], sigma=theta[2], t0=1.0), h, nsteps, w)
    assert abs(Jt - J(theta)) < 1e-12 * abs(Jt)
    assert np.abs(g - fd).max() < 1e-7 * np.abs(fd).max()


# --- Pade-accelerated transforms (the short-time spectral technique the paper cites, Sec. 1) ---

def _damped_modes(k, dt, modes):
    return sum(A * np.exp(-g * k * dt) * np.sin(w * k * dt) for A, w, g in modes)


def test_pade_transform_is_the_infinite_time_sum_of_damped_modes():
    """For a signal that is a sum of damped exponentials the diagonal Pade approximant of its
    power series is the closed-form infinite sum; the truncated sum over the same 41 samples is not."""
    dt, modes = 0.1, [(0.3, 0.81, 0.02), (0.1, 1.37, 0.05)]
    om = np.linspace(0.2, 2.0, 400)
    z = np.exp(1j * om * dt)
    exact = 0.0
    for A, w, g in modes:
        p, q = np.exp((1j * w - g) * dt), np.exp((-1j * w - g) * dt)
        exact = exact + A / 2j * (1.0 / (1.0 - p * z) - 1.0 / (1.0 - q * z))
    c = _damped_modes(np.arange(41), dt, modes)
    err = np.abs(spectrum.pade_transform(c, z) - exact).max() / np.abs(exact).max()
    assert err < 1e-9
    truncated = np.exp(1j * np.outer(om, dt * np.arange(41))) @ c
    assert np.abs(truncated - exact).max() / np.abs(exact).max() > 0.1


def test_pade_spectrum_resolves_peaks_from_a_short_record():
    """A 12 au record of two modes 0.15 Eh apart (below the 2 pi / 12 = 0.52 Eh Fourier
    resolution): the Pade spectrum puts its two peaks on the mode frequencies."""
    dt = 0.05
    t = dt * np.arange(241)
    mu = np.zeros((len(t), 3))
    mu[:, 2] = 0.4 * np.sin(1.00 * t) + 0.3 * np.sin(1.15 * t)
    om = np.linspace(0.6, 1.6, 2001)
    I = spectrum.pade_spectrum(t, mu, om, (0, 0, 1), kappa=1.0, gamma=0.01)
    peaks = [om[k] for k in range(1, len(om) - 1) if I[k] > I[k - 1] and I[k] > I[k + 1] and I[k] > 0.2 * I.max()]
    assert len(peaks) == 2
    assert abs(peaks[0] - 1.00) < 2e-3 and abs(peaks[1] - 1.15) < 2e-3
    Id = spectrum.spectrum(t, mu, om, (0, 0, 1), kappa=1.0, gamma=0.01)
    pd = [om[k] for k in range(1, len(om) - 1) if Id[k] > Id[k - 1] and Id[k] > Id[k + 1] and Id[k] > 0.2 * Id.max()]
    assert len(pd) < 2   # the plain transform of the same record does not separate them


# --- implicit Gauss-Legendre RK (the paper's integrator library names implicit/symplectic RK) ---

def test_gauss_legendre_tableau_is_the_exact_order_four_collocation():
    sp = pytest.importorskip("sympy")
    r = sp.sqrt(3) / 6
    c = [sp.Rational(1, 2) - r, sp.Rational(1, 2) + r]
    A = [[sp.Rational(1, 4), sp.Rational(1, 4) - r], [sp.Rational(1, 4) + r, sp.Rational(1, 4)]]
    b = [sp.Rational(1, 2), sp.Rational(1, 2)]
    tab = rk.GL2_TABLE
    for i in range(2):
        assert abs(tab["c"][i] - float(c[i])) < 1e-16 and abs(tab["b"][i] - float(b[i])) < 1e-16
        for j in range(2):
            assert abs(tab["a"][i][j] - float(A[i][j])) < 1e-16
    # collocation: sum_j a_ij c_j^(k-1) = c_i^k / k (k = 1, 2); Gauss nodes: sum_i b_i c_i^(k-1) = 1/k, k <= 4
    for i in range(2):
        for k in (1, 2):
            assert sp.simplify(sum(A[i][j] * c[j] ** (k - 1) for j in range(2)) - c[i] ** k / k) == 0
    rng = range(2)
    conds = [sum(b) - 1, sum(b[i] * c[i] for i in rng) - sp.Rational(1, 2),
             sum(b[i] * c[i] ** 2 for i in rng) - sp.Rational(1, 3),
             sum(b[i] * A[i][j] * c[j] for i in rng for j in rng) - sp.Rational(1, 6),
             sum(b[i] * c[i] ** 3 for i in rng) - sp.Rational(1, 4),
             sum(b[i] * c[i] * A[i][j] * c[j] for i in rng for j in rng) - sp.Rational(1, 8),
             sum(b[i] * A[i][j] * c[j] ** 2 for i in rng for j in rng) - sp.Rational(1, 12),
             sum(b[i] * A[i][j] * A[j][k] * c[k] for i in rng for j in rng for k in rng) - sp.Rational(1, 24)]
    assert all(sp.simplify(x) == 0 for x in conds)
    assert sp.simplify(sum(b[i] * c[i] ** 4 for i in rng) - sp.Rational(1, 5)) != 0   # not fifth order


def test_gauss_legendre_is_unitary_for_hermitian_dynamics_and_fourth_order():
    """For y' = -i H y with H Hermitian the Gauss-Legendre stability function (the diagonal Pade
    approximant of exp) has modulus one on the imaginary axis: the norm is kept exactly, which
    RK4 does not; the global error falls as h^4."""
    rng = np.random.default_rng(3)
    X = rng.standard_normal((6, 6)) + 1j * rng.standard_normal((6, 6))
    H = (X + X.conj().T) / 2

    class Lin(rk.RTCC):
        def __init__(self):
            pass

        def rhs(self, tt, y, fld):
            return -1j * (H @ y)

    s = Lin()
    y0 = rng.standard_normal(6) + 1j * rng.standard_normal(6)
    w, U = np.linalg.eigh(H)
    exact = U @ (np.exp(-1j * w * 2.0) * (U.conj().T @ y0))
    errs = []
    for h in (0.05, 0.025):
        y, z = y0.copy(), y0.copy()
        for n in range(int(round(2.0 / h))):
            y = s.gl2_step(n * h, y, h, None)
            z = s.rk4_step(n * h, z, h, None)
        assert abs(np.linalg.norm(y) - np.linalg.norm(y0)) < 1e-12 * np.linalg.norm(y0)
        assert abs(np.linalg.norm(z) - np.linalg.norm(y0)) > 1e-9 * np.linalg.norm(y0)
        errs.append(np.abs(y - exact).max())
    assert 14.0 < errs[0] / errs[1] < 18.0


def test_gauss_legendre_rtcc_follows_fci_with_h4_error(two_electron):
    """The implicit integrator on the RT-CC equations of motion: mu(t) -> FCI mu(t) (CCSD is
    exact for two electrons) with the order-4 error ratio, like RK4."""
    s, y0, _, F, _, psi0, _ = two_electron
    fld = rk.Field(E0=0.05, omega=0.5, sigma=0.5, t0=1.0)
    T = 2.0
    _, mf = F.propagate(psi0, fld, T, 1e-4, 1000)
    errs = []
    for h in (0.1, 0.05):
        _, mm, _, _ = rk.propagate(s, y0, fld, rk.Integrator(method="gl2", h=h, nsteps=int(round(T / h))))
        errs.append(np.abs(mm[-1] - mf[-1]).max())
    assert errs[1] < 1e-6
    assert 10.0 < errs[0] / errs[1] < 25.0


# --- the per-term flop counter (roofline's algorithmic work) ---------------------------

def _numpy_naive_flops(subs, shapes):
    """numpy's own real-flop count of an einsum, from einsum_path's report."""
    import re
    rep = np.einsum_path(subs, *[np.empty(s) for s in shapes], optimize=False)[1]
    return float(re.search(r"Naive FLOP count:\s*([0-9.eE+-]+)", rep).group(1))


def test_flop_counter_agrees_with_numpy_einsum_path_term_by_term():
    """Every counted term: the counter's real flops equal numpy's naive flop count of the same
    einsum (2 per product over a summed label, 1 for an outer product) times the real products
    per complex product (1, 2 or 4), so a wrong extent, a missed label or a wrong complex factor
    fails here."""
    from oracle import flops
    recs = flops.records(2, 3)
    rows = flops.term_table(2, 3)
    assert len(recs) == len(rows) > 50
    for r, row in zip(recs, rows):
        mine = row[2] * 2.0 ** row[3] * 3.0 ** row[4]
        assert mine == r["cfac"] * _numpy_naive_flops(r["subs"], r["shapes"]), r["subs"]
    # both residuals are counted: the reverse sweep has every forward contraction's adjoints
    assert {r["phase"] for r in recs} == {"omega", "lambda"}


def test_flop_counter_ladder_and_shape_independence():
    """The particle-particle ladder is the only o^2 v^4 class: a complex-by-real contraction of
    o^2 v^4 products in Omega and its adjoint in R, 2 x 4 o^2 v^4 flops in all.  The term table
    taken at (2, 3) reproduces a direct count at (3, 5), so the program and the o/v assignment of
    every label do not depend on the shape."""
    from oracle import flops
    o, v = 30, 114
    r = flops.rhs_flops(o, v)
    assert r["o2v4"] == 8.0 * o ** 2 * v ** 4
    direct = sum(x["cfac"] * _numpy_naive_flops(x["subs"], x["shapes"]) for x in flops.records(3, 5))
    assert flops.rhs_flops(3, 5)["total"] == direct


def test_stored_flop_table_is_the_counters():
    """tests/golden/rhs_flops.json (read by the benchmark) is what the counter gives now."""
    import json
    import os

    from oracle import flops
    doc = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "rhs_flops.json")))
    assert [tuple(r) for r in doc["rows"]] == [tuple(r) for r in flops.term_table()]


def test_gauss_legendre_newton_is_the_pade_stability_function_beyond_the_fixed_point_limit():
    """y' = -i H y, H Hermitian, at h ||H|| = 4: the Gauss-Legendre step is R(-i h H) y with R the
    (2, 2) Pade approximant of exp, R(z) = (1 + z/2 + z^2/12) / (1 - z/2 + z^2/12) (a closed form),
    which keeps the norm.  Newton's method reaches it; the fixed-point iteration diverges there."""
    rng = np.random.default_rng(8)
    X = rng.standard_normal((6, 6)) + 1j * rng.standard_normal((6, 6))
    H = (X + X.conj().T) / 2
    H = H * (4.0 / np.abs(np.linalg.eigvalsh(H)).max())

    class Lin(rk.RTCC):
        def __init__(self):
            pass

        def rhs(self, tt, y, fld):
            return -1j * (H @ y)

    s = Lin()
    y0 = rng.standard_normal(6) + 1j * rng.standard_normal(6)
    h = 1.0
    w, U = np.linalg.eigh(H)
    z = -1j * h * w
    R = (1 + z / 2 + z * z / 12) / (1 - z / 2 + z * z / 12)
    exact = U @ (R * (U.conj().T @ y0))
    y1 = s.gl2_step_newton(0.0, y0, h, None)
    assert np.abs(y1 - exact).max() < 1e-12 * np.abs(y0).max()
    assert abs(np.linalg.norm(y1) - np.linalg.norm(y0)) < 1e-12 * np.linalg.norm(y0)
    with pytest.raises(RuntimeError):
        s.gl2_step(0.0, y0, h, None, maxiter=60)


def test_gauss_legendre_newton_equals_fixed_point_and_solves_collocation_rtcc():
    """On the RT-CC equations (o = 1, v = 3, strong field): where the fixed-point iteration
    converges, Newton's method gives the same step; at a step 4x longer it still satisfies the
    collocation equations K_i = f(t + c_i h, y + h sum_j a_ij K_j) to rounding."""
    o, v = 1, 3
    f, B, mu = synth.make_system(o, v, seed=9)
    s = rk.RTCC(f, B, mu, o)
    y0, _, _ = s.ground_state(tol=1e-12)
    fld = rk.Field(E0=2.0, omega=0.5, sigma=0.5, t0=1.0)
    ya = s.gl2_step(0.9, y0, 0.05, fld)
    yb = s.gl2_step_newton(0.9, y0, 0.05, fld)
    assert np.abs(ya - yb).max() < 1e-12
    # the longer step: the returned stages satisfy the stage equations and give the step
    c, a = rk.GL2_TABLE["c"], rk.GL2_TABLE["a"]
    h = 0.2
    y1, K = s.gl2_step_newton(0.9, y0, h, fld, return_stages=True)
    assert np.all(np.isfinite(y1)) and np.abs(y1 - y0).max() > 1e-4
    assert np.abs(y0 + h * (K[0] + K[1]) / 2 - y1).max() < 1e-13
    resid = [K[i] - s.rhs(0.9 + c[i] * h, y0 + h * (a[i][0] * K[0] + a[i][1] * K[1]), fld) for i in range(2)]
    assert max(np.abs(r).max() for r in resid) < 1e-12


def test_stored_gauss_legendre_newton_record_starts_from_the_oracle_ground_state():
    """The stored dense-Newton record (tests/golden/gl2n_o2v6_h04.json) starts from the oracle's
    ground state of the seeded system, samples every h, and its first dipole is that state's."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "gl2n_o2v6_h04.json")) as fh:
        doc = json.load(fh)
    o, v = doc["o"], doc["v"]
    f, B, mu = synth.make_system(o, v, seed=doc["seed"])
    s = rk.RTCC(f, B, mu, o)
    y0, _, _ = s.ground_state(tol=1e-12)
    ys = np.array([complex(a, b) for a, b in doc["y0"]])
    assert np.abs(ys - y0).max() < 1e-10
    assert np.allclose(doc["t"], doc["h"] * np.arange(doc["nsteps"] + 1), atol=1e-14)
    m0 = s.dipole(ys)
    assert np.abs(np.array(doc["mu"][0][0::2]) + 1j * np.array(doc["mu"][0][1::2]) - m0).max() < 1e-13
    assert np.isfinite(doc["mu"]).all()
