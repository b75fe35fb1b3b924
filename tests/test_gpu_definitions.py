"""The CUDA path against the definitions of the method, with no closed-shell oracle in between.

The closed-shell oracle (oracle/closed.py) follows the same intermediates as the device program,
so these tests check the device directly against tiers and identities that share nothing with it:

* brute force in the full determinant space (oracle/brute.py): the ket residual
  Omega_mu = <mu|e^-T H(t) e^T|0> (Eq. derivT), the bra residual
  R_mu = <0|(1+Lambda)[Hbar, tau_mu]|0> (Eq. derivL) and the dipole Tr(rho mu_x) (Eq. dipole),
  on random complex amplitudes under a field (so f_ov != 0), mapped between the closed-shell and
  spin-orbital forms by the embedding that the oracle pins against brute force;
* the spin-orbital residual with Stanton-Gauss intermediates (oracle/spinorb.py, pinned to brute
  force) at shapes where the reduced-precision modes run their contractions on the tensor cores;
* two identities evaluated on the device alone: R = dL/dt for L = E + l.Omega (five-point stencil
  in a complex scalar, exact for the quartic Lagrangian, built from the device's own Omega), and
  the dipole as the one-body Lagrangian, mu_x = <0|mu_x bar|0> + l.Omega[f -> mu_x, ERI -> 0].
"""
import numpy as np
import pytest

from oracle import brute, spinorb
from paper_2205_05175_gb300 import synth
from tests.gpu_common import rel_err, state_from, system

pytestmark = pytest.mark.gpu

# max |device - reference| / max |reference| per precision mode (same bounds as the closed-shell tests)
TOL = {0: 1e-12, 1: 3e-3, 2: 3e-6, 3: 3e-5}

E0, OMEGA, SIGMA, T0, POL = 0.4, 0.5, 0.5, 1.0, (0.3, 0.5, 0.8)


def _amp(t, E0=E0):
    """Eq. field: E(t) = E0 exp(-(t-t0)^2 / (2 sigma^2)) sin(omega (t-t0)) (sine carrier, sign +1)."""
    x = t - T0
    return E0 * np.exp(-0.5 * x * x / SIGMA ** 2) * np.sin(OMEGA * x)


def _fock_at(f, mu, t, E0=E0):
    """f(t) = f - E(t) . mu (Sec. 2.2, V = -mu . E)."""
    a = _amp(t, E0)
    return f - a * sum(p * mu[x] for x, p in enumerate(POL))


def _split(dydt, o, v):
    """dy/dt = (-i Omega1, -i Omega2, +i R1, +i R2) -> (Omega1, Omega2, R1, R2)."""
    n1, n2 = o * v, o * o * v * v
    y = np.asarray(dydt)
    om1 = 1j * y[:n1].reshape(o, v)
    om2 = 1j * y[n1:n1 + n2].reshape(o, o, v, v)
    r1 = -1j * y[n1 + n2:2 * n1 + n2].reshape(o, v)
    r2 = -1j * y[2 * n1 + n2:].reshape(o, o, v, v)
    return om1, om2, r1, r2


def _device_rhs(f, B, mu, o, v, prec, ys, times, E0s):
    from paper_2205_05175_gb300 import rtcc
    fields = [rtcc.make_field(E0=e, omega=OMEGA, sigma=SIGMA, t0=T0, pol=POL) for e in E0s]
    with rtcc.Handle(f, B, mu, o, v, ntraj=len(ys), prec=prec) as h:
        out = h.rhs(np.stack(ys), fields, np.array(times, dtype=float))
    return [_split(out[z], o, v) for z in range(len(ys))]


# --- brute force (determinant space) ---------------------------------------------------

@pytest.fixture(scope="module", params=[(2, 2), (2, 3)], ids=["o2v2", "o2v3"])
def brute_case(request):
    """Random complex amplitudes and multipliers of a 4-electron system under a field at t = 0.8,
    with the brute-force Omega, R and dipole of the embedded spin-orbital amplitudes."""
    o, v = request.param
    f, B, mu = system(o, v, seed=91)
    f = f + synth.random_symmetric(synth.rng_for(92), o + v, 0.05)
    t1, t2 = synth.random_amplitudes(o, v, seed=93, s1=0.1, s2=0.08)
    l1, l2 = synth.random_amplitudes(o, v, seed=94, s1=0.1, s2=0.08)
    tt = 0.8
    fso, w = spinorb.spin_orbital_operators(_fock_at(f, mu, tt), spinorb.eri_chemist(B))
    bc = brute.BruteCC(fso, w, 2 * o)
    ts, ls = spinorb.embed_amplitudes(t1, t2), spinorb.embed_multipliers(l1, l2)
    b1, b2, _ = bc.omega(*ts)
    R1s, R2s = bc.lambda_residual(*ts, *ls)
    rho = bc.density(*ts, *ls)
    dip = np.array([np.sum(rho * spinorb.spin_orbital_one_body(mu[x])) for x in range(3)])
    assert np.abs(b2).max() > 1e-2 and np.abs(R2s).max() > 1e-2    # non-trivial values
    return dict(o=o, v=v, f=f, B=B, mu=mu, t=(t1, t2), l=(l1, l2), tt=tt, omega=spinorb.restrict(b1, b2),
                R=(R1s, R2s), dip=dip)


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_residuals_match_brute_force(brute_case, prec):
    """Omega (Eq. derivT) and R (Eq. derivL) of the device against the determinant-space
    definitions; R is compared in the spin-orbital form through the multiplier embedding."""
    c = brute_case
    o, v = c["o"], c["v"]
    y = state_from(*c["t"], *c["l"])
    om1, om2, r1, r2 = _device_rhs(c["f"], c["B"], c["mu"], o, v, prec, [y], [c["tt"]], [E0])[0]
    ref_o1, ref_o2 = c["omega"]
    scale = max(np.abs(ref_o1).max(), np.abs(ref_o2).max())
    assert np.abs(om1 - ref_o1).max() / scale < TOL[prec]
    assert np.abs(om2 - ref_o2).max() / scale < TOL[prec]
    q1, q2 = spinorb.embed_multipliers(r1, r2)
    R1s, R2s = c["R"]
    scale = max(np.abs(R1s).max(), np.abs(R2s).max())
    assert np.abs(q1 - R1s).max() / scale < TOL[prec]
    assert np.abs(q2 - R2s).max() / scale < TOL[prec]


def test_dipole_matches_brute_force_density(brute_case):
    """mu_x = <0|(1+Lambda) e^-T mu_x e^T|0> = Tr(rho mu_x) (Eq. dipole), float64 device path."""
    from paper_2205_05175_gb300 import rtcc
    c = brute_case
    o, v = c["o"], c["v"]
    with rtcc.Handle(c["f"], c["B"], c["mu"], o, v, ntraj=1, prec=rtcc.P64) as h:
        h.set_state(0, state_from(*c["t"], *c["l"]))
        d = h.dipole()[0]
    assert np.abs(d - c["dip"]).max() < 1e-12 * max(1.0, np.abs(c["dip"]).max())


# --- spin-orbital residual at tensor-core shapes --------------------------------------

SHAPES = [(4, 24), (5, 30)]


@pytest.fixture(scope="module", params=SHAPES, ids=[f"o{o}v{v}" for o, v in SHAPES])
def so_case(request):
    """Two trajectories (different field strengths and times) with their spin-orbital residuals."""
    o, v = request.param
    f, B, mu = system(o, v)
    eri = spinorb.eri_chemist(B)
    cases = []
    for z, (e0, tt) in enumerate(((E0, 0.8), (2.5 * E0, 1.7))):
        t1, t2 = synth.random_amplitudes(o, v, seed=300 + z, s1=0.05, s2=0.02)
        l1, l2 = synth.random_amplitudes(o, v, seed=400 + z, s1=0.05, s2=0.02)
        fso, w = spinorb.spin_orbital_operators(_fock_at(f, mu, tt, e0), eri)
        s1, s2, _ = spinorb.omega(fso, w, 2 * o, *spinorb.embed_amplitudes(t1, t2))
        cases.append(dict(y=state_from(t1, t2, l1, l2), tt=tt, e0=e0, omega=spinorb.restrict(s1, s2)))
    return dict(o=o, v=v, f=f, B=B, mu=mu, eri=eri, cases=cases)


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_omega_matches_spin_orbital_residual(so_case, prec):
    """Eq. derivT for two batched trajectories against the spin-orbital residual (pinned to brute
    force); in the reduced modes the ladder and ring products take the tcgen05 GEMM here."""
    c = so_case
    o, v = c["o"], c["v"]
    got = _device_rhs(c["f"], c["B"], c["mu"], o, v, prec, [k["y"] for k in c["cases"]],
                      [k["tt"] for k in c["cases"]], [k["e0"] for k in c["cases"]])
    for z, k in enumerate(c["cases"]):
        ref1, ref2 = k["omega"]
        scale = max(np.abs(ref1).max(), np.abs(ref2).max())
        assert np.abs(got[z][0] - ref1).max() / scale < TOL[prec], (z, "singles")
        assert np.abs(got[z][1] - ref2).max() / scale < TOL[prec], (z, "doubles")


def _closed_energy(f, eri, o, t1, t2):
    """Closed-shell CC energy E = 2 sum f_ia t_ia + sum (2<ij|ab> - <ij|ba>) (t2 + t1 t1)_ijab,
    with <ij|ab> = (ia|jb); checked against the spin-orbital energy (pinned to brute force)."""
    ov = eri[:o, o:, :o, o:]                                   # (ia|jb)
    L = 2.0 * ov.transpose(0, 2, 1, 3) - ov.transpose(0, 2, 3, 1)   # [i,j,a,b]
    tau = t2 + np.einsum("ia,jb->ijab", t1, t1)
    return 2.0 * np.sum(f[:o, o:] * t1) + np.sum(L * tau)


def test_lambda_is_gradient_of_device_lagrangian(so_case):
    """Eq. derivL as R = dL/dt with L = E + l.Omega: the device's R contracted with a pair-symmetric
    direction u equals the five-point derivative in s of L(t + s u), where every Omega comes from
    the device (float64 mode).  The stencil is exact for the quartic Lagrangian."""
    c = so_case
    o, v = c["o"], c["v"]
    k = c["cases"][0]
    n1, n2 = o * v, o * o * v * v
    t1 = k["y"][:n1].reshape(o, v)
    t2 = k["y"][n1:n1 + n2].reshape(o, o, v, v)
    l1 = k["y"][n1 + n2:2 * n1 + n2].reshape(o, v)
    l2 = k["y"][2 * n1 + n2:].reshape(o, o, v, v)
    u1, u2 = synth.random_amplitudes(o, v, seed=501, s1=0.5, s2=0.2)
    ft = _fock_at(c["f"], c["mu"], k["tt"], k["e0"])
    # the test's energy formula against the spin-orbital energy
    fso, w = spinorb.spin_orbital_operators(ft, c["eri"])
    e_so = spinorb.omega(fso, w, 2 * o, *spinorb.embed_amplitudes(t1, t2))[2]
    e_cs = _closed_energy(ft, c["eri"], o, t1, t2)
    assert abs(e_cs - e_so) < 1e-12 * max(1.0, abs(e_so))
    h = 0.2
    shifts = (-2 * h, -h, h, 2 * h)
    ys = [k["y"]] + [state_from(t1 + s * u1, t2 + s * u2, l1, l2) for s in shifts]
    out = _device_rhs(c["f"], c["B"], c["mu"], o, v, 0, ys, [k["tt"]] * 5, [k["e0"]] * 5)
    L = []
    for s, res in zip(shifts, out[1:]):
        L.append(_closed_energy(ft, c["eri"], o, t1 + s * u1, t2 + s * u2) + np.sum(l1 * res[0]) + np.sum(l2 * res[1]))
    d = (L[0] - 8 * L[1] + 8 * L[2] - L[3]) / (12 * h)
    r1, r2 = out[0][2], out[0][3]
    g = np.sum(r1 * u1) + np.sum(r2 * u2)
    assert abs(g - d) < 1e-10 * max(1.0, abs(d)), (g, d)
    assert abs(d) > 1e-3


def test_dipole_is_one_body_lagrangian_on_device(so_case):
    """Eq. dipole: mu_x = 2 sum_i mu_x,ii + 2 sum mu_x,ia t_ia + l . Omega[f -> mu_x, ERI -> 0].
    The one-body residuals come from a second handle with zero integrals whose field makes
    f(t) = mu_x exactly (f = 0, cos carrier at t = t0, E0 = 1, sign -1, polarisation e_x)."""
    from paper_2205_05175_gb300 import rtcc
    c = so_case
    o, v = c["o"], c["v"]
    nmo = o + v
    y = c["cases"][0]["y"]
    n1, n2 = o * v, o * o * v * v
    t1 = y[:n1].reshape(o, v)
    l1 = y[n1 + n2:2 * n1 + n2].reshape(o, v)
    l2 = y[2 * n1 + n2:].reshape(o, o, v, v)
    mu = c["mu"]
    with rtcc.Handle(c["f"], c["B"], mu, o, v, ntraj=1, prec=rtcc.P64) as h:
        h.set_state(0, y)
        d = h.dipole()[0]
    pols = ((1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0))
    fields = [rtcc.make_field(E0=1.0, omega=0.0, sigma=1.0, t0=0.0, pol=p, carrier=rtcc.CARRIER_COS, sign=-1.0)
              for p in pols]
    zeros_B = np.zeros((4, nmo, nmo))
    with rtcc.Handle(np.zeros((nmo, nmo)), zeros_B, mu, o, v, ntraj=3, prec=rtcc.P64) as h0:
        out = h0.rhs(np.stack([y] * 3), fields, np.zeros(3))
    ref = np.zeros(3, complex)
    for x in range(3):
        om1, om2, _, _ = _split(out[x], o, v)
        ref[x] = 2.0 * np.trace(mu[x][:o, :o]) + 2.0 * np.sum(mu[x][:o, o:] * t1) + np.sum(l1 * om1) + np.sum(l2 * om2)
    assert np.abs(d - ref).max() < 1e-11 * max(1.0, np.abs(ref).max()), (d, ref)
