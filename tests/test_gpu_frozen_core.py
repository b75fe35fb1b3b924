"""Frozen core (the paper freezes the O 1s orbitals of its water clusters, Sec. 3): the lowest nfc
occupied orbitals stay doubly occupied and uncorrelated.  By definition the correlated problem is
then the one on the active orbitals, with the active blocks of f, B and mu, and the core adds the
constant 2 sum_c mu_cc to the dipole.  The oracle is run on exactly that active problem."""
import numpy as np
import pytest

from oracle import rk
from tests.gpu_common import system

pytestmark = pytest.mark.gpu


def _active(f, B, mu, nfc):
    return f[nfc:, nfc:].copy(), B[:, nfc:, nfc:].copy(), mu[:, nfc:, nfc:].copy()


@pytest.mark.parametrize("nfc", [1, 2])
def test_frozen_core_ground_state_and_trajectory(nfc):
    from paper_2205_05175_gb300 import rtcc
    o, v = 5, 19
    f, B, mu = system(o, v)
    fa, Ba, mua = _active(f, B, mu, nfc)
    core = 2.0 * np.array([mu[x, :nfc, :nfc].trace() for x in range(3)])
    s = rk.RTCC(fa, Ba, mua, o - nfc)
    y0, ec, _ = s.ground_state(tol=1e-11)
    mu0 = s.dipole(y0).real + core
    fld = rk.Field(E0=0.05, omega=0.5, sigma=0.5, t0=1.0, pol=(0.0, 0.0, 1.0))
    integ = rk.Integrator(method="rk4", h=0.05, nsteps=6)
    _, mus_ref, _, _ = rk.propagate(s, y0, fld, integ)
    with rtcc.Handle(f, B, mu, o, v, ntraj=1, prec=rtcc.P64, nfc=nfc) as h:
        assert h.o == o - nfc
        e, m0 = h.ground_state(tol=1e-11)
        yg = h.get_state(0)[0]
        _, mus, n = h.propagate([rtcc.make_field(E0=0.05, omega=0.5, sigma=0.5, t0=1.0, pol=(0.0, 0.0, 1.0))],
                                rtcc.make_integrator(rtcc.RK4, h=0.05, nsteps=6), 7)
    assert abs(e - ec.real) < 1e-10
    assert np.abs(yg - y0).max() < 1e-9
    assert np.abs(m0 - mu0).max() < 1e-10
    assert n[0] == 7
    assert np.abs(mus[0, :7] - (np.asarray(mus_ref) + core)).max() < 1e-9


@pytest.mark.last
def test_frozen_core_with_the_papers_isotropic_pulse():
    """The paper's setup in one run: frozen core (Sec. 3) and the pulse of Eq. field as printed,
    E(t) = -E0 exp(-(t - nu)^2 / (2 sigma^2)) cos(omega (t - nu)) n, along the isotropic
    direction n = (1, 1, 1)/sqrt(3) of Eq. iso-field, so every dipole component responds."""
    from paper_2205_05175_gb300 import rtcc
    o, v, nfc = 5, 19, 1
    f, B, mu = system(o, v)
    fa, Ba, mua = _active(f, B, mu, nfc)
    core = 2.0 * np.array([mu[x, :nfc, :nfc].trace() for x in range(3)])
    n = tuple(np.ones(3) / np.sqrt(3.0))
    s = rk.RTCC(fa, Ba, mua, o - nfc)
    y0, _, _ = s.ground_state(tol=1e-11)
    fld = rk.Field(E0=0.05, omega=0.5, sigma=0.5, t0=1.0, pol=n, carrier="cos", sign=-1.0)
    _, mus_ref, _, _ = rk.propagate(s, y0, fld, rk.Integrator(method="rk4", h=0.05, nsteps=8))
    with rtcc.Handle(f, B, mu, o, v, ntraj=1, prec=rtcc.P64, nfc=nfc) as h:
        h.set_state(0, y0)
        _, mus, k = h.propagate([rtcc.make_field(E0=0.05, omega=0.5, sigma=0.5, t0=1.0, pol=n,
                                                 carrier=rtcc.CARRIER_COS, sign=-1.0)],
                                rtcc.make_integrator(rtcc.RK4, h=0.05, nsteps=8), 9)
    ref = np.asarray(mus_ref) + core
    assert k[0] == 9
    assert np.abs(mus[0, :9] - ref).max() < 1e-9
    assert np.all(np.abs(ref[-1].real - ref[0].real) > 1e-6)     # all three components respond


def test_frozen_core_zero_is_the_plain_handle():
    from paper_2205_05175_gb300 import rtcc
    o, v = 3, 7
    f, B, mu = system(o, v)
    with rtcc.Handle(f, B, mu, o, v, prec=rtcc.P64) as a, rtcc.Handle(f, B, mu, o, v, prec=rtcc.P64, nfc=0) as b:
        ea, ma = a.ground_state(tol=1e-11)
        eb, mb = b.ground_state(tol=1e-11)
    # same computation (split-K partial sums are added atomically, so not bit-identical)
    assert abs(ea - eb) < 1e-13 and np.abs(ma - mb).max() < 1e-13


@pytest.mark.parametrize("nfc", [-1, 3])
def test_frozen_core_count_out_of_range(nfc):
    from paper_2205_05175_gb300 import rtcc
    o, v = 3, 7
    f, B, mu = system(o, v)
    with pytest.raises(rtcc.RtccError) as ei:
        rtcc.Handle(f, B, mu, o, v, prec=rtcc.P64, nfc=nfc)
    assert ei.value.status == "INVALID_ARG"
