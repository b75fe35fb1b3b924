"""Parity of one right-hand-side evaluation (Eqs. derivT/derivL), the dipole (Eq. dipole) and the
ground state between the CUDA path (through the C-ABI) and the CPU oracle."""
import numpy as np
import pytest

from oracle import closed, rk
from paper_2205_05175_gb300 import synth
from tests.gpu_common import rel_err, state_from, system

pytestmark = pytest.mark.gpu

# max |GPU - oracle| / max |oracle| per precision mode for one RHS evaluation
RHS_TOL = {0: 1e-11, 1: 3e-3, 2: 3e-6, 3: 3e-5}


def _oracle_rhs(f, B, mu, o, y, fld, t):
    s = rk.RTCC(f, B, mu, o)
    return s.rhs(t, y, fld)


@pytest.mark.parametrize("o,v,ntraj", [(2, 5, 1), (3, 7, 2), (5, 19, 1), (3, 30, 2), (5, 30, 1)])
@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_rhs_parity(o, v, ntraj, prec):
    """(3, 30): contractions over o*v*v >= 2048 indices into o x o outputs take the staged
    small-output reduction in the reduced-precision modes; (5, 30): products with K = N = o over
    o*v*v >= 4096 rows take the one-thread-per-row kernel."""
    from paper_2205_05175_gb300 import rtcc
    f, B, mu = system(o, v)
    fields, times, ys, refs = [], [], [], []
    for z in range(ntraj):
        t1, t2 = synth.random_amplitudes(o, v, seed=100 + z, s1=0.05, s2=0.02)
        l1, l2 = synth.random_amplitudes(o, v, seed=200 + z, s1=0.05, s2=0.02)
        y = state_from(t1, t2, l1, l2)
        E0 = 0.3 * (z + 1)
        fld = rk.Field(E0=E0, omega=0.5, sigma=0.5, t0=1.0, pol=(0.3, 0.5, 0.8))
        tt = 0.8 + 0.1 * z
        refs.append(_oracle_rhs(f, B, mu, o, y, fld, tt))
        ys.append(y)
        fields.append(rtcc.make_field(E0=E0, omega=0.5, sigma=0.5, t0=1.0, pol=(0.3, 0.5, 0.8)))
        times.append(tt)
    with rtcc.Handle(f, B, mu, o, v, ntraj=ntraj, prec=prec) as h:
        out = h.rhs(np.stack(ys), fields, np.array(times))
    for z in range(ntraj):
        assert rel_err(out[z], refs[z]) < RHS_TOL[prec], (z, rel_err(out[z], refs[z]))


@pytest.mark.parametrize("o,v", [(2, 5), (5, 19)])
def test_dipole_parity(o, v):
    from paper_2205_05175_gb300 import rtcc
    f, B, mu = system(o, v)
    t1, t2 = synth.random_amplitudes(o, v, seed=31, s1=0.05, s2=0.02)
    l1, l2 = synth.random_amplitudes(o, v, seed=32, s1=0.05, s2=0.02)
    ref = closed.dipole(t1, t2, l1, l2, mu, o)
    with rtcc.Handle(f, B, mu, o, v, ntraj=1, prec=0) as h:
        h.set_state(0, state_from(t1, t2, l1, l2))
        d = h.dipole()[0]
    assert np.abs(d - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())


def test_ground_state_parity_monomer_shape():
    from paper_2205_05175_gb300 import rtcc
    o, v = 5, 19
    f, B, mu = system(o, v)
    s = rk.RTCC(f, B, mu, o)
    y0, ec, _ = s.ground_state(tol=1e-11)
    mu0 = s.dipole(y0)
    with rtcc.Handle(f, B, mu, o, v, ntraj=2, prec=1) as h:
        e, m0 = h.ground_state(tol=1e-11)
        yg, tg, _ = h.get_state(1)
    assert abs(e - ec.real) < 1e-10
    assert np.abs(yg - y0).max() < 1e-9
    assert np.abs(m0 - mu0.real).max() < 1e-10
    assert tg == 0.0
