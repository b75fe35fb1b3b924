"""Trajectory parity (RK4, Cash-Karp, mixed-step RK4, Gauss-Legendre by sweeps and by Newton) of the CUDA path against the oracle, the
zero-field fixed point, two-electron exactness against FCI, and batched-trajectory independence."""
import numpy as np
import pytest

from oracle import fci, rk
from paper_2205_05175_gb300 import synth
from tests.gpu_common import system

pytestmark = pytest.mark.gpu


def _gpu_traj(o, v, f, B, mu, fields, integ, max_out, prec=0, y0=None, tol=1e-11):
    from paper_2205_05175_gb300 import rtcc
    with rtcc.Handle(f, B, mu, o, v, ntraj=len(fields), prec=prec) as h:
        if y0 is None:
            h.ground_state(tol=tol)
        else:
            for z in range(len(fields)):
                h.set_state(z, y0, 0.0, 0.0)
        t, m, n = h.propagate(fields, integ, max_out)
        stats = h.last_stats()
    return t, m, n, stats


def test_rk4_monomer_shape_matches_oracle():
    """Config: o=5, v=19, z-polarised sine pulse E0=0.01, omega=0.5, sigma=0.5, t0=1, RK4 h=0.05, 40 steps."""
    from paper_2205_05175_gb300 import rtcc
    o, v = 5, 19
    f, B, mu = system(o, v)
    s = rk.RTCC(f, B, mu, o)
    y0, _, _ = s.ground_state(tol=1e-11)
    fld = rk.Field(E0=0.01, omega=0.5, sigma=0.5, t0=1.0)
    tt, mm, _, _ = rk.propagate(s, y0, fld, rk.Integrator(method="rk4", h=0.05, nsteps=40))
    t, m, n, _ = _gpu_traj(o, v, f, B, mu, [rtcc.make_field()], rtcc.make_integrator(rtcc.RK4, h=0.05, nsteps=40),
                           64, prec=0, y0=y0)
    assert n[0] == 41
    assert np.abs(t[0, :41] - tt).max() < 1e-12
    assert np.abs(m[0, :41] - mm).max() < 1e-10


# 1e-5 au: the dipole noise level below which the spectrum is unchanged (Sec. 4.1, Fig. sp-noise).
# The split-precision modes meet it; a single TF32 pass (10-bit operands) lands near 1.3e-5 au
# over these 40 steps, so it is held to 5e-5 au and reported as not meeting the target.
@pytest.mark.parametrize("prec,tol", [(1, 5e-5), (2, 1e-5), (3, 1e-5)])
def test_rk4_reduced_precision_dipole_error(prec, tol):
    from paper_2205_05175_gb300 import rtcc
    o, v = 5, 19
    f, B, mu = system(o, v)
    s = rk.RTCC(f, B, mu, o)
    y0, _, _ = s.ground_state(tol=1e-11)
    fld = rk.Field(E0=0.01, omega=0.5, sigma=0.5, t0=1.0)
    _, mm, _, _ = rk.propagate(s, y0, fld, rk.Integrator(method="rk4", h=0.05, nsteps=40))
    _, m, n, _ = _gpu_traj(o, v, f, B, mu, [rtcc.make_field()], rtcc.make_integrator(rtcc.RK4, h=0.05, nsteps=40),
                           64, prec=prec, y0=y0)
    assert np.abs(m[0, :41] - mm).max() < tol


def test_cash_karp_matches_oracle():
    from paper_2205_05175_gb300 import rtcc
    o, v = 2, 6
    f, B, mu = system(o, v)
    s = rk.RTCC(f, B, mu, o)
    y0, _, _ = s.ground_state(tol=1e-11)
    fld = rk.Field(E0=0.5, omega=0.5, sigma=0.3, t0=1.0)
    integ = rk.Integrator(method="ck", h=0.01, tol=1e-6, t_end=2.5)
    tt, mm, _, st = rk.propagate(s, y0, fld, integ)
    t, m, n, stats = _gpu_traj(o, v, f, B, mu, [rtcc.make_field(E0=0.5, sigma=0.3)],
                               rtcc.make_integrator(rtcc.CK, h=0.01, tol=1e-6, t_end=2.5), 4096, prec=0, y0=y0)
    assert n[0] == len(tt)
    assert stats[0] == st["accepted"] and stats[1] == st["rejected"]
    # Delta is the difference of two nearly equal solutions: its relative rounding error
    # (~1e-16 |R| h / Delta ~ 1e-9) moves h_new, hence the sample times, at the 1e-11 level
    assert np.abs(t[0, :n[0]] - tt).max() < 1e-9
    assert np.abs(m[0, :n[0]] - mm).max() < 1e-9


def test_mixed_step_matches_oracle():
    from paper_2205_05175_gb300 import rtcc
    o, v = 2, 6
    f, B, mu = system(o, v)
    s = rk.RTCC(f, B, mu, o)
    y0, _, _ = s.ground_state(tol=1e-11)
    fld = rk.Field(E0=0.5, omega=0.5, sigma=0.3, t0=1.8)
    integ = rk.Integrator(method="mixed", h1=0.005, h2=0.05, t_switch=3.6, t_end=4.0)
    tt, mm, _, _ = rk.propagate(s, y0, fld, integ)
    t, m, n, _ = _gpu_traj(o, v, f, B, mu, [rtcc.make_field(E0=0.5, sigma=0.3, t0=1.8)],
                           rtcc.make_integrator(rtcc.MIXED_RK4, h1=0.005, h2=0.05, t_switch=3.6, t_end=4.0),
                           4096, prec=0, y0=y0)
    assert n[0] == len(tt)
    assert np.abs(t[0, :n[0]] - tt).max() < 1e-12
    assert np.abs(m[0, :n[0]] - mm).max() < 1e-10


@pytest.mark.last
def test_gauss_legendre_matches_oracle():
    """Implicit two-stage Gauss-Legendre: the device's Gauss-Seidel sweeps and the oracle's
    fixed-point iteration converge to the same collocation solution."""
    from paper_2205_05175_gb300 import rtcc
    o, v = 3, 7
    f, B, mu = system(o, v)
    s = rk.RTCC(f, B, mu, o)
    y0, _, _ = s.ground_state(tol=1e-11)
    fld = rk.Field(E0=0.05, omega=0.5, sigma=0.5, t0=0.5)
    tt, mm, _, _ = rk.propagate(s, y0, fld, rk.Integrator(method="gl2", h=0.05, nsteps=20))
    t, m, n, stats = _gpu_traj(o, v, f, B, mu, [rtcc.make_field(E0=0.05, t0=0.5)],
                               rtcc.make_integrator(rtcc.GL2, h=0.05, nsteps=20, sweeps=20), 64, prec=0, y0=y0)
    assert n[0] == 21
    assert stats[2] == 20 * (1 + 2 * 20)
    assert np.abs(t[0, :21] - tt).max() < 1e-12
    assert np.abs(m[0, :21] - mm).max() < 1e-10


@pytest.mark.last
def test_gauss_legendre_newton_beyond_the_fixed_point_limit_matches_oracle():
    """h = 0.4 at o = 1, v = 4, where the Gauss-Seidel sweeps of the stage equations diverge: the
    device's simplified Newton iterations with GMRES reach the collocation solution that the
    oracle's dense Newton solve gives; the sweeps stop with NOCONV; the Krylov size is checked."""
    from paper_2205_05175_gb300 import rtcc
    o, v = 1, 4
    f, B, mu = system(o, v)
    s = rk.RTCC(f, B, mu, o)
    y0, _, _ = s.ground_state(tol=1e-11)
    fld = rk.Field(E0=0.05, omega=0.5, sigma=0.5, t0=0.5)
    nsteps = 4
    tt, mm, _, _ = rk.propagate(s, y0, fld, rk.Integrator(method="gl2n", h=0.4, nsteps=nsteps))
    field = [rtcc.make_field(E0=0.05, t0=0.5)]
    integ = rtcc.make_integrator(rtcc.GL2_NEWTON, h=0.4, nsteps=nsteps, tol=1e-12)
    t, m, n, stats = _gpu_traj(o, v, f, B, mu, field, integ, 16, prec=0, y0=y0)
    assert n[0] == nsteps + 1
    assert stats[2] == nsteps * (1 + 6 * (2 + 2 * 12))
    assert np.abs(t[0, :n[0]] - tt).max() < 1e-12
    assert np.abs(m[0, :n[0]] - mm).max() < 1e-10
    # the split-precision right-hand side: the same solution to the mode's accuracy
    _, mb, nb, _ = _gpu_traj(o, v, f, B, mu, field, rtcc.make_integrator(rtcc.GL2_NEWTON, h=0.4, nsteps=nsteps, tol=1e-6),
                             16, prec=rtcc.P32_BF16X3, y0=y0)
    assert nb[0] == nsteps + 1 and np.abs(mb[0, :nb[0]] - mm).max() < 1e-5
    with rtcc.Handle(f, B, mu, o, v, ntraj=1, prec=0) as h:
        h.set_state(0, y0, 0.0, 0.0)
        with pytest.raises(rtcc.RtccError) as e:
            h.propagate(field, rtcc.make_integrator(rtcc.GL2, h=0.4, nsteps=nsteps, tol=1e-8, sweeps=20), 16)
        assert e.value.status == "NOCONV"
        with pytest.raises(rtcc.RtccError) as e:
            h.propagate(field, rtcc.make_integrator(rtcc.GL2_NEWTON, h=0.4, nsteps=1, krylov=33), 16)
        assert e.value.status == "INVALID_ARG"


def test_gauss_legendre_newton_trajectories_solve_independent_systems():
    """Two trajectories with different fields in one handle: every Krylov inner product, rotation
    and back substitution is per trajectory, so each equals the same trajectory run alone."""
    from paper_2205_05175_gb300 import rtcc
    o, v = 1, 4
    f, B, mu = system(o, v)
    s = rk.RTCC(f, B, mu, o)
    y0, _, _ = s.ground_state(tol=1e-11)
    fields = [rtcc.make_field(E0=0.05, t0=0.5), rtcc.make_field(E0=0.5, omega=0.9, t0=0.3, pol=(1.0, 0.0, 0.0))]
    # the strong field needs more simplified-Newton iterations than the default six (the Jacobian
    # is frozen at the step's start): twelve bring h max|dK_2| to ~1e-16 at this step
    integ = rtcc.make_integrator(rtcc.GL2_NEWTON, h=0.4, nsteps=3, tol=1e-10, sweeps=12)
    _, mb, nb, _ = _gpu_traj(o, v, f, B, mu, fields, integ, 8, prec=0, y0=y0)
    for z in range(2):
        _, m1, n1, _ = _gpu_traj(o, v, f, B, mu, [fields[z]], integ, 8, prec=0, y0=y0)
        assert nb[z] == n1[0] == 4
        assert np.abs(mb[z, :4] - m1[0, :4]).max() < 1e-12
    assert np.abs(mb[0, :4] - mb[1, :4]).max() > 1e-4


@pytest.mark.last
def test_gauss_legendre_newton_at_o2_v6_matches_the_stored_oracle_record():
    """o = 2, v = 6, h = 0.4 (the sweeps diverge there): the device's Newton-Krylov steps against the
    oracle's dense-Newton record written by tests/golden/make_gl2n_reference.py."""
    import json
    import os

    from paper_2205_05175_gb300 import rtcc
    with open(os.path.join(os.path.dirname(__file__), "golden", "gl2n_o2v6_h04.json")) as fh:
        doc = json.load(fh)
    o, v = doc["o"], doc["v"]
    f, B, mu = synth.make_system(o, v, seed=doc["seed"])
    y0 = np.array([complex(a, b) for a, b in doc["y0"]])
    tt = np.array(doc["t"])
    mm = np.array([[complex(r[2 * x], r[2 * x + 1]) for x in range(3)] for r in doc["mu"]])
    fl = doc["field"]
    integ = rtcc.make_integrator(rtcc.GL2_NEWTON, h=doc["h"], nsteps=doc["nsteps"], tol=1e-12, sweeps=10, krylov=20)
    t, m, n, _ = _gpu_traj(o, v, f, B, mu, [rtcc.make_field(E0=fl["E0"], omega=fl["omega"], sigma=fl["sigma"],
                                                             t0=fl["t0"])], integ, 8, prec=0, y0=y0)
    assert n[0] == doc["nsteps"] + 1
    assert np.abs(t[0, :n[0]] - tt).max() < 1e-12
    assert np.abs(m[0, :n[0]] - mm).max() < 1e-10


def test_zero_field_fixed_point_on_device():
    from paper_2205_05175_gb300 import rtcc
    o, v = 5, 19
    f, B, mu = system(o, v)
    t, m, n, _ = _gpu_traj(o, v, f, B, mu, [rtcc.make_field(E0=0.0)], rtcc.make_integrator(rtcc.RK4, h=0.05, nsteps=40),
                           64, prec=0, tol=1e-12)
    assert np.abs(m[0, :n[0]] - m[0, 0]).max() < 1e-10


def test_two_electron_dipole_follows_fci_on_device():
    from paper_2205_05175_gb300 import rtcc
    o, v = 1, 4
    f, B, mu = synth.make_system(o, v, seed=5)
    F = fci.FCI(f, B, mu, o)
    _, psi0, _, _ = F.ground()
    fld = rk.Field(E0=0.05, omega=0.5, sigma=0.5, t0=1.0)
    _, mf = F.propagate(psi0, fld, 2.0, 1e-4, 1000)
    errs = []
    for hh in (0.1, 0.05):
        t, m, n, _ = _gpu_traj(o, v, f, B, mu, [rtcc.make_field(E0=0.05)],
                               rtcc.make_integrator(rtcc.RK4, h=hh, nsteps=int(round(2.0 / hh))), 64, prec=0)
        errs.append(np.abs(m[0, n[0] - 1] - mf[-1]).max())
        assert np.abs(m[0, n[0] - 1].imag).max() < 1e-8
    assert errs[1] < 1e-6 and 10 < errs[0] / errs[1] < 25


def test_batched_trajectories_are_independent():
    """x/y/z polarisations in one batch equal three single-trajectory runs."""
    from paper_2205_05175_gb300 import rtcc
    o, v = 3, 8
    f, B, mu = system(o, v)
    pols = [(1.0, 0, 0), (0, 1.0, 0), (0, 0, 1.0)]
    integ = rtcc.make_integrator(rtcc.RK4, h=0.05, nsteps=20)
    fields = [rtcc.make_field(E0=0.05, pol=p) for p in pols]
    _, mb, nb, _ = _gpu_traj(o, v, f, B, mu, fields, integ, 32, prec=0)
    for z in range(3):
        _, ms, ns, _ = _gpu_traj(o, v, f, B, mu, [fields[z]], integ, 32, prec=0)
        assert nb[z] == ns[0] == 21
        assert np.abs(mb[z, :21] - ms[0, :21]).max() < 1e-12


@pytest.mark.last
def test_cash_karp_checkpoint_resume_across_handles():
    """Checkpoint/resume: the state, time and trial step read from one handle and written into a
    fresh one continue the Cash-Karp run exactly as the first handle continues it (h = 0 keeps
    each trajectory's stored step)."""
    from paper_2205_05175_gb300 import rtcc
    o, v = 2, 6
    f, B, mu = system(o, v)
    fld = [rtcc.make_field(E0=0.5, sigma=0.3, t0=1.0)]
    first = rtcc.make_integrator(rtcc.CK, h=0.01, tol=1e-6, t_end=1.5)
    rest = rtcc.make_integrator(rtcc.CK, h=0.0, tol=1e-6, t_end=3.0)
    with rtcc.Handle(f, B, mu, o, v, ntraj=1, prec=rtcc.P64) as a:
        a.ground_state(tol=1e-11)
        a.propagate(fld, first, 4096)
        y, t, hs = a.get_state(0)
        ta, ma, na = a.propagate(fld, rest, 4096)
    assert abs(t - 1.5) < 1e-12 and hs > 0
    with rtcc.Handle(f, B, mu, o, v, ntraj=1, prec=rtcc.P64) as b:
        with pytest.raises(rtcc.RtccError) as e:          # nothing stored yet: h = 0 is refused
            b.propagate(fld, rest, 4096)
        assert e.value.status == "INVALID_ARG"
        b.set_state(0, y, t, hs)
        tb, mb, nb = b.propagate(fld, rest, 4096)
    assert na[0] == nb[0] > 10
    assert ta[0, 0] == t and abs(ta[0, na[0] - 1] - 3.0) < 1e-12
    assert np.abs(ta[0, :na[0]] - tb[0, :nb[0]]).max() < 1e-9
    assert np.abs(ma[0, :na[0]] - mb[0, :nb[0]]).max() < 1e-9


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (2, 1e-5), (3, 1e-5)])
def test_narrow_strong_pulse_mixed_step_matches_oracle(prec, tol):
    """The narrow strong pulse of Sec. 4.2 (E0 = 100 au, sigma = 1e-6 au, a kick of 2.5e-4 au) through
    mixed-step RK4 with h1 = 1e-7 au while the pulse is on (120 steps to t_switch = 1.2e-5 au, where
    the cut step lands) and h2 = 0.05 au after it, to 1 au: the dipole of every sample against the
    oracle, in float64 and in the split-precision modes (1e-5 au, the noise level below which the
    spectrum is unchanged, Sec. 4.1)."""
    from paper_2205_05175_gb300 import rtcc
    o, v = 2, 6
    f, B, mu = system(o, v)
    s = rk.RTCC(f, B, mu, o)
    y0, _, _ = s.ground_state(tol=1e-11)
    E0, sigma, t0 = 100.0, 1e-6, 6e-6
    fld = rk.Field(E0=E0, omega=0.0, sigma=sigma, t0=t0, carrier="cos")
    integ = rk.Integrator(method="mixed", h1=1e-7, h2=0.05, t_switch=2 * t0, t_end=1.0)
    tt, mm, _, _ = rk.propagate(s, y0, fld, integ)
    t, m, n, _ = _gpu_traj(o, v, f, B, mu,
                           [rtcc.make_field(E0=E0, omega=0.0, sigma=sigma, t0=t0, carrier=rtcc.CARRIER_COS)],
                           rtcc.make_integrator(rtcc.MIXED_RK4, h1=1e-7, h2=0.05, t_switch=2 * t0, t_end=1.0),
                           512, prec=prec, y0=y0)
    assert n[0] == len(tt) and len(tt) > 130
    assert np.abs(t[0, :n[0]] - tt).max() < 1e-12
    # the kick moves the dipole by far more than the tolerance
    assert np.abs(mm.real - mm[0].real).max() > 1e-3
    assert np.abs(m[0, :n[0]] - mm).max() < tol


# float64: equal to rounding; BF16x3: split-K partial sums are added in a run-dependent order, so
# the same trajectory alone and in a batch agree to the contraction's resolution only
@pytest.mark.parametrize("prec,tol_t,tol", [(0, 1e-14, 1e-12), (3, 1e-6, 1e-6)])
def test_cash_karp_compaction_keeps_every_trajectory_exact(prec, tol_t, tol):
    """Per-trajectory Cash-Karp steps (Eqs. ck-h, ck-h-final) in t_end mode: weak-field trajectories
    take longer steps and finish first, are moved behind the running ones, and the remaining
    attempts run over the running trajectories only.  Every trajectory of the batch (given in an
    order that interleaves strong and weak fields) must equal the same trajectory run alone, sample
    by sample, and the handle's slots must hold the trajectories in their own order afterwards."""
    from paper_2205_05175_gb300 import rtcc
    o, v = 3, 8
    f, B, mu = system(o, v)
    e0s = [0.5, 0.001, 0.2, 0.01, 0.5]
    pols = [(0, 0, 1.0), (1.0, 0, 0), (0, 1.0, 0), (0, 0, 1.0), (1.0, 0, 0)]
    fields = [rtcc.make_field(E0=e, sigma=0.3, pol=p) for e, p in zip(e0s, pols)]
    integ = rtcc.make_integrator(rtcc.CK, h=0.01, tol=1e-7, t_end=2.0)
    with rtcc.Handle(f, B, mu, o, v, ntraj=len(fields), prec=prec) as h:
        h.ground_state(tol=1e-11)
        y0 = h.get_state(0)[0]
        tb, mb, nb = h.propagate(fields, integ, 4096)
        ends = [h.get_state(z) for z in range(len(fields))]
    assert len(set(nb.tolist())) >= 3          # trajectories took different numbers of steps
    for z in range(len(fields)):
        with rtcc.Handle(f, B, mu, o, v, ntraj=1, prec=prec) as h1:
            h1.set_state(0, y0, 0.0, 0.0)
            ts, ms, ns = h1.propagate([fields[z]], integ, 4096)
            end1 = h1.get_state(0)
        assert nb[z] == ns[0]
        assert np.abs(tb[z, :nb[z]] - ts[0, :ns[0]]).max() < tol_t
        assert np.abs(mb[z, :nb[z]] - ms[0, :ns[0]]).max() < tol
        assert np.abs(ends[z][0] - end1[0]).max() < tol and abs(ends[z][1] - 2.0) < 1e-12
        assert abs(ends[z][2] - end1[2]) <= tol_t * end1[2]   # the stored trial step came back to its trajectory
