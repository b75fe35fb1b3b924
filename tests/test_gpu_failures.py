"""Failure detection without a GPU fault: faults are made on the host (non-finite states, impossible
controller settings, too few iterations) or by a bounded device wait on a flag nothing sets; the
library reports a status and the context stays usable."""
import numpy as np
import pytest

from paper_2205_05175_gb300 import synth

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives():
    from paper_2205_05175_gb300 import rtcc
    assert rtcc.rtcc_selftest_timeout(0.2) == "TIMEOUT"
    a = np.random.default_rng(0).standard_normal((1, 40, 64))
    c = rtcc.rtcc_selftest_gemm(0, a, a)          # the context is still usable
    assert np.allclose(c, np.einsum("bmk,bnk->bmn", a, a))


def test_nonfinite_state_is_reported_as_diverged():
    from paper_2205_05175_gb300 import rtcc
    o, v = 2, 5
    f, B, mu = synth.make_system(o, v)
    with rtcc.Handle(f, B, mu, o, v, ntraj=2, prec=0) as H:
        H.ground_state(tol=1e-10)
        y, _, _ = H.get_state(1)
        y[3] = np.nan
        H.set_state(1, y, 0.0, 0.0)
        with pytest.raises(rtcc.RtccError) as e:
            H.propagate([rtcc.make_field()] * 2, rtcc.make_integrator(rtcc.RK4, h=0.05, nsteps=5), 8)
        assert e.value.status == "DIVERGED" and "trajectory 1" in rtcc.rtcc_last_error()
        H.ground_state(tol=1e-10)                 # the handle recovers
        _, m, n = H.propagate([rtcc.make_field()] * 2, rtcc.make_integrator(rtcc.RK4, h=0.05, nsteps=2), 4)
        assert (n == 3).all() and np.isfinite(m[:, :3]).all()


def test_step_size_underflow_is_reported():
    from paper_2205_05175_gb300 import rtcc
    o, v = 2, 5
    f, B, mu = synth.make_system(o, v)
    with rtcc.Handle(f, B, mu, o, v, ntraj=1, prec=0) as H:
        H.ground_state(tol=1e-10)
        integ = rtcc.make_integrator(rtcc.CK, h=0.5, tol=1e-14, h_min=0.4, h_max=1.0, max_rejects=2, t_end=3.0)
        with pytest.raises(rtcc.RtccError) as e:
            H.propagate([rtcc.make_field(E0=1.0)], integ, 16)
        assert e.value.status == "STEP_UNDERFLOW"


def test_ground_state_nonconvergence_is_reported():
    from paper_2205_05175_gb300 import rtcc
    o, v = 2, 5
    f, B, mu = synth.make_system(o, v)
    with rtcc.Handle(f, B, mu, o, v, ntraj=1, prec=0) as H:
        with pytest.raises(rtcc.RtccError) as e:
            H.ground_state(tol=1e-12, maxiter=2)
        assert e.value.status == "NOCONV"


@pytest.mark.last
def test_unconverged_implicit_stages_are_reported():
    """Gauss-Legendre stages solved by fixed-point sweeps: at o=2, v=6 the sweeps stop contracting
    between h = 0.3 and 0.4 (the same sweeps run on the oracle leave h |dK_2| near 4 after 20
    sweeps at h = 0.4, finite), so the step is refused with NOCONV instead of being taken."""
    from paper_2205_05175_gb300 import rtcc
    o, v = 2, 6
    f, B, mu = synth.make_system(o, v)
    fld = [rtcc.make_field(E0=0.05, t0=0.5)]
    with rtcc.Handle(f, B, mu, o, v, ntraj=1, prec=0) as H:
        H.ground_state(tol=1e-11)
        with pytest.raises(rtcc.RtccError) as e:
            H.propagate(fld, rtcc.make_integrator(rtcc.GL2, h=0.4, nsteps=1, tol=1e-6, sweeps=20), 4)
        assert e.value.status == "NOCONV" and "implicit stages" in rtcc.rtcc_last_error()
        H.ground_state(tol=1e-11)                 # the handle recovers
        _, m, n = H.propagate(fld, rtcc.make_integrator(rtcc.GL2, h=0.05, nsteps=2, tol=1e-6), 4)
        assert n[0] == 3 and np.isfinite(m[0, :3]).all()
