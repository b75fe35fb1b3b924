"""rtcc_spectrum (spline resampling, damping, DFT, division by the pulse's transform) against the oracle."""
import numpy as np
import pytest

from oracle import rk, spectrum

pytestmark = pytest.mark.gpu


def _signal(t):
    mu = np.zeros((len(t), 3))
    mu[:, 0] = 0.1 * np.sin(0.9 * t) * np.exp(-0.002 * t)
    mu[:, 2] = 0.3 * np.sin(0.7 * t) + 0.05 * np.sin(1.6 * t) + 0.2
    return mu


def test_delta_pulse_uniform_samples():
    from paper_2205_05175_gb300 import rtcc
    t = 0.05 * np.arange(3000)
    mu = _signal(t)
    om = np.linspace(0.1, 2.0, 1200)
    ref = spectrum.spectrum(t, mu, om, (0, 0, 1), kappa=0.5, gamma=0.01)
    got = rtcc.rtcc_spectrum(t, mu, rtcc.make_field(pol=(0, 0, 1)), om, kappa=0.5, gamma=0.01)
    assert np.abs(got - ref).max() < 1e-9 * np.abs(ref).max()


def test_finite_pulse_division():
    from paper_2205_05175_gb300 import rtcc
    t = 0.02 * np.arange(2000)
    mu = _signal(t)
    fld = rk.Field(E0=0.01, omega=0.5, sigma=0.5, t0=1.0, pol=(0.0, 0.6, 0.8))
    om = np.linspace(0.2, 1.5, 500)
    ref = spectrum.spectrum(t, mu, om, fld.pol, field_amp=fld.amplitude, gamma=0.02)
    got = rtcc.rtcc_spectrum(t, mu, rtcc.make_field(E0=0.01, omega=0.5, sigma=0.5, t0=1.0, pol=(0.0, 0.6, 0.8)), om,
                             kappa=0.0, gamma=0.02)
    assert np.abs(got - ref).max() < 1e-9 * np.abs(ref).max()


def test_nonuniform_samples_are_resampled_by_natural_spline():
    from paper_2205_05175_gb300 import rtcc
    rng = np.random.default_rng(3)
    steps = rng.uniform(0.01, 0.05, 1500)
    t = np.concatenate([[0.0], np.cumsum(steps)])
    mu = _signal(t)
    om = np.linspace(0.2, 1.8, 800)
    dt = 0.01
    tu, mu_u = spectrum.uniform_resample(t, mu, dt)
    ref = spectrum.spectrum(tu, mu_u, om, (0, 0, 1), kappa=1.0, gamma=0.01, dt=dt)
    got = rtcc.rtcc_spectrum(t, mu, rtcc.make_field(pol=(0, 0, 1)), om, kappa=1.0, gamma=0.01, dt=dt)
    assert np.abs(got - ref).max() < 1e-8 * np.abs(ref).max()
    # the peaks sit at the oscillation frequencies of the signal
    k = int(np.argmax(got))
    assert abs(om[k] - 0.7) < 0.01
