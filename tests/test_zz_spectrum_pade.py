"""rtcc_spectrum_pade (Pade-accelerated spectra: Jacobi-SVD least squares for the denominator,
numerator convolution, evaluation on the frequency grid, all on the device) against the oracle's
pade_spectrum.  The same arithmetic built for the host matches the oracle to 1e-10 or better on
these series (tests/test_pade_core.py); the device runs the same functions with the lanes of each
warp, and the warps of a block, in parallel."""
import numpy as np
import pytest

from oracle import rk, spectrum

pytestmark = [pytest.mark.gpu, pytest.mark.last]


def _peaks(om, I):
    return [om[k] for k in range(1, len(om) - 1) if I[k] > I[k - 1] and I[k] > I[k + 1] and I[k] > 0.2 * I.max()]


@pytest.mark.parametrize("n", [241, 240])
def test_delta_pulse_short_record_matches_oracle_and_resolves_both_modes(n):
    """Two modes 0.15 Eh apart in a 12 au record (below the plain transform's resolution); an
    even count drops the last sample on both sides."""
    from paper_2205_05175_gb300 import rtcc
    dt = 0.05
    t = dt * np.arange(n)
    mu = np.zeros((n, 3))
    mu[:, 2] = 0.4 * np.sin(1.00 * t) + 0.3 * np.sin(1.15 * t)
    om = np.linspace(0.6, 1.6, 2001)
    ref = spectrum.pade_spectrum(t, mu, om, (0, 0, 1), kappa=1.0, gamma=0.01)
    got = rtcc.rtcc_spectrum_pade(t, mu, rtcc.make_field(pol=(0.0, 0.0, 1.0)), om, kappa=1.0, gamma=0.01)
    assert np.abs(got - ref).max() < 1e-8 * np.abs(ref).max()
    p = _peaks(om, got)
    assert len(p) == 2 and abs(p[0] - 1.00) < 2e-3 and abs(p[1] - 1.15) < 2e-3


def test_finite_pulse_division_matches_oracle():
    """The pulse's samples get their own approximant (they decay to underflow within the record)."""
    from paper_2205_05175_gb300 import rtcc
    dt, n = 0.1, 1025
    t = dt * np.arange(n)
    mu = np.zeros((n, 3))
    mu[:, 1] = 0.1 * np.sin(0.9 * t) * np.exp(-0.002 * t)
    mu[:, 2] = 0.3 * np.sin(0.7 * t) + 0.05 * np.sin(1.6 * t) + 0.2
    fld = rk.Field(E0=0.01, omega=0.5, sigma=0.5, t0=1.0, pol=(0.0, 0.6, 0.8))
    om = np.linspace(0.2, 1.5, 300)
    ref = spectrum.pade_spectrum(t, mu, om, fld.pol, field_amp=fld.amplitude, gamma=0.02)
    got = rtcc.rtcc_spectrum_pade(t, mu, rtcc.make_field(E0=0.01, omega=0.5, sigma=0.5, t0=1.0, pol=(0.0, 0.6, 0.8)),
                                  om, kappa=0.0, gamma=0.02)
    assert np.abs(got - ref).max() < 1e-8 * np.abs(ref).max()
