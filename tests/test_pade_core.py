"""The Pade core of the library (csrc/pade_core.cuh: Toeplitz least-squares by one-sided Jacobi
SVD, minimum-norm cut, numerator convolution, Horner evaluation) built for the host with the
warp's lanes and shuffle reduction replayed in order, against the oracle's Pade transform and
closed forms.  The device kernels run exactly these functions."""
import os
import subprocess

import numpy as np
import pytest

from oracle import spectrum

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    exe = tmp_path_factory.mktemp("pade") / "pade_harness"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2205_05175_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "native", "pade_harness.cpp"), "-o", str(exe)], check=True)
    return str(exe)


def _run(exe, text):
    return subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout.split("\n")


def _pade(exe, c, z):
    text = "pade %d %s %d %s" % (len(c), " ".join("%.17g" % x for x in c), len(z),
                                 " ".join("%.17g %.17g" % (v.real, v.imag) for v in z))
    out = _run(exe, text)
    return int(out[0]), np.array([complex(*map(float, line.split())) for line in out[1:] if line.strip()])


@pytest.mark.parametrize("n", [2, 4, 6, 16, 64])
def test_tournament_pairs_every_column_once_per_sweep(harness, n):
    rows = [tuple(map(int, line.split())) for line in _run(harness, "pairs %d" % n) if line.strip()]
    assert len(rows) == (n - 1) * (n // 2)
    for r in range(n - 1):
        cols = [c for rr, p, q in rows if rr == r for c in (p, q)]
        assert sorted(cols) == list(range(n))            # disjoint and covering in every round
    pairs = {(p, q) for _, p, q in rows}
    assert len(pairs) == n * (n - 1) // 2 and all(p < q for p, q in pairs)


def test_damped_modes_give_the_closed_form_sum(harness):
    """Rank-deficient case (two modes, M = 20): the minimum-norm solution still gives the exact
    rational function, as the oracle's least-squares solver does."""
    dt, modes = 0.1, [(0.3, 0.81, 0.02), (0.1, 1.37, 0.05)]
    k = np.arange(41)
    c = sum(A * np.exp(-g * k * dt) * np.sin(w * k * dt) for A, w, g in modes)
    z = np.exp(1j * np.linspace(0.2, 2.0, 400) * dt)
    exact = 0.0
    for A, w, g in modes:
        p, q = np.exp((1j * w - g) * dt), np.exp((-1j * w - g) * dt)
        exact = exact + A / 2j * (1.0 / (1.0 - p * z) - 1.0 / (1.0 - q * z))
    sweeps, v = _pade(harness, c, z)
    assert 0 < sweeps < 60
    assert np.abs(v - exact).max() < 1e-9 * np.abs(exact).max()
    o = spectrum.pade_transform(c, z)
    assert np.abs(v - o).max() < 1e-9 * np.abs(o).max()


def test_short_two_mode_record_matches_the_oracle(harness):
    dt = 0.05
    t = dt * np.arange(241)
    d = (0.4 * np.sin(1.0 * t) + 0.3 * np.sin(1.15 * t)) * np.exp(-0.01 * t)
    z = np.exp(1j * np.linspace(0.6, 1.6, 2001) * dt)
    _, v = _pade(harness, d, z)
    o = spectrum.pade_transform(d, z)
    assert np.abs(v - o).max() < 1e-10 * np.abs(o).max()


@pytest.mark.parametrize("n", [3, 5, 31, 101])
def test_full_rank_series_match_the_oracle(harness, n):
    c = np.random.default_rng(n).standard_normal(n)
    z = np.exp(1j * np.linspace(0.1, 3.0, 50) * 0.1)
    _, v = _pade(harness, c, z)
    o = spectrum.pade_transform(c, z)
    assert np.abs(v - o).max() < 1e-11 * np.abs(o).max()


def test_pulse_record_that_decays_to_underflow_converges(harness):
    """The samples of a Gaussian pulse fall to ~1e-300 long before the record ends (1025 samples,
    the largest accepted): columns of negligible size are left alone, so the sweeps stop early,
    and the transform still matches the oracle's."""
    from oracle import rk
    fld = rk.Field(E0=0.01, omega=0.5, sigma=0.5, t0=1.0)
    t = 0.1 * np.arange(1025)
    e = fld.amplitude(t)
    z = np.exp(1j * np.linspace(0.2, 1.5, 300) * 0.1)
    sweeps, v = _pade(harness, e, z)
    assert sweeps < 30
    o = spectrum.pade_transform(e, z)
    assert np.abs(v - o).max() < 1e-12 * np.abs(o).max()
