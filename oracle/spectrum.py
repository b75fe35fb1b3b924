"""Absorption spectrum post-processing (Sec. 2.2, Eqs. dipole ... ; Sec. 4.2 interpolation).

Test infrastructure only: nothing on the product path imports this module.

The steps, in the paper's order:
1. non-uniform samples (adaptive Cash-Karp steps) are interpolated onto a
   uniform grid (natural cubic spline, written out below);
2. the induced dipole d_x(t) = Re mu_x(t) - Re mu_x(t_0), damped by exp(-gamma (t-t_0));
3. Fourier transform D_x(w) = dt sum_k d_x(t_k) exp(i w t_k) evaluated directly on the
   requested frequency grid (a plain DFT; no FFT reordering);
4. alpha(w) = n.D(w) / E(w) with E(w) the same transform of the scalar pulse
   amplitude (or kappa for a delta pulse), and I(w) = Im alpha(w).
Also a matrix-pencil fit (Hua & Sarkar) that recovers the oscillation
frequencies of a sampled sum of exponentials below the Fourier resolution, and Pade-accelerated
transforms (the Pade approach to short-time spectra that the paper cites among spectral
techniques, Sec. 1): the Fourier sum sum_k d_k z^k, z = exp(i w dt), is replaced by the diagonal
Pade approximant of the power series, which is exact for a signal that is a sum of at most M
damped exponentials and resolves peaks from much shorter records than the plain sum.
"""
from __future__ import annotations

import numpy as np


def natural_cubic_spline(x, y, xn):
    """Natural cubic spline through (x, y) evaluated at xn (x strictly increasing)."""
    x = np.asarray(x, float)
    y = np.asarray(y, float)
    n = len(x)
    h = np.diff(x)
    # second derivatives M with M_0 = M_{n-1} = 0: tridiagonal system
    A = np.zeros((n, n))
    r = np.zeros(n)
    A[0, 0] = A[-1, -1] = 1.0
    for i in range(1, n - 1):
        A[i, i - 1] = h[i - 1]
        A[i, i] = 2.0 * (h[i - 1] + h[i])
        A[i, i + 1] = h[i]
        r[i] = 6.0 * ((y[i + 1] - y[i]) / h[i] - (y[i] - y[i - 1]) / h[i - 1])
    M = np.linalg.solve(A, r)
    k = np.clip(np.searchsorted(x, xn, side="right") - 1, 0, n - 2)
    dx = xn - x[k]
    hk = h[k]
    a = (M[k + 1] - M[k]) / (6.0 * hk)
    b = M[k] / 2.0
    c = (y[k + 1] - y[k]) / hk - hk * (2.0 * M[k] + M[k + 1]) / 6.0
    return y[k] + c * dx + b * dx * dx + a * dx * dx * dx


def uniform_resample(t, mu, dt=None):
    t = np.asarray(t, float)
    if dt is None:
        dt = float(np.min(np.diff(t)))
    n = int(np.floor((t[-1] - t[0]) / dt + 1e-9)) + 1
    tu = t[0] + dt * np.arange(n)
    mu = np.asarray(mu)
    out = np.stack([natural_cubic_spline(t, mu[:, x], tu) for x in range(mu.shape[1])], axis=1)
    return tu, out


def dft(t, d, omegas, dt):
    phase = np.exp(1j * np.outer(omegas, t))
    return dt * (phase @ d)


def spectrum(t, mu_re, omegas, pol, field_amp=None, kappa=None, gamma=0.01, dt=None, uniform=True):
    """I(w) = Im[ n.D(w) / E(w) ] for real dipole samples mu_re[n,3]."""
    t = np.asarray(t, float)
    mu_re = np.asarray(mu_re, float)
    if not uniform:
        t, mu_re = uniform_resample(t, mu_re, dt)
    if dt is None:
        dt = t[1] - t[0]
    d = (mu_re - mu_re[0]) * np.exp(-gamma * (t - t[0]))[:, None]
    dn = d @ np.asarray(pol, float)
    D = dft(t, dn, omegas, dt)
    if kappa is not None:
        Ew = kappa
    else:
        Ew = dft(t, field_amp(t), omegas, dt)
    return np.imag(D / Ew)


def matrix_pencil(y, dt, order, L=None):
    """Frequencies w (and decay) of y_k = sum_m c_m exp(-i w_m k dt): returns complex w_m."""
    y = np.asarray(y, complex)
    N = len(y)
    L = N // 2 if L is None else L
    Y = np.array([y[i:i + L + 1] for i in range(N - L)])
    U, s, Vh = np.linalg.svd(Y, full_matrices=False)
    V = Vh[:order, :].T          # row-space basis of Y (no conjugation)
    V1, V2 = V[:-1, :], V[1:, :]
    z = np.linalg.eigvals(np.linalg.pinv(V1) @ V2)
    return 1j * np.log(z) / dt


def pade_transform(c, z):
    """Diagonal [M/M] Pade approximant of the power series sum_k c_k z^k, built from c_0 .. c_2M,
    evaluated at the points z.  Q(z) = sum_{m=0..M} b_m z^m with b_0 = 1 is fixed by requiring
    P/Q to reproduce the series through z^{2M}: sum_{m=0..M} b_m c_{k-m} = 0 for k = M+1 .. 2M;
    then P(z) = sum_{k=0..M} a_k z^k with a_k = sum_{m=0..k} b_m c_{k-m}.  The linear system is
    solved in the least-squares sense (a signal with fewer than M exponentials makes it singular)."""
    c = np.asarray(c, complex)
    M = (len(c) - 1) // 2
    G = np.array([[c[k - m] for m in range(1, M + 1)] for k in range(M + 1, 2 * M + 1)])
    b = np.concatenate([[1.0 + 0j], np.linalg.lstsq(G, -c[M + 1:2 * M + 1], rcond=None)[0]])
    a = np.array([np.dot(b[:k + 1], c[k::-1]) for k in range(M + 1)])
    z = np.asarray(z, complex)
    return np.polyval(a[::-1], z) / np.polyval(b[::-1], z)


def pade_spectrum(t, mu_re, omegas, pol, field_amp=None, kappa=None, gamma=0.01):
    """I(w) as in spectrum(), with each Fourier sum over the uniform samples replaced by its
    diagonal Pade approximant in z = exp(i w dt) (odd sample counts use all samples)."""
    t = np.asarray(t, float)
    mu_re = np.asarray(mu_re, float)
    dt = t[1] - t[0]
    n = len(t) if len(t) % 2 == 1 else len(t) - 1
    t, mu_re = t[:n], mu_re[:n]
    d = (mu_re - mu_re[0]) * np.exp(-gamma * (t - t[0]))[:, None]
    dn = d @ np.asarray(pol, float)
    z = np.exp(1j * np.asarray(omegas, float) * dt)
    shift = dt * np.exp(1j * np.asarray(omegas, float) * t[0])
    D = shift * pade_transform(dn, z)
    Ew = kappa if kappa is not None else shift * pade_transform(field_amp(t), z)
    return np.imag(D / Ew)

