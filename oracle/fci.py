"""Exact references for tiny systems: FCI propagation and the CC Jacobian.

Test infrastructure only: nothing on the product path imports this module.

* ``FCI``: the time-dependent Schroedinger equation (Eq. TDSE) for the same
  Hamiltonian H(t) = H0 - E(t).mu as the RT-CC oracle, in the full
  determinant space of ``oracle/brute.py``.  For two electrons CCSD is exact,
  so the RT-CCSD dipole must follow <Psi(t)|mu|Psi(t)> / <Psi|Psi>.
* ``jacobian``: the closed-shell CC Jacobian A = d Omega / d t on the
  pair-symmetric amplitude space, built column by column from the five-point
  central difference in a complex scalar, which is exact for polynomials up to
  degree four (the CCSD residual is at most quartic in t).  Its eigenvalues are
  the EOM-CCSD excitation energies (the paper's stick spectra).
"""
from __future__ import annotations

import itertools

import numpy as np

from . import brute, closed, spinorb


class FCI:
    def __init__(self, f, B, mu, o):
        g = spinorb.eri_chemist(B)
        fso, w = spinorb.spin_orbital_operators(f, g)
        self.bc = brute.BruteCC(fso, w, 2 * o)
        self.H0 = self.bc.H
        self.M = [self.bc.sp.one_body(spinorb.spin_orbital_one_body(mu[x])) for x in range(3)]
        self.ref = self.bc.sp.ref

    def ground(self):
        w, U = np.linalg.eigh(self.H0)
        k = int(np.argmax(np.abs(U[self.ref, :])))
        psi = U[:, k] / U[self.ref, k] * abs(U[self.ref, k])
        return w[k], psi / np.linalg.norm(psi), w, U

    def dipole(self, psi):
        nrm = np.vdot(psi, psi)
        return np.array([np.vdot(psi, M @ psi) / nrm for M in self.M])

    def hamiltonian(self, fld, t):
        if fld is None:
            return self.H0
        e = fld.vector(t)
        return self.H0 - sum(e[x] * self.M[x] for x in range(3))

    def propagate(self, psi0, fld, t_end, h, sample_every):
        """Classic RK4 on d psi/dt = -i H(t) psi with a fine step h; returns samples."""
        psi = psi0.astype(complex)
        tt = 0.0
        nsteps = int(round(t_end / h))
        times, mus = [0.0], [self.dipole(psi)]
        f = lambda s, x: -1j * (self.hamiltonian(fld, s) @ x)
        for n in range(1, nsteps + 1):
            k1 = f(tt, psi)
            k2 = f(tt + h / 2, psi + h / 2 * k1)
            k3 = f(tt + h / 2, psi + h / 2 * k2)
            k4 = f(tt + h, psi + h * k3)
            psi = psi + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
            tt = n * h
            if n % sample_every == 0:
                times.append(tt)
                mus.append(self.dipole(psi))
        return np.array(times), np.array(mus)


def symmetric_basis(o, v):
    """Basis of the pair-symmetric amplitude space: singles e_ia, doubles e_ijab + e_jiba."""
    basis = []
    for i in range(o):
        for a in range(v):
            x1 = np.zeros((o, v), complex)
            x1[i, a] = 1.0
            basis.append((x1, np.zeros((o, o, v, v), complex)))
    pairs = list(itertools.product(range(o), range(v)))
    for p, q in itertools.combinations_with_replacement(range(len(pairs)), 2):
        (i, a), (j, b) = pairs[p], pairs[q]
        x2 = np.zeros((o, o, v, v), complex)
        x2[i, j, a, b] = 1.0
        x2[j, i, b, a] = 1.0
        basis.append((np.zeros((o, v), complex), x2))
    return basis


def coords(x1, x2, o, v):
    """Coordinates of a pair-symmetric vector in `symmetric_basis` (inverse map)."""
    out = [x1[i, a] for i in range(o) for a in range(v)]
    pairs = list(itertools.product(range(o), range(v)))
    for p, q in itertools.combinations_with_replacement(range(len(pairs)), 2):
        (i, a), (j, b) = pairs[p], pairs[q]
        out.append(x2[i, j, a, b])
    return np.array(out)


def jacobian(t1, t2, f, V):
    o, v = t1.shape
    basis = symmetric_basis(o, v)
    cols = []
    for u1, u2 in basis:
        def om(s):
            r1, r2, _ = closed.omega(t1 + s * u1, t2 + s * u2, f, V)
            return coords(r1, r2, o, v)
        hstep = 0.25
        d = (om(-2 * hstep) - 8 * om(-hstep) + 8 * om(hstep) - om(2 * hstep)) / (12 * hstep)
        cols.append(d)
    return np.array(cols).T
