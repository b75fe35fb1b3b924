"""O0: brute-force coupled cluster in the full determinant space (tiny systems).

Test infrastructure only: nothing on the product path imports this module.

Everything here is the definition written out with explicit matrices over all
N-electron Slater determinants of a spin-orbital basis:

* the similarity-transformed Hamiltonian  Hbar = e^{-T} H e^{T}      (Eq. simtranH)
* the ket residual    Omega_mu = <mu| Hbar |0>                        (Eq. derivT)
* the bra residual    R_mu     = <0|(1+Lambda)[Hbar, tau_mu]|0>       (Eq. derivL)
* the dipole          mu_x     = <0|(1+Lambda) e^{-T} mu_x e^{T}|0>   (Eq. dipole)

The Hamiltonian is built from a Fock matrix f and antisymmetrised integrals
<pq||rs> as H = sum h_pq p^+ q + 1/4 sum <pq||rs> p^+ q^+ s r with
h = f - sum_i <pi||qi>, so that the Fock operator of the reference is exactly
the supplied f (the frozen-orbital, field-dressed Fock matrix of Sec. 2.2,
f(t) = f - sum_alpha E_alpha(t) mu_alpha).  Determinants are bit strings;
|d> = a+_{p1} a+_{p2} ... |vac> with p1 < p2 < ..., so a+_p / a_p carry the
sign (-1)^(number of occupied orbitals below p).

Spin orbitals are indexed 0..n-1; the first N are occupied in the reference.
Amplitude tensors use occupied indices 0..N-1 and virtual indices 0..n-N-1
(virtual spin orbital a sits at N + a).  Doubles tensors are antisymmetric
and T2 = 1/4 sum t_ij^ab a+_a a+_b a_j a_i.
"""
from __future__ import annotations

import itertools
from math import factorial

import numpy as np


def _sign_below(det: int, p: int) -> int:
    return -1 if bin(det & ((1 << p) - 1)).count("1") & 1 else 1


def ann(p: int, det: int):
    if not (det >> p) & 1:
        return 0, 0
    return _sign_below(det, p), det ^ (1 << p)


def cre(p: int, det: int):
    if (det >> p) & 1:
        return 0, 0
    return _sign_below(det, p), det | (1 << p)


def apply_string(ops, det):
    """Apply operators right-to-left: ops = [(p, dagger), ...] listed left-to-right."""
    sign = 1
    for p, dag in reversed(ops):
        s, det = (cre if dag else ann)(p, det)
        if s == 0:
            return 0, 0
        sign *= s
    return sign, det


class Space:
    """All determinants with `nel` electrons in `n` spin orbitals."""

    def __init__(self, n: int, nel: int):
        self.n, self.nel = n, nel
        self.dets = [sum(1 << p for p in c) for c in itertools.combinations(range(n), nel)]
        self.index = {d: k for k, d in enumerate(self.dets)}
        self.dim = len(self.dets)
        self.ref = self.index[(1 << nel) - 1]

    def occ(self, det):
        return [p for p in range(self.n) if (det >> p) & 1]

    def vir(self, det):
        return [p for p in range(self.n) if not (det >> p) & 1]

    # --- operators as dense matrices -------------------------------------------------
    def one_body(self, h):
        """Matrix of sum_pq h[p,q] p^+ q."""
        M = np.zeros((self.dim, self.dim), dtype=complex)
        for col, d in enumerate(self.dets):
            for q in self.occ(d):
                s1, d1 = ann(q, d)
                for p in range(self.n):
                    if h[p, q] == 0:
                        continue
                    s2, d2 = cre(p, d1)
                    if s2:
                        M[self.index[d2], col] += s1 * s2 * h[p, q]
        return M

    def two_body(self, w):
        """Matrix of 1/4 sum_pqrs w[p,q,r,s] p^+ q^+ s r (w antisymmetric)."""
        M = np.zeros((self.dim, self.dim), dtype=complex)
        for col, d in enumerate(self.dets):
            occ = self.occ(d)
            for r in occ:
                s1, d1 = ann(r, d)
                for s in occ:
                    if s == r:
                        continue
                    s2, d2 = ann(s, d1)
                    for q in range(self.n):
                        s3, d3 = cre(q, d2)
                        if not s3:
                            continue
                        for p in range(self.n):
                            val = w[p, q, r, s]
                            if val == 0:
                                continue
                            s4, d4 = cre(p, d3)
                            if s4:
                                M[self.index[d4], col] += 0.25 * s1 * s2 * s3 * s4 * val
        return M

    def excitation_matrix(self, t1, t2):
        """Matrix of T = sum t_i^a a+_a a_i + 1/4 sum t_ij^ab a+_a a+_b a_j a_i."""
        N = self.nel
        T = np.zeros((self.dim, self.dim), dtype=complex)
        nocc, nvir = t1.shape
        for col, d in enumerate(self.dets):
            for i in range(nocc):
                for a in range(nvir):
                    if t1[i, a] != 0:
                        s, d2 = apply_string([(N + a, True), (i, False)], d)
                        if s:
                            T[self.index[d2], col] += s * t1[i, a]
            for i, j in itertools.combinations(range(nocc), 2):
                for a, b in itertools.combinations(range(nvir), 2):
                    if t2[i, j, a, b] != 0:
                        s, d2 = apply_string([(N + a, True), (N + b, True), (j, False), (i, False)], d)
                        if s:
                            T[self.index[d2], col] += s * t2[i, j, a, b]
        return T


def expm_nilpotent(T):
    """exp(T) for a nilpotent excitation matrix, by its finite power series."""
    out = np.eye(T.shape[0], dtype=complex)
    term = np.eye(T.shape[0], dtype=complex)
    k = 0
    while True:
        k += 1
        term = term @ T / k
        if not np.any(term):
            return out
        out = out + term
        if k > 64:
            raise RuntimeError("excitation operator is not nilpotent")


def spin_orbital_hamiltonian(f_so, w_so, nel):
    """One-body part h = f - sum_i <pi||qi> so that the reference Fock operator is f."""
    h = f_so - np.einsum("piqi->pq", w_so[:, :nel, :, :nel])
    return h


class BruteCC:
    """Brute-force CC quantities for one Hamiltonian (f_so, w_so) with `nel` electrons."""

    def __init__(self, f_so, w_so, nel):
        n = f_so.shape[0]
        self.sp = Space(n, nel)
        self.nel, self.n = nel, n
        h = spin_orbital_hamiltonian(f_so, w_so, nel)
        self.H = self.sp.one_body(h) + self.sp.two_body(w_so)
        self.Eref = self.H[self.sp.ref, self.sp.ref]
        # unique excitations mu -> (det index, sign of tau_mu|0>)
        N, nv = nel, n - nel
        ref_det = self.sp.dets[self.sp.ref]
        self.singles, self.doubles = [], []
        for i in range(N):
            for a in range(nv):
                s, d = apply_string([(N + a, True), (i, False)], ref_det)
                self.singles.append((i, a, self.sp.index[d], s))
        for i, j in itertools.combinations(range(N), 2):
            for a, b in itertools.combinations(range(nv), 2):
                s, d = apply_string([(N + a, True), (N + b, True), (j, False), (i, False)], ref_det)
                self.doubles.append((i, j, a, b, self.sp.index[d], s))

    def hbar(self, t1, t2):
        T = self.sp.excitation_matrix(t1, t2)
        return expm_nilpotent(-T) @ self.H @ expm_nilpotent(T), T

    def omega(self, t1, t2):
        """Ket residuals (Omega1[i,a], Omega2[i,j,a,b] antisymmetric) and E_corr."""
        Hb, _ = self.hbar(t1, t2)
        x = Hb[:, self.sp.ref]
        N, nv = self.nel, self.n - self.nel
        o1 = np.zeros((N, nv), complex)
        o2 = np.zeros((N, N, nv, nv), complex)
        for i, a, k, s in self.singles:
            o1[i, a] = s * x[k]
        for i, j, a, b, k, s in self.doubles:
            val = s * x[k]
            o2[i, j, a, b] = val
            o2[j, i, a, b] = -val
            o2[i, j, b, a] = -val
            o2[j, i, b, a] = val
        return o1, o2, x[self.sp.ref] - self.Eref

    def bra(self, l1, l2):
        """Row vector <0|(1 + Lambda), Lambda = sum_mu lambda_mu tau_mu^+ (no conjugation)."""
        L = np.zeros(self.sp.dim, complex)
        L[self.sp.ref] = 1.0
        for i, a, k, s in self.singles:
            L[k] += s * l1[i, a]
        for i, j, a, b, k, s in self.doubles:
            L[k] += s * l2[i, j, a, b]
        return L

    def _tau_apply(self, ops, vec):
        out = np.zeros_like(vec)
        for k in np.nonzero(vec)[0]:
            s, d = apply_string(ops, self.sp.dets[k])
            if s:
                out[self.sp.index[d]] += s * vec[k]
        return out

    def lambda_residual(self, t1, t2, l1, l2):
        """R_mu = <0|(1+Lambda)[Hbar, tau_mu]|0> for every unique mu (Eq. derivL)."""
        Hb, _ = self.hbar(t1, t2)
        L = self.bra(l1, l2)
        u = L @ Hb
        x = Hb[:, self.sp.ref]
        N, nv = self.nel, self.n - self.nel
        r1 = np.zeros((N, nv), complex)
        r2 = np.zeros((N, N, nv, nv), complex)
        for i, a, k, s in self.singles:
            r1[i, a] = s * u[k] - L @ self._tau_apply([(N + a, True), (i, False)], x)
        for i, j, a, b, k, s in self.doubles:
            val = s * u[k] - L @ self._tau_apply([(N + a, True), (N + b, True), (j, False), (i, False)], x)
            r2[i, j, a, b] = val
            r2[j, i, a, b] = -val
            r2[i, j, b, a] = -val
            r2[j, i, b, a] = val
        return r1, r2

    def expectation(self, t1, t2, l1, l2, op_so):
        """<0|(1+Lambda) e^{-T} O e^{T}|0> for a one-body operator O = sum o_pq p^+ q (Eq. dipole)."""
        T = self.sp.excitation_matrix(t1, t2)
        M = self.sp.one_body(op_so)
        L = self.bra(l1, l2)
        ket = expm_nilpotent(T)[:, self.sp.ref]
        return (L @ expm_nilpotent(-T)) @ (M @ ket)

    def density(self, t1, t2, l1, l2):
        """rho_pq = <0|(1+Lambda) e^{-T} p^+ q e^{T}|0> over all spin orbitals."""
        T = self.sp.excitation_matrix(t1, t2)
        L = self.bra(l1, l2) @ expm_nilpotent(-T)
        ket = expm_nilpotent(T)[:, self.sp.ref]
        rho = np.zeros((self.n, self.n), complex)
        for p in range(self.n):
            for q in range(self.n):
                rho[p, q] = L @ self._tau_apply([(p, True), (q, False)], ket)
        return rho
