"""O1: spin-orbital CCSD ket residual and the closed-shell <-> spin-orbital maps.

Test infrastructure only: nothing on the product path imports this module.

The ket residual Omega_mu = <mu|e^{-T} H e^{T}|0> (Eq. derivT) is written with
the Stanton-Gauss (1991) intermediates for a general (non-canonical,
non-Hartree-Fock) reference: the full field-dressed Fock matrix enters the
F_ae / F_mi intermediates (diagonal included), so the result is the complete
residual rather than "right-hand side minus D*t".  Complex amplitudes are
used holomorphically (no conjugation anywhere), as the phase-isolated
time-dependent ansatz of Sec. 2 requires.

Spin orbitals are ordered 2p + sigma (sigma = 0 alpha, 1 beta) over spatial
orbitals p, occupied spatial orbitals first.
"""
from __future__ import annotations

import numpy as np


def eri_chemist(B):
    """(pq|rs) = sum_P B[P,p,q] B[P,r,s] (density-fitting factors)."""
    return np.einsum("Ppq,Prs->pqrs", B, B, optimize=True)


def spin_orbital_operators(f, g):
    """Spin-orbital Fock matrix and antisymmetrised <pq||rs> from spatial f and (pq|rs)."""
    nmo = f.shape[0]
    n = 2 * nmo
    spat = np.arange(n) // 2
    spin = np.arange(n) % 2
    same = (spin[:, None] == spin[None, :]).astype(float)
    f_so = f[np.ix_(spat, spat)] * same
    gs = g[np.ix_(spat, spat, spat, spat)]
    # <pq|rs> = (pr|qs) delta(sp,sr) delta(sq,ss)
    v = gs.transpose(0, 2, 1, 3) * same[:, None, :, None] * same[None, :, None, :]
    w = v - v.transpose(0, 1, 3, 2)
    return f_so, w


def spin_orbital_one_body(op):
    nmo = op.shape[0]
    n = 2 * nmo
    spat = np.arange(n) // 2
    spin = np.arange(n) % 2
    return op[np.ix_(spat, spat)] * (spin[:, None] == spin[None, :])


# --- closed-shell embedding -----------------------------------------------------------

def _delta_spin(nsp):
    s = np.arange(2 * nsp) % 2
    return s


def embed_amplitudes(x1, x2):
    """Spin-adapted closed-shell amplitudes -> spin-orbital amplitudes.

    x_{i s1, a s3} = delta(s1,s3) x[i,a]
    x_{i s1 j s2, a s3 b s4} = delta(s1,s3) delta(s2,s4) x[i,j,a,b] - delta(s1,s4) delta(s2,s3) x[i,j,b,a]
    """
    o, v = x1.shape
    so, sv = np.arange(2 * o) % 2, np.arange(2 * v) % 2
    po, pv = np.arange(2 * o) // 2, np.arange(2 * v) // 2
    d_ov = (so[:, None] == sv[None, :])
    x1s = x1[np.ix_(po, pv)] * d_ov
    X = x2[np.ix_(po, po, pv, pv)]
    Xs = x2.transpose(0, 1, 3, 2)[np.ix_(po, po, pv, pv)]
    d13 = d_ov[:, None, :, None]
    d24 = d_ov[None, :, None, :]
    d14 = d_ov[:, None, None, :]
    d23 = d_ov[None, :, :, None]
    x2s = d13 * d24 * X - d14 * d23 * Xs
    return x1s, x2s


def embed_multipliers(l1, l2):
    """Closed-shell multipliers (paired with the closed-shell residual by a plain dot
    product) -> spin-orbital multipliers paired with the spin-orbital residual over
    unique excitations, so that both Lagrangians coincide."""
    return embed_amplitudes(0.5 * l1, (2.0 * l2 + l2.transpose(0, 1, 3, 2)) / 3.0)


def restrict(r1s, r2s):
    """Spin-orbital residual -> closed-shell components (i alpha, a alpha) and (i alpha j beta, a alpha b beta)."""
    return r1s[0::2, 0::2], r2s[0::2, 1::2, 0::2, 1::2]


# --- spin-orbital CCSD residual ---------------------------------------------------------

def omega(f_so, w, nocc, t1, t2):
    """Spin-orbital CCSD residuals (Omega1[i,a], Omega2[i,j,a,b]) and correlation energy."""
    o = slice(0, nocc)
    v = slice(nocc, f_so.shape[0])
    fov, foo, fvv = f_so[o, v], f_so[o, o], f_so[v, v]
    ein = lambda s, *a: np.einsum(s, *a, optimize=True)
    tt = ein("ia,jb->ijab", t1, t1)
    tt = tt - tt.transpose(0, 1, 3, 2)
    tau = t2 + tt
    taut = t2 + 0.5 * tt

    Fae = fvv - 0.5 * ein("me,ma->ae", fov, t1) + ein("mf,mafe->ae", t1, w[o, v, v, v]) \
        - 0.5 * ein("mnaf,mnef->ae", taut, w[o, o, v, v])
    Fmi = foo + 0.5 * ein("ie,me->mi", t1, fov) + ein("ne,mnie->mi", t1, w[o, o, o, v]) \
        + 0.5 * ein("inef,mnef->mi", taut, w[o, o, v, v])
    Fme = fov + ein("nf,mnef->me", t1, w[o, o, v, v])

    Wmnij = w[o, o, o, o] + ein("je,mnie->mnij", t1, w[o, o, o, v]) \
        - ein("ie,mnje->mnij", t1, w[o, o, o, v]) + 0.25 * ein("ijef,mnef->mnij", tau, w[o, o, v, v])
    Wabef = w[v, v, v, v] - ein("mb,amef->abef", t1, w[v, o, v, v]) \
        + ein("ma,bmef->abef", t1, w[v, o, v, v]) + 0.25 * ein("mnab,mnef->abef", tau, w[o, o, v, v])
    Wmbej = w[o, v, v, o] + ein("jf,mbef->mbej", t1, w[o, v, v, v]) - ein("nb,mnej->mbej", t1, w[o, o, v, o]) \
        - ein("jnfb,mnef->mbej", 0.5 * t2 + ein("jf,nb->jnfb", t1, t1), w[o, o, v, v])

    r1 = fov.copy() + ein("ie,ae->ia", t1, Fae) - ein("ma,mi->ia", t1, Fmi) + ein("imae,me->ia", t2, Fme) \
        - ein("nf,naif->ia", t1, w[o, v, o, v]) - 0.5 * ein("imef,maef->ia", t2, w[o, v, v, v]) \
        - 0.5 * ein("mnae,nmei->ia", t2, w[o, o, v, o])

    Xbe = Fae - 0.5 * ein("mb,me->be", t1, Fme)
    Zmj = Fmi + 0.5 * ein("je,me->mj", t1, Fme)
    pab = ein("ijae,be->ijab", t2, Xbe)
    pij = ein("imab,mj->ijab", t2, Zmj)
    ring = ein("imae,mbej->ijab", t2, Wmbej) - ein("ie,ma,mbej->ijab", t1, t1, w[o, v, v, o])
    r2 = w[o, o, v, v].copy()
    r2 = r2 + pab - pab.transpose(0, 1, 3, 2)
    r2 = r2 - pij + pij.transpose(1, 0, 2, 3)
    r2 = r2 + 0.5 * ein("mnab,mnij->ijab", tau, Wmnij) + 0.5 * ein("ijef,abef->ijab", tau, Wabef)
    r2 = r2 + ring - ring.transpose(1, 0, 2, 3) - ring.transpose(0, 1, 3, 2) + ring.transpose(1, 0, 3, 2)
    pe = ein("ie,abej->ijab", t1, w[v, v, v, o])
    r2 = r2 + pe - pe.transpose(1, 0, 2, 3)
    pm = ein("ma,mbij->ijab", t1, w[o, v, o, o])
    r2 = r2 - pm + pm.transpose(0, 1, 3, 2)

    e = ein("ia,ia->", fov, t1) + 0.25 * ein("ijab,ijab->", w[o, o, v, v], t2) \
        + 0.5 * ein("ijab,ia,jb->", w[o, o, v, v], t1, t1)
    return r1, r2, e
