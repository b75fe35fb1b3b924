"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module only draws random numbers.  It holds none of the method's
arithmetic (no integrals are contracted, no residual is formed): it produces

* a canonical Fock matrix ``f`` (nmo x nmo, diagonal),
* density-fitting factors ``B`` (naux x nmo x nmo, symmetric in the last two
  indices) from which both sides build their own electron-repulsion integrals
  ``(pq|rs) = sum_P B[P,p,q] B[P,r,s]``,
* three symmetric dipole matrices ``mu`` (3 x nmo x nmo),
* random complex amplitude sets with the closed-shell pair symmetry
  ``x[i,j,a,b] == x[j,i,b,a]`` for residual-level tests.

The shapes follow the paper's water-cluster workloads (occupied o = 5n,
virtual v = 19n for (H2O)n in cc-pVDZ, all electrons correlated); the real
water integrals (Psi4, cc-pVDZ) are not available, so these seeded draws stand
in for them.  Orbital order is occupied first, then virtual.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 2205_05175

# (o, v) shapes of the water-cluster-shaped workloads.
SHAPES = {
    "monomer": (5, 19),
    "dimer": (10, 38),
    "tetramer": (20, 76),
    "hexamer": (30, 114),
}


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def b_sigma(o: int, v: int, naux: int) -> float:
    """Standard deviation of the density-fitting factors.

    0.05 for the monomer shape (o=5, v=19, naux=96).  For other shapes the
    variance is scaled so that the collective coupling sqrt(o v naux) sigma^2 of
    the dense random integrals stays at the monomer's value: with a fixed 0.05,
    (pq|pq) = naux sigma^2 grows with the basis and from the dimer shape on the
    CCSD ground-state equations have no convergent Jacobi/DIIS solution.
    """
    return 0.05 * (95.0 * 96.0 / (o * v * naux)) ** 0.25


def make_system(o: int, v: int, seed: int = SEED_BASE, naux: int | None = None):
    """Draw (f, B, mu) for a closed-shell system with o occupied and v virtual orbitals.

    f  : float64 (nmo, nmo), diag(sorted U[-1.4,-0.3] occupied, sorted U[0.15,3.0] virtual)
    B  : float64 (naux, nmo, nmo), entries N(0, b_sigma^2), symmetric in (p, q); naux = 4*nmo
    mu : float64 (3, nmo, nmo), entries N(0, 0.3^2), symmetric
    """
    if o <= 0 or v <= 0:
        raise ValueError("o and v must be positive")
    rng = rng_for(seed)
    nmo = o + v
    naux = 4 * nmo if naux is None else int(naux)
    eps_o = np.sort(rng.uniform(-1.4, -0.3, o))
    eps_v = np.sort(rng.uniform(0.15, 3.0, v))
    f = np.diag(np.concatenate([eps_o, eps_v])).astype(np.float64)
    raw = rng.normal(0.0, b_sigma(o, v, naux), (naux, nmo, nmo))
    upper = np.triu(raw)
    B = upper + np.transpose(np.triu(raw, 1), (0, 2, 1))
    rawm = rng.normal(0.0, 0.3, (3, nmo, nmo))
    mu = np.triu(rawm) + np.transpose(np.triu(rawm, 1), (0, 2, 1))
    return f, np.ascontiguousarray(B), np.ascontiguousarray(mu)


def random_complex(rng: np.random.Generator, shape, scale: float) -> np.ndarray:
    return scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))


def random_amplitudes(o: int, v: int, seed: int, s1: float = 0.05, s2: float = 0.02):
    """Random complex (x1[o,v], x2[o,o,v,v]) with x2[i,j,a,b] == x2[j,i,b,a]."""
    rng = rng_for(seed)
    x1 = random_complex(rng, (o, v), s1)
    raw = random_complex(rng, (o, o, v, v), s2)
    x2 = 0.5 * (raw + raw.transpose(1, 0, 3, 2))
    return x1, x2


def random_general_so_amplitudes(nocc: int, nvir: int, seed: int, s1=0.05, s2=0.02):
    """Random complex spin-orbital amplitudes, antisymmetric in (i,j) and in (a,b).

    Used only by tests that exercise a spin-orbital formulation away from the
    closed-shell manifold.
    """
    rng = rng_for(seed)
    x1 = random_complex(rng, (nocc, nvir), s1)
    raw = random_complex(rng, (nocc, nocc, nvir, nvir), s2)
    x2 = raw - raw.transpose(1, 0, 2, 3)
    x2 = x2 - x2.transpose(0, 1, 3, 2)
    return x1, 0.25 * x2


def random_symmetric(rng: np.random.Generator, n: int, scale: float) -> np.ndarray:
    a = rng.normal(0.0, scale, (n, n))
    return np.triu(a) + np.triu(a, 1).T
