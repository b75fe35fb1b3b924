"""Forward-mode tangent of the RK4 propagation with respect to the pulse parameters.

Test infrastructure only (imported by tests; never by the product path).

The objective is J = sum_n sum_x w[n][x] Re mu_x(t_n) over the RK4 samples t_n = t_start + n h
(the propagation of Sec. 2.1, Eqs. rk_y / rk_k, driven by the pulse of Eq. field with
theta = (E0, omega, sigma)).  Its gradient is formed by differentiating every RK4 step forward:

    Y_i  = y + h sum_j a_ij k_j,        dY_i = dy + h sum_j a_ij dk_j
    k_i  = f(t_i, Y_i),                 dk_i = J_f(t_i, Y_i) dY_i + (df/dA)(t_i, Y_i) dA/dtheta(t_i)
    y'   = y + h sum_i b_i k_i,         dy'  = dy + h sum_i b_i dk_i
    dJ  += sum_x w[n][x] Re (dmu_x/dy . dy_n)

* J_f v: five-point central difference of the right-hand side along v.  The right-hand side is a
  polynomial of degree <= 4 in the amplitudes and multipliers (Omega is quartic in t; the Lambda
  residual is cubic in t and linear in lambda), so the stencil is exact up to rounding.  The
  same holds for the dipole (degree <= 3).
* df/dA: the right-hand side is affine in the field-dressed Fock matrix f(t) = f - A(t) P with
  P = sum_x pol_x mu_x, so df/dA = f(F - P) - f(F) at any F.
* dA/dtheta: the analytic derivatives of A(t) = sign E0 exp(-(t-t0)^2 / (2 sigma^2)) car(omega (t-t0)).

Pinned by central finite differences of the oracle's own propagation (tests/test_oracle_pins.py).
"""
from __future__ import annotations

import numpy as np

from . import closed
from .rk import RK4_TABLE, Field, as_float, fock_at, pack, unpack


def amplitude_gradient(fld: Field, t: float) -> np.ndarray:
    """d A(t) / d(E0, omega, sigma) of the pulse amplitude (Eq. field)."""
    x = t - fld.t0
    env = np.exp(-0.5 * x * x / (fld.sigma * fld.sigma))
    if fld.carrier == "sin":
        car, dcar = np.sin(fld.omega * x), x * np.cos(fld.omega * x)
    else:
        car, dcar = np.cos(fld.omega * x), -x * np.sin(fld.omega * x)
    s = fld.sign
    return np.array([s * env * car, s * fld.E0 * env * dcar, s * fld.E0 * env * car * x * x / fld.sigma ** 3])


def _five_point(fun, y, v):
    """Directional derivative of a polynomial map of degree <= 4 (exact up to rounding)."""
    scale = float(np.abs(v).max())
    if scale == 0.0:
        return np.zeros_like(fun(y))
    e = 0.25 / scale
    return (fun(y - 2 * e * v) - 8 * fun(y - e * v) + 8 * fun(y + e * v) - fun(y + 2 * e * v)) / (12 * e)


def _rhs_fock(sys, y, F):
    t1, t2, l1, l2 = unpack(y, sys.o, sys.v)
    return pack(*closed.rhs(t1, t2, l1, l2, F, sys.V))


def tangent_gradient(sys, y0, fld: Field, h: float, nsteps: int, w, t_start: float = 0.0):
    """(J, dJ/d(E0, omega, sigma)) of J = sum_n w[n] . Re mu(t_n) over nsteps RK4 steps of size h."""
    w = np.asarray(w, float).reshape(nsteps + 1, 3)
    tab = as_float(RK4_TABLE)
    P = np.einsum("x,xpq->pq", np.asarray(fld.pol, float), sys.mu)
    y = np.asarray(y0, complex).copy()
    dy = np.zeros((3, y.size), complex)

    def observe(n, y, dy):
        J = float(np.sum(w[n] * sys.dipole(y).real))
        dJ = np.array([float(np.sum(w[n] * _five_point(sys.dipole, y, dy[p]).real)) for p in range(3)])
        return J, dJ

    J, dJ = observe(0, y, dy)
    tt = t_start
    for n in range(1, nsteps + 1):
        ks, dks = [], []
        for i, ci in enumerate(tab["c"]):
            ys, dys = y.copy(), dy.copy()
            for j, aij in enumerate(tab["a"][i]):
                if aij != 0.0:
                    ys = ys + h * aij * ks[j]
                    dys = dys + h * aij * dks[j]
            ti = tt + ci * h
            F = fock_at(sys.f, sys.mu, fld, ti)
            k = _rhs_fock(sys, ys, F)
            dfdA = _rhs_fock(sys, ys, F - P) - k
            dA = amplitude_gradient(fld, ti)
            dk = np.array([_five_point(lambda u: _rhs_fock(sys, u, F), ys, dys[p]) + dfdA * dA[p] for p in range(3)])
            ks.append(k)
            dks.append(dk)
        y = y + h * sum(b * k for b, k in zip(tab["b"], ks))
        dy = dy + h * sum(b * dk for b, dk in zip(tab["b"], dks))
        tt += h
        Jn, dJn = observe(n, y, dy)
        J += Jn
        dJ += dJn
    return J, dJ
