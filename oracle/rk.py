"""O3: field, Runge-Kutta tableaus, step controller, ground state and RT-CC propagation.

Test infrastructure only: nothing on the product path imports this module.

* Field (Eq. field): E(t) = sign * E0 * exp(-(t-t0)^2 / (2 sigma^2)) * carrier(omega (t-t0)) * n,
  carrier = cos (the paper's form, sign = -1) or sin (the z-polarised sine pulse of
  the benchmark workloads, sign = +1); n a unit polarisation vector (Eq. iso-field
  gives the isotropic choice).
* Time-dependent Fock matrix (Sec. 2.2, V = -mu.E): f(t) = f - sum_x E_x(t) mu_x.
* Explicit RK (Eqs. rk_y, rk_k): classic RK4 (Eq. rk4truncation, with the step h
  multiplying the stage sum) and Cash-Karp (Eqs. ck-k, ck-y) with the two
  coefficient corrections the row-sum condition sum_j a_ij = c_i forces
  (a42 = -9/10, a63 = +575/13824, hence c4 = 3/5, c5 = 1); the 37/378 weights are
  the fifth-order solution and are propagated, 2825/27648 is the embedded fourth
  order one.  The error estimate is Delta = max_k |y5_k - y4_k| over all complex
  components of (t1, t2, l1, l2).
* Controller (Eq. ck-h-final): h_new = 0.84 h (tol/Delta)^(1/5) after an accepted
  attempt, 0.84 h (tol/Delta)^(1/4) after a rejected one (which is repeated);
  h_new is clamped to [0.2 h, 5 h] and to [h_min, h_max]; the last step is cut to
  land on t_end.
* Mixed-step RK4 (Sec. 4.2): h1 while t < t_switch (the step that would cross
  t_switch is cut to land on it), h2 afterwards.
* Implicit Gauss-Legendre RK (two stages, order 4; Sec. 1 lists implicit and symplectic
  methods among the integrators for RT-CC without giving coefficients): the Gauss points and
  collocation matrix of [0, 1]; the coupled stage equations are solved by fixed-point iteration.
* Ground state: Jacobi updates t <- t + Omega/D, l <- l + R/D with
  D = f_ii(+f_jj) - f_aa(-f_bb) of the field-free Fock matrix, plus DIIS.
"""
from __future__ import annotations

from dataclasses import dataclass, field as dc_field
from fractions import Fraction as Fr

import numpy as np

from . import closed

# --- Butcher tableaus (exact rationals) ---------------------------------------------

RK4_TABLE = {
    "c": [Fr(0), Fr(1, 2), Fr(1, 2), Fr(1)],
    "a": [[], [Fr(1, 2)], [Fr(0), Fr(1, 2)], [Fr(0), Fr(0), Fr(1)]],
    "b": [Fr(1, 6), Fr(1, 3), Fr(1, 3), Fr(1, 6)],
}

CK_TABLE = {
    "c": [Fr(0), Fr(1, 5), Fr(3, 10), Fr(3, 5), Fr(1), Fr(7, 8)],
    "a": [[],
          [Fr(1, 5)],
          [Fr(3, 40), Fr(9, 40)],
          [Fr(3, 10), Fr(-9, 10), Fr(6, 5)],
          [Fr(-11, 54), Fr(5, 2), Fr(-70, 27), Fr(35, 27)],
          [Fr(1631, 55296), Fr(175, 512), Fr(575, 13824), Fr(44275, 110592), Fr(253, 4096)]],
    "b5": [Fr(37, 378), Fr(0), Fr(250, 621), Fr(125, 594), Fr(0), Fr(512, 1771)],
    "b4": [Fr(2825, 27648), Fr(0), Fr(18575, 48384), Fr(13525, 55296), Fr(277, 14336), Fr(1, 4)],
}


# Two-stage Gauss-Legendre collocation (implicit, order 4, A-stable and symplectic: the paper's
# "library of integrators", Sec. 1, names implicit and symplectic Runge-Kutta methods without
# coefficients).  Nodes are the Gauss points of [0, 1], c = 1/2 -+ sqrt(3)/6; A is the
# collocation matrix; b = (1/2, 1/2).  Irrational, so kept in floating point.
_SQ3_6 = np.sqrt(3.0) / 6.0
GL2_TABLE = {
    "c": [0.5 - _SQ3_6, 0.5 + _SQ3_6],
    "a": [[0.25, 0.25 - _SQ3_6], [0.25 + _SQ3_6, 0.25]],
    "b": [0.5, 0.5],
}


def as_float(tab):
    return {k: ([[float(x) for x in row] for row in v] if k == "a" else [float(x) for x in v])
            for k, v in tab.items()}


# --- field -----------------------------------------------------------------------------

@dataclass
class Field:
    E0: float = 0.01
    omega: float = 0.5
    sigma: float = 0.5
    t0: float = 1.0
    pol: tuple = (0.0, 0.0, 1.0)
    carrier: str = "sin"      # "sin" or "cos"
    sign: float = 1.0

    def amplitude(self, t):
        x = t - self.t0
        env = np.exp(-0.5 * x * x / (self.sigma * self.sigma))
        car = np.sin(self.omega * x) if self.carrier == "sin" else np.cos(self.omega * x)
        return self.sign * self.E0 * env * car

    def vector(self, t):
        return self.amplitude(t) * np.asarray(self.pol, dtype=float)


def fock_at(f, mu, fld: Field | None, t):
    if fld is None:
        return f
    e = fld.vector(t)
    return f - np.einsum("x,xpq->pq", e, mu)


# --- state packing -------------------------------------------------------------------

def pack(t1, t2, l1, l2):
    return np.concatenate([t1.ravel(), t2.ravel(), l1.ravel(), l2.ravel()]).astype(complex)


def unpack(y, o, v):
    n1, n2 = o * v, o * o * v * v
    t1 = y[:n1].reshape(o, v)
    t2 = y[n1:n1 + n2].reshape(o, o, v, v)
    l1 = y[n1 + n2:2 * n1 + n2].reshape(o, v)
    l2 = y[2 * n1 + n2:].reshape(o, o, v, v)
    return t1, t2, l1, l2


# --- RT-CC system ----------------------------------------------------------------------

class RTCC:
    def __init__(self, f, B, mu, o):
        self.f = np.asarray(f, float)
        self.mu = np.asarray(mu, float)
        self.o = o
        self.v = self.f.shape[0] - o
        self.V = closed.Integrals(B, o)

    def rhs(self, tt, y, fld):
        t1, t2, l1, l2 = unpack(y, self.o, self.v)
        ft = fock_at(self.f, self.mu, fld, tt)
        return pack(*closed.rhs(t1, t2, l1, l2, ft, self.V))

    def dipole(self, y):
        t1, t2, l1, l2 = unpack(y, self.o, self.v)
        return closed.dipole(t1, t2, l1, l2, self.mu, self.o)

    # -- ground state --------------------------------------------------------------
    def denominators(self):
        eo = np.diag(self.f)[:self.o]
        ev = np.diag(self.f)[self.o:]
        d1 = eo[:, None] - ev[None, :]
        d2 = eo[:, None, None, None] + eo[None, :, None, None] - ev[None, None, :, None] - ev[None, None, None, :]
        return d1, d2

    def ground_state(self, tol=1e-12, maxiter=200, ndiis=8):
        o, v = self.o, self.v
        d1, d2 = self.denominators()
        t1 = np.zeros((o, v), complex)
        t2 = np.zeros((o, o, v, v), complex)

        def solve(update, x1, x2):
            hist_x, hist_e = [], []
            for it in range(maxiter):
                r1, r2 = update(x1, x2)
                err = max(np.abs(r1).max(), np.abs(r2).max())
                if err < tol:
                    return x1, x2, it
                n1 = x1 + r1 / d1
                n2 = x2 + r2 / d2
                xv = np.concatenate([n1.ravel(), n2.ravel()])
                ev = np.concatenate([(r1 / d1).ravel(), (r2 / d2).ravel()])
                hist_x.append(xv)
                hist_e.append(ev)
                if len(hist_x) > ndiis:
                    hist_x.pop(0)
                    hist_e.pop(0)
                if len(hist_x) >= 3:
                    m = len(hist_x)
                    Bm = -np.ones((m + 1, m + 1), complex)
                    Bm[m, m] = 0
                    for a in range(m):
                        for b in range(m):
                            Bm[a, b] = np.vdot(hist_e[a], hist_e[b])
                    rhs = np.zeros(m + 1, complex)
                    rhs[m] = -1
                    try:
                        cvec = np.linalg.solve(Bm, rhs)[:m]
                        xv = sum(c * x for c, x in zip(cvec, hist_x))
                    except np.linalg.LinAlgError:
                        pass
                x1 = xv[:o * v].reshape(o, v)
                x2 = xv[o * v:].reshape(o, o, v, v)
                x2 = closed.sym_pair(x2)
            raise RuntimeError("ground state did not converge")

        t1, t2, nt = solve(lambda a, b: closed.omega(a, b, self.f, self.V)[:2], t1, t2)
        l1, l2, nl = solve(lambda a, b: closed.lambda_residual(t1, t2, a, b, self.f, self.V),
                           np.zeros_like(t1), np.zeros_like(t2))
        ecorr = closed.omega(t1, t2, self.f, self.V)[2]
        return pack(t1, t2, l1, l2), ecorr, (nt, nl)

    # -- integrators -----------------------------------------------------------------
    def stages(self, tab, tt, y, h, fld):
        ks = []
        for i, ci in enumerate(tab["c"]):
            ys = y.copy()
            for j, aij in enumerate(tab["a"][i]):
                if aij != 0.0:
                    ys = ys + h * aij * ks[j]
            ks.append(self.rhs(tt + ci * h, ys, fld))
        return ks

    def rk4_step(self, tt, y, h, fld):
        tab = as_float(RK4_TABLE)
        ks = self.stages(tab, tt, y, h, fld)
        return y + h * sum(b * k for b, k in zip(tab["b"], ks))

    def gl2_step(self, tt, y, h, fld, tol=1e-14, maxiter=200):
        """One Gauss-Legendre step: the stage derivatives K_i = f(t + c_i h, y + h sum_j a_ij K_j)
        (a fully implicit system) solved by fixed-point iteration from K_i = f(t, y)."""
        c, a, b = GL2_TABLE["c"], GL2_TABLE["a"], GL2_TABLE["b"]
        k0 = self.rhs(tt, y, fld)
        K = [k0.copy(), k0.copy()]
        for _ in range(maxiter):
            Kn = [self.rhs(tt + c[i] * h, y + h * (a[i][0] * K[0] + a[i][1] * K[1]), fld) for i in range(2)]
            delta = max(float(np.abs(Kn[i] - K[i]).max()) for i in range(2))
            K = Kn
            if delta <= tol * max(1.0, max(float(np.abs(k).max()) for k in K)):
                break
        else:
            raise RuntimeError("implicit stages did not converge")
        return y + h * (b[0] * K[0] + b[1] * K[1])

    def jacobian(self, tt, y, fld, step=0.1):
        """J = d rhs / d y at (tt, y), one column per unit vector by the five-point stencil in a
        complex scalar; exact up to rounding because the right-hand side is a polynomial of degree
        at most four in y (and holomorphic: no conjugates)."""
        n = y.size
        J = np.empty((n, n), dtype=complex)
        for k in range(n):
            e = np.zeros(n, dtype=complex)
            e[k] = step
            J[:, k] = (self.rhs(tt, y - 2 * e, fld) - 8 * self.rhs(tt, y - e, fld) + 8 * self.rhs(tt, y + e, fld)
                       - self.rhs(tt, y + 2 * e, fld)) / (12 * step)
        return J

    def gl2_step_newton(self, tt, y, h, fld, tol=1e-13, maxiter=30, return_stages=False):
        """The same collocation system as gl2_step, K_i = f(t + c_i h, y + h sum_j a_ij K_j), solved
        by Newton's method: G_i(K) = K_i - f(...) with the exact Jacobian dG_i/dK_j = delta_ij -
        h a_ij J(t + c_i h, Y_i) and a dense solve per iteration.  Converges for steps where the
        fixed-point iteration diverges."""
        c, a, b = GL2_TABLE["c"], GL2_TABLE["a"], GL2_TABLE["b"]
        k0 = self.rhs(tt, y, fld)
        K = [k0.copy(), k0.copy()]
        n = y.size
        for _ in range(maxiter):
            Y = [y + h * (a[i][0] * K[0] + a[i][1] * K[1]) for i in range(2)]
            G = [K[i] - self.rhs(tt + c[i] * h, Y[i], fld) for i in range(2)]
            if max(float(np.abs(g).max()) for g in G) <= tol * max(1.0, max(float(np.abs(k).max()) for k in K)):
                y1 = y + h * (b[0] * K[0] + b[1] * K[1])
                return (y1, K) if return_stages else y1
            J = [self.jacobian(tt + c[i] * h, Y[i], fld) for i in range(2)]
            M = np.zeros((2 * n, 2 * n), dtype=complex)
            for i in range(2):
                for j in range(2):
                    M[i * n:(i + 1) * n, j * n:(j + 1) * n] = (np.eye(n) if i == j else 0) - h * a[i][j] * J[i]
            d = np.linalg.solve(M, -np.concatenate(G))
            K = [K[0] + d[:n], K[1] + d[n:]]
        raise RuntimeError("Newton iterations of the implicit stages did not converge")

    def ck_attempt(self, tt, y, h, fld):
        tab = as_float(CK_TABLE)
        ks = self.stages(tab, tt, y, h, fld)
        y5 = y + h * sum(b * k for b, k in zip(tab["b5"], ks))
        y4 = y + h * sum(b * k for b, k in zip(tab["b4"], ks))
        return y5, float(np.abs(y5 - y4).max())


@dataclass
class Integrator:
    method: str = "rk4"          # "rk4", "ck", "mixed", "gl2" (implicit Gauss-Legendre, fixed point),
                                 # "gl2n" (the same, Newton)
    h: float = 0.05
    h1: float = 0.005
    h2: float = 0.05
    t_switch: float = 0.0
    tol: float = 1e-6
    safety: float = 0.84
    h_min: float = 1e-9
    h_max: float = 1.0
    max_rejects: int = 50
    nsteps: int = 0              # rk4/mixed: number of steps if > 0, else run to t_end
    t_end: float = 0.0


def ck_controller(h, delta, tol, safety=0.84, h_min=1e-9, h_max=1.0):
    """Returns (accept, h_new) per Eq. ck-h-final with clamping to [0.2h, 5h] and [h_min, h_max]."""
    accept = delta <= tol
    if delta == 0.0:
        fac = 5.0
    else:
        fac = safety * (tol / delta) ** (0.2 if accept else 0.25)
    fac = min(5.0, max(0.2, fac))
    return accept, min(h_max, max(h_min, h * fac))


def propagate(sys: RTCC, y0, fld: Field, integ: Integrator, t_start=0.0):
    """Returns (times, dipoles[n,3] complex, final y, stats) with a sample at t_start."""
    tt, y = t_start, y0.copy()
    times, mus = [tt], [sys.dipole(y)]
    stats = {"accepted": 0, "rejected": 0, "rhs_evals": 0}
    eps = 1e-12
    if integ.method in ("rk4", "mixed", "gl2", "gl2n"):
        step = 0
        while True:
            if integ.nsteps > 0 and step >= integ.nsteps:
                break
            if integ.nsteps <= 0 and tt >= integ.t_end - eps:
                break
            if integ.method in ("rk4", "gl2", "gl2n"):
                h = integ.h
            else:
                h = integ.h1 if tt < integ.t_switch - eps else integ.h2
                if tt < integ.t_switch - eps:
                    h = min(h, integ.t_switch - tt)
            if integ.nsteps <= 0:
                h = min(h, integ.t_end - tt)
            if integ.method == "gl2":
                y = sys.gl2_step(tt, y, h, fld)
            elif integ.method == "gl2n":
                y = sys.gl2_step_newton(tt, y, h, fld)
            else:
                y = sys.rk4_step(tt, y, h, fld)
            tt = tt + h
            step += 1
            stats["accepted"] += 1
            stats["rhs_evals"] += 4
            times.append(tt)
            mus.append(sys.dipole(y))
    elif integ.method == "ck":
        h = integ.h
        rejects = 0
        while tt < integ.t_end - eps:
            hs = min(h, integ.t_end - tt)
            y5, delta = sys.ck_attempt(tt, y, hs, fld)
            stats["rhs_evals"] += 6
            accept, hn = ck_controller(hs, delta, integ.tol, integ.safety, integ.h_min, integ.h_max)
            if accept:
                y, tt = y5, tt + hs
                times.append(tt)
                mus.append(sys.dipole(y))
                stats["accepted"] += 1
                rejects = 0
            else:
                stats["rejected"] += 1
                rejects += 1
                if rejects > integ.max_rejects or hn <= integ.h_min:
                    raise RuntimeError("step size underflow")
            h = hn
    else:
        raise ValueError(integ.method)
    return np.array(times), np.array(mus), y, stats
