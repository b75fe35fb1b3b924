"""O2: closed-shell (spin-adapted) RT-CCSD right-hand side, energy and dipole.

Test infrastructure only: the product path never imports, calls or links this
module; only tests, the smoke check and the benchmark's CPU-baseline leg do.

What is computed (all complex128, plain NumPy einsum, no blocking or fusion):

* ``omega``: the closed-shell ket residual Omega(t) = <mu~|e^{-T} H(t) e^{T}|0>
  (Eq. derivT), with Omega1[i,a] the (i alpha -> a alpha) component and
  Omega2[i,j,a,b] the (i alpha j beta -> a alpha b beta) component of the
  spin-orbital residual, so that i dt/dt = Omega holds component-wise.  The
  expressions are the spin integration of the Stanton-Gauss spin-orbital
  equations (see ``oracle/spinorb.py``) with the full field-dressed Fock matrix.
* ``lambda_residual``: R(t, l) = <0|(1+Lambda)[Hbar, tau_mu]|0> (Eq. derivL).
  Because d Hbar / d t_mu = [Hbar, tau_mu], R is the holomorphic gradient of the
  Lagrangian  L(t, l) = E(t) + l1.Omega1(t) + l2.Omega2(t)  with respect to t
  (doubles gradient symmetrised over the (ia)<->(jb) pair), where the
  multipliers l are paired with Omega by a plain dot product.  The gradient is
  taken by exact reverse-mode differentiation of the einsum program below
  (class ``Tape``), so no separate Lambda equations are transcribed.
* ``dipole``: mu_x(t) = <0|(1+Lambda) e^{-T} mu_x e^{T}|0> (Eq. dipole) =
  2 sum_i mu_ii + E[mu](t) + l.Omega[mu](t), i.e. the Lagrangian evaluated with
  the one-body operator mu_x in place of f and no two-electron part.
* ``rhs``: the propagated vector field of Eq. IVP: dt/dt = -i Omega,
  dl/dt = +i R.

Integrals: (pq|rs) = sum_P B[P,p,q] B[P,r,s]; physicist v[p,q,r,s] = <pq|rs> = (pr|qs).
"""
from __future__ import annotations

import numpy as np


# --- a minimal reverse-mode tape over einsum ---------------------------------------

class Node:
    __slots__ = ("value", "parents", "idx")

    def __init__(self, value, parents, idx):
        self.value, self.parents, self.idx = value, parents, idx


class Tape:
    """Records einsum / linear-combination nodes; `grad` runs them backwards.

    For C = alpha * einsum('A,B->C', a, b) the adjoints are
    da += alpha * einsum('C,B->A', dC, b) and db += alpha * einsum('A,C->B', a, dC)
    (holomorphic: no conjugation).  Every label of an operand must appear in the
    output or in the other operand.
    """

    def __init__(self):
        self.nodes = []

    def var(self, value):
        n = Node(np.asarray(value, dtype=complex), [], len(self.nodes))
        self.nodes.append(n)
        return n

    @staticmethod
    def _val(x):
        return x.value if isinstance(x, Node) else x

    def ein(self, subs, *ops, alpha=1.0):
        ins, out = subs.split("->")
        in_list = ins.split(",")
        vals = [self._val(x) for x in ops]
        value = alpha * np.einsum(subs, *vals, optimize=True)
        parents = []
        for k, x in enumerate(ops):
            if not isinstance(x, Node):
                continue
            others = [(in_list[m], vals[m]) for m in range(len(ops)) if m != k]
            sub_k = ",".join([out] + [s for s, _ in others]) + "->" + in_list[k]
            ovals = [v for _, v in others]

            def vjp(gout, sub_k=sub_k, ovals=ovals):
                return alpha * np.einsum(sub_k, gout, *ovals, optimize=True)

            parents.append((x.idx, vjp))
        n = Node(np.asarray(value, dtype=complex), parents, len(self.nodes))
        self.nodes.append(n)
        return n

    def lin(self, *terms):
        """sum of coef * x over (coef, x) pairs; x a Node or a constant array."""
        value = 0
        parents = []
        for c, x in terms:
            value = value + c * self._val(x)
            if isinstance(x, Node):
                parents.append((x.idx, lambda gout, c=c: c * gout))
        n = Node(np.asarray(value, dtype=complex), parents, len(self.nodes))
        self.nodes.append(n)
        return n

    def grad(self, seeds, wrt):
        g = {}
        for node, s in seeds:
            g[node.idx] = g.get(node.idx, 0) + s
        for n in reversed(self.nodes):
            gn = g.get(n.idx)
            if gn is None:
                continue
            for pidx, vjp in n.parents:
                g[pidx] = g.get(pidx, 0) + vjp(gn)
        return [np.asarray(g.get(x.idx, np.zeros_like(x.value))) for x in wrt]


# --- integrals -------------------------------------------------------------------------

class Integrals:
    """Physicist blocks <pq|rs> built on demand from density-fitting factors."""

    def __init__(self, B, o):
        self.B = np.asarray(B, dtype=float)
        self.o = o
        self.nmo = self.B.shape[1]
        self._cache = {}

    def _sl(self, c):
        return slice(0, self.o) if c == "o" else slice(self.o, self.nmo)

    def __call__(self, blk):
        if blk not in self._cache:
            p, q, r, s = (self._sl(c) for c in blk)
            # <pq|rs> = (pr|qs)
            self._cache[blk] = np.einsum("Ppr,Pqs->pqrs", self.B[:, p, r], self.B[:, q, s], optimize=True)
        return self._cache[blk]


def zero_integrals(o, nmo):
    class _Zero:
        def __init__(self):
            self.o, self.nmo = o, nmo

        def __call__(self, blk):
            dims = [o if c == "o" else nmo - o for c in blk]
            return np.zeros(dims)
    return _Zero()


# --- the closed-shell residual program -------------------------------------------------

def residual_program(tp: Tape, t1, t2, f, V, onebody_only=False):
    """Build Omega1, Omega2 and E_corr on tape `tp` for the closed-shell CCSD ket equations.

    t1 (o,v), t2 (o,o,v,v) are tape nodes; f is the (nmo,nmo) one-body operator
    (Fock matrix, or a dipole matrix when evaluating E[mu], Omega[mu]); V gives the
    physicist integral blocks.  With onebody_only the two-electron terms are skipped
    (they are identically zero for a one-body operator).
    """
    o = t1.value.shape[0]
    fov, foo, fvv = f[:o, o:], f[:o, :o], f[o:, o:]
    E = tp.ein
    two = not onebody_only

    tt = E("ia,jb->ijab", t1, t1)
    tau = tp.lin((1.0, t2), (1.0, tt))
    taut = tp.lin((1.0, t2), (0.5, tt))

    # one-body intermediates
    fae = [(1.0, fvv), (-0.5, E("me,ma->ae", fov, t1))]
    fmi = [(1.0, foo), (0.5, E("ie,me->mi", t1, fov))]
    fme = [(1.0, fov)]
    if two:
        Lovvv = 2.0 * V("ovvv") - V("ovvv").transpose(0, 1, 3, 2)      # L_mafe = 2<ma|fe> - <ma|ef>
        Loovv = 2.0 * V("oovv") - V("oovv").transpose(0, 1, 3, 2)      # L_mnef = 2<mn|ef> - <mn|fe>
        Looov = 2.0 * V("ooov") - V("oovo").transpose(0, 1, 3, 2)      # L_mnie = 2<mn|ie> - <mn|ei>
        fae += [(1.0, E("mf,mafe->ae", t1, Lovvv)), (-1.0, E("mnaf,mnef->ae", taut, Loovv))]
        fmi += [(1.0, E("ne,mnie->mi", t1, Looov)), (1.0, E("inef,mnef->mi", taut, Loovv))]
        fme += [(1.0, E("nf,mnef->me", t1, Loovv))]
    Fae, Fmi, Fme = tp.lin(*fae), tp.lin(*fmi), tp.lin(*fme)

    # singles
    t2t = tp.lin((2.0, t2), (-1.0, E("imea->imae", t2)))                # 2 t_imae - t_imea
    r1 = [(1.0, fov), (1.0, E("ie,ae->ia", t1, Fae)), (-1.0, E("ma,mi->ia", t1, Fmi)),
          (1.0, E("imae,me->ia", t2t, Fme))]
    if two:
        Lovvo = 2.0 * V("ovvo") - V("ovov").transpose(0, 1, 3, 2)      # 2<na|fi> - <na|if>
        Loovo = 2.0 * V("oovo") - V("ooov").transpose(0, 1, 3, 2)      # 2<nm|ei> - <nm|ie>
        r1 += [(1.0, E("nf,nafi->ia", t1, Lovvo)), (1.0, E("imef,mafe->ia", t2, Lovvv)),
               (-1.0, E("mnae,nmei->ia", t2, Loovo))]
    Om1 = tp.lin(*r1)

    # doubles: Omega2 = S + S^(ij,ab swapped), S collects every term
    Xbe = tp.lin((1.0, Fae), (-0.5, E("mb,me->be", t1, Fme)))
    Zmj = tp.lin((1.0, Fmi), (0.5, E("je,me->mj", t1, Fme)))
    s = [(1.0, E("ijae,be->ijab", t2, Xbe)), (-1.0, E("imab,mj->ijab", t2, Zmj))]
    if two:
        voovv = V("oovv")
        # particle-particle ladder and hole-hole ladder (symmetric; half goes into S)
        lad = E("ijef,abef->ijab", tau, V("vvvv"))
        Wmnij = tp.lin((1.0, V("oooo")), (1.0, E("je,mnie->mnij", t1, V("ooov"))),
                       (1.0, E("ie,mnej->mnij", t1, V("oovo"))), (1.0, E("ijef,mnef->mnij", tau, voovv)))
        hh = E("mnab,mnij->ijab", tau, Wmnij)
        # t1-corrections of the ladder: Z_ijmb = sum_ef tau_ijef <mb|ef>
        Zijmb = E("ijef,mbef->ijmb", tau, V("ovvv"))
        # ring intermediates: the (m alpha b beta e alpha j beta) and (m alpha b beta e beta j alpha) blocks of W_mbej
        t1t1 = E("jf,nb->jnfb", t1, t1)
        Wa = tp.lin((1.0, V("ovvo")), (1.0, E("jf,mbef->mbej", t1, V("ovvv"))),
                    (-1.0, E("nb,mnej->mbej", t1, V("oovo"))), (-1.0, E("jnfb,mnef->mbej", t1t1, voovv)),
                    (0.5, E("jnbf,mnef->mbej", t2, Loovv)), (-0.5, E("jnfb,mnef->mbej", t2, voovv)))
        U = tp.lin((-1.0, V("ovov").transpose(0, 1, 3, 2)), (-1.0, E("jf,mbfe->mbej", t1, V("ovvv"))),
                   (1.0, E("nb,mnje->mbej", t1, V("ooov"))),
                   (1.0, E("jnfb,mnfe->mbej", tp.lin((0.5, t2), (1.0, t1t1)), voovv)))
        s += [(0.5, voovv), (0.5, lad), (0.5, hh),
              (-1.0, E("ma,ijmb->ijab", t1, Zijmb)),
              (1.0, E("imae,mbej->ijab", t2t, Wa)), (1.0, E("imae,mbej->ijab", t2, U)),
              (1.0, E("mjae,mbei->ijab", t2, U)),
              (-1.0, E("ma,mbij->ijab", t1, E("ie,mbej->mbij", t1, V("ovvo")))),
              (-1.0, E("ma,mbji->ijab", t1, E("je,mbie->mbji", t1, V("ovov")))),
              (1.0, E("ie,abej->ijab", t1, V("vvvo"))),
              (-1.0, E("ma,mbij->ijab", t1, V("ovoo")))]
    S = tp.lin(*s)
    Om2 = tp.lin((1.0, S), (1.0, E("jiba->ijab", S)))

    # correlation energy E = 2 sum f_ia t_ia + sum (2<ij|ab> - <ij|ba>) tau_ijab
    e = [(2.0, E("ia,ia->", fov, t1))]
    if two:
        e += [(1.0, E("ijab,ijab->", Loovv, tau))]
    En = tp.lin(*e)
    return Om1, Om2, En


def _run(t1, t2, f, V, onebody_only=False):
    tp = Tape()
    n1, n2 = tp.var(t1), tp.var(t2)
    o1, o2, e = residual_program(tp, n1, n2, f, V, onebody_only)
    return tp, (n1, n2), (o1, o2, e)


def omega(t1, t2, f, V):
    """Closed-shell ket residual (Omega1, Omega2) and correlation energy."""
    _, _, (o1, o2, e) = _run(t1, t2, f, V)
    return o1.value, o2.value, complex(e.value)


def sym_pair(x2):
    return 0.5 * (x2 + x2.transpose(1, 0, 3, 2))


def lambda_residual(t1, t2, l1, l2, f, V):
    """R(t, l) = d/dt [E + l.Omega] (holomorphic), doubles symmetrised over (ia)<->(jb)."""
    tp, (n1, n2), (o1, o2, e) = _run(t1, t2, f, V)
    g1, g2 = tp.grad([(e, 1.0), (o1, l1), (o2, l2)], [n1, n2])
    return g1, sym_pair(g2)


def lagrangian(t1, t2, l1, l2, f, V):
    o1, o2, e = omega(t1, t2, f, V)
    return e + np.sum(l1 * o1) + np.sum(l2 * o2)


def dipole(t1, t2, l1, l2, mu, o):
    """mu_x = 2 sum_i mu_ii + E[mu_x] + l.Omega[mu_x] for x = 0,1,2 (complex)."""
    out = np.zeros(3, complex)
    V0 = zero_integrals(o, mu.shape[1])
    for x in range(3):
        _, _, (o1, o2, e) = _run(t1, t2, mu[x], V0, onebody_only=True)
        out[x] = 2.0 * np.trace(mu[x][:o, :o]) + e.value + np.sum(l1 * o1.value) + np.sum(l2 * o2.value)
    return out


def rhs(t1, t2, l1, l2, f, V):
    """Right-hand side of the RT-CC equations of motion (Eqs. derivT, derivL):
    dt/dt = -i Omega(t),  dl/dt = +i R(t, l)."""
    o1, o2, _ = omega(t1, t2, f, V)
    r1, r2 = lambda_residual(t1, t2, l1, l2, f, V)
    return -1j * o1, -1j * o2, 1j * r1, 1j * r2
