"""Algorithmic floating-point work of one right-hand-side evaluation, counted term by term.

Test infrastructure only: nothing on the product path imports this module.  A committed
script (tests/golden/make_rhs_flops.py) writes its per-term table to a JSON file that the
benchmark reads for the roofline's algorithmic flops.

What is counted: the closed-shell oracle's einsum program (oracle/closed.py) for the ket
residual Omega (Eq. derivT) and, by its reverse sweep, the bra residual R = dL/dt (Eq. derivL)
of one trajectory.  A two-operand einsum C = A B over the label set S is prod_{l in S} n_l
products, counted as numpy's einsum_path counts real flops (2 per product when a label is
summed, a multiply and an add; 1 for an outer product), times the real products per complex
one: 1 between real operands, 2 when one operand is complex, 4 when both are.  One-operand
permutations and linear combinations move data and cost no flops.  Each label's extent is
either o or v, so a term costs c * o^p * v^q flops; the table keeps (c, p, q) per term and
evaluates at any shape.

The count is that of the plain program, with no symmetry used: the particle-particle ladder
over all (e, f), both operands of every product differentiated where they depend on t.
Kernels that exploit a symmetry (the pair-symmetric ladder) execute fewer flops than this.
"""
from __future__ import annotations

import numpy as np

from oracle import closed


class CountingTape(closed.Tape):
    """A Tape that records, for every einsum it evaluates (forward, and each vector-Jacobian
    product when `grad` runs it), the subscripts, the extent of every label, and the complex
    factor of the real multiply-adds."""

    def __init__(self):
        super().__init__()
        self.records = []

    def _record(self, subs, vals, phase):
        ins, _ = subs.split("->")
        terms = ins.split(",")
        if len(terms) < 2:
            return
        ext = {}
        for t, x in zip(terms, vals):
            for lab, n in zip(t, np.shape(x)):
                ext[lab] = n
        ncplx = sum(1 for x in vals if np.iscomplexobj(x) and np.any(np.imag(x) != 0))
        cfac = {0: 1, 1: 2, 2: 4}[min(ncplx, 2)]
        inner = any(lab not in subs.split("->")[1] for lab in ext)
        self.records.append({"subs": subs, "ext": ext, "cfac": cfac, "phase": phase, "inner": inner,
                             "shapes": [np.shape(x) for x in vals]})

    def ein(self, subs, *ops, alpha=1.0):
        vals = [self._val(x) for x in ops]
        self._record(subs, vals, "omega")
        node = super().ein(subs, *ops, alpha=alpha)
        # wrap the vector-Jacobian products so that their einsums are counted when they run
        ins, out = subs.split("->")
        in_list = ins.split(",")
        wrapped = []
        nodes = [k for k, x in enumerate(ops) if isinstance(x, closed.Node)]
        for (pidx, vjp), k in zip(node.parents, nodes):
            others = [(in_list[m], vals[m]) for m in range(len(ops)) if m != k]
            sub_k = ",".join([out] + [s for s, _ in others]) + "->" + in_list[k]

            def counted(gout, vjp=vjp, sub_k=sub_k, ovals=[v for _, v in others]):
                self._record(sub_k, [gout] + ovals, "lambda")
                return vjp(gout)

            wrapped.append((pidx, counted))
        node.parents = wrapped
        return node


def term_table(o=2, v=3, seed=5):
    """Per-term records of one Omega + R evaluation at a shape where o != v, each label
    classified as occupied or virtual by its extent: [(subs, phase, c, p, q)], the term costing
    c * o^p * v^q real flops (c = complex factor x 2 for a contraction, x 1 for an outer product)."""
    assert o != v
    rows = []
    for r in records(o, v, seed):
        p = sum(1 for n in r["ext"].values() if n == o)
        q = sum(1 for n in r["ext"].values() if n == v)
        assert p + q == len(r["ext"]), r
        rows.append((r["subs"], r["phase"], r["cfac"] * (2 if r["inner"] else 1), p, q))
    return rows


def records(o=2, v=3, seed=5):
    """The raw records of term_table (subscripts, label extents, operand shapes, factors)."""
    from paper_2205_05175_gb300 import synth
    f, B, _ = synth.make_system(o, v, seed=seed)
    f = f + synth.random_symmetric(synth.rng_for(seed + 1), o + v, 0.05)
    t1, t2 = synth.random_amplitudes(o, v, seed=seed + 2, s1=0.1, s2=0.1)
    l1, l2 = synth.random_amplitudes(o, v, seed=seed + 3, s1=0.1, s2=0.1)
    tp = CountingTape()
    n1, n2 = tp.var(t1), tp.var(t2)
    o1, o2, e = closed.residual_program(tp, n1, n2, f, closed.Integrals(B, o))
    tp.grad([(e, 1.0), (o1, l1), (o2, l2)], [n1, n2])
    return tp.records


def rhs_flops(o, v, table=None):
    """Real flops of one Omega + R evaluation of one trajectory at shape (o, v), split by phase
    and by scaling class."""
    rows = term_table() if table is None else table
    out = {"omega": 0.0, "lambda": 0.0, "o2v4": 0.0, "o3v3": 0.0, "other": 0.0}
    for _, phase, c, p, q in rows:
        fl = c * float(o) ** p * float(v) ** q
        out[phase] += fl
        key = "o2v4" if (p, q) == (2, 4) else ("o3v3" if (p, q) == (3, 3) else "other")
        out[key] += fl
    out["total"] = out["omega"] + out["lambda"]
    return out
