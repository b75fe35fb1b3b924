"""Writes rhs_flops.json: the per-term flop table of one right-hand-side evaluation (Omega by
Eq. derivT and R by Eq. derivL, one trajectory) from the oracle's counter (oracle/flops.py).

Each row is [subscripts, phase, c, p, q]: the term costs c * o^p * v^q real flops.  The benchmark
evaluates the table at its shape for the roofline's algorithmic flops.  Calls only oracle/.
Usage: python tests/golden/make_rhs_flops.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import flops  # noqa: E402


def main():
    rows = flops.term_table()
    at = {f"{o},{v}": flops.rhs_flops(o, v, rows) for o, v in ((5, 19), (10, 38), (20, 76), (30, 114))}
    doc = {"what": "real flops of one Omega + R evaluation of one trajectory, per einsum term of the oracle's "
                   "program (forward terms: phase omega; reverse sweep: phase lambda); term cost c * o^p * v^q",
           "source": "oracle/flops.py term_table(o=2, v=3)",
           "rows": [list(r) for r in rows], "totals": at}
    with open(os.path.join(HERE, "rhs_flops.json"), "w") as fh:
        json.dump(doc, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()
