"""Writes gl2n_o2v6_h04.json: a dipole record of the implicit two-stage Gauss-Legendre method at a
step where fixed-point iteration of its stage equations diverges, from the oracle's dense Newton
solve (oracle/rk.py gl2_step_newton), for the device's Newton-Krylov integrator to be compared
against without re-running the (minutes-long) dense solve.

System: o = 2, v = 6 from the seeded generator (seed SEED_BASE), the oracle's ground state as the
initial state (stored), sine pulse E0 = 0.05, omega = 0.5, sigma = 0.5, t0 = 0.5 along z, h = 0.4,
three steps.  Calls only oracle/ (and the seeded input generator).
Usage: python tests/golden/make_gl2n_reference.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import rk  # noqa: E402
from paper_2205_05175_gb300 import synth  # noqa: E402

O, V, H, NSTEPS = 2, 6, 0.4, 3
FIELD = dict(E0=0.05, omega=0.5, sigma=0.5, t0=0.5)


def main():
    f, B, mu = synth.make_system(O, V, seed=synth.SEED_BASE)
    s = rk.RTCC(f, B, mu, O)
    y0, _, _ = s.ground_state(tol=1e-12)
    tt, mm, _, _ = rk.propagate(s, y0, rk.Field(**FIELD), rk.Integrator(method="gl2n", h=H, nsteps=NSTEPS))
    doc = {"what": "implicit two-stage Gauss-Legendre (stages by dense Newton) dipole record beyond the "
                   "fixed-point limit; mu[k] = [Re mu_x, Im mu_x, Re mu_y, Im mu_y, Re mu_z, Im mu_z] at t[k]",
           "source": "oracle/rk.py propagate(method='gl2n') from oracle ground_state(tol=1e-12)",
           "o": O, "v": V, "h": H, "nsteps": NSTEPS, "field": FIELD, "seed": synth.SEED_BASE,
           "y0": [[float(z.real), float(z.imag)] for z in y0],
           "t": [float(x) for x in tt],
           "mu": [[float(c) for z in row for c in (z.real, z.imag)] for row in mm]}
    with open(os.path.join(HERE, "gl2n_o2v6_h04.json"), "w") as fh:
        json.dump(doc, fh)
        fh.write("\n")


if __name__ == "__main__":
    main()
