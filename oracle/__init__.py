"""CPU reference (oracle) for the RT-CCSD hot path — TEST INFRASTRUCTURE ONLY.

Plain, slow, FP64/complex128 NumPy code written from the paper's definitions
(Eqs. derivT, derivL, simtranH, dipole, rk_y/rk_k, rk4truncation, ck-k/ck-y,
ck-h-final, field).  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it.  The CUDA path shares no code with
it: the only common module is the seeded input generator
``paper_2205_05175_gb300.synth``, which holds none of the method's arithmetic.

Modules and their pins (tests/test_oracle_pins.py):
  brute     O0  determinant-space definitions (pins everything below)
  spinorb   O1  spin-orbital CCSD residual         <- brute force
  closed    O2  closed-shell residual, Lambda, dipole <- spinorb, brute force, 5-point identity
  rk        O3  field, tableaus, controller, ground state, propagation <- printed values,
                exact order conditions, h^4 scaling, two-electron FCI, zero-field stationarity
  fci           exact two-electron dynamics and the CC Jacobian
  spectrum      spline, DFT spectrum, matrix pencil <- closed forms
"""
