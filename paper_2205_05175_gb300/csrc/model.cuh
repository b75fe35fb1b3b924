// RT-CCSD model programs built on the contraction engine.
#pragma once
#include "engine.cuh"

namespace rtcc {

// Physicist integral blocks <pq|rs> = (pr|qs) (float64, device, contiguous) and the
// exchange combinations L = 2<..> - <..> that the closed-shell equations use.
struct IntegralStore {
  int o = 0, v = 0, naux = 0;
  double* blk[16] = {nullptr};
  enum Blk { OOOO, OOOV, OOVO, OOVV, OVOV, OVVO, OVOO, OVVV, VVVO, VVVV, LOVVV, LOOVV, LOOOV, LOVVO, LOOVO, NBLK };
  std::vector<void*> owned;
  size_t bytes = 0;
  ~IntegralStore();
};

// Builds every block on the device from density-fitting factors B[naux][nmo][nmo]
// (device pointer) with a float64 setup program.
void build_integrals(IntegralStore& S, const double* dB, int naux, int o, int v, cudaStream_t stream);

// Tensor ids of the integral blocks registered in one engine.
struct IntIds {
  int b[IntegralStore::NBLK];
};
IntIds register_integrals(Engine& E, const IntegralStore& S);

// Closed-shell RT-CCSD right-hand side over nz trajectories:
//   fwd : Omega1/Omega2 of the state views (t1,t2) written into the output views
//   rev : R = d/dt [E + l.Omega] (l1, l2 views), doubles symmetrised, into the output views
// The state buffer is [nz][ns] complex, the Fock buffer [nz][nmo][nmo] real, the output
// buffer [nz][ns] complex (Omega1 | Omega2 | R1 | R2 in the state layout).
struct RhsPrograms {
  Program fwd, rev;
  int t1, t2, l1, l2;      // input views
  int foo, fov, fvv;       // Fock views
  int r1, r2, rl1, rl2;    // output views
  int tau;                 // tau intermediate (used by the energy program)
  int fwd_arena = -1, rev_arena = -1;   // arenas of the intermediates and of the reverse sweep
};
// fwd_arena / rev_arena >= 0 reuse those arenas from their start (programs of several batch sizes
// over the same buffers share them); -1 creates new ones.
RhsPrograms build_rhs(Engine& E, const IntIds& I, int nz, int o, int v, double* state, double* fock,
                      double* out, bool with_lambda, int fwd_arena = -1, int rev_arena = -1);

// Dipole of the state views: for each component x, mu_xz = E[mu_x] + l.Omega[mu_x]
// (one-body programs; the reference term 2 sum_i mu_ii is added by the caller).
struct DipolePrograms {
  Program prog;
  double* fdummy = nullptr;   // placeholder operator buffer (owned by the caller's allocation list)
  int y1, y2, y3, y4;          // state views (t1, t2, l1, l2)
  int dip;                     // output [3][nz]
  int fwd_arena = -1, rev_arena = -1;
};
DipolePrograms build_dipole(Engine& E, int nz, int o, int v, double* state, const double* mu_dev,
                            double* dip_out, int fwd_arena = -1, int rev_arena = -1);

// Vector-Jacobian product of one right-hand-side evaluation (the programs in R, last run on
// the state in R's input buffer): given the cotangent `cot` of the raw output (Omega | R) in the
// state layout, accumulate ybar = (dOut/dy)^T cot (state layout) and fbar = (dOut/df)^T cot
// (Fock layout [nz][nmo][nmo], oo/ov/vv blocks).  Holomorphic: no conjugation.
Program build_rhs_vjp(Engine& E, const RhsPrograms& R, int nz, int o, int v, double* cot, double* ybar,
                      double* fbar);

// Vector-Jacobian product of the dipole program D (last run on its state buffer): given weights
// wdip[3][nz] (complex) of the dipole components, ybar += (d mu / dy)^T w (state layout).
Program build_dipole_vjp(Engine& E, const DipolePrograms& D, int nz, int o, int v, double* wdip, double* ybar);

// Correlation energy E = 2 sum f_ia t_ia + sum L_ijab tau_ijab (after `fwd` has run).
Program build_energy(Engine& E, const IntIds& I, const RhsPrograms& R, int nz, int o, int v, double* fock,
                     double* e_out);

}  // namespace rtcc
