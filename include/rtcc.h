/*
 * rtcc.h — C-ABI of the GB300 (sm_103a) real-time CCSD propagation library.
 *
 * The library evaluates the closed-shell RT-CCSD equations of motion
 *     i dt_mu/dt      = <mu| e^{-T} H(t) e^{T} |0>            (Sec. 2, Eq. derivT)
 *    -i dlambda_mu/dt = <0|(1+Lambda)[Hbar(t), tau_mu]|0>      (Sec. 2, Eq. derivL)
 * with H(t) = H0 - mu.E(t) in frozen molecular orbitals (Sec. 2.2), propagates them
 * with Runge-Kutta integrators (Sec. 2.1 Eqs. rk_y/rk_k; Sec. 4.2 RK4, Cash-Karp
 * Eqs. ck-k/ck-y/ck-h-final, mixed-step RK4; the implicit two-stage Gauss-Legendre method
 * from the integrator library of Sec. 1) and records the dipole
 * mu_x(t) = <0|(1+Lambda) e^{-T} mu_x e^{T}|0> (Sec. 2.2, Eq. dipole), from which it forms
 * absorption spectra by a direct transform or a Pade-accelerated one (Sec. 2.2; Sec. 1).
 *
 * Conventions shared by every call
 *  - Orbitals are ordered occupied (o) then virtual (v); nmo = o + v.
 *  - Matrices are row-major float64.  Complex numbers are interleaved (re, im) float64.
 *  - One "state" of a trajectory is the complex vector
 *        y = [ t1[o][v] | t2[o][o][v][v] | l1[o][v] | l2[o][o][v][v] ]
 *    of length rtcc_state_size(); t2 and l2 obey x[i][j][a][b] == x[j][i][b][a].
 *    t2[i][j][a][b] is the (i alpha, j beta -> a alpha, b beta) amplitude; the
 *    multipliers l are paired with the residual by a plain (unconjugated) dot product.
 *  - A handle holds ntraj independent trajectories that share one integral set and
 *    are stacked into the same GEMMs.
 *  - Ownership: the caller owns every buffer it passes.  The library copies inputs on
 *    entry and keeps no caller pointer after a call returns.  Output buffers are
 *    caller-allocated.  Pointers documented "host or device" may be either; the
 *    library inspects them with cudaPointerGetAttributes.
 *  - A handle is bound to the CUDA device that was current at rtcc_create and to a
 *    stream owned by the library; it is not thread-safe.  Every call is synchronous
 *    with respect to the host unless stated otherwise.
 *  - Errors: every call returns an rtcc_status_t; rtcc_last_error() returns a
 *    thread-local message describing the most recent failure.  No call aborts the
 *    process.  There is no CPU fallback: without a usable sm_103a GPU, rtcc_create
 *    returns RTCC_ERR_CUDA.
 */
#ifndef RTCC_H
#define RTCC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RTCC_OK = 0,
    RTCC_ERR_INVALID_ARG = 1,   /* bad size, null pointer, asymmetric input, unknown enum */
    RTCC_ERR_OOM = 2,           /* device allocation failed */
    RTCC_ERR_CUDA = 3,          /* CUDA runtime/driver error (no device, launch failure) */
    RTCC_ERR_NOCONV = 4,        /* ground-state iterations or implicit stage sweeps did not converge */
    RTCC_ERR_DIVERGED = 5,      /* NaN/Inf or norm blow-up in a propagated state */
    RTCC_ERR_STEP_UNDERFLOW = 6,/* Cash-Karp step fell below h_min or too many rejects */
    RTCC_ERR_TIMEOUT = 7,       /* a bounded device-side wait expired (kernel returned early) */
    RTCC_ERR_UNSUPPORTED = 8    /* option not available in this build */
} rtcc_status_t;

/* Arithmetic of the residual contractions.  The propagated state, the controller and the
 * dipole reduction are float64 in every mode (Sec. 4.1 studies single vs double precision).
 * In the three reduced modes the intermediates of the residual are stored as float32
 * (complex64), small contractions and sums run in float32, and the RK stage combinations form
 * the weighted sum of the right-hand sides (and the error estimate) in float32 before adding
 * h times it to the float64 state; all of these resolve far more than the split products do. */
typedef enum {
    RTCC_P64 = 0,         /* float64 contractions (SIMT DFMA) */
    RTCC_P32_TF32 = 1,    /* one TF32 tcgen05 pass, float32 accumulate */
    RTCC_P32_3XTF32 = 2,  /* split hi/lo TF32 (3 passes), float32 accumulate */
    RTCC_P32_BF16X3 = 3   /* split hi/lo BF16 (3 passes), float32 accumulate */
} rtcc_precision_t;

typedef enum { RTCC_CARRIER_SIN = 0, RTCC_CARRIER_COS = 1 } rtcc_carrier_t;

/* Gaussian-envelope pulse (Sec. 3, Eq. field):
 *   E(t) = sign * E0 * exp(-(t-t0)^2/(2 sigma^2)) * carrier(omega (t-t0)) * pol
 * The paper's form is carrier = cos, sign = -1; pol = (1,1,1)/sqrt(3) is Eq. iso-field. */
typedef struct {
    double E0, omega, sigma, t0;
    double pol[3];
    int carrier;    /* rtcc_carrier_t */
    double sign;    /* +1 or -1 */
} rtcc_field_t;

typedef enum { RTCC_RK4 = 0, RTCC_CK = 1, RTCC_MIXED_RK4 = 2, RTCC_GL2 = 3, RTCC_GL2_NEWTON = 4 } rtcc_method_t;

/* Integrator settings (Sec. 2.1, Sec. 4.2).
 *   RK4:        fixed step h.
 *   CK:         Cash-Karp with the 37/378 (fifth-order) solution propagated, error
 *               Delta = max |y5 - y4| over all complex components, accept if Delta <= tol,
 *               h_new = safety*h*(tol/Delta)^(1/5) (accept) or ^(1/4) (reject, repeat),
 *               clamped to [0.2h, 5h] and [h_min, h_max]; h is the first trial step, and
 *               h = 0 continues every trajectory with its stored trial step (the one the
 *               previous call ended with, or rtcc_set_state's hstep), so that a run resumed
 *               from rtcc_get_state takes the same steps as one that never stopped
 *               (INVALID_ARG if a stored step lies outside [h_min, h_max]).
 *   MIXED_RK4:  RK4 with h1 while t < t_switch (the crossing step is cut to land on
 *               t_switch), h2 afterwards.
 *   GL2:        implicit two-stage Gauss-Legendre collocation (order 4, A-stable; Sec. 1
 *               lists implicit RK among the integrators, without coefficients) with fixed
 *               step h: c = 1/2 -+ sqrt(3)/6, the collocation matrix of [0, 1], b = (1/2, 1/2).
 *               The stage equations K_i = f(t + c_i h, y + h sum_j a_ij K_j) are solved by
 *               `sweeps` Gauss-Seidel fixed-point sweeps from K_i = f(t, y) (0: 20 sweeps;
 *               each sweep costs two right-hand sides).  A step whose last sweep still moves
 *               h K_2 by more than tol (max over components) stops the call with
 *               RTCC_ERR_NOCONV.  The sweeps contract only for steps of the order of RK4's
 *               stability limit, so they do not lengthen the usable step; what GL2 adds is
 *               that it conserves quadratic invariants (the norm, for Hermitian linear
 *               dynamics), which RK4 does not.
 *   GL2_NEWTON: the same collocation method with the stage equations solved by `sweeps`
 *               simplified Newton iterations (0: 6): the residuals G_i = K_i - f(t + c_i h,
 *               y + h sum_j a_ij K_j) and a correction from (I - h A x J) dK = -G, where J is
 *               the Jacobian of f at (t, y) applied by a forward difference of the library's own
 *               right-hand side and the linear system is solved by GMRES with `krylov` Arnoldi
 *               vectors (0: 12; at most 32; Hermitian inner product, classical Gram-Schmidt done
 *               twice, Givens rotations, all on the device).  Each Newton iteration costs
 *               2 + 2 krylov right-hand sides (one more per step for f(t, y)).  A step whose last
 *               Newton correction still moves h K_2 by more than tol stops the call with
 *               RTCC_ERR_NOCONV.  This converges for steps well beyond RK4's stability limit
 *               (at o = 2, v = 6: h = 0.4, where the sweeps of GL2 diverge).  Device memory:
 *               2 krylov + 9 state-sized complex vectors per trajectory, allocated on first use.
 * Stop after nsteps accepted steps if nsteps > 0, else at t_end (last step cut to land). */
typedef struct {
    int method;        /* rtcc_method_t */
    double h, h1, h2, t_switch;
    double tol, safety, h_min, h_max;
    int max_rejects;
    int nsteps;
    double t_end;
    int sweeps;        /* GL2: fixed-point sweeps; GL2_NEWTON: Newton iterations */
    int krylov;        /* GL2_NEWTON only: Arnoldi vectors of the GMRES solve */
} rtcc_integrator_t;

typedef struct rtcc_ctx* rtcc_handle_t;

/* Create a handle (Sec. 3; Sec. 4.1 describes the per-term integral uploads this replaces with residency).
 *  f   : host, nmo*nmo float64, symmetric field-free Fock matrix.
 *  B   : host, naux*nmo*nmo float64, density-fitting factors symmetric in the last two
 *        indices; the library forms (pq|rs) = sum_P B[P][p][q] B[P][r][s] on the device
 *        for every block the residual needs and keeps them resident.
 *  mu  : host, 3*nmo*nmo float64, symmetric dipole matrices (x, y, z).
 *  o,v : occupied / virtual counts (o >= 1, v >= 1).   ntraj: trajectories (>= 1).
 *  prec: rtcc_precision_t of the contractions.
 *  out : receives the handle.  All trajectories start at y = 0 (no ground state) and time 0.
 * Errors: INVALID_ARG (sizes, null, asymmetric f/B/mu), OOM, CUDA. */
rtcc_status_t rtcc_create(const double* f, const double* B, int naux, const double* mu,
                          int o, int v, int ntraj, int prec, rtcc_handle_t* out);

/* Create a handle with a frozen core (the paper's water runs freeze the O 1s orbitals, Sec. 3).
 * Same inputs as rtcc_create over all nmo = o + v orbitals; the lowest nfc occupied orbitals
 * (0 <= nfc < o) stay doubly occupied and are not correlated.  The handle then works in the
 * active space: o - nfc occupied and v virtual orbitals (the state layout, rtcc_state_size and
 * every amplitude index refer to the active orbitals only), with the active blocks of f (which
 * already carries the core's mean field), of B and of mu.  Every dipole the handle reports
 * includes the core's constant contribution 2 sum_c mu_x[c][c].  nfc = 0 is rtcc_create.
 * Errors: as rtcc_create; INVALID_ARG for nfc outside [0, o). */
rtcc_status_t rtcc_create_frozen_core(const double* f, const double* B, int naux, const double* mu,
                                      int o, int v, int nfc, int ntraj, int prec,
                                      rtcc_handle_t* out);

/* Free every device resource of the handle.  Null is accepted. */
rtcc_status_t rtcc_destroy(rtcc_handle_t h);

/* Number of complex elements of one trajectory's state y (2*o*v + 2*o*o*v*v). */
rtcc_status_t rtcc_state_size(rtcc_handle_t h, size_t* n);

/* Field-free ground state (Sec. 2.1: y0 is the ground-state T and Lambda solution),
 * float64 on the device whatever the handle's precision: Jacobi updates with
 * orbital-energy denominators plus DIIS until max|Omega| and max|R| < tol.
 * Every trajectory is set to the result at time 0.  e_corr (host, may be null)
 * receives the correlation energy, mu0 (host, 3 doubles, may be null) the real dipole.
 * Errors: NOCONV after maxiter iterations, CUDA. */
rtcc_status_t rtcc_ground_state(rtcc_handle_t h, double tol, int maxiter,
                                double* e_corr, double* mu0);

/* Copy one trajectory's state, time and current step size out of / into the handle.
 * y: host or device, rtcc_state_size() complex numbers.  time/hstep may be null (get)
 * or are applied (set).  traj in [0, ntraj).  Used for checkpoint/resume and tests. */
rtcc_status_t rtcc_get_state(rtcc_handle_t h, int traj, double* y, double* time, double* hstep);
rtcc_status_t rtcc_set_state(rtcc_handle_t h, int traj, const double* y, double time, double hstep);

/* One evaluation of the right-hand side of Eq. IVP for every trajectory:
 *   dt/dt = -i Omega(t; f(t)),  dl/dt = +i R(t, l; f(t))   with f(t) = f - E(t_z).mu
 * y    : host or device, ntraj * state_size complex (trajectory-major).
 * fields, times: host, ntraj entries (field of trajectory z evaluated at times[z]).
 * dydt : host or device, ntraj * state_size complex (output).
 * This is exactly the function every Runge-Kutta stage calls (Eqs. derivT/derivL). */
rtcc_status_t rtcc_rhs(rtcc_handle_t h, const double* y, const rtcc_field_t* fields,
                       const double* times, double* dydt);

/* Tile autotuning (performance only; results do not depend on it).  The reduced-precision
 * modes run their large contractions on a tcgen05 GEMM whose N tile (64, 128 or 256 columns)
 * is chosen per contraction shape by timing each usable tile on this GPU; rtcc_propagate does
 * this the first time it runs a given number of unfinished trajectories, the ground state and
 * the adjoint when their engines are built.  rtcc_autotune tunes every batch size of the handle
 * now, so that later propagations spend no time on it.  Tuning runs kernels that overwrite
 * intermediates only, never the state.  tuned_gemms (host, may be null): distinct GEMM shapes
 * tuned so far.  Setting RTCC_NO_AUTOTUNE=1 keeps the default tiles.  Errors: CUDA, TIMEOUT. */
rtcc_status_t rtcc_autotune(rtcc_handle_t h, int* tuned_gemms);

/* Vector-Jacobian product of the right-hand side rtcc_rhs computes (Eqs. derivT/derivL; the
 * transposed Jacobian is what the adjoint of the propagation applies at every stage):
 *   ybar_z = (d dydt_z / d y_z)^T u_z      (holomorphic: no complex conjugation)
 * at the states y, the fields and the times of rtcc_rhs.  y, u: host or device, ntraj *
 * state_size complex; ybar: host or device, same size (output).  Uses the handle's adjoint
 * engine (built on the first call).  Errors: INVALID_ARG, OOM, CUDA, TIMEOUT. */
rtcc_status_t rtcc_rhs_vjp(rtcc_handle_t h, const double* y, const rtcc_field_t* fields,
                           const double* times, const double* u, double* ybar);

/* Dipole of every trajectory's current state (Eq. dipole): mu_out host or device,
 * ntraj*3 complex. */
rtcc_status_t rtcc_dipole(rtcc_handle_t h, double* mu_out);

/* Propagate every trajectory from its current state and time (Sec. 2.1, Sec. 4.2).
 * fields : host, ntraj pulses.   integ: host, shared integrator settings.
 * max_out: samples per trajectory the output arrays hold (>= 1).
 * t_out  : host or device, ntraj*max_out float64 times (sample 0 = start time).
 * mu_out : host or device, ntraj*max_out*3 complex dipoles (re, im).
 * n_out  : host, ntraj ints: samples written per trajectory.
 * Each trajectory carries its own step size (Cash-Karp) and time; all trajectories
 * share every GEMM.  Sampling stops silently when max_out is reached; propagation
 * continues to the end.  Errors: DIVERGED, STEP_UNDERFLOW, NOCONV (GL2 stages), TIMEOUT, CUDA. */
rtcc_status_t rtcc_propagate(rtcc_handle_t h, const rtcc_field_t* fields,
                             const rtcc_integrator_t* integ, int max_out,
                             double* t_out, double* mu_out, int* n_out);

/* Gradient of a dipole-trajectory objective with respect to the pulse parameters, by the
 * discrete adjoint of RK4 (the paper has no adjoint; it differentiates the propagation of
 * Sec. 2.1 Eqs. rk_y/rk_k with the Eq. field pulse):
 *   J_z = sum_{n=0..nsteps} sum_x w[n][x] Re mu_x(t_n),  t_n = t_start + n h,
 *   grad[z] = dJ_z / d(E0, omega, sigma) of trajectory z's field.
 * Starts from every trajectory's current state and time; leaves them unchanged.
 * w: host, (nsteps+1)*3.  The forward sweep keeps a checkpoint every ckpt_every steps; the
 * reverse sweep recomputes each segment and applies the transposed stages with the
 * vector-Jacobian products of the right-hand side (state and Fock matrix) and of the dipole.
 * grad: host, ntraj*3 (output); J: host, ntraj (output).  Errors: INVALID_ARG, OOM, CUDA. */
rtcc_status_t rtcc_propagate_vjp(rtcc_handle_t h, const rtcc_field_t* fields, double hstep, int nsteps,
                                 const double* w, int ckpt_every, double* grad, double* J);

/* Counters of the last rtcc_propagate: accepted steps, rejected attempts and
 * right-hand-side evaluations summed over trajectories, and the number of kernels the
 * library launched (host, each may be null). */
rtcc_status_t rtcc_last_stats(rtcc_handle_t h, long long* accepted, long long* rejected,
                              long long* rhs_evals, long long* launches);

/* Launch profile (Sec. 4.1 reports time per step; this splits it by kernel class).
 * Class index: 0 tcgen05 GEMM, 1 float64 GEMM, 2 pack, 3 unpack, 4 direct contraction
 * (small terms, outer products, short-K row kernel), 5 reductions over a long K (split-K and
 * staged few-output kernels), 6 add/permute, 7 Runge-Kutta/field/controller kernels.
 * flops: algorithmic real flops of the launches (GEMMs: 2 x rows x cols x unpadded K of the
 * packed product); bytes: algorithmic bytes moved (memory-bound classes). */
typedef struct {
    long long launches[8];
    double ms[8];
    double flops[8];
    double bytes[8];
} rtcc_profile_t;

/* enable = 1: start timing every library launch of this handle with CUDA events on its
 * stream (rtcc_propagate then runs without CUDA-graph replay).  enable = 0: stop, wait for
 * the recorded events and write the per-class totals since the start into *out (may be null). */
rtcc_status_t rtcc_profile(rtcc_handle_t h, int enable, rtcc_profile_t* out);

/* Absorption spectrum (Sec. 2.2: I(w) = Im Tr alpha(w); Sec. 4.2: non-uniform samples
 * are interpolated onto a uniform grid).  Runs on the current CUDA device.
 *  t      : host, n sample times (increasing; need not be uniform).
 *  mu     : host, n*3 float64 real parts of the dipole.
 *  field  : host; the scalar pulse amplitude E(t) of this field is transformed and
 *           divided out, unless kappa > 0 (delta pulse: alpha = mu(w)/kappa).
 *  gamma  : exponential damping exp(-gamma (t - t_0)) applied to mu(t) - mu(t_0).
 *  dt     : uniform grid spacing for the interpolation (<= 0: smallest sample spacing).
 *  omega  : host, n_omega frequencies;  I : host, n_omega outputs
 *           I(w) = Im[ (pol . D(w)) / E(w) ],  D(w) = dt sum_k d(t_k) exp(i w t_k).
 * Errors: INVALID_ARG, CUDA. */
rtcc_status_t rtcc_spectrum(const double* t, const double* mu, int n, const rtcc_field_t* field,
                            double kappa, double gamma, double dt, const double* omega,
                            int n_omega, double* I);

/* Pade-accelerated absorption spectrum (Sec. 1 cites Pade approximants for spectra from short
 * propagations): as rtcc_spectrum, but each Fourier sum dt sum_k d_k e^{i w t_k} over the
 * samples is replaced by dt e^{i w t_0} P(z)/Q(z), z = e^{i w dt}, the diagonal [M/M] Pade
 * approximant of the power series sum_k d_k z^k built from 2M + 1 samples (all samples when n is
 * odd, the first n - 1 otherwise).  The denominator solves its Toeplitz system in the
 * least-squares sense with the minimum-norm solution (singular values at or below
 * 2.2e-16 * M * sigma_max are dropped), by a one-sided Jacobi SVD on the device.  The pulse's
 * samples E(t_k) get the same treatment unless kappa > 0 (delta pulse: alpha = D(w)/kappa).
 *  t      : host, n sample times, increasing and uniformly spaced (relative 1e-9); 3 <= n <= 1025.
 *  mu     : host, n*3 float64 real parts of the dipole.
 *  field  : host; its pol projects the dipole, its amplitude is the pulse (kappa <= 0).
 *  gamma  : damping exp(-gamma (t - t_0)) applied to mu(t) - mu(t_0).
 *  omega  : host, n_omega frequencies;  I : host, n_omega outputs I(w) = Im[ D(w) / E(w) ].
 * Errors: INVALID_ARG (sizes, non-uniform samples), NOCONV (Jacobi sweeps did not converge),
 * CUDA. */
rtcc_status_t rtcc_spectrum_pade(const double* t, const double* mu, int n, const rtcc_field_t* field,
                                 double kappa, double gamma, const double* omega, int n_omega, double* I);

/* Thread-local description of the most recent error (never null). */
const char* rtcc_last_error(void);

/* Library self-test of failure reporting (not part of the method): a kernel waits on a device
 * flag that nothing sets, gives up after `seconds` (bounded, 0..10) and reports it; the call
 * returns RTCC_ERR_TIMEOUT and the CUDA context stays usable.  Errors: INVALID_ARG, CUDA. */
rtcc_status_t rtcc_selftest_timeout(double seconds);

/* Library self-test of the contraction core (not part of the method): computes
 * C[b][m][n] = sum_k A[b][m][k] * Bm[b][n][k] for host or device inputs with the
 * handle-independent GEMM path of precision `prec` (TF32/3xTF32/BF16x3 run on the
 * tcgen05 tensor cores, P64 on the float64 path).  cplx bit 0: A is complex
 * (interleaved re, im), bit 1: Bm is complex; C (host or device) is complex when either
 * operand is.  Internally the product is formed four times, into two zeroed temporaries laid
 * out m-major and n-major (each first stored, then accumulated in place), and C is a quarter
 * of their sum, so every output path of the contraction core is exercised.
 * Errors: INVALID_ARG, CUDA, TIMEOUT. */
rtcc_status_t rtcc_selftest_gemm(int prec, int cplx, int batch, int M, int N, int K, const double* A,
                                 const double* Bm, double* C);

/* Allocation-free tensor-core GEMM (the paper has no counterpart: this serves callers that
 * cannot let a library allocate device memory, e.g. applications that own all device memory
 * through their own pool).  Computes C[b][m][n] = sum_k A[b][m][k] * Bm[b][n][k] with the same
 * packing and tcgen05 kernels as rtcc_selftest_gemm, in precision prec = TF32, 3xTF32 or BF16x3
 * (RTCC_P64 is rejected).  cplx bit 0: A complex (interleaved), bit 1: Bm complex; C is complex
 * when either is.  A, Bm and C are DEVICE pointers owned by the caller; C is overwritten.  The
 * call runs on `stream` (a cudaStream_t, null = default stream) and returns after completion.
 * It calls no cudaMalloc, cudaFree or allocating library routine: the packed operands live in a
 * 64 MiB file-scope device array that every GPU loading the library keeps until process exit.
 * batch*(planesA*M + planesB*N)*Kpad*element_size must fit in it (planes = 1 or 2 components x
 * 1 split part for TF32, 2 parts otherwise; Kpad = K rounded up to 32 (TF32) or 64 (BF16)
 * elements; 4-byte elements for TF32 modes, 2-byte for BF16x3), else RTCC_ERR_INVALID_ARG.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) and
 * should come before any stream capture.  All calls share the array, which keeps the previous
 * call's contents: calls that overlap on the GPU (other streams, other host threads) race.
 * Errors: INVALID_ARG, CUDA, TIMEOUT. */
rtcc_status_t rtcc_gemm_noalloc(int prec, int cplx, int batch, int M, int N, int K, const double* A,
                                const double* Bm, double* C, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RTCC_H */
