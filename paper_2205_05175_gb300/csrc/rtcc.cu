// C-ABI of the RT-CCSD library (include/rtcc.h): handle, ground state, Runge-Kutta
// propagation with a device-side step controller, dipole recording, spectrum.
#include "model.cuh"
#include "pade_core.cuh"
#include <algorithm>
#include <vector>
#include "../../include/rtcc.h"
#include <cmath>
#include <type_traits>
#include <cstring>
#include <memory>
#include <cstdio>
#include <cstdlib>

namespace rtcc {
namespace {

thread_local std::string g_last_error = "no error";

constexpr int kMaxStages = 6;
enum TrajStatus : int { TS_RUN = 0, TS_DONE = 1, TS_DIVERGED = 2, TS_UNDERFLOW = 3, TS_NOCONV = 4 };

// Butcher tableaus (Sec. 2.1 Eqs. rk_y/rk_k; Sec. 4.2 Eq. rk4truncation, Eqs. ck-k/ck-y with
// the row sums sum_j a_ij = c_i restored: a42 = -9/10, a63 = +575/13824, c4 = 3/5, c5 = 1).
struct Tableau {
  int s;
  double c[kMaxStages];
  double a[kMaxStages][kMaxStages];
  double b[kMaxStages];    // propagated solution
  double e[kMaxStages];    // b - b_embedded (error weights), zero for RK4
  bool adaptive;
  bool implicit = false;   // full A: stages solved by fixed-point sweeps
  int sweeps = 0;
  bool newton = false;     // implicit stages solved by simplified Newton iterations with GMRES
  int krylov = 0;          // Arnoldi vectors per GMRES solve
};

Tableau rk4_tableau() {
  Tableau t{};
  t.s = 4;
  t.c[0] = 0; t.c[1] = 0.5; t.c[2] = 0.5; t.c[3] = 1.0;
  t.a[1][0] = 0.5;
  t.a[2][1] = 0.5;
  t.a[3][2] = 1.0;
  t.b[0] = 1.0 / 6; t.b[1] = 1.0 / 3; t.b[2] = 1.0 / 3; t.b[3] = 1.0 / 6;
  t.adaptive = false;
  return t;
}

// Two-stage Gauss-Legendre collocation (implicit, order 4): Gauss points of [0, 1] and the
// collocation matrix; the stage system is solved by Gauss-Seidel fixed-point sweeps.
Tableau gl2_tableau(int sweeps) {
  Tableau t{};
  const double r = std::sqrt(3.0) / 6.0;
  t.s = 2;
  t.c[0] = 0.5 - r; t.c[1] = 0.5 + r;
  t.a[0][0] = 0.25; t.a[0][1] = 0.25 - r;
  t.a[1][0] = 0.25 + r; t.a[1][1] = 0.25;
  t.b[0] = 0.5; t.b[1] = 0.5;
  t.adaptive = false;
  t.implicit = true;
  t.sweeps = sweeps > 0 ? sweeps : 20;
  return t;
}

constexpr int kKrylovMax = 32;

// The same collocation method with the stage equations solved by `newton` simplified Newton
// iterations, each correction from a GMRES solve with `krylov` Arnoldi vectors.
Tableau gl2_newton_tableau(int newton, int krylov) {
  Tableau t = gl2_tableau(0);
  t.implicit = false;
  t.newton = true;
  t.sweeps = newton > 0 ? newton : 6;
  t.krylov = krylov > 0 ? krylov : 12;
  return t;
}

Tableau ck_tableau() {
  Tableau t{};
  t.s = 6;
  const double c[6] = {0, 1.0 / 5, 3.0 / 10, 3.0 / 5, 1.0, 7.0 / 8};
  for (int i = 0; i < 6; ++i) t.c[i] = c[i];
  t.a[1][0] = 1.0 / 5;
  t.a[2][0] = 3.0 / 40; t.a[2][1] = 9.0 / 40;
  t.a[3][0] = 3.0 / 10; t.a[3][1] = -9.0 / 10; t.a[3][2] = 6.0 / 5;
  t.a[4][0] = -11.0 / 54; t.a[4][1] = 5.0 / 2; t.a[4][2] = -70.0 / 27; t.a[4][3] = 35.0 / 27;
  t.a[5][0] = 1631.0 / 55296; t.a[5][1] = 175.0 / 512; t.a[5][2] = 575.0 / 13824;
  t.a[5][3] = 44275.0 / 110592; t.a[5][4] = 253.0 / 4096;
  const double b5[6] = {37.0 / 378, 0, 250.0 / 621, 125.0 / 594, 0, 512.0 / 1771};
  const double b4[6] = {2825.0 / 27648, 0, 18575.0 / 48384, 13525.0 / 55296, 277.0 / 14336, 1.0 / 4};
  for (int i = 0; i < 6; ++i) {
    t.b[i] = b5[i];
    t.e[i] = b5[i] - b4[i];
  }
  t.adaptive = true;
  return t;
}

// ---------------------------------------------------------------------------------------
// Device kernels of the integrator (all float64)

__device__ __forceinline__ double field_amp(const rtcc_field_t& f, double t) {
  const double x = t - f.t0;
  const double env = exp(-0.5 * x * x / (f.sigma * f.sigma));
  const double car = (f.carrier == RTCC_CARRIER_COS) ? cos(f.omega * x) : sin(f.omega * x);
  return f.sign * f.E0 * env * car;
}

// F[z] = f0 - E_z(t_z + c h_z) . mu   (Sec. 2.2, V = -mu.E; Eq. field)
__global__ void k_fock(double* F, const double* f0, const double* mu, const rtcc_field_t* fields,
                       const double* tz, const double* hz, double c, int nz, int n2) {
  const int z = blockIdx.y;
  const double tt = tz[z] + c * hz[z];
  const rtcc_field_t fl = fields[z];
  const double amp = field_amp(fl, tt);
  const double ex = amp * fl.pol[0], ey = amp * fl.pol[1], ez = amp * fl.pol[2];
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n2; k += gridDim.x * blockDim.x)
    F[(size_t)z * n2 + k] = f0[k] - ex * mu[k] - ey * mu[n2 + k] - ez * mu[2 * n2 + k];
}

struct StageArgs {
  const double* R[kMaxStages];   // raw right-hand sides (Omega | R) of the stages used
  double coef[kMaxStages];
  int nterms;
  const double* copy_src;        // the most recent right-hand side, saved to copy_dst
  double* copy_dst;
};

// y_out = y + h_z * sum_j coef_j * D R_j, with D = -i on the T part and +i on the Lambda part
// (dt/dt = -i Omega, dl/dt = +i R).  Optionally saves the newest right-hand side.
// F32 (reduced-precision handles, whose right-hand sides resolve far less than float32): the
// weighted sum of the right-hand sides is formed in float32 from integer-rounded values and only
// y + h * increment is float64, which keeps the kernel off the float64 pipe; otherwise float64.
template <bool F32>
__global__ void k_stage(double* __restrict__ yout, const double* __restrict__ y, StageArgs A, const double* hz,
                        long long ns, long long nT) {
  using R = typename std::conditional<F32, float, double>::type;
  const int z = blockIdx.y;
  const double h = hz[z];
  const size_t base = (size_t)z * ns;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < ns; k += (long long)gridDim.x * blockDim.x) {
    const size_t e = base + k;
    R sr = 0, si = 0;
    for (int j = 0; j < A.nterms; ++j) {
      const double2 rv = reinterpret_cast<const double2*>(A.R[j])[e];
      const R c = (R)A.coef[j];
      if constexpr (F32) {
        sr = fmaf(c, f64_to_f32_bits(rv.x), sr);
        si = fmaf(c, f64_to_f32_bits(rv.y), si);
      } else {
        sr += c * rv.x;
        si += c * rv.y;
      }
    }
    if (A.copy_dst) reinterpret_cast<double2*>(A.copy_dst)[e] = reinterpret_cast<const double2*>(A.copy_src)[e];
    // D * s: -i (sr + i si) = si - i sr ; +i (sr + i si) = -si + i sr
    double dr, di;
    if constexpr (F32) {
      dr = f32_to_f64_bits((k < nT) ? si : -si);
      di = f32_to_f64_bits((k < nT) ? -sr : sr);
    } else {
      dr = (k < nT) ? si : -si;
      di = (k < nT) ? -sr : sr;
    }
    const double2 yv = reinterpret_cast<const double2*>(y)[e];
    reinterpret_cast<double2*>(yout)[e] = make_double2(yv.x + h * dr, yv.y + h * di);
  }
}

// Final combination: ynew = y + h sum b_j D R_j; err_z = max |h sum e_j R_j|; non-finite -> +inf.
// F32 as in k_stage; the error estimate then also sums in float32 (it only steers the step size).
template <bool F32>
__global__ void k_final(double* __restrict__ ynew, const double* __restrict__ y, StageArgs B, StageArgs Ew,
                        const double* hz, long long ns, long long nT, unsigned long long* err_bits, int adaptive) {
  using R = typename std::conditional<F32, float, double>::type;
  const int z = blockIdx.y;
  const double h = hz[z];
  const size_t base = (size_t)z * ns;
  double emax = 0.0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < ns; k += (long long)gridDim.x * blockDim.x) {
    const size_t e = base + k;
    R sr = 0, si = 0, er = 0, ei = 0;
    for (int j = 0; j < B.nterms; ++j) {
      const double2 rv = reinterpret_cast<const double2*>(B.R[j])[e];
      R rr, ri;
      if constexpr (F32) {
        rr = f64_to_f32_bits(rv.x);
        ri = f64_to_f32_bits(rv.y);
      } else {
        rr = rv.x;
        ri = rv.y;
      }
      const R bc = (R)B.coef[j];
      sr += bc * rr;
      si += bc * ri;
      if (adaptive) {
        const R ec = (R)Ew.coef[j];
        er += ec * rr;
        ei += ec * ri;
      }
    }
    double dr, di;
    if constexpr (F32) {
      dr = f32_to_f64_bits((k < nT) ? si : -si);
      di = f32_to_f64_bits((k < nT) ? -sr : sr);
    } else {
      dr = (k < nT) ? si : -si;
      di = (k < nT) ? -sr : sr;
    }
    const double2 yv = reinterpret_cast<const double2*>(y)[e];
    const double yr = yv.x + h * dr, yi = yv.y + h * di;
    reinterpret_cast<double2*>(ynew)[e] = make_double2(yr, yi);
    double ek = 0.0;
    if (adaptive) {
      if constexpr (F32) ek = (double)((float)h * sqrtf(er * er + ei * ei));
      else ek = h * sqrt(er * er + ei * ei);
    }
    if (!isfinite(yr) || !isfinite(yi) || !isfinite(ek)) ek = INFINITY;
    emax = fmax(emax, ek);
  }
  for (int off = 16; off > 0; off >>= 1) emax = fmax(emax, __shfl_down_sync(0xffffffffu, emax, off));
  if ((threadIdx.x & 31) == 0) atomicMax(&err_bits[z], (unsigned long long)__double_as_longlong(emax));
}

struct Ctl {
  double* t;          // current time per trajectory
  double* h;          // next trial step (CK) per trajectory
  double* htry;       // step of the current attempt
  int* status;
  int* accepted;      // 1 if the current attempt was accepted
  int* steps;         // accepted steps
  int* rejects;       // consecutive rejects
  unsigned long long* err_bits;
  long long* counters;   // [0] accepted, [1] rejected (summed over trajectories)
  int* nout;
  int* perm;          // trajectory held by each slot (slots are compacted while propagating)
};

__global__ void k_prestep(Ctl c, rtcc_integrator_t in, int nz) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= nz) return;
  c.err_bits[z] = 0ull;
  c.accepted[z] = 0;
  if (c.status[z] != TS_RUN) {
    c.htry[z] = 0.0;
    return;
  }
  const double t = c.t[z];
  const double eps = 1e-12;
  double hs;
  if (in.method == RTCC_RK4 || in.method == RTCC_GL2 || in.method == RTCC_GL2_NEWTON) hs = in.h;
  else if (in.method == RTCC_MIXED_RK4) hs = (t < in.t_switch - eps) ? fmin(in.h1, in.t_switch - t) : in.h2;
  else hs = c.h[z];
  if (in.nsteps <= 0) hs = fmin(hs, in.t_end - t);
  c.htry[z] = hs;
}

__global__ void k_controller(Ctl c, rtcc_integrator_t in, int nz) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= nz || c.status[z] != TS_RUN) return;
  const double delta = __longlong_as_double((long long)c.err_bits[z]);
  const double hs = c.htry[z];
  const double eps = 1e-12;
  if (!isfinite(delta)) {
    c.status[z] = TS_DIVERGED;
    return;
  }
  if ((in.method == RTCC_GL2 || in.method == RTCC_GL2_NEWTON) && delta > in.tol) {
    // the last Gauss-Seidel sweep still moved h K_2 by more than tol: the stages have not converged
    c.status[z] = TS_NOCONV;
    return;
  }
  bool acc = true;
  if (in.method == RTCC_CK) {
    // Eq. ck-h-final: safety * h * (tol/Delta)^(1/5) after an accepted attempt, ^(1/4) after a rejected one
    acc = delta <= in.tol;
    double fac = (delta == 0.0) ? 5.0 : in.safety * pow(in.tol / delta, acc ? 0.2 : 0.25);
    fac = fmin(5.0, fmax(0.2, fac));
    const double hn = fmin(in.h_max, fmax(in.h_min, hs * fac));
    c.h[z] = hn;
    if (!acc) {
      c.rejects[z] += 1;
      atomicAdd((unsigned long long*)&c.counters[1], 1ull);
      if (c.rejects[z] > in.max_rejects || hn <= in.h_min) c.status[z] = TS_UNDERFLOW;
      return;
    }
    c.rejects[z] = 0;
  }
  c.accepted[z] = 1;
  c.t[z] += hs;
  c.steps[z] += 1;
  atomicAdd((unsigned long long*)&c.counters[0], 1ull);
  const bool done = (in.nsteps > 0) ? (c.steps[z] >= in.nsteps) : (c.t[z] >= in.t_end - eps);
  if (done) c.status[z] = TS_DONE;
}

__global__ void k_accept(double* __restrict__ y, const double* __restrict__ ynew, const int* accepted, long long ns) {
  const int z = blockIdx.y;
  if (!accepted[z]) return;
  const size_t base = 2 * (size_t)z * ns;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < 2 * ns; k += (long long)gridDim.x * blockDim.x)
    y[base + k] = ynew[base + k];
}

// Append (t, mu) for trajectories accepted in this attempt (or all when force).
__global__ void k_record(Ctl c, const double* dip, double r0, double r1, double r2, double* tout, double* muout,
                         int max_out, int nz, int force) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= nz) return;
  if (!force && !c.accepted[z]) return;
  const int n = c.nout[z];
  if (n >= max_out) return;
  const int tr = c.perm[z];   // outputs are indexed by trajectory, not by slot
  tout[(size_t)tr * max_out + n] = c.t[z];
  const double ref[3] = {r0, r1, r2};
  for (int x = 0; x < 3; ++x) {
    const size_t q = 2 * ((size_t)x * nz + z);
    muout[2 * (((size_t)tr * max_out + n) * 3 + x)] = dip[q] + ref[x];
    muout[2 * (((size_t)tr * max_out + n) * 3 + x) + 1] = dip[q + 1];
  }
  c.nout[z] = n + 1;
}

// dydt = D * R (D = -i on the T part, +i on the Lambda part)
__global__ void k_apply_D(double* out, const double* R, long long ns, long long nT, int nz) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < (long long)nz * ns;
       k += (long long)gridDim.x * blockDim.x) {
    const long long kk = k % ns;
    const double rr = R[2 * k], ri = R[2 * k + 1];
    out[2 * k] = (kk < nT) ? ri : -ri;
    out[2 * k + 1] = (kk < nT) ? -rr : rr;
  }
}

// Ground state: x += r / D over one amplitude block (singles then doubles) of one state.
__global__ void k_jacobi(double* x, const double* r, const double* f0, int o, int v, int nmo, double* e_out) {
  const long long n1 = (long long)o * v, n2 = n1 * o * v;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n1 + n2; k += (long long)gridDim.x * blockDim.x) {
    double d;
    if (k < n1) {
      const int i = (int)(k / v), a = (int)(k % v);
      d = f0[(size_t)i * nmo + i] - f0[(size_t)(o + a) * nmo + o + a];
    } else {
      long long q = k - n1;
      const int b = (int)(q % v); q /= v;
      const int a = (int)(q % v); q /= v;
      const int j = (int)(q % o);
      const int i = (int)(q / o);
      d = f0[(size_t)i * nmo + i] + f0[(size_t)j * nmo + j] - f0[(size_t)(o + a) * nmo + o + a] -
          f0[(size_t)(o + b) * nmo + o + b];
    }
    const double er = r[2 * k] / d, ei = r[2 * k + 1] / d;
    x[2 * k] += er;
    x[2 * k + 1] += ei;
    if (e_out) {
      e_out[2 * k] = er;
      e_out[2 * k + 1] = ei;
    }
  }
}

__global__ void k_maxabs(const double* r, long long n, unsigned long long* out) {
  double m = 0.0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const double a = sqrt(r[2 * k] * r[2 * k] + r[2 * k + 1] * r[2 * k + 1]);
    m = isfinite(a) ? fmax(m, a) : INFINITY;
  }
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// Re sum conj(a) b
__global__ void k_dot(const double* a, const double* b, long long n, double* out) {
  double s = 0.0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
    s += a[2 * k] * b[2 * k] + a[2 * k + 1] * b[2 * k + 1];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

struct Combo {
  const double* x[12];
  double c[12];
  int m;
};
__global__ void k_combine(double* out, Combo C, long long n) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < 2 * n; k += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < C.m; ++j) s += C.c[j] * C.x[j][k];
    out[k] = s;
  }
}

// x2 <- (x2 + x2^(ij,ab swapped)) / 2 for the doubles block of one state (keeps DIIS iterates pair-symmetric)
__global__ void k_sym_pair(double* x2, int o, int v) {
  const long long n = (long long)o * o * v * v;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    long long q = k;
    const int b = (int)(q % v); q /= v;
    const int a = (int)(q % v); q /= v;
    const int j = (int)(q % o);
    const int i = (int)(q / o);
    const long long kt = (((long long)j * o + i) * v + b) * v + a;
    if (kt <= k) continue;
    const double r = 0.5 * (x2[2 * k] + x2[2 * kt]), im = 0.5 * (x2[2 * k + 1] + x2[2 * kt + 1]);
    x2[2 * k] = r; x2[2 * kt] = r;
    x2[2 * k + 1] = im; x2[2 * kt + 1] = im;
  }
}

// Spectrum (Sec. 2.2; Sec. 4.2 interpolation): natural cubic spline second derivatives per
// component by the tridiagonal (Thomas) recursion, evaluation on a uniform grid, direct DFT.
__global__ void k_spline_m(const double* t, const double* y, int n, double* M, double* cp, double* dp) {
  const int x = threadIdx.x;   // component
  if (x >= 3) return;
  double* Mx = M + (size_t)x * n;
  double* c = cp + (size_t)x * n;
  double* d = dp + (size_t)x * n;
  auto Y = [&](int k) { return y[(size_t)k * 3 + x]; };
  // rows 1..n-2: h_{k-1} M_{k-1} + 2 (h_{k-1} + h_k) M_k + h_k M_{k+1} = r_k ; M_0 = M_{n-1} = 0
  c[0] = 0.0;
  d[0] = 0.0;
  for (int k = 1; k < n - 1; ++k) {
    const double hl = t[k] - t[k - 1], hr = t[k + 1] - t[k];
    const double r = 6.0 * ((Y(k + 1) - Y(k)) / hr - (Y(k) - Y(k - 1)) / hl);
    const double den = 2.0 * (hl + hr) - hl * c[k - 1];
    c[k] = hr / den;
    d[k] = (r - hl * d[k - 1]) / den;
  }
  Mx[n - 1] = 0.0;
  for (int k = n - 2; k >= 1; --k) Mx[k] = d[k] - c[k] * Mx[k + 1];
  Mx[0] = 0.0;
}

__global__ void k_spline_eval(const double* t, const double* y, const double* M, int n, double t0, double dt, int nu,
                              double* yu) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nu; q += gridDim.x * blockDim.x) {
    const double tq = t0 + dt * q;
    int lo = 0, hi = n - 1;
    while (hi - lo > 1) {
      const int mid = (lo + hi) / 2;
      if (t[mid] <= tq) lo = mid;
      else hi = mid;
    }
    const double h = t[lo + 1] - t[lo], dx = tq - t[lo];
    for (int x = 0; x < 3; ++x) {
      const double* Mx = M + (size_t)x * n;
      const double y0 = y[(size_t)lo * 3 + x], y1 = y[(size_t)(lo + 1) * 3 + x];
      const double a = (Mx[lo + 1] - Mx[lo]) / (6.0 * h), b = Mx[lo] / 2.0;
      const double c = (y1 - y0) / h - h * (2.0 * Mx[lo] + Mx[lo + 1]) / 6.0;
      yu[(size_t)q * 3 + x] = y0 + c * dx + b * dx * dx + a * dx * dx * dx;
    }
  }
}

// I(w) = Im[ (pol . D(w)) / E(w) ], D(w) = dt sum_k d(t_k) e^{i w t_k}, d = (mu - mu_0) e^{-gamma (t - t_0)}
__global__ void k_dft(const double* t, const double* y, int n, double dt, rtcc_field_t fld, double kappa, double gamma,
                      const double* omega, int nw, double* I) {
  const int w = blockIdx.x;
  if (w >= nw) return;
  const double om = omega[w];
  double dr = 0, di = 0, er = 0, ei = 0;
  const double t0 = t[0];
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const double tk = t[k];
    const double damp = exp(-gamma * (tk - t0));
    const double d = ((y[(size_t)k * 3] - y[0]) * fld.pol[0] + (y[(size_t)k * 3 + 1] - y[1]) * fld.pol[1] +
                      (y[(size_t)k * 3 + 2] - y[2]) * fld.pol[2]) * damp;
    double s, c;
    sincos(om * tk, &s, &c);
    dr += d * c;
    di += d * s;
    if (kappa <= 0.0) {
      const double e = field_amp(fld, tk);
      er += e * c;
      ei += e * s;
    }
  }
  __shared__ double sh[4][32];
  for (int off = 16; off > 0; off >>= 1) {
    dr += __shfl_down_sync(0xffffffffu, dr, off);
    di += __shfl_down_sync(0xffffffffu, di, off);
    er += __shfl_down_sync(0xffffffffu, er, off);
    ei += __shfl_down_sync(0xffffffffu, ei, off);
  }
  const int wi = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sh[0][wi] = dr; sh[1][wi] = di; sh[2][wi] = er; sh[3][wi] = ei; }
  __syncthreads();
  if (threadIdx.x == 0) {
    dr = di = er = ei = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { dr += sh[0][q]; di += sh[1][q]; er += sh[2][q]; ei += sh[3][q]; }
    dr *= dt; di *= dt;
    if (kappa > 0.0) { er = kappa; ei = 0.0; }
    else { er *= dt; ei *= dt; }
    // Im[(dr + i di) / (er + i ei)] = (di er - dr ei) / |E|^2
    I[w] = (di * er - dr * ei) / (er * er + ei * ei);
  }
}

// Pade-accelerated spectrum (Sec. 1 cites Pade approximants among the short-time spectral
// techniques): the Fourier sum dt sum_k d_k e^{i w t_k} over uniform samples is replaced by
// dt e^{i w t_0} P(z)/Q(z), z = e^{i w dt}, the diagonal Pade approximant of sum_k d_k z^k
// (arithmetic in pade_core.cuh).
// series[0][k] = (pol . (mu_k - mu_0)) e^{-gamma (t_k - t_0)}; series[1][k] = E(t_k) when the
// pulse's own transform is divided out.
__global__ void k_pade_series(const double* t, const double* y, int N, rtcc_field_t fld, double gamma, int with_field,
                              double* series) {
  const double t0 = t[0];
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    const double tk = t[k];
    const double damp = exp(-gamma * (tk - t0));
    series[k] = ((y[(size_t)k * 3] - y[0]) * fld.pol[0] + (y[(size_t)k * 3 + 1] - y[1]) * fld.pol[1] +
                 (y[(size_t)k * 3 + 2] - y[2]) * fld.pol[2]) * damp;
    if (with_field) series[N + k] = field_amp(fld, tk);
  }
}

// Sum over a warp, the same value on every lane (shuffle-down tree into lane 0, then broadcast).
struct WarpSum {
  __device__ double operator()(double x) const {
    for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
    return __shfl_sync(0xffffffffu, x, 0);
  }
};

// One CTA per series (N = 2M + 1 coefficients): one warp per column pair of each tournament
// round, a block barrier between rounds, sweeps until no pair rotates (at most
// pade::kMaxSweeps; info = 1 if that bound is reached); then the minimum-norm denominator and
// the numerator.  coef[s] = a_0 .. a_M, b_0 .. b_M.  work: pade::work_doubles(M) per series.
constexpr int kPadeThreads = 512, kPadeMaxOrder = 512;
__global__ void __launch_bounds__(kPadeThreads) k_pade_solve(const double* series, int M, double* work, double* coef,
                                                             int* info) {
  using namespace pade;
  const int sid = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  const int N = 2 * M + 1, M2 = padded(M);
  const double* c = series + (size_t)sid * N;
  double* U = work + (size_t)sid * work_doubles(M);
  double* V = U + (size_t)M * M2;
  double* rhs = V + (size_t)M2 * M2;
  double* s2 = rhs + M2;
  double* w = s2 + M2;
  __shared__ int s_rot;
  __shared__ double s_red[32];
  const WarpSum sum;
  fill(c, M, U, V, rhs, tid, blockDim.x);
  {
    double f = fro2_partial(c, M, tid, blockDim.x);
    f = sum(f);
    if (lane == 0) s_red[warp] = f;
  }
  __syncthreads();
  double fro2 = 0.0;
  for (int i = 0; i < nwarp; ++i) fro2 += s_red[i];
  const double fl = floor2(fro2);
  __syncthreads();
  int sweep = 0;
  for (; sweep < kMaxSweeps; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int r = 0; r < M2 - 1; ++r) {
      for (int k = warp; k < M2 / 2; k += nwarp) {
        int p, q;
        pair_of(M2, r, k, p, q);
        double a, b, g;
        pair_dots(U, M, p, q, lane, 32, a, b, g);
        a = sum(a);
        b = sum(b);
        g = sum(g);
        double cs, sn;
        if (rotation(a, b, g, fl, cs, sn)) {
          pair_apply(U, V, M, M2, p, q, cs, sn, lane, 32);
          if (lane == 0) s_rot = 1;
        }
      }
      __syncthreads();
    }
    const int any = s_rot;
    __syncthreads();
    if (!any) break;
  }
  if (tid == 0) info[sid] = (sweep >= kMaxSweeps) ? 1 : 0;
  for (int j = warp; j < M2; j += nwarp) {
    double x, y;
    col_dots(U, rhs, M, j, lane, 32, x, y);
    x = sum(x);
    y = sum(y);
    if (lane == 0) {
      s2[j] = x;
      w[j] = y;
    }
  }
  __syncthreads();
  double mx = 0.0;
  for (int j = tid; j < M2; j += blockDim.x) mx = fmax(mx, s2[j]);
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, off));
  if (lane == 0) s_red[warp] = mx;
  __syncthreads();
  if (tid == 0) {
    double m = 0.0;
    for (int i = 0; i < nwarp; ++i) m = fmax(m, s_red[i]);
    s_red[0] = m;
  }
  __syncthreads();
  const double cut = cut2(M, s_red[0]);
  for (int j = tid; j < M2; j += blockDim.x) w[j] = (s2[j] > cut) ? w[j] / s2[j] : 0.0;
  __syncthreads();
  double* out = coef + (size_t)sid * 2 * (M + 1);
  double* bq = out + (M + 1);
  for (int i = tid; i < M; i += blockDim.x) bq[i + 1] = denominator(V, w, M2, i);
  if (tid == 0) bq[0] = 1.0;
  __syncthreads();
  for (int k = tid; k <= M; k += blockDim.x) out[k] = numerator(bq, c, k);
}

// I(w) = Im[ D(w) / E(w) ] with D = dt e^{i w t_0} P_0/Q_0 and E = kappa (delta pulse) or the
// same approximant of the pulse's samples (series 1).
__global__ void k_pade_eval(const double* coef, int M, double dt, double t0, double kappa, const double* omega, int nw,
                            double* I) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nw; q += gridDim.x * blockDim.x) {
    const double om = omega[q];
    double zs, zc, ss, sc;
    sincos(om * dt, &zs, &zc);
    sincos(om * t0, &ss, &sc);
    double pr, pi;
    pade::ratio(coef, coef + M + 1, M, zc, zs, pr, pi);
    const double dr = dt * (sc * pr - ss * pi), di = dt * (sc * pi + ss * pr);
    double er = kappa, ei = 0.0;
    if (kappa <= 0.0) {
      const double* c1 = coef + 2 * (M + 1);
      double fr, fi;
      pade::ratio(c1, c1 + M + 1, M, zc, zs, fr, fi);
      er = dt * (sc * fr - ss * fi);
      ei = dt * (sc * fi + ss * fr);
    }
    I[q] = (di * er - dr * ei) / (er * er + ei * ei);
  }
}

// ---------------------------------------------------------------------------------------
// Newton-Krylov kernels of the implicit Gauss-Legendre stages.  A Krylov vector holds both stage
// blocks, each [nz][ns] complex; `bstride` is the distance (in doubles) between the two blocks and
// blockIdx.y is the trajectory.  Every inner product is Hermitian: <v, w> = sum conj(v) w.

// out[z][k] += <V_k, w>_z for k = blockIdx.z (V_k at V + k * vstride); out has ldo entries per z
__global__ void k_zdots(const double* __restrict__ V, long long vstride, const double* __restrict__ w,
                        long long bstride, long long ns, int ldo, double* out) {
  const int z = blockIdx.y, k = blockIdx.z;
  double sr = 0.0, si = 0.0;
  for (int b = 0; b < 2; ++b) {
    const double* vb = V + (size_t)k * vstride + (size_t)b * bstride + (size_t)z * 2 * ns;
    const double* wb = w + (size_t)b * bstride + (size_t)z * 2 * ns;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ns; i += (long long)gridDim.x * blockDim.x) {
      const double vr = vb[2 * i], vi = vb[2 * i + 1], wr = wb[2 * i], wi = wb[2 * i + 1];
      sr += vr * wr + vi * wi;
      si += vr * wi - vi * wr;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    sr += __shfl_down_sync(0xffffffffu, sr, off);
    si += __shfl_down_sync(0xffffffffu, si, off);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&out[2 * ((size_t)z * ldo + k)], sr);
    atomicAdd(&out[2 * ((size_t)z * ldo + k) + 1], si);
  }
}

// w += alpha * sum_{k < nvec} coef[z][k] V_k   (coef complex, ldo entries per z)
__global__ void k_zupdate(double* __restrict__ w, const double* __restrict__ V, long long vstride, int nvec,
                          const double* __restrict__ coef, int ldo, double alpha, long long bstride, long long ns) {
  const int z = blockIdx.y;
  for (int b = 0; b < 2; ++b) {
    double* wb = w + (size_t)b * bstride + (size_t)z * 2 * ns;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ns; i += (long long)gridDim.x * blockDim.x) {
      double ar = 0.0, ai = 0.0;
      for (int k = 0; k < nvec; ++k) {
        const double* vb = V + (size_t)k * vstride + (size_t)b * bstride + (size_t)z * 2 * ns;
        const double cr = coef[2 * ((size_t)z * ldo + k)], ci = coef[2 * ((size_t)z * ldo + k) + 1];
        const double vr = vb[2 * i], vi = vb[2 * i + 1];
        ar += cr * vr - ci * vi;
        ai += cr * vi + ci * vr;
      }
      wb[2 * i] += alpha * ar;
      wb[2 * i + 1] += alpha * ai;
    }
  }
}

// out = scale[z] * in over both stage blocks
__global__ void k_zscale(double* __restrict__ out, const double* __restrict__ in, const double* __restrict__ scale,
                         long long bstride, long long ns) {
  const int z = blockIdx.y;
  const double sc = scale[z];
  for (int b = 0; b < 2; ++b) {
    const size_t base = (size_t)b * bstride + (size_t)z * 2 * ns;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 2 * ns; i += (long long)gridDim.x * blockDim.x)
      out[base + i] = sc * in[base + i];
  }
}

// out = x - h_z (c0 u0 + c1 u1) over one block [nz][ns] complex
__global__ void k_lincomb_h(double* __restrict__ out, const double* __restrict__ x, const double* __restrict__ u0,
                            const double* __restrict__ u1, double c0, double c1, const double* __restrict__ hz,
                            long long ns) {
  const int z = blockIdx.y;
  const double h = hz[z];
  const size_t base = (size_t)z * 2 * ns;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 2 * ns; i += (long long)gridDim.x * blockDim.x)
    out[base + i] = x[base + i] - h * (c0 * u0[base + i] + c1 * u1[base + i]);
}

// GMRES start: beta = |r0| (nrm holds <r0, r0>), V_0 = r0 / beta = -G / beta (scale), g = beta e_1
__global__ void k_gm_start(const double* nrm, double* scale, double* g, int m, int nz) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= nz) return;
  const double beta = sqrt(fmax(0.0, nrm[2 * z]));
  scale[z] = (beta > 1e-300) ? -1.0 / beta : 0.0;
  for (int k = 0; k <= m; ++k) {
    g[2 * ((size_t)z * (m + 1) + k)] = (k == 0) ? beta : 0.0;
    g[2 * ((size_t)z * (m + 1) + k) + 1] = 0.0;
  }
}

// Column j of the Hessenberg matrix from the two Gram-Schmidt passes (d1 + d2) and |w|, the earlier
// Givens rotations applied to it, a new rotation that zeroes H[j+1][j], and the rotated right-hand
// side g; scale = 1 / H[j+1][j] normalises the next Arnoldi vector (0 after a breakdown).
// Rotation k: [c_k, s_k; -conj(s_k), c_k] with c_k real.
__global__ void k_gm_col(int j, int m, const double* d1, const double* d2, int ldo, const double* nrm, double* H,
                         double* cs, double* sn, double* g, double* scale, int nz) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= nz) return;
  double* Hz = H + 2 * (size_t)z * (m + 1) * m;          // H[r][c] at 2 * (r * m + c)
  double* csz = cs + (size_t)z * m;
  double* snz = sn + 2 * (size_t)z * m;
  double* gz = g + 2 * (size_t)z * (m + 1);
  for (int r = 0; r <= j; ++r) {
    Hz[2 * (r * m + j)] = d1[2 * ((size_t)z * ldo + r)] + d2[2 * ((size_t)z * ldo + r)];
    Hz[2 * (r * m + j) + 1] = d1[2 * ((size_t)z * ldo + r) + 1] + d2[2 * ((size_t)z * ldo + r) + 1];
  }
  const double hn = sqrt(fmax(0.0, nrm[2 * z]));
  for (int k = 0; k < j; ++k) {
    const double c = csz[k], sr = snz[2 * k], si = snz[2 * k + 1];
    const double xr = Hz[2 * (k * m + j)], xi = Hz[2 * (k * m + j) + 1];
    const double yr = Hz[2 * ((k + 1) * m + j)], yi = Hz[2 * ((k + 1) * m + j) + 1];
    // x' = c x + s y ; y' = -conj(s) x + c y
    Hz[2 * (k * m + j)] = c * xr + (sr * yr - si * yi);
    Hz[2 * (k * m + j) + 1] = c * xi + (sr * yi + si * yr);
    Hz[2 * ((k + 1) * m + j)] = -(sr * xr + si * xi) + c * yr;
    Hz[2 * ((k + 1) * m + j) + 1] = -(sr * xi - si * xr) + c * yi;
  }
  const double ar = Hz[2 * (j * m + j)], ai = Hz[2 * (j * m + j) + 1];
  const double aa = sqrt(ar * ar + ai * ai);
  const double r = sqrt(aa * aa + hn * hn);
  double c, sr, si;
  if (r == 0.0) {
    c = 1.0; sr = 0.0; si = 0.0;
  } else if (aa == 0.0) {
    c = 0.0; sr = 1.0; si = 0.0;
  } else {
    c = aa / r;
    sr = ar / aa * hn / r;
    si = ai / aa * hn / r;
  }
  csz[j] = c;
  snz[2 * j] = sr;
  snz[2 * j + 1] = si;
  Hz[2 * (j * m + j)] = c * ar + sr * hn;
  Hz[2 * (j * m + j) + 1] = c * ai + si * hn;
  Hz[2 * ((j + 1) * m + j)] = 0.0;      // the rotation zeroes H[j+1][j]
  Hz[2 * ((j + 1) * m + j) + 1] = 0.0;
  const double gr = gz[2 * j], gi = gz[2 * j + 1];
  gz[2 * (j + 1)] = -(sr * gr + si * gi);
  gz[2 * (j + 1) + 1] = -(sr * gi - si * gr);
  gz[2 * j] = c * gr;
  gz[2 * j + 1] = c * gi;
  scale[z] = (hn > 1e-300) ? 1.0 / hn : 0.0;
}

// Back substitution R y = g over the first m rows (a zero pivot contributes nothing)
__global__ void k_gm_solve(int m, const double* H, const double* g, double* y, int ldo, int nz) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= nz) return;
  const double* Hz = H + 2 * (size_t)z * (m + 1) * m;
  const double* gz = g + 2 * (size_t)z * (m + 1);
  double* yz = y + 2 * (size_t)z * ldo;
  for (int k = m - 1; k >= 0; --k) {
    double br = gz[2 * k], bi = gz[2 * k + 1];
    for (int l = k + 1; l < m; ++l) {
      const double hr = Hz[2 * (k * m + l)], hi = Hz[2 * (k * m + l) + 1];
      br -= hr * yz[2 * l] - hi * yz[2 * l + 1];
      bi -= hr * yz[2 * l + 1] + hi * yz[2 * l];
    }
    const double pr = Hz[2 * (k * m + k)], pi = Hz[2 * (k * m + k) + 1];
    const double den = pr * pr + pi * pi;
    if (den > 0.0) {
      yz[2 * k] = (br * pr + bi * pi) / den;
      yz[2 * k + 1] = (bi * pr - br * pi) / den;
    } else {
      yz[2 * k] = 0.0;
      yz[2 * k + 1] = 0.0;
    }
  }
}

// y += alpha * x over complex state-sized buffers (alpha real)
__global__ void k_axpy(double* __restrict__ y, const double* __restrict__ x, double alpha, long long n) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < 2 * n; k += (long long)gridDim.x * blockDim.x)
    y[k] += alpha * x[k];
}

// dE/dtheta of the pulse amplitude at time t for theta = (E0, omega, sigma)
__device__ __forceinline__ void field_grad(const rtcc_field_t& f, double t, double g[3]) {
  const double x = t - f.t0;
  const double env = exp(-0.5 * x * x / (f.sigma * f.sigma));
  const bool cosc = f.carrier == RTCC_CARRIER_COS;
  const double car = cosc ? cos(f.omega * x) : sin(f.omega * x);
  const double dcar = cosc ? -x * sin(f.omega * x) : x * cos(f.omega * x);   // d carrier / d omega
  g[0] = f.sign * env * car;
  g[1] = f.sign * f.E0 * env * dcar;
  g[2] = f.sign * f.E0 * env * car * (x * x) / (f.sigma * f.sigma * f.sigma);
}

// grad[z][j] += Re( -dE/dtheta_j(t_z) * sum_pq fbar[z][p][q] (pol_z . mu)[p][q] ) for one stage
__global__ void k_theta_grad(double* grad, const double* fbar, const double* mu, const rtcc_field_t* fields,
                             const double* tz, double c, const double* hz, int n2) {
  const int z = blockIdx.x;
  const rtcc_field_t fl = fields[z];
  double pr = 0.0, pi = 0.0;
  for (int k = threadIdx.x; k < n2; k += blockDim.x) {
    const double m = fl.pol[0] * mu[k] + fl.pol[1] * mu[n2 + k] + fl.pol[2] * mu[2 * n2 + k];
    pr += fbar[2 * ((size_t)z * n2 + k)] * m;
    pi += fbar[2 * ((size_t)z * n2 + k) + 1] * m;
  }
  __shared__ double sh[2][32];
  for (int off = 16; off > 0; off >>= 1) {
    pr += __shfl_down_sync(0xffffffffu, pr, off);
    pi += __shfl_down_sync(0xffffffffu, pi, off);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = pr;
    sh[1][threadIdx.x >> 5] = pi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    pr = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) pr += sh[0][w];
    double g[3];
    field_grad(fl, tz[z] + c * hz[z], g);
    for (int j = 0; j < 3; ++j) grad[3 * z + j] += -g[j] * pr;   // real part of -dE/dtheta * P
  }
}

// Bounded wait on a flag that nothing sets: returns after `ns` nanoseconds with a status word.
__global__ void k_wait_flag(const volatile int* flag, unsigned long long ns, int* status) {
  unsigned long long t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  while (*flag == 0) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > ns) {
      *status = 1;
      return;
    }
  }
  *status = 0;
}

inline unsigned blocks_for(long long n, int threads = 256) {
  long long b = (n + threads - 1) / threads;
  return (unsigned)std::max(1ll, std::min(b, (long long)device_sm_count() * 32));
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

void set_last_error(const std::string& msg) { g_last_error = msg; }

}  // namespace rtcc

using namespace rtcc;

struct GroundEngine {
  std::unique_ptr<Engine> E;
  RhsPrograms rhs;
  Program energy;
  double *Y = nullptr, *R = nullptr, *F = nullptr, *Ec = nullptr;
  double *hx = nullptr, *he = nullptr, *dots = nullptr;   // DIIS history (one amplitude block)
  double* DIP = nullptr;
  DipolePrograms dip;
  unsigned long long* scratch = nullptr;
};

struct AdjointEngine {
  std::unique_ptr<Engine> E;
  RhsPrograms rhs;
  DipolePrograms dip;
  Program vjp, dvjp;
  double *Ys = nullptr, *F = nullptr, *Rout = nullptr, *cot = nullptr, *ybar = nullptr, *fbar = nullptr;
  double *Yd = nullptr, *DIP = nullptr, *wdip = nullptr, *ybar_obs = nullptr;
  double *k[4] = {nullptr}, *sin[4] = {nullptr}, *kbar[4] = {nullptr};
  double *y = nullptr, *abar = nullptr, *anew = nullptr;
  double *tdev = nullptr, *hdev = nullptr, *grad = nullptr;
};

struct rtcc_ctx {
  int dev = 0;
  cudaStream_t stream = nullptr;
  int o = 0, v = 0, nmo = 0, naux = 0, nz = 0;
  Prec prec = Prec::P64;
  long long ns = 0, nT = 0;
  double *f0 = nullptr, *Bd = nullptr, *mu = nullptr;
  double mu_ref[3] = {0, 0, 0};
  std::unique_ptr<IntegralStore> ints;
  std::unique_ptr<Engine> E;
  RhsPrograms rhs;
  DipolePrograms dip;
  // programs over the first k slots (k = 1 .. nz-1) of the same buffers: finished trajectories are
  // moved behind the running ones and the attempts run on the running slots only
  std::vector<RhsPrograms> rhs_k;
  std::vector<DipolePrograms> dip_k;
  double *Y = nullptr, *Ys = nullptr, *Ynew = nullptr, *Rout = nullptr, *Rk[kMaxStages] = {nullptr}, *F = nullptr,
         *DIP = nullptr;
  rtcc_field_t* d_fields = nullptr;
  Ctl ctl{};
  std::vector<void*> allocs;
  // Newton-Krylov work of the implicit Gauss-Legendre stages (allocated on first use)
  struct Krylov {
    int m = 0;
    long long bstride = 0;                       // doubles per [nz][ns] complex block
    double *V = nullptr, *W = nullptr, *DL = nullptr, *U = nullptr, *raw0 = nullptr;
    double *d1 = nullptr, *d2 = nullptr, *nrm = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr,
           *y = nullptr, *scale = nullptr, *eps = nullptr;
  } kry;
  std::unique_ptr<GroundEngine> gs[4];   // per precision, one trajectory
  std::unique_ptr<AdjointEngine> adj;
  long long last_stats[4] = {0, 0, 0, 0};
  long long last_slot_attempts = 0;   // sum over attempts of the slots they ran (last rtcc_propagate)
  void* out_stage = nullptr;          // device staging of host-side propagation outputs
  size_t out_stage_bytes = 0;
  Profiler prof;
  ~rtcc_ctx() {
    adj.reset();
    for (auto& g : gs) g.reset();
    E.reset();
    ints.reset();
    for (void* p : allocs) cudaFree(p);
    if (out_stage) cudaFree(out_stage);
    if (stream) cudaStreamDestroy(stream);
  }
  template <class T>
  T* alloc(size_t n) {
    T* p = static_cast<T*>(dev_alloc(n * sizeof(T)));
    allocs.push_back(p);
    RTCC_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), stream));
    return p;
  }
};

namespace {

rtcc_status_t fail(int code, const std::string& msg) {
  g_last_error = msg;
  return (rtcc_status_t)code;
}

template <class F>
rtcc_status_t guarded(F&& f) {
  try {
    f();
    return RTCC_OK;
  } catch (const Error& e) {
    return fail(e.status, e.what());
  } catch (const std::exception& e) {
    return fail(RTCC_ERR_CUDA, e.what());
  }
}

void copy_in(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  RTCC_CUDA(cudaMemcpyAsync(dst, src, bytes, is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
}
void copy_out(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  RTCC_CUDA(cudaMemcpyAsync(dst, src, bytes, is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
}

void run_dipole(rtcc_ctx* h, int nact = 0) {
  h->E->run((nact <= 0 || nact == h->nz) ? h->dip.prog : h->dip_k[nact].prog);
}

const RhsPrograms& rhs_for(rtcc_ctx* h, int nact) { return (nact == h->nz) ? h->rhs : h->rhs_k[nact]; }

bool autotune_on() {
  const char* e = std::getenv("RTCC_NO_AUTOTUNE");
  return !(e && e[0] == '1');
}

// Tensor-core tiles of the programs over nact slots, chosen on first use (Engine::autotune).
void tune_slots(rtcc_ctx* h, int nact) {
  if (!autotune_on() || h->prec == Prec::P64) return;
  RhsPrograms& r = (nact == h->nz) ? h->rhs : h->rhs_k[nact];
  DipolePrograms& d = (nact == h->nz) ? h->dip : h->dip_k[nact];
  h->E->autotune(r.fwd);
  h->E->autotune(r.rev);
  h->E->autotune(d.prog);
}

// Step of the forward-difference Jacobian products of the Newton-Krylov stage solve (the Krylov
// vectors have unit norm): small in float64; in the split modes large enough that the
// right-hand side's rounding (about 1e-6 of it) stays well below the difference.
double kry_eps(Prec p) { return p == Prec::P64 ? 1e-6 : 1e-3; }

// Krylov work for m Arnoldi vectors over all slots (grown when a later call asks for more).
void ensure_krylov(rtcc_ctx* h, int m) {
  rtcc_ctx::Krylov& K = h->kry;
  if (K.m >= m) return;
  RTCC_CUDA(cudaStreamSynchronize(h->stream));
  for (double* p : {K.V, K.W, K.DL, K.U, K.raw0, K.d1, K.d2, K.nrm, K.H, K.cs, K.sn, K.g, K.y, K.scale, K.eps}) {
    if (!p) continue;
    auto it = std::find(h->allocs.begin(), h->allocs.end(), (void*)p);
    if (it != h->allocs.end()) h->allocs.erase(it);
    cudaFree(p);
  }
  const size_t nz = h->nz, ldo = kKrylovMax + 1;
  K.bstride = 2 * h->ns * (long long)nz;
  const size_t bs = (size_t)K.bstride;
  K.V = h->alloc<double>(2 * bs * (m + 1));
  K.W = h->alloc<double>(2 * bs);
  K.DL = h->alloc<double>(2 * bs);
  K.U = h->alloc<double>(2 * bs);
  K.raw0 = h->alloc<double>(bs);
  K.d1 = h->alloc<double>(2 * nz * ldo);
  K.d2 = h->alloc<double>(2 * nz * ldo);
  K.y = h->alloc<double>(2 * nz * ldo);
  K.nrm = h->alloc<double>(2 * nz);
  K.H = h->alloc<double>(2 * nz * (m + 1) * m);
  K.cs = h->alloc<double>(nz * m);
  K.sn = h->alloc<double>(2 * nz * m);
  K.g = h->alloc<double>(2 * nz * (m + 1));
  K.scale = h->alloc<double>(nz);
  K.eps = h->alloc<double>(nz);
  std::vector<double> e(nz, kry_eps(h->prec));
  RTCC_CUDA(cudaMemcpyAsync(K.eps, e.data(), sizeof(double) * nz, cudaMemcpyHostToDevice, h->stream));
  RTCC_CUDA(cudaStreamSynchronize(h->stream));
  K.m = m;
}

// One Runge-Kutta attempt over the first nact slots (stages, combination, controller, accept, dipole, record).
void run_attempt(rtcc_ctx* h, const Tableau& tb, const rtcc_integrator_t& in, double* tout, double* muout, int max_out,
                 int nact) {
  cudaStream_t s = h->stream;
  Profiler& pr = h->prof;
  const int nz = nact;
  const RhsPrograms& rp = rhs_for(h, nact);
  const long long ns = h->ns, nT = h->nT;
  const double sb = 16.0 * (double)ns * nz;   // bytes of one state-sized complex buffer
  const dim3 gst(blocks_for(ns) / nz + 1 > 4096 ? 4096 : blocks_for(ns) / nz + 1, nz);
  pr.start(s);
  k_prestep<<<(nz + 127) / 128, 128, 0, s>>>(h->ctl, in, nz);
  pr.stop(s, KC_RK, 0, 0);
  auto stage_rhs = [&](const StageArgs& A, double c) {
    pr.start(s);
    if (h->prec != Prec::P64) k_stage<true><<<gst, 256, 0, s>>>(h->Ys, h->Y, A, h->ctl.htry, ns, nT);
    else k_stage<false><<<gst, 256, 0, s>>>(h->Ys, h->Y, A, h->ctl.htry, ns, nT);
    pr.stop(s, KC_RK, 0, sb * (A.nterms + 2));
    pr.start(s);
    k_fock<<<dim3(blocks_for((long long)h->nmo * h->nmo), nz), 256, 0, s>>>(h->F, h->f0, h->mu, h->d_fields, h->ctl.t,
                                                                           h->ctl.htry, c, nz, h->nmo * h->nmo);
    pr.stop(s, KC_RK, 0, 8.0 * h->nmo * h->nmo * (4 + nz));
    h->E->run(rp.fwd);
    h->E->run(rp.rev);
  };
  const size_t rbytes = sizeof(double) * 2 * (size_t)ns * nz;
  if (tb.implicit) {
    // K_1 = K_2 = f(t, y), then Gauss-Seidel sweeps K_i <- f(t + c_i h, y + h sum_j a_ij D K_j)
    StageArgs A0{};
    stage_rhs(A0, 0.0);
    RTCC_CUDA(cudaMemcpyAsync(h->Rk[0], h->Rout, rbytes, cudaMemcpyDeviceToDevice, s));
    RTCC_CUDA(cudaMemcpyAsync(h->Rk[1], h->Rout, rbytes, cudaMemcpyDeviceToDevice, s));
    for (int sw = 0; sw < tb.sweeps; ++sw)
      for (int st = 0; st < tb.s; ++st) {
        StageArgs A{};
        A.nterms = tb.s;
        for (int j = 0; j < tb.s; ++j) {
          A.R[j] = h->Rk[j];
          A.coef[j] = tb.a[st][j];
        }
        stage_rhs(A, tb.c[st]);
        // the last evaluation stays in Rout, so Rk[1] keeps the previous sweep's K_2 for the
        // convergence measure h max |K_2(new) - K_2(old)| formed by the final combination
        if (sw < tb.sweeps - 1 || st < tb.s - 1)
          RTCC_CUDA(cudaMemcpyAsync(h->Rk[st], h->Rout, rbytes, cudaMemcpyDeviceToDevice, s));
      }
  }
  if (tb.newton) {
    // Simplified Newton on G_i(K) = K_i - f(t + c_i h, y + h sum_j a_ij D K_j) (raw right-hand sides K_i),
    // each correction from (I - h A x J) dK = -G with J = df/dy at (t, y), J v = (f(t, y + eps D v) -
    // f(t, y)) / eps, solved by GMRES(m) from dK = 0: Arnoldi with classical Gram-Schmidt done twice,
    // Givens rotations and the back substitution per trajectory on the device.
    rtcc_ctx::Krylov& K = h->kry;
    const int m = tb.krylov;
    const long long bs = K.bstride;
    const int ldo = kKrylovMax + 1;
    const dim3 gv(gst.x, nz);
    const unsigned gx = std::min<unsigned>(gst.x, 128u);
    const unsigned gsc = (unsigned)((nz + 127) / 128);
    auto jvp_stage = [&](const double* v) {   // Ys = y + eps_z D v
      StageArgs A{};
      A.nterms = 1;
      A.R[0] = v;
      A.coef[0] = 1.0;
      if (h->prec != Prec::P64) k_stage<true><<<gst, 256, 0, s>>>(h->Ys, h->Y, A, K.eps, ns, nT);
      else k_stage<false><<<gst, 256, 0, s>>>(h->Ys, h->Y, A, K.eps, ns, nT);
      k_fock<<<dim3(blocks_for((long long)h->nmo * h->nmo), nz), 256, 0, s>>>(h->F, h->f0, h->mu, h->d_fields, h->ctl.t,
                                                                             h->ctl.htry, 0.0, nz, h->nmo * h->nmo);
      h->E->run(rp.fwd);
      h->E->run(rp.rev);
    };
    auto dots = [&](const double* V, int nvec, const double* w, double* out, int ld) {
      RTCC_CUDA(cudaMemsetAsync(out, 0, sizeof(double) * 2 * (size_t)nz * ld, s));
      k_zdots<<<dim3(gx, nz, nvec), 256, 0, s>>>(V, 2 * bs, w, bs, ns, ld, out);
    };
    StageArgs A0{};
    stage_rhs(A0, 0.0);   // f(t, y): the starting stages and the base point of the Jacobian products
    RTCC_CUDA(cudaMemcpyAsync(K.raw0, h->Rout, rbytes, cudaMemcpyDeviceToDevice, s));
    RTCC_CUDA(cudaMemcpyAsync(h->Rk[0], h->Rout, rbytes, cudaMemcpyDeviceToDevice, s));
    RTCC_CUDA(cudaMemcpyAsync(h->Rk[1], h->Rout, rbytes, cudaMemcpyDeviceToDevice, s));
    for (int it = 0; it < tb.sweeps; ++it) {
      for (int st = 0; st < 2; ++st) {   // G_i into W (block i)
        StageArgs A{};
        A.nterms = 2;
        for (int j = 0; j < 2; ++j) {
          A.R[j] = h->Rk[j];
          A.coef[j] = tb.a[st][j];
        }
        stage_rhs(A, tb.c[st]);
        Combo C{};
        C.m = 2;
        C.x[0] = h->Rk[st];
        C.c[0] = 1.0;
        C.x[1] = h->Rout;
        C.c[1] = -1.0;
        k_combine<<<blocks_for(ns * nz), 256, 0, s>>>(K.W + st * bs, C, ns * nz);
      }
      dots(K.W, 1, K.W, K.nrm, 1);
      k_gm_start<<<gsc, 128, 0, s>>>(K.nrm, K.scale, K.g, m, nz);
      k_zscale<<<gv, 256, 0, s>>>(K.V, K.W, K.scale, bs, ns);   // V_0 = -G / |G|
      for (int j = 0; j < m; ++j) {
        const double* Vj = K.V + (size_t)j * 2 * bs;
        for (int jj = 0; jj < 2; ++jj) {   // u_jj = J D V_j[jj]
          jvp_stage(Vj + jj * bs);
          Combo C{};
          C.m = 2;
          C.x[0] = h->Rout;
          C.c[0] = 1.0 / kry_eps(h->prec);
          C.x[1] = K.raw0;
          C.c[1] = -1.0 / kry_eps(h->prec);
          k_combine<<<blocks_for(ns * nz), 256, 0, s>>>(K.U + jj * bs, C, ns * nz);
        }
        for (int i = 0; i < 2; ++i)   // W_i = V_j[i] - h sum_jj a_i,jj u_jj
          k_lincomb_h<<<gv, 256, 0, s>>>(K.W + i * bs, Vj + i * bs, K.U, K.U + bs, tb.a[i][0], tb.a[i][1],
                                         h->ctl.htry, ns);
        dots(K.V, j + 1, K.W, K.d1, ldo);
        k_zupdate<<<gv, 256, 0, s>>>(K.W, K.V, 2 * bs, j + 1, K.d1, ldo, -1.0, bs, ns);
        dots(K.V, j + 1, K.W, K.d2, ldo);
        k_zupdate<<<gv, 256, 0, s>>>(K.W, K.V, 2 * bs, j + 1, K.d2, ldo, -1.0, bs, ns);
        dots(K.W, 1, K.W, K.nrm, 1);
        k_gm_col<<<gsc, 128, 0, s>>>(j, m, K.d1, K.d2, ldo, K.nrm, K.H, K.cs, K.sn, K.g, K.scale, nz);
        k_zscale<<<gv, 256, 0, s>>>(K.V + (size_t)(j + 1) * 2 * bs, K.W, K.scale, bs, ns);
      }
      k_gm_solve<<<gsc, 128, 0, s>>>(m, K.H, K.g, K.y, ldo, nz);
      RTCC_CUDA(cudaMemsetAsync(K.DL, 0, rbytes, s));
      RTCC_CUDA(cudaMemsetAsync(K.DL + bs, 0, rbytes, s));
      k_zupdate<<<gv, 256, 0, s>>>(K.DL, K.V, 2 * bs, m, K.y, ldo, 1.0, bs, ns);
      k_axpy<<<blocks_for(ns * nz), 256, 0, s>>>(h->Rk[0], K.DL, 1.0, ns * nz);
      k_axpy<<<blocks_for(ns * nz), 256, 0, s>>>(h->Rk[1], K.DL + bs, 1.0, ns * nz);
    }
  }
  for (int st = 0; st < ((tb.implicit || tb.newton) ? 0 : tb.s); ++st) {
    StageArgs A{};
    A.nterms = 0;
    for (int j = 0; j < st; ++j) {
      if (tb.a[st][j] == 0.0 && j != st - 1) continue;
      A.R[A.nterms] = (j == st - 1) ? h->Rout : h->Rk[j];
      A.coef[A.nterms] = tb.a[st][j];
      ++A.nterms;
    }
    if (st > 0) {
      A.copy_src = h->Rout;
      A.copy_dst = h->Rk[st - 1];
    }
    pr.start(s);
    if (h->prec != Prec::P64) k_stage<true><<<gst, 256, 0, s>>>(h->Ys, h->Y, A, h->ctl.htry, ns, nT);
    else k_stage<false><<<gst, 256, 0, s>>>(h->Ys, h->Y, A, h->ctl.htry, ns, nT);
    pr.stop(s, KC_RK, 0, sb * (A.nterms + 2 + (st > 0 ? 1 : 0)));
    pr.start(s);
    k_fock<<<dim3(blocks_for((long long)h->nmo * h->nmo), nz), 256, 0, s>>>(h->F, h->f0, h->mu, h->d_fields, h->ctl.t,
                                                                           h->ctl.htry, tb.c[st], nz, h->nmo * h->nmo);
    pr.stop(s, KC_RK, 0, 8.0 * h->nmo * h->nmo * (4 + nz));
    h->E->run(rp.fwd);
    h->E->run(rp.rev);
  }
  StageArgs B{}, Ew{};
  for (int j = 0; j < tb.s; ++j) {
    B.R[j] = (j == tb.s - 1) ? h->Rout : h->Rk[j];
    B.coef[j] = tb.b[j];
    Ew.coef[j] = tb.e[j];
  }
  B.nterms = tb.s;
  if (tb.newton) {
    // the converged stages; error slot: h max |last Newton correction of K_2|
    B.R[0] = h->Rk[0];
    B.R[1] = h->Rk[1];
    B.R[2] = h->kry.DL + h->kry.bstride;
    B.coef[0] = tb.b[0];
    B.coef[1] = tb.b[1];
    B.coef[2] = 0.0;
    Ew.coef[0] = Ew.coef[1] = 0.0;
    Ew.coef[2] = 1.0;
    B.nterms = 3;
  }
  if (tb.implicit) {
    // error slot: +1 on the newest K_2 (Rout), -1 on the previous sweep's K_2 (Rk[1], weight 0 in y)
    for (int j = 0; j < tb.s; ++j) Ew.coef[j] = (j == tb.s - 1) ? 1.0 : 0.0;
    B.R[tb.s] = h->Rk[tb.s - 1];
    B.coef[tb.s] = 0.0;
    Ew.coef[tb.s] = -1.0;
    B.nterms = tb.s + 1;
  }
  const int measure = (tb.adaptive || tb.implicit || tb.newton) ? 1 : 0;
  pr.start(s);
  if (h->prec != Prec::P64)
    k_final<true><<<gst, 256, 0, s>>>(h->Ynew, h->Y, B, Ew, h->ctl.htry, ns, nT, h->ctl.err_bits, measure);
  else
    k_final<false><<<gst, 256, 0, s>>>(h->Ynew, h->Y, B, Ew, h->ctl.htry, ns, nT, h->ctl.err_bits, measure);
  pr.stop(s, KC_RK, 0, sb * (B.nterms + 2));
  pr.start(s);
  k_controller<<<(nz + 127) / 128, 128, 0, s>>>(h->ctl, in, nz);
  pr.stop(s, KC_RK, 0, 0);
  pr.start(s);
  k_accept<<<gst, 256, 0, s>>>(h->Y, h->Ynew, h->ctl.accepted, ns);
  pr.stop(s, KC_RK, 0, 2 * sb);
  run_dipole(h, nact);
  pr.start(s);
  k_record<<<(nz + 127) / 128, 128, 0, s>>>(h->ctl, h->DIP, h->mu_ref[0], h->mu_ref[1], h->mu_ref[2], tout, muout, max_out,
                                            nz, 0);
  pr.stop(s, KC_RK, 0, 0);
  RTCC_CUDA(cudaGetLastError());
}

long long total_count(const Profiler& p) {
  long long c = 0;
  for (int k = 0; k < KC_N; ++k) c += p.count[k];
  return c;
}

constexpr int kDiis = 8;

GroundEngine* ground_engine(rtcc_ctx* h, Prec p) {
  auto& slot = h->gs[(int)p];
  if (slot) return slot.get();
  auto g = std::make_unique<GroundEngine>();
  g->E = std::make_unique<Engine>(p, h->stream);
  Engine& E = *g->E;
  const IntIds I = register_integrals(E, *h->ints);
  g->Y = h->alloc<double>(2 * h->ns);
  g->R = h->alloc<double>(2 * h->ns);
  g->F = h->alloc<double>((size_t)h->nmo * h->nmo);
  g->Ec = h->alloc<double>(2);
  g->hx = h->alloc<double>((size_t)2 * h->nT * kDiis);
  g->he = h->alloc<double>((size_t)2 * h->nT * kDiis);
  g->dots = h->alloc<double>(kDiis);
  g->scratch = h->alloc<unsigned long long>(1);
  RTCC_CUDA(cudaMemcpyAsync(g->F, h->f0, sizeof(double) * h->nmo * h->nmo, cudaMemcpyDeviceToDevice, h->stream));
  g->rhs = build_rhs(E, I, 1, h->o, h->v, g->Y, g->F, g->R, true);
  g->energy = build_energy(E, I, g->rhs, 1, h->o, h->v, g->F, g->Ec);
  g->DIP = h->alloc<double>(6);
  if (p == Prec::P64) {
    g->dip = build_dipole(E, 1, h->o, h->v, g->Y, h->mu, g->DIP);
    h->allocs.push_back(g->dip.fdummy);
    E.finalize({&g->rhs.fwd, &g->rhs.rev, &g->energy, &g->dip.prog});
  } else {
    E.finalize({&g->rhs.fwd, &g->rhs.rev, &g->energy});
  }
  if (autotune_on() && p != Prec::P64) {
    E.autotune(g->rhs.fwd);
    E.autotune(g->rhs.rev);
  }
  slot = std::move(g);
  return slot.get();
}

double read_max(rtcc_ctx* h, const double* r, long long n, unsigned long long* scratch) {
  RTCC_CUDA(cudaMemsetAsync(scratch, 0, sizeof(unsigned long long), h->stream));
  k_maxabs<<<blocks_for(n), 256, 0, h->stream>>>(r, n, scratch);
  unsigned long long bits = 0;
  RTCC_CUDA(cudaMemcpyAsync(&bits, scratch, sizeof(bits), cudaMemcpyDeviceToHost, h->stream));
  RTCC_CUDA(cudaStreamSynchronize(h->stream));
  double m;
  std::memcpy(&m, &bits, sizeof(m));
  return m;
}

// Jacobi + DIIS on one amplitude block (T or Lambda) of a ground-state engine.  Returns the final
// max-abs residual.  With `floor_ok` the iteration also stops (without error) once the residual
// has not improved for 10 iterations: the rounding floor of a reduced-precision engine.
double solve_block(rtcc_ctx* h, GroundEngine* g, bool lambda, double tol, int maxiter, bool floor_ok) {
  const long long nT = h->nT;
  double* x = g->Y + (lambda ? 2 * nT : 0);
  double* r = g->R + (lambda ? 2 * nT : 0);
  int count = 0;
  double Bm[kDiis][kDiis] = {};
  double best = INFINITY;
  int since_best = 0;
  if (lambda) g->E->run(g->rhs.fwd);   // intermediates of the converged t stay valid
  for (int it = 0; it < maxiter; ++it) {
    if (lambda) g->E->run(g->rhs.rev);
    else g->E->run(g->rhs.fwd);
    const double err = read_max(h, r, nT, g->scratch);
    if (std::getenv("RTCC_VERBOSE"))
      std::fprintf(stderr, "[rtcc] ground state %s prec=%d iter %d max|residual| %.3e\n", lambda ? "Lambda" : "T",
                   (int)g->E->prec(), it, err);
    if (!std::isfinite(err)) throw Error(RTCC_ERR_DIVERGED, "ground-state residual is not finite");
    if (err < tol) return err;
    if (err < 0.999 * best) {
      best = err;
      since_best = 0;
    } else if (floor_ok && ++since_best >= 10) {
      return err;
    }
    const int slot = count % kDiis;
    double* xs = g->hx + (size_t)2 * nT * slot;
    double* es = g->he + (size_t)2 * nT * slot;
    k_jacobi<<<blocks_for(nT), 256, 0, h->stream>>>(x, r, h->f0, h->o, h->v, h->nmo, es);
    RTCC_CUDA(cudaMemcpyAsync(xs, x, sizeof(double) * 2 * nT, cudaMemcpyDeviceToDevice, h->stream));
    ++count;
    const int m = std::min(count, kDiis);
    RTCC_CUDA(cudaMemsetAsync(g->dots, 0, sizeof(double) * kDiis, h->stream));
    for (int j = 0; j < m; ++j)
      k_dot<<<blocks_for(nT), 256, 0, h->stream>>>(es, g->he + (size_t)2 * nT * j, nT, g->dots + j);
    double row[kDiis];
    RTCC_CUDA(cudaMemcpyAsync(row, g->dots, sizeof(double) * kDiis, cudaMemcpyDeviceToHost, h->stream));
    RTCC_CUDA(cudaStreamSynchronize(h->stream));
    for (int j = 0; j < m; ++j) Bm[slot][j] = Bm[j][slot] = row[j];
    if (m >= 3) {
      // DIIS: minimise |sum c_j e_j| with sum c_j = 1, i.e. [B -1; -1 0][c; l] = [0; -1]
      // (Gauss-Jordan elimination with partial pivoting on the (m+1) x (m+1) system)
      const int N = m + 1;
      double A[kDiis + 1][kDiis + 2] = {};
      for (int i = 0; i < m; ++i) {
        for (int j = 0; j < m; ++j) A[i][j] = Bm[i][j];
        A[i][m] = -1.0;
        A[m][i] = -1.0;
      }
      A[m][N] = -1.0;
      bool ok = true;
      for (int c = 0; c < N && ok; ++c) {
        int p = c;
        for (int i = c + 1; i < N; ++i)
          if (std::fabs(A[i][c]) > std::fabs(A[p][c])) p = i;
        if (std::fabs(A[p][c]) < 1e-300) {
          ok = false;
          break;
        }
        for (int j = 0; j <= N; ++j) std::swap(A[c][j], A[p][j]);
        for (int i = 0; i < N; ++i) {
          if (i == c) continue;
          const double f = A[i][c] / A[c][c];
          for (int j = c; j <= N; ++j) A[i][j] -= f * A[c][j];
        }
      }
      if (ok) {
        Combo C{};
        C.m = m;
        for (int j = 0; j < m; ++j) {
          C.x[j] = g->hx + (size_t)2 * nT * j;
          C.c[j] = A[j][N] / A[j][j];
        }
        k_combine<<<blocks_for(2 * nT), 256, 0, h->stream>>>(x, C, nT);
      }
    }
    k_sym_pair<<<blocks_for(nT), 256, 0, h->stream>>>(x + 2ll * h->o * h->v, h->o, h->v);
  }
  if (floor_ok) return best;
  throw Error(RTCC_ERR_NOCONV, std::string("ground-state ") + (lambda ? "Lambda" : "T") + " equations did not converge");
}


// ---------------------------------------------------------------------------------------
// Adjoint of RK4 (discrete, checkpointed): gradients of J = sum_n sum_x w[n][x] Re mu_x(t_n)
// with respect to the pulse parameters (E0, omega, sigma).  Every map is holomorphic in the
// complex state, so the adjoint uses unconjugated VJPs and dJ/dtheta = Re dG/dtheta.

AdjointEngine* adjoint_engine(rtcc_ctx* h) {
  if (h->adj) return h->adj.get();
  auto a = std::make_unique<AdjointEngine>();
  a->E = std::make_unique<Engine>(h->prec, h->stream);
  Engine& E = *a->E;
  const IntIds I = register_integrals(E, *h->ints);
  const size_t nsz = (size_t)2 * h->ns * h->nz;
  const size_t n2 = (size_t)h->nmo * h->nmo;
  a->Ys = h->alloc<double>(nsz);
  a->Rout = h->alloc<double>(nsz);
  a->cot = h->alloc<double>(nsz);
  a->ybar = h->alloc<double>(nsz);
  a->Yd = h->alloc<double>(nsz);
  a->ybar_obs = h->alloc<double>(nsz);
  a->y = h->alloc<double>(nsz);
  a->abar = h->alloc<double>(nsz);
  a->anew = h->alloc<double>(nsz);
  for (int s = 0; s < 4; ++s) {
    a->k[s] = h->alloc<double>(nsz);
    a->sin[s] = h->alloc<double>(nsz);
    a->kbar[s] = h->alloc<double>(nsz);
  }
  a->F = h->alloc<double>(n2 * h->nz);
  a->fbar = h->alloc<double>(2 * n2 * h->nz);
  a->DIP = h->alloc<double>((size_t)6 * h->nz);
  a->wdip = h->alloc<double>((size_t)6 * h->nz);
  a->tdev = h->alloc<double>(h->nz);
  a->hdev = h->alloc<double>(h->nz);
  a->grad = h->alloc<double>((size_t)3 * h->nz);
  a->rhs = build_rhs(E, I, h->nz, h->o, h->v, a->Ys, a->F, a->Rout, true);
  a->vjp = build_rhs_vjp(E, a->rhs, h->nz, h->o, h->v, a->cot, a->ybar, a->fbar);
  a->dip = build_dipole(E, h->nz, h->o, h->v, a->Yd, h->mu, a->DIP);
  h->allocs.push_back(a->dip.fdummy);
  a->dvjp = build_dipole_vjp(E, a->dip, h->nz, h->o, h->v, a->wdip, a->ybar_obs);
  E.finalize({&a->rhs.fwd, &a->rhs.rev, &a->vjp, &a->dip.prog, &a->dvjp});
  if (autotune_on() && h->prec != Prec::P64)
    for (Program* P : {&a->rhs.fwd, &a->rhs.rev, &a->vjp, &a->dip.prog, &a->dvjp}) E.autotune(*P);
  h->adj = std::move(a);
  return h->adj.get();
}

void adj_set_time(rtcc_ctx* h, AdjointEngine* a, double t, double hs) {
  std::vector<double> tv(h->nz, t), hv(h->nz, hs);
  RTCC_CUDA(cudaMemcpyAsync(a->tdev, tv.data(), sizeof(double) * h->nz, cudaMemcpyHostToDevice, h->stream));
  RTCC_CUDA(cudaMemcpyAsync(a->hdev, hv.data(), sizeof(double) * h->nz, cudaMemcpyHostToDevice, h->stream));
}

// stage st of RK4 from state y: Ys = y + h sum_j a_sj D k_j, f(t + c h), right-hand side -> Rout
void adj_stage(rtcc_ctx* h, AdjointEngine* a, const Tableau& tb, const double* y, int st) {
  cudaStream_t s = h->stream;
  const long long ns = h->ns, nT = h->nT;
  const int nz = h->nz;
  const dim3 gst(blocks_for(ns) / nz + 1 > 4096 ? 4096 : blocks_for(ns) / nz + 1, nz);
  StageArgs A{};
  for (int j = 0; j < st; ++j) {
    if (tb.a[st][j] == 0.0) continue;
    A.R[A.nterms] = a->k[j];
    A.coef[A.nterms] = tb.a[st][j];
    ++A.nterms;
  }
  k_stage<false><<<gst, 256, 0, s>>>(a->Ys, y, A, a->hdev, ns, nT);
  k_fock<<<dim3(blocks_for((long long)h->nmo * h->nmo), nz), 256, 0, s>>>(a->F, h->f0, h->mu, h->d_fields, a->tdev,
                                                                         a->hdev, tb.c[st], nz, h->nmo * h->nmo);
  a->E->run(a->rhs.fwd);
  a->E->run(a->rhs.rev);
}

// one RK4 step from y (device) into ynew, keeping the stage inputs and right-hand sides
void adj_step(rtcc_ctx* h, AdjointEngine* a, const Tableau& tb, const double* y, double* ynew) {
  cudaStream_t s = h->stream;
  const size_t bytes = sizeof(double) * 2 * h->ns * h->nz;
  for (int st = 0; st < 4; ++st) {
    adj_stage(h, a, tb, y, st);
    RTCC_CUDA(cudaMemcpyAsync(a->sin[st], a->Ys, bytes, cudaMemcpyDeviceToDevice, s));
    RTCC_CUDA(cudaMemcpyAsync(a->k[st], a->Rout, bytes, cudaMemcpyDeviceToDevice, s));
  }
  StageArgs B{}, Ew{};
  for (int j = 0; j < 4; ++j) {
    B.R[j] = a->k[j];
    B.coef[j] = tb.b[j];
  }
  B.nterms = 4;
  const dim3 gst(blocks_for(h->ns) / h->nz + 1 > 4096 ? 4096 : blocks_for(h->ns) / h->nz + 1, h->nz);
  k_final<false><<<gst, 256, 0, s>>>(ynew, y, B, Ew, a->hdev, h->ns, h->nT, h->ctl.err_bits, 0);
  RTCC_CUDA(cudaGetLastError());
}

// dipoles of state y (device) into host mu[z][x] (real parts) and the observable VJP seed
void adj_dipole(rtcc_ctx* h, AdjointEngine* a, const double* y, std::vector<double>& mu) {
  const size_t bytes = sizeof(double) * 2 * h->ns * h->nz;
  RTCC_CUDA(cudaMemcpyAsync(a->Yd, y, bytes, cudaMemcpyDeviceToDevice, h->stream));
  a->E->run(a->dip.prog);
  std::vector<double> d((size_t)6 * h->nz);
  RTCC_CUDA(cudaMemcpyAsync(d.data(), a->DIP, sizeof(double) * d.size(), cudaMemcpyDeviceToHost, h->stream));
  RTCC_CUDA(cudaStreamSynchronize(h->stream));
  mu.assign((size_t)3 * h->nz, 0.0);
  for (int z = 0; z < h->nz; ++z)
    for (int x = 0; x < 3; ++x) mu[3 * z + x] = d[2 * (x * h->nz + z)] + h->mu_ref[x];
}

// abar += (d mu / dy)^T w_n at state y (the dipole program must have run on y)
void adj_observable(rtcc_ctx* h, AdjointEngine* a, const double* wn, double* abar) {
  std::vector<double> wd((size_t)6 * h->nz, 0.0);
  for (int x = 0; x < 3; ++x)
    for (int z = 0; z < h->nz; ++z) wd[2 * (x * h->nz + z)] = wn[x];
  RTCC_CUDA(cudaMemcpyAsync(a->wdip, wd.data(), sizeof(double) * wd.size(), cudaMemcpyHostToDevice, h->stream));
  RTCC_CUDA(cudaMemsetAsync(a->ybar_obs, 0, sizeof(double) * 2 * h->ns * h->nz, h->stream));
  a->E->run(a->dvjp);
  k_axpy<<<blocks_for(h->ns * h->nz), 256, 0, h->stream>>>(abar, a->ybar_obs, 1.0, h->ns * h->nz);
}

}  // namespace

extern "C" {

const char* rtcc_last_error(void) { return g_last_error.c_str(); }

rtcc_status_t rtcc_create(const double* f, const double* B, int naux, const double* mu, int o, int v, int ntraj,
                          int prec, rtcc_handle_t* out) {
  return rtcc_create_frozen_core(f, B, naux, mu, o, v, 0, ntraj, prec, out);
}

rtcc_status_t rtcc_create_frozen_core(const double* f_all, const double* B_all, int naux, const double* mu_all,
                                      int o_all, int v, int nfc, int ntraj, int prec, rtcc_handle_t* out) {
  if (!out) return fail(RTCC_ERR_INVALID_ARG, "out is null");
  *out = nullptr;
  if (!f_all || !B_all || !mu_all) return fail(RTCC_ERR_INVALID_ARG, "null input pointer");
  if (nfc < 0 || nfc >= o_all) return fail(RTCC_ERR_INVALID_ARG, "frozen-core count must be in [0, o)");
  if (o_all < 1 || v < 1 || naux < 1) return fail(RTCC_ERR_INVALID_ARG, "bad sizes");
  // Frozen core: the lowest nfc occupied orbitals stay doubly occupied and uncorrelated.  The
  // active problem uses the active blocks of f (which already carries the core's mean field),
  // of the factors B and of mu; the core's constant dipole 2 sum_c mu_cc joins the reference term.
  const int na = o_all + v, nact = na - nfc;
  std::vector<double> fa, Ba, mua;
  const double *f = f_all, *B = B_all, *mu = mu_all;
  double core_ref[3] = {0, 0, 0};
  if (nfc > 0) {
    fa.resize((size_t)nact * nact);
    Ba.resize((size_t)naux * nact * nact);
    mua.resize((size_t)3 * nact * nact);
    for (int p = 0; p < nact; ++p)
      for (int q = 0; q < nact; ++q) {
        const size_t src = (size_t)(p + nfc) * na + (q + nfc), dst = (size_t)p * nact + q;
        fa[dst] = f_all[src];
        for (int P = 0; P < naux; ++P) Ba[(size_t)P * nact * nact + dst] = B_all[(size_t)P * na * na + src];
        for (int x = 0; x < 3; ++x) mua[(size_t)x * nact * nact + dst] = mu_all[(size_t)x * na * na + src];
      }
    for (int x = 0; x < 3; ++x)
      for (int c = 0; c < nfc; ++c) core_ref[x] += 2.0 * mu_all[(size_t)x * na * na + (size_t)c * na + c];
    f = fa.data();
    B = Ba.data();
    mu = mua.data();
  }
  const int o = o_all - nfc;
  *out = nullptr;
  if (o < 1 || v < 1 || naux < 1 || ntraj < 1 || ntraj > 4096) return fail(RTCC_ERR_INVALID_ARG, "bad sizes");
  if (prec < 0 || prec > 3) return fail(RTCC_ERR_INVALID_ARG, "unknown precision");
  const int n = o + v;
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < p; ++q) {
      if (f[p * n + q] != f[q * n + p]) return fail(RTCC_ERR_INVALID_ARG, "Fock matrix is not symmetric");
      for (int x = 0; x < 3; ++x)
        if (mu[(size_t)x * n * n + p * n + q] != mu[(size_t)x * n * n + q * n + p])
          return fail(RTCC_ERR_INVALID_ARG, "dipole matrix is not symmetric");
      for (int P = 0; P < naux; ++P)
        if (B[(size_t)P * n * n + p * n + q] != B[(size_t)P * n * n + q * n + p])
          return fail(RTCC_ERR_INVALID_ARG, "density-fitting factors are not symmetric");
    }
  auto* h = new rtcc_ctx();
  rtcc_status_t st = guarded([&] {
    int ndev = 0;
    RTCC_CUDA(cudaGetDeviceCount(&ndev));
    if (ndev < 1) throw Error(RTCC_ERR_CUDA, "no CUDA device");
    RTCC_CUDA(cudaGetDevice(&h->dev));
    cudaDeviceProp prop;
    RTCC_CUDA(cudaGetDeviceProperties(&prop, h->dev));
    if (prop.major < 10) throw Error(RTCC_ERR_CUDA, "this library needs an sm_103a (Blackwell) GPU");
    RTCC_CUDA(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    h->o = o;
    h->v = v;
    h->nmo = n;
    h->naux = naux;
    h->nz = ntraj;
    h->prec = (Prec)prec;
    h->nT = (long long)o * v + (long long)o * o * v * v;
    h->ns = 2 * h->nT;
    h->f0 = h->alloc<double>((size_t)n * n);
    h->mu = h->alloc<double>((size_t)3 * n * n);
    h->Bd = h->alloc<double>((size_t)naux * n * n);
    copy_in(h->f0, f, sizeof(double) * n * n, h->stream);
    copy_in(h->mu, mu, sizeof(double) * 3 * n * n, h->stream);
    copy_in(h->Bd, B, sizeof(double) * naux * n * n, h->stream);
    for (int x = 0; x < 3; ++x) {
      double tr = 0;
      for (int i = 0; i < o; ++i) tr += mu[(size_t)x * n * n + i * n + i];
      h->mu_ref[x] = 2.0 * tr + core_ref[x];
    }
    h->ints = std::make_unique<IntegralStore>();
    build_integrals(*h->ints, h->Bd, naux, o, v, h->stream);
    const size_t nsz = (size_t)2 * h->ns * h->nz;
    h->Y = h->alloc<double>(nsz);
    h->Ys = h->alloc<double>(nsz);
    h->Ynew = h->alloc<double>(nsz);
    h->Rout = h->alloc<double>(nsz);
    for (int s = 0; s < kMaxStages - 1; ++s) h->Rk[s] = h->alloc<double>(nsz);
    h->F = h->alloc<double>((size_t)h->nz * n * n);
    h->DIP = h->alloc<double>((size_t)2 * 3 * h->nz);
    h->d_fields = h->alloc<rtcc_field_t>(h->nz);
    h->ctl.t = h->alloc<double>(h->nz);
    h->ctl.h = h->alloc<double>(h->nz);
    h->ctl.htry = h->alloc<double>(h->nz);
    h->ctl.status = h->alloc<int>(h->nz);
    h->ctl.accepted = h->alloc<int>(h->nz);
    h->ctl.steps = h->alloc<int>(h->nz);
    h->ctl.rejects = h->alloc<int>(h->nz);
    h->ctl.err_bits = h->alloc<unsigned long long>(h->nz);
    h->ctl.counters = h->alloc<long long>(4);
    h->ctl.nout = h->alloc<int>(h->nz);
    h->ctl.perm = h->alloc<int>(h->nz);
    {
      std::vector<int> id(h->nz);
      for (int z = 0; z < h->nz; ++z) id[z] = z;
      RTCC_CUDA(cudaMemcpyAsync(h->ctl.perm, id.data(), sizeof(int) * h->nz, cudaMemcpyHostToDevice, h->stream));
      RTCC_CUDA(cudaStreamSynchronize(h->stream));
    }
    h->E = std::make_unique<Engine>(h->prec, h->stream);
    const IntIds I = register_integrals(*h->E, *h->ints);
    h->rhs = build_rhs(*h->E, I, h->nz, o, v, h->Ys, h->F, h->Rout, true);
    h->dip = build_dipole(*h->E, h->nz, o, v, h->Y, h->mu, h->DIP);
    h->allocs.push_back(h->dip.fdummy);
    std::vector<Program*> progs = {&h->rhs.fwd, &h->rhs.rev, &h->dip.prog};
    // the same programs over the first k slots share the arenas (and every constant pack)
    h->rhs_k.resize(h->nz);
    h->dip_k.resize(h->nz);
    for (int k = 1; k < h->nz; ++k) {
      h->rhs_k[k] = build_rhs(*h->E, I, k, o, v, h->Ys, h->F, h->Rout, true, h->rhs.fwd_arena, h->rhs.rev_arena);
      h->dip_k[k] = build_dipole(*h->E, k, o, v, h->Y, h->mu, h->DIP, h->dip.fwd_arena, h->dip.rev_arena);
      h->allocs.push_back(h->dip_k[k].fdummy);
      progs.insert(progs.end(), {&h->rhs_k[k].fwd, &h->rhs_k[k].rev, &h->dip_k[k].prog});
    }
    h->E->finalize(progs);
    h->E->set_profiler(&h->prof);
    RTCC_CUDA(cudaStreamSynchronize(h->stream));
  });
  if (st != RTCC_OK) {
    delete h;
    return st;
  }
  *out = h;
  return RTCC_OK;
}

rtcc_status_t rtcc_destroy(rtcc_handle_t h) {
  if (!h) return RTCC_OK;
  cudaStreamSynchronize(h->stream);
  delete h;
  return RTCC_OK;
}

rtcc_status_t rtcc_state_size(rtcc_handle_t h, size_t* n) {
  if (!h || !n) return fail(RTCC_ERR_INVALID_ARG, "null argument");
  *n = (size_t)h->ns;
  return RTCC_OK;
}

rtcc_status_t rtcc_get_state(rtcc_handle_t h, int traj, double* y, double* time, double* hstep) {
  if (!h || !y || traj < 0 || traj >= h->nz) return fail(RTCC_ERR_INVALID_ARG, "bad argument");
  return guarded([&] {
    copy_out(y, h->Y + (size_t)2 * h->ns * traj, sizeof(double) * 2 * h->ns, h->stream);
    if (time) RTCC_CUDA(cudaMemcpyAsync(time, h->ctl.t + traj, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (hstep) RTCC_CUDA(cudaMemcpyAsync(hstep, h->ctl.h + traj, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    RTCC_CUDA(cudaStreamSynchronize(h->stream));
  });
}

rtcc_status_t rtcc_set_state(rtcc_handle_t h, int traj, const double* y, double time, double hstep) {
  if (!h || !y || traj < 0 || traj >= h->nz) return fail(RTCC_ERR_INVALID_ARG, "bad argument");
  return guarded([&] {
    copy_in(h->Y + (size_t)2 * h->ns * traj, y, sizeof(double) * 2 * h->ns, h->stream);
    RTCC_CUDA(cudaMemcpyAsync(h->ctl.t + traj, &time, sizeof(double), cudaMemcpyHostToDevice, h->stream));
    RTCC_CUDA(cudaMemcpyAsync(h->ctl.h + traj, &hstep, sizeof(double), cudaMemcpyHostToDevice, h->stream));
    RTCC_CUDA(cudaStreamSynchronize(h->stream));
  });
}

rtcc_status_t rtcc_rhs(rtcc_handle_t h, const double* y, const rtcc_field_t* fields, const double* times, double* dydt) {
  if (!h || !y || !fields || !times || !dydt) return fail(RTCC_ERR_INVALID_ARG, "null argument");
  return guarded([&] {
    const size_t bytes = sizeof(double) * 2 * h->ns * h->nz;
    copy_in(h->Ys, y, bytes, h->stream);
    RTCC_CUDA(cudaMemcpyAsync(h->d_fields, fields, sizeof(rtcc_field_t) * h->nz, cudaMemcpyHostToDevice, h->stream));
    RTCC_CUDA(cudaMemcpyAsync(h->ctl.htry, times, sizeof(double) * h->nz, cudaMemcpyHostToDevice, h->stream));
    RTCC_CUDA(cudaMemsetAsync(h->ctl.err_bits, 0, sizeof(double) * h->nz, h->stream));
    // F = f0 - E(times).mu : use t = 0 and c = 1 with htry = times
    double* zeros = reinterpret_cast<double*>(h->ctl.err_bits);
    k_fock<<<dim3(blocks_for((long long)h->nmo * h->nmo), h->nz), 256, 0, h->stream>>>(
        h->F, h->f0, h->mu, h->d_fields, zeros, h->ctl.htry, 1.0, h->nz, h->nmo * h->nmo);
    h->E->run(h->rhs.fwd);
    h->E->run(h->rhs.rev);
    k_apply_D<<<blocks_for(h->ns * h->nz), 256, 0, h->stream>>>(h->Ynew, h->Rout, h->ns, h->nT, h->nz);
    RTCC_CUDA(cudaGetLastError());
    h->E->check_error();
    copy_out(dydt, h->Ynew, bytes, h->stream);
    RTCC_CUDA(cudaStreamSynchronize(h->stream));
  });
}

rtcc_status_t rtcc_autotune(rtcc_handle_t h, int* tuned_gemms) {
  if (!h) return fail(RTCC_ERR_INVALID_ARG, "null handle");
  return guarded([&] {
    if (h->prec != Prec::P64)
      for (int k = 1; k <= h->nz; ++k) {
        RhsPrograms& r = (k == h->nz) ? h->rhs : h->rhs_k[k];
        DipolePrograms& d = (k == h->nz) ? h->dip : h->dip_k[k];
        h->E->autotune(r.fwd);
        h->E->autotune(r.rev);
        h->E->autotune(d.prog);
      }
    RTCC_CUDA(cudaStreamSynchronize(h->stream));
    if (tuned_gemms) *tuned_gemms = h->E->tuned_gemms();
  });
}

rtcc_status_t rtcc_rhs_vjp(rtcc_handle_t h, const double* y, const rtcc_field_t* fields, const double* times,
                           const double* u, double* ybar) {
  if (!h || !y || !fields || !times || !u || !ybar) return fail(RTCC_ERR_INVALID_ARG, "null argument");
  return guarded([&] {
    AdjointEngine* a = adjoint_engine(h);
    cudaStream_t s = h->stream;
    const size_t bytes = sizeof(double) * 2 * h->ns * h->nz;
    copy_in(a->Ys, y, bytes, s);
    RTCC_CUDA(cudaMemcpyAsync(h->d_fields, fields, sizeof(rtcc_field_t) * h->nz, cudaMemcpyHostToDevice, s));
    RTCC_CUDA(cudaMemcpyAsync(a->tdev, times, sizeof(double) * h->nz, cudaMemcpyHostToDevice, s));
    RTCC_CUDA(cudaMemsetAsync(a->hdev, 0, sizeof(double) * h->nz, s));
    k_fock<<<dim3(blocks_for((long long)h->nmo * h->nmo), h->nz), 256, 0, s>>>(a->F, h->f0, h->mu, h->d_fields,
                                                                              a->tdev, a->hdev, 0.0, h->nz,
                                                                              h->nmo * h->nmo);
    // the VJP program reads the intermediates of the last forward and reverse sweeps at y
    a->E->run(a->rhs.fwd);
    a->E->run(a->rhs.rev);
    // dydt = D raw with D = diag(-i on the T part, +i on the Lambda part), so the cotangent of the
    // raw output is D u (D is diagonal and its own transpose)
    copy_in(a->abar, u, bytes, s);
    k_apply_D<<<blocks_for(h->ns * h->nz), 256, 0, s>>>(a->cot, a->abar, h->ns, h->nT, h->nz);
    a->E->run(a->vjp);
    RTCC_CUDA(cudaGetLastError());
    a->E->check_error();
    copy_out(ybar, a->ybar, bytes, s);
    RTCC_CUDA(cudaStreamSynchronize(s));
  });
}

rtcc_status_t rtcc_dipole(rtcc_handle_t h, double* mu_out) {
  if (!h || !mu_out) return fail(RTCC_ERR_INVALID_ARG, "null argument");
  return guarded([&] {
    run_dipole(h);
    std::vector<double> d((size_t)6 * h->nz);
    RTCC_CUDA(cudaMemcpyAsync(d.data(), h->DIP, sizeof(double) * d.size(), cudaMemcpyDeviceToHost, h->stream));
    RTCC_CUDA(cudaStreamSynchronize(h->stream));
    h->E->check_error();
    std::vector<double> o((size_t)6 * h->nz);
    for (int z = 0; z < h->nz; ++z)
      for (int x = 0; x < 3; ++x) {
        o[2 * (z * 3 + x)] = d[2 * (x * h->nz + z)] + h->mu_ref[x];
        o[2 * (z * 3 + x) + 1] = d[2 * (x * h->nz + z) + 1];
      }
    copy_in(h->Ynew, o.data(), sizeof(double) * o.size(), h->stream);
    copy_out(mu_out, h->Ynew, sizeof(double) * o.size(), h->stream);
    RTCC_CUDA(cudaStreamSynchronize(h->stream));
  });
}

rtcc_status_t rtcc_ground_state(rtcc_handle_t h, double tol, int maxiter, double* e_corr, double* mu0) {
  if (!h || tol <= 0 || maxiter < 1) return fail(RTCC_ERR_INVALID_ARG, "bad argument");
  return guarded([&] {
    GroundEngine* g = ground_engine(h, Prec::P64);
    RTCC_CUDA(cudaMemsetAsync(g->Y, 0, sizeof(double) * 2 * h->ns, h->stream));
    if (h->prec != Prec::P64) {
      // reduced-precision iterations down to their rounding floor, then float64 cleanup iterations
      GroundEngine* gl = ground_engine(h, h->prec);
      RTCC_CUDA(cudaMemsetAsync(gl->Y, 0, sizeof(double) * 2 * h->ns, h->stream));
      solve_block(h, gl, false, std::max(tol, 1e-9), maxiter, true);
      solve_block(h, gl, true, std::max(tol, 1e-9), maxiter, true);
      RTCC_CUDA(cudaMemcpyAsync(g->Y, gl->Y, sizeof(double) * 2 * h->ns, cudaMemcpyDeviceToDevice, h->stream));
    }
    solve_block(h, g, false, tol, maxiter, false);
    solve_block(h, g, true, tol, maxiter, false);
    g->E->run(g->rhs.fwd);
    g->E->run(g->energy);
    double ec[2];
    RTCC_CUDA(cudaMemcpyAsync(ec, g->Ec, sizeof(ec), cudaMemcpyDeviceToHost, h->stream));
    for (int z = 0; z < h->nz; ++z)
      RTCC_CUDA(cudaMemcpyAsync(h->Y + (size_t)2 * h->ns * z, g->Y, sizeof(double) * 2 * h->ns,
                                cudaMemcpyDeviceToDevice, h->stream));
    RTCC_CUDA(cudaMemsetAsync(h->ctl.t, 0, sizeof(double) * h->nz, h->stream));
    RTCC_CUDA(cudaStreamSynchronize(h->stream));
    g->E->check_error();
    if (e_corr) *e_corr = ec[0];
    if (mu0) {
      g->E->run(g->dip.prog);
      double d[6];
      RTCC_CUDA(cudaMemcpyAsync(d, g->DIP, sizeof(d), cudaMemcpyDeviceToHost, h->stream));
      RTCC_CUDA(cudaStreamSynchronize(h->stream));
      for (int x = 0; x < 3; ++x) mu0[x] = d[2 * x] + h->mu_ref[x];
    }
  });
}

rtcc_status_t rtcc_propagate(rtcc_handle_t h, const rtcc_field_t* fields, const rtcc_integrator_t* integ, int max_out,
                             double* t_out, double* mu_out, int* n_out) {
  if (!h || !fields || !integ || max_out < 1 || !t_out || !mu_out || !n_out)
    return fail(RTCC_ERR_INVALID_ARG, "null argument or max_out < 1");
  const rtcc_integrator_t in = *integ;
  if (in.method < 0 || in.method > 4) return fail(RTCC_ERR_INVALID_ARG, "unknown integrator");
  if (in.method == RTCC_GL2 && (!(in.h > 0) || !(in.tol > 0) || in.sweeps < 0 || in.sweeps > 1000))
    return fail(RTCC_ERR_INVALID_ARG, "Gauss-Legendre needs h > 0, tol > 0 and 0 <= sweeps <= 1000");
  if (in.method == RTCC_GL2_NEWTON &&
      (!(in.h > 0) || !(in.tol > 0) || in.sweeps < 0 || in.sweeps > 100 || in.krylov < 0 || in.krylov > kKrylovMax))
    return fail(RTCC_ERR_INVALID_ARG,
                "Gauss-Legendre (Newton) needs h > 0, tol > 0, 0 <= sweeps <= 100 and 0 <= krylov <= 32");
  if (in.nsteps <= 0 && !(in.t_end > 0)) return fail(RTCC_ERR_INVALID_ARG, "need nsteps > 0 or t_end > 0");
  if (in.method == RTCC_RK4 && !(in.h > 0)) return fail(RTCC_ERR_INVALID_ARG, "h must be positive");
  if (in.method == RTCC_MIXED_RK4 && !(in.h1 > 0 && in.h2 > 0)) return fail(RTCC_ERR_INVALID_ARG, "h1, h2 must be positive");
  if (in.method == RTCC_CK && !(in.h >= 0 && in.tol > 0 && in.safety > 0 && in.h_min > 0 && in.h_max >= in.h_min))
    return fail(RTCC_ERR_INVALID_ARG, "bad Cash-Karp settings");
  return guarded([&] {
    cudaStream_t s = h->stream;
    const int nz = h->nz;
    const bool dev_out = is_device_ptr(t_out);
    // device staging of host outputs: one buffer on the handle, grown when a call needs more
    double* tout = t_out;
    double* muout = mu_out;
    if (!dev_out) {
      const size_t need = sizeof(double) * (size_t)nz * max_out * 7;
      if (h->out_stage_bytes < need) {
        if (h->out_stage) {
          RTCC_CUDA(cudaStreamSynchronize(s));
          cudaFree(h->out_stage);
          h->out_stage = nullptr;
          h->out_stage_bytes = 0;
        }
        h->out_stage = dev_alloc(need);
        h->out_stage_bytes = need;
      }
      tout = static_cast<double*>(h->out_stage);
      muout = tout + (size_t)nz * max_out;
      RTCC_CUDA(cudaMemsetAsync(tout, 0, sizeof(double) * nz * max_out, s));
      RTCC_CUDA(cudaMemsetAsync(muout, 0, sizeof(double) * nz * max_out * 6, s));
    }
    RTCC_CUDA(cudaMemcpyAsync(h->d_fields, fields, sizeof(rtcc_field_t) * nz, cudaMemcpyHostToDevice, s));
    RTCC_CUDA(cudaMemsetAsync(h->ctl.status, 0, sizeof(int) * nz, s));
    RTCC_CUDA(cudaMemsetAsync(h->ctl.steps, 0, sizeof(int) * nz, s));
    RTCC_CUDA(cudaMemsetAsync(h->ctl.rejects, 0, sizeof(int) * nz, s));
    RTCC_CUDA(cudaMemsetAsync(h->ctl.nout, 0, sizeof(int) * nz, s));
    RTCC_CUDA(cudaMemsetAsync(h->ctl.counters, 0, sizeof(long long) * 4, s));
    if (in.method == RTCC_CK) {
      if (in.h > 0) {
        std::vector<double> h0(nz, in.h);
        RTCC_CUDA(cudaMemcpyAsync(h->ctl.h, h0.data(), sizeof(double) * nz, cudaMemcpyHostToDevice, s));
      } else {
        // h = 0: every trajectory continues with its stored trial step (resume)
        std::vector<double> hz(nz);
        RTCC_CUDA(cudaMemcpyAsync(hz.data(), h->ctl.h, sizeof(double) * nz, cudaMemcpyDeviceToHost, s));
        RTCC_CUDA(cudaStreamSynchronize(s));
        for (int z = 0; z < nz; ++z)
          if (!(hz[z] >= in.h_min && hz[z] <= in.h_max))
            throw Error(RTCC_ERR_INVALID_ARG, "trajectory " + std::to_string(z) +
                                                  " has no stored Cash-Karp step in [h_min, h_max]; pass h > 0");
      }
    }
    const Tableau tb = (in.method == RTCC_CK)           ? ck_tableau()
                       : (in.method == RTCC_GL2)        ? gl2_tableau(in.sweeps)
                       : (in.method == RTCC_GL2_NEWTON) ? gl2_newton_tableau(in.sweeps, in.krylov)
                                                        : rk4_tableau();
    if (tb.newton) ensure_krylov(h, tb.krylov);
    run_dipole(h);
    k_record<<<(nz + 127) / 128, 128, 0, s>>>(h->ctl, h->DIP, h->mu_ref[0], h->mu_ref[1], h->mu_ref[2], tout, muout,
                                             max_out, nz, 1);
    RTCC_CUDA(cudaGetLastError());
    const char* ng = std::getenv("RTCC_NO_GRAPH");
    const bool use_graph = !(ng && ng[0] == '1') && !h->prof.on();
    // Slots: trajectories that have finished are moved behind the running ones between attempts
    // (permuting the state, field and controller entries of every slot), and the attempts then run
    // over the running slots only, with the programs built for that many slots.  The slot order is
    // restored when the call ends, normally or by an error.
    struct SlotOrder {
      rtcc_ctx* h;
      std::vector<int> perm;   // trajectory held by each slot
      bool moved = false;
      explicit SlotOrder(rtcc_ctx* hh) : h(hh), perm(hh->nz) {
        for (int z = 0; z < hh->nz; ++z) perm[z] = z;
      }
      // new slot i takes the contents of old slot order[i] (i < n)
      void apply(const std::vector<int>& order) {
        const int n = (int)order.size();
        cudaStream_t st = h->stream;
        const size_t sb = sizeof(double) * 2 * (size_t)h->ns;
        bool any = false;
        for (int i = 0; i < n; ++i) any |= (order[i] != i);
        if (!any) return;
        moved = true;
        // the state through Ynew (free between attempts), the small per-slot arrays through the host
        for (int i = 0; i < n; ++i)
          if (order[i] != i)
            RTCC_CUDA(cudaMemcpyAsync(h->Ynew + (size_t)2 * h->ns * i, h->Y + (size_t)2 * h->ns * order[i], sb,
                                      cudaMemcpyDeviceToDevice, st));
        for (int i = 0; i < n; ++i)
          if (order[i] != i)
            RTCC_CUDA(cudaMemcpyAsync(h->Y + (size_t)2 * h->ns * i, h->Ynew + (size_t)2 * h->ns * i, sb,
                                      cudaMemcpyDeviceToDevice, st));
        auto permute = [&](auto* dev) {
          using T = std::remove_pointer_t<decltype(dev)>;
          std::vector<T> a(n), b(n);
          RTCC_CUDA(cudaMemcpyAsync(a.data(), dev, sizeof(T) * n, cudaMemcpyDeviceToHost, st));
          RTCC_CUDA(cudaStreamSynchronize(st));
          for (int i = 0; i < n; ++i) b[i] = a[order[i]];
          RTCC_CUDA(cudaMemcpyAsync(dev, b.data(), sizeof(T) * n, cudaMemcpyHostToDevice, st));
          RTCC_CUDA(cudaStreamSynchronize(st));
        };
        permute(h->d_fields);
        permute(h->ctl.t);
        permute(h->ctl.h);
        permute(h->ctl.status);
        permute(h->ctl.steps);
        permute(h->ctl.rejects);
        permute(h->ctl.nout);
        std::vector<int> p2(h->nz);
        for (int i = 0; i < h->nz; ++i) p2[i] = (i < n) ? perm[order[i]] : perm[i];
        perm = p2;
        RTCC_CUDA(cudaMemcpyAsync(h->ctl.perm, perm.data(), sizeof(int) * h->nz, cudaMemcpyHostToDevice, st));
        RTCC_CUDA(cudaStreamSynchronize(st));
      }
      void restore() {
        if (!moved) return;
        std::vector<int> order(h->nz);
        for (int i = 0; i < h->nz; ++i) order[perm[i]] = i;   // slot j takes the slot holding trajectory j
        apply(order);
        moved = false;
      }
      ~SlotOrder() {
        try {
          restore();
        } catch (...) {
        }
      }
    } slots(h);
    // one captured attempt per slot count in use (its first attempt runs eagerly: kernel
    // attributes are set and the launches of one attempt counted)
    struct Graphs {
      std::vector<cudaGraphExec_t> e;
      ~Graphs() {
        for (auto x : e)
          if (x) cudaGraphExecDestroy(x);
      }
    } graphs;
    graphs.e.assign(nz + 1, nullptr);
    std::vector<long long> per_attempt(nz + 1, -1), attempts_at(nz + 1, 0);
    auto attempt = [&](int nact) {
      if (per_attempt[nact] < 0) {
        tune_slots(h, nact);
        const long long c0 = total_count(h->prof);
        run_attempt(h, tb, in, tout, muout, max_out, nact);
        per_attempt[nact] = total_count(h->prof) - c0;
        if (use_graph) {
          cudaGraph_t graph = nullptr;
          RTCC_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
          try {
            run_attempt(h, tb, in, tout, muout, max_out, nact);
          } catch (...) {
            cudaStreamEndCapture(s, &graph);
            if (graph) cudaGraphDestroy(graph);
            throw;
          }
          RTCC_CUDA(cudaStreamEndCapture(s, &graph));
          const cudaError_t ie = cudaGraphInstantiate(&graphs.e[nact], graph, 0);
          cudaGraphDestroy(graph);
          RTCC_CUDA(ie);
        }
      } else if (graphs.e[nact]) {
        RTCC_CUDA(cudaGraphLaunch(graphs.e[nact], s));
      } else {
        run_attempt(h, tb, in, tout, muout, max_out, nact);
      }
      attempts_at[nact] += 1;
    };
    int nact = nz;
    attempt(nact);
    long long attempts = 1;
    std::vector<int> stat(nz), stp(nz);
    std::vector<double> tz(nz), hz(nz);
    const long long max_attempts = (in.nsteps > 0) ? (long long)in.nsteps * 64 + 64 : (1ll << 40);
    int check_every = 4;
    while (true) {
      RTCC_CUDA(cudaMemcpyAsync(stat.data(), h->ctl.status, sizeof(int) * nact, cudaMemcpyDeviceToHost, s));
      RTCC_CUDA(cudaMemcpyAsync(stp.data(), h->ctl.steps, sizeof(int) * nact, cudaMemcpyDeviceToHost, s));
      RTCC_CUDA(cudaMemcpyAsync(tz.data(), h->ctl.t, sizeof(double) * nact, cudaMemcpyDeviceToHost, s));
      RTCC_CUDA(cudaMemcpyAsync(hz.data(), h->ctl.h, sizeof(double) * nact, cudaMemcpyDeviceToHost, s));
      RTCC_CUDA(cudaStreamSynchronize(s));
      h->E->check_error();
      int running = 0;
      for (int z = 0; z < nact; ++z) {
        const std::string who = "trajectory " + std::to_string(slots.perm[z]);
        if (stat[z] == TS_DIVERGED) throw Error(RTCC_ERR_DIVERGED, who + " diverged");
        if (stat[z] == TS_NOCONV) throw Error(RTCC_ERR_NOCONV, who + ": implicit stages did not converge");
        if (stat[z] == TS_UNDERFLOW) throw Error(RTCC_ERR_STEP_UNDERFLOW, who + ": step size underflow");
        running += (stat[z] == TS_RUN);
      }
      if (running == 0) break;
      if (attempts >= max_attempts) throw Error(RTCC_ERR_TIMEOUT, "attempt limit reached");
      if (running < nact) {
        // running slots first (in their order), finished ones after them
        std::vector<int> order;
        for (int z = 0; z < nact; ++z)
          if (stat[z] == TS_RUN) order.push_back(z);
        for (int z = 0; z < nact; ++z)
          if (stat[z] != TS_RUN) order.push_back(z);
        slots.apply(order);
        std::vector<int> st2(nact), sp2(nact);
        std::vector<double> t2(nact), h2(nact);
        for (int i = 0; i < nact; ++i) {
          st2[i] = stat[order[i]];
          sp2[i] = stp[order[i]];
          t2[i] = tz[order[i]];
          h2[i] = hz[order[i]];
        }
        std::copy(st2.begin(), st2.end(), stat.begin());
        std::copy(sp2.begin(), sp2.end(), stp.begin());
        std::copy(t2.begin(), t2.end(), tz.begin());
        std::copy(h2.begin(), h2.end(), hz.begin());
        nact = running;
      }
      // every running trajectory needs at least `need` more attempts: replay that many before polling
      long long need = 1ll << 40;
      for (int z = 0; z < nact; ++z) {
        long long nz_need;
        if (in.nsteps > 0) nz_need = in.nsteps - stp[z];
        else {
          const double hstep = (in.method == RTCC_CK) ? hz[z] * 5.0
                               : ((in.method == RTCC_RK4 || in.method == RTCC_GL2 || in.method == RTCC_GL2_NEWTON)
                                      ? in.h
                                      : std::max(in.h1, in.h2));
          nz_need = (long long)std::floor((in.t_end - tz[z]) / hstep);
        }
        need = std::min(need, nz_need);
      }
      const long long k = std::max(1ll, std::min<long long>(need, check_every));
      for (long long q = 0; q < k; ++q) attempt(nact);
      attempts += k;
      check_every = std::min(check_every * 2, 64);
    }
    slots.restore();
    std::vector<int> nout(nz);
    long long cnt[4];
    RTCC_CUDA(cudaMemcpyAsync(nout.data(), h->ctl.nout, sizeof(int) * nz, cudaMemcpyDeviceToHost, s));
    RTCC_CUDA(cudaMemcpyAsync(cnt, h->ctl.counters, sizeof(cnt), cudaMemcpyDeviceToHost, s));
    if (!dev_out) {
      RTCC_CUDA(cudaMemcpyAsync(t_out, tout, sizeof(double) * nz * max_out, cudaMemcpyDeviceToHost, s));
      RTCC_CUDA(cudaMemcpyAsync(mu_out, muout, sizeof(double) * nz * max_out * 6, cudaMemcpyDeviceToHost, s));
    }
    RTCC_CUDA(cudaStreamSynchronize(s));
    for (int z = 0; z < nz; ++z) n_out[z] = nout[z];
    long long launches = 0, slot_attempts = 0;
    for (int k = 1; k <= nz; ++k) {
      launches += std::max(0ll, per_attempt[k]) * attempts_at[k];
      slot_attempts += (long long)k * attempts_at[k];
    }
    h->last_stats[0] = cnt[0];
    h->last_stats[1] = cnt[1];
    const long long per_attempt_rhs = tb.implicit ? 1 + (long long)tb.s * tb.sweeps
                                      : tb.newton ? 1 + (long long)tb.sweeps * (2 + 2 * tb.krylov)
                                                  : tb.s;
    h->last_stats[2] = (cnt[0] + cnt[1]) * per_attempt_rhs;
    h->last_stats[3] = launches;
    h->last_slot_attempts = slot_attempts;
  });
}


rtcc_status_t rtcc_propagate_vjp(rtcc_handle_t h, const rtcc_field_t* fields, double hstep, int nsteps,
                                 const double* w, int ckpt_every, double* grad, double* J) {
  if (!h || !fields || !w || !grad || !J || nsteps < 1 || !(hstep > 0) || ckpt_every < 1)
    return fail(RTCC_ERR_INVALID_ARG, "bad argument");
  return guarded([&] {
    cudaStream_t s = h->stream;
    AdjointEngine* a = adjoint_engine(h);
    const int nz = h->nz;
    const size_t st_bytes = sizeof(double) * 2 * h->ns * nz;
    const Tableau tb = rk4_tableau();
    RTCC_CUDA(cudaMemcpyAsync(h->d_fields, fields, sizeof(rtcc_field_t) * nz, cudaMemcpyHostToDevice, s));
    double t0 = 0.0;
    RTCC_CUDA(cudaMemcpyAsync(&t0, h->ctl.t, sizeof(double), cudaMemcpyDeviceToHost, s));
    RTCC_CUDA(cudaStreamSynchronize(s));
    const int nck = nsteps / ckpt_every + 1;
    std::vector<double*> ck(nck, nullptr);
    std::vector<void*> tmp;
    auto cleanup = [&] {
      for (void* p : tmp) cudaFree(p);
    };
    try {
      for (int c = 0; c < nck; ++c) {
        ck[c] = static_cast<double*>(dev_alloc(st_bytes));
        tmp.push_back(ck[c]);
      }
      double* seg = static_cast<double*>(dev_alloc(st_bytes * (size_t)ckpt_every));
      tmp.push_back(seg);
      // forward sweep with checkpoints; J from the dipoles at every step
      std::vector<double> Jz(nz, 0.0), mu;
      RTCC_CUDA(cudaMemcpyAsync(a->y, h->Y, st_bytes, cudaMemcpyDeviceToDevice, s));
      for (int n = 0; n <= nsteps; ++n) {
        if (n % ckpt_every == 0)
          RTCC_CUDA(cudaMemcpyAsync(ck[n / ckpt_every], a->y, st_bytes, cudaMemcpyDeviceToDevice, s));
        adj_dipole(h, a, a->y, mu);
        for (int z = 0; z < nz; ++z)
          for (int x = 0; x < 3; ++x) Jz[z] += w[3 * n + x] * mu[3 * z + x];
        if (n == nsteps) break;
        adj_set_time(h, a, t0 + n * hstep, hstep);
        adj_step(h, a, tb, a->y, a->anew);
        RTCC_CUDA(cudaMemcpyAsync(a->y, a->anew, st_bytes, cudaMemcpyDeviceToDevice, s));
      }
      // abar = dG/dy_N: the observable at the last step (the dipole program ran on y_N last)
      RTCC_CUDA(cudaMemsetAsync(a->abar, 0, st_bytes, s));
      adj_observable(h, a, w + 3 * nsteps, a->abar);
      RTCC_CUDA(cudaMemsetAsync(a->grad, 0, sizeof(double) * 3 * nz, s));
      const long long nst = h->ns * nz;
      const unsigned nb = blocks_for(nst);
      for (int c = (nsteps - 1) / ckpt_every; c >= 0; --c) {
        const int n0 = c * ckpt_every, n1 = std::min(nsteps, n0 + ckpt_every);
        // recompute the segment's states from its checkpoint
        RTCC_CUDA(cudaMemcpyAsync(a->y, ck[c], st_bytes, cudaMemcpyDeviceToDevice, s));
        for (int n = n0; n < n1; ++n) {
          RTCC_CUDA(cudaMemcpyAsync(seg + (size_t)(n - n0) * 2 * nst, a->y, st_bytes, cudaMemcpyDeviceToDevice, s));
          if (n + 1 < n1) {
            adj_set_time(h, a, t0 + n * hstep, hstep);
            adj_step(h, a, tb, a->y, a->anew);
            RTCC_CUDA(cudaMemcpyAsync(a->y, a->anew, st_bytes, cudaMemcpyDeviceToDevice, s));
          }
        }
        for (int n = n1 - 1; n >= n0; --n) {
          const double* yn = seg + (size_t)(n - n0) * 2 * nst;
          adj_set_time(h, a, t0 + n * hstep, hstep);
          adj_step(h, a, tb, yn, a->anew);   // stage inputs and right-hand sides of step n
          RTCC_CUDA(cudaMemcpyAsync(a->anew, a->abar, st_bytes, cudaMemcpyDeviceToDevice, s));   // identity part
          for (int st = 0; st < 4; ++st) RTCC_CUDA(cudaMemsetAsync(a->kbar[st], 0, st_bytes, s));
          for (int st = 3; st >= 0; --st) {
            k_axpy<<<nb, 256, 0, s>>>(a->kbar[st], a->abar, hstep * tb.b[st], nst);
            if (st != 3) {   // restore this stage's intermediates
              RTCC_CUDA(cudaMemcpyAsync(a->Ys, a->sin[st], st_bytes, cudaMemcpyDeviceToDevice, s));
              k_fock<<<dim3(blocks_for((long long)h->nmo * h->nmo), nz), 256, 0, s>>>(
                  a->F, h->f0, h->mu, h->d_fields, a->tdev, a->hdev, tb.c[st], nz, h->nmo * h->nmo);
              a->E->run(a->rhs.fwd);
              a->E->run(a->rhs.rev);
            }
            k_apply_D<<<nb, 256, 0, s>>>(a->cot, a->kbar[st], h->ns, h->nT, nz);   // F = D R, D symmetric
            a->E->run(a->vjp);
            k_theta_grad<<<nz, 256, 0, s>>>(a->grad, a->fbar, h->mu, h->d_fields, a->tdev, tb.c[st], a->hdev,
                                            h->nmo * h->nmo);
            k_axpy<<<nb, 256, 0, s>>>(a->anew, a->ybar, 1.0, nst);
            for (int j = 0; j < st; ++j)
              if (tb.a[st][j] != 0.0) k_axpy<<<nb, 256, 0, s>>>(a->kbar[j], a->ybar, hstep * tb.a[st][j], nst);
          }
          // observable at step n
          adj_dipole(h, a, yn, mu);
          adj_observable(h, a, w + 3 * n, a->anew);
          RTCC_CUDA(cudaMemcpyAsync(a->abar, a->anew, st_bytes, cudaMemcpyDeviceToDevice, s));
        }
      }
      std::vector<double> g((size_t)3 * nz);
      RTCC_CUDA(cudaMemcpyAsync(g.data(), a->grad, sizeof(double) * g.size(), cudaMemcpyDeviceToHost, s));
      RTCC_CUDA(cudaStreamSynchronize(s));
      a->E->check_error();
      for (int z = 0; z < nz; ++z) {
        J[z] = Jz[z];
        for (int j = 0; j < 3; ++j) grad[3 * z + j] = g[3 * z + j];
      }
    } catch (...) {
      cleanup();
      throw;
    }
    cleanup();
  });
}

rtcc_status_t rtcc_last_stats(rtcc_handle_t h, long long* accepted, long long* rejected, long long* rhs_evals,
                              long long* launches) {
  if (!h) return fail(RTCC_ERR_INVALID_ARG, "null handle");
  if (accepted) *accepted = h->last_stats[0];
  if (rejected) *rejected = h->last_stats[1];
  if (rhs_evals) *rhs_evals = h->last_stats[2];
  if (launches) *launches = h->last_stats[3];
  return RTCC_OK;
}

rtcc_status_t rtcc_profile(rtcc_handle_t h, int enable, rtcc_profile_t* out) {
  if (!h) return fail(RTCC_ERR_INVALID_ARG, "null handle");
  return guarded([&] {
    if (enable) {
      h->prof.begin();
      return;
    }
    rtcc_profile_t p{};
    h->prof.end(p.launches, p.ms, p.flops, p.bytes);
    if (out) *out = p;
  });
}

rtcc_status_t rtcc_spectrum(const double* t, const double* mu, int n, const rtcc_field_t* field, double kappa,
                            double gamma, double dt, const double* omega, int n_omega, double* I) {
  if (!t || !mu || !field || !omega || !I || n < 4 || n_omega < 1) return fail(RTCC_ERR_INVALID_ARG, "bad argument");
  for (int k = 1; k < n; ++k)
    if (!(t[k] > t[k - 1])) return fail(RTCC_ERR_INVALID_ARG, "sample times must increase");
  return guarded([&] {
    bool uniform = true;
    double hmin = t[1] - t[0];
    for (int k = 1; k < n; ++k) {
      const double hk = t[k] - t[k - 1];
      hmin = std::min(hmin, hk);
      if (std::fabs(hk - (t[1] - t[0])) > 1e-9 * std::fabs(t[1] - t[0])) uniform = false;
    }
    if (dt <= 0) dt = hmin;
    cudaStream_t s;
    RTCC_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    std::vector<void*> al;
    auto A = [&](size_t bytes) {
      void* p = dev_alloc(bytes);
      al.push_back(p);
      return static_cast<double*>(p);
    };
    try {
      double* dt_ = A(sizeof(double) * n);
      double* dy = A(sizeof(double) * 3 * n);
      double* dw = A(sizeof(double) * n_omega);
      double* dI = A(sizeof(double) * n_omega);
      RTCC_CUDA(cudaMemcpyAsync(dt_, t, sizeof(double) * n, cudaMemcpyHostToDevice, s));
      RTCC_CUDA(cudaMemcpyAsync(dy, mu, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
      RTCC_CUDA(cudaMemcpyAsync(dw, omega, sizeof(double) * n_omega, cudaMemcpyHostToDevice, s));
      const double* ts = dt_;
      const double* ys = dy;
      int nu = n;
      double step = t[1] - t[0];
      if (!uniform) {
        nu = (int)std::floor((t[n - 1] - t[0]) / dt + 1e-9) + 1;
        double* M = A(sizeof(double) * 3 * n);
        double* cp = A(sizeof(double) * 3 * n);
        double* dp = A(sizeof(double) * 3 * n);
        double* tu = A(sizeof(double) * nu);
        double* yu = A(sizeof(double) * 3 * nu);
        k_spline_m<<<1, 32, 0, s>>>(dt_, dy, n, M, cp, dp);
        k_spline_eval<<<blocks_for(nu), 256, 0, s>>>(dt_, dy, M, n, t[0], dt, nu, yu);
        std::vector<double> th(nu);
        for (int q = 0; q < nu; ++q) th[q] = t[0] + dt * q;
        RTCC_CUDA(cudaMemcpyAsync(tu, th.data(), sizeof(double) * nu, cudaMemcpyHostToDevice, s));
        ts = tu;
        ys = yu;
        step = dt;
        RTCC_CUDA(cudaStreamSynchronize(s));
      }
      k_dft<<<n_omega, 256, 0, s>>>(ts, ys, nu, step, *field, kappa, gamma, dw, n_omega, dI);
      RTCC_CUDA(cudaGetLastError());
      RTCC_CUDA(cudaMemcpyAsync(I, dI, sizeof(double) * n_omega, cudaMemcpyDeviceToHost, s));
      RTCC_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
      for (void* p : al) cudaFree(p);
      cudaStreamDestroy(s);
      throw;
    }
    for (void* p : al) cudaFree(p);
    cudaStreamDestroy(s);
  });
}

rtcc_status_t rtcc_spectrum_pade(const double* t, const double* mu, int n, const rtcc_field_t* field, double kappa,
                                 double gamma, const double* omega, int n_omega, double* I) {
  if (!t || !mu || !field || !omega || !I || n < 3 || n_omega < 1) return fail(RTCC_ERR_INVALID_ARG, "bad argument");
  const double h0 = t[1] - t[0];
  for (int k = 1; k < n; ++k) {
    const double hk = t[k] - t[k - 1];
    if (!(hk > 0.0) || std::fabs(hk - h0) > 1e-9 * h0)
      return fail(RTCC_ERR_INVALID_ARG, "Pade spectra need increasing, uniformly spaced sample times");
  }
  const int N = (n % 2 == 1) ? n : n - 1;   // 2M + 1 samples
  const int M = (N - 1) / 2;
  if (M > kPadeMaxOrder) return fail(RTCC_ERR_INVALID_ARG, "Pade spectra take at most 1025 samples");
  const int nser = (kappa > 0.0) ? 1 : 2;
  return guarded([&] {
    cudaStream_t s;
    RTCC_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    std::vector<void*> al;
    auto A = [&](size_t bytes) {
      void* p = dev_alloc(bytes);
      al.push_back(p);
      return p;
    };
    std::vector<int> info(nser, 0);
    try {
      double* dt_ = static_cast<double*>(A(sizeof(double) * N));
      double* dy = static_cast<double*>(A(sizeof(double) * 3 * N));
      double* dw = static_cast<double*>(A(sizeof(double) * n_omega));
      double* dI = static_cast<double*>(A(sizeof(double) * n_omega));
      double* ser = static_cast<double*>(A(sizeof(double) * nser * N));
      double* work = static_cast<double*>(A(sizeof(double) * nser * pade::work_doubles(M)));
      double* coef = static_cast<double*>(A(sizeof(double) * nser * 2 * (M + 1)));
      int* dinfo = static_cast<int*>(A(sizeof(int) * nser));
      RTCC_CUDA(cudaMemcpyAsync(dt_, t, sizeof(double) * N, cudaMemcpyHostToDevice, s));
      RTCC_CUDA(cudaMemcpyAsync(dy, mu, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, s));
      RTCC_CUDA(cudaMemcpyAsync(dw, omega, sizeof(double) * n_omega, cudaMemcpyHostToDevice, s));
      k_pade_series<<<blocks_for(N), 256, 0, s>>>(dt_, dy, N, *field, gamma, nser > 1 ? 1 : 0, ser);
      k_pade_solve<<<nser, kPadeThreads, 0, s>>>(ser, M, work, coef, dinfo);
      k_pade_eval<<<blocks_for(n_omega), 256, 0, s>>>(coef, M, h0, t[0], kappa, dw, n_omega, dI);
      RTCC_CUDA(cudaGetLastError());
      RTCC_CUDA(cudaMemcpyAsync(I, dI, sizeof(double) * n_omega, cudaMemcpyDeviceToHost, s));
      RTCC_CUDA(cudaMemcpyAsync(info.data(), dinfo, sizeof(int) * nser, cudaMemcpyDeviceToHost, s));
      RTCC_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
      for (void* p : al) cudaFree(p);
      cudaStreamDestroy(s);
      throw;
    }
    for (void* p : al) cudaFree(p);
    cudaStreamDestroy(s);
    for (int x : info)
      if (x) throw Error(RTCC_ERR_NOCONV, "Pade denominator: Jacobi sweeps did not converge");
  });
}

rtcc_status_t rtcc_selftest_timeout(double seconds) {
  if (!(seconds >= 0.0) || seconds > 10.0) return fail(RTCC_ERR_INVALID_ARG, "seconds must be in [0, 10]");
  return guarded([&] {
    int* d = static_cast<int*>(dev_alloc(2 * sizeof(int)));
    cudaError_t e = cudaMemset(d, 0, 2 * sizeof(int));
    if (e == cudaSuccess) {
      k_wait_flag<<<1, 1>>>(d, (unsigned long long)(seconds * 1e9), d + 1);
      e = cudaDeviceSynchronize();
    }
    int st = -1;
    if (e == cudaSuccess) e = cudaMemcpy(&st, d + 1, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) throw Error(RTCC_ERR_CUDA, cudaGetErrorString(e));
    if (st != 0) throw Error(RTCC_ERR_TIMEOUT, "bounded device wait expired (flag never set)");
  });
}

rtcc_status_t rtcc_selftest_gemm(int prec, int cplx, int batch, int M, int N, int K, const double* A,
                                 const double* Bm, double* C) {
  if (prec < 0 || prec > 3 || cplx < 0 || cplx > 3 || batch < 1 || M < 1 || N < 1 || K < 1 || !A || !Bm || !C)
    return fail(RTCC_ERR_INVALID_ARG, "bad argument");
  return guarded([&] {
    cudaStream_t s;
    RTCC_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    std::vector<void*> al;
    try {
      auto Al = [&](size_t bytes) {
        void* p = dev_alloc(bytes);
        al.push_back(p);
        return static_cast<double*>(p);
      };
      const bool ac = cplx & 1, bc = (cplx >> 1) & 1, cc = ac || bc;
      const size_t na = (size_t)batch * M * K * (ac ? 2 : 1), nb = (size_t)batch * N * K * (bc ? 2 : 1);
      const size_t nc = (size_t)batch * M * N * (cc ? 2 : 1);
      double* dA = Al(na * 8);
      double* dB = Al(nb * 8);
      double* dC = Al(nc * 8);
      copy_in(dA, A, na * 8, s);
      copy_in(dB, Bm, nb * 8, s);
      RTCC_CUDA(cudaMemsetAsync(dC, 0, nc * 8, s));
      Engine E((Prec)prec, s);
      E.set_force_gemm(true);
      const int ta = E.external("A", {batch, M, K}, ac, dA);
      const int tb = E.external("B", {batch, N, K}, bc, dB);
      const int tc = E.external("C", {batch, M, N}, cc, dC);
      // T[zmn] and U[znm] (output unit stride along n, then along m) are zeroed temporaries:
      // the first product of each is stored, the second added in place; C = (T + U) / 4
      const int arena = E.new_arena();
      const int tt = E.temp(arena, "T", {batch, M, N}, cc);
      const int tu = E.temp(arena, "U", {batch, N, M}, cc);
      Program P;
      P.name = "selftest";
      P.zero_arenas = {arena};
      Engine::ein(P, tt, "zmn", ta, "zmk", tb, "znk");
      Engine::ein(P, tt, "zmn", ta, "zmk", tb, "znk");
      Engine::ein(P, tu, "znm", ta, "zmk", tb, "znk");
      Engine::ein(P, tu, "znm", ta, "zmk", tb, "znk");
      Engine::add(P, tc, "zmn", tt, "zmn", 0.25);
      Engine::add(P, tc, "zmn", tu, "znm", 0.25);
      E.finalize({&P});
      E.run(P);
      E.check_error();
      copy_out(C, dC, nc * 8, s);
      RTCC_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
      for (void* p : al) cudaFree(p);
      cudaStreamDestroy(s);
      throw;
    }
    for (void* p : al) cudaFree(p);
    cudaStreamDestroy(s);
  });
}

}  // extern "C"
