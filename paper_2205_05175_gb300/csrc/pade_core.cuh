// Diagonal Pade approximant of a real power series sum_k c_k z^k from c_0 .. c_2M (the
// Pade-accelerated Fourier transform the paper cites among short-time spectral techniques,
// Sec. 1): the denominator Q(z) = sum_m b_m z^m, b_0 = 1, solves
//     sum_{m=1..M} b_m c_{k-m} = -c_k   for k = M+1 .. 2M           (Toeplitz, M x M)
// in the least-squares sense with the minimum-norm solution (the system is singular when the
// series is a sum of fewer than M exponentials), and the numerator is the convolution
// a_k = sum_{m<=k} b_m c_{k-m}, k = 0 .. M.
//
// The least-squares solve is a one-sided Jacobi SVD (Hestenes): plane rotations orthogonalise
// the columns of U = G while V accumulates them, so G = U V^T with orthogonal columns U_j of
// norm sigma_j, and the minimum-norm solution is b = sum_j v_j (U_j . r) / sigma_j^2 over the
// columns with sigma_j > eps * M * sigma_max (the default cut of a float64 least-squares
// solver).  The columns are paired by the circle-method tournament, so the pairs of one round
// are disjoint and rotate concurrently.
//
// Every function here is plain arithmetic on one lane's share of the rows (lane, nl): the device
// kernels call them with one warp per column pair, and a host build of this header runs the
// same arithmetic lane by lane in the tests.
#pragma once
#include <math.h>
#include <stddef.h>

#if defined(__CUDACC__)
#define PADE_HD __host__ __device__ inline
#else
#define PADE_HD inline
#endif

namespace rtcc {
namespace pade {

constexpr double kEps = 2.220446049250313e-16;   // float64 unit roundoff x 2 (machine epsilon)
constexpr double kOrthTol = 1e-15;               // columns count as orthogonal below this cosine
constexpr int kMaxSweeps = 60;

// Column count padded to even (a zero column when M is odd; it never rotates).
PADE_HD int padded(int M) { return M + (M & 1); }

// Workspace doubles per series: U (M x M2), V (M2 x M2), right-hand side, sigma^2, weights.
PADE_HD size_t work_doubles(int M) {
  const size_t M2 = (size_t)padded(M);
  return (size_t)M * M2 + M2 * M2 + 3 * M2;
}

// Circle-method tournament over n (even) columns: in round r (0 <= r < n-1), pair k
// (0 <= k < n/2) joins columns p < q.  Column n-1 stays put, the others rotate.
PADE_HD void pair_of(int n, int r, int k, int& p, int& q) {
  const int m = n - 1;
  int x, y;
  if (k == 0) {
    x = m;
    y = r;
  } else {
    x = (r + k) % m;
    y = (r - k + m) % m;
  }
  p = x < y ? x : y;
  q = x < y ? y : x;
}

// U column-major with M rows (U[j*M + r] = G[r][j] = c[M + r - j]), the padding column zero;
// V = identity (M2 x M2); rhs[r] = -c[M + 1 + r].  Threads tid of nt share the entries.
PADE_HD void fill(const double* c, int M, double* U, double* V, double* rhs, long long tid, long long nt) {
  const int M2 = padded(M);
  for (long long i = tid; i < (long long)M * M2; i += nt) {
    const long long j = i / M, r = i - j * M;
    U[i] = (j < M) ? c[M + r - j] : 0.0;
  }
  for (long long i = tid; i < (long long)M2 * M2; i += nt) V[i] = (i / M2 == i % M2) ? 1.0 : 0.0;
  for (long long r = tid; r < M2; r += nt) rhs[r] = (r < M) ? -c[M + 1 + r] : 0.0;
}

// This lane's partial |U_p|^2, |U_q|^2 and U_p . U_q.
PADE_HD void pair_dots(const double* U, int M, int p, int q, int lane, int nl, double& a, double& b, double& g) {
  const double* up = U + (size_t)p * M;
  const double* uq = U + (size_t)q * M;
  a = b = g = 0.0;
  for (int r = lane; r < M; r += nl) {
    const double x = up[r], y = uq[r];
    a += x * x;
    b += y * y;
    g += x * y;
  }
}

// This thread's share of |G|_F^2 = sum_k (M - |k - M|) c_k^2 (c_k fills M - |k - M| entries).
PADE_HD double fro2_partial(const double* c, int M, long long tid, long long nt) {
  double s = 0.0;
  for (long long k = 1 + tid; k <= 2LL * M - 1; k += nt) {
    const double m = (double)(M - (k > M ? k - M : M - k));
    s += m * c[k] * c[k];
  }
  return s;
}

// Columns with norm^2 at or below eps^2 |G|_F^2 take part in no rotation: they end below the
// least-squares cut (whose square is at least eps^2 M^2 |G|_F^2 / (M + 1)) and stay there.
// Without this floor, columns of negligible size (a pulse record that has decayed to
// underflow) keep rotating among themselves for many sweeps.
PADE_HD double floor2(double fro2) { return kEps * kEps * fro2; }

// The rotation that makes columns p and q orthogonal, from the full a, b, g; false when they
// already are (cosine below kOrthTol), when either is below the floor, or for non-finite input.
PADE_HD bool rotation(double a, double b, double g, double fl, double& cs, double& sn) {
  if (!(a > fl && b > fl)) return false;
  if (!(fabs(g) > kOrthTol * sqrt(a * b))) return false;
  const double zeta = (b - a) / (2.0 * g);
  const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  cs = 1.0 / sqrt(1.0 + t * t);
  sn = cs * t;
  return true;
}

// Applies the rotation to this lane's rows of columns p, q of U (M rows) and V (M2 rows).
PADE_HD void pair_apply(double* U, double* V, int M, int M2, int p, int q, double cs, double sn, int lane, int nl) {
  double* up = U + (size_t)p * M;
  double* uq = U + (size_t)q * M;
  for (int r = lane; r < M; r += nl) {
    const double x = up[r], y = uq[r];
    up[r] = cs * x - sn * y;
    uq[r] = sn * x + cs * y;
  }
  double* vp = V + (size_t)p * M2;
  double* vq = V + (size_t)q * M2;
  for (int r = lane; r < M2; r += nl) {
    const double x = vp[r], y = vq[r];
    vp[r] = cs * x - sn * y;
    vq[r] = sn * x + cs * y;
  }
}

// This lane's partial |U_j|^2 and U_j . rhs.
PADE_HD void col_dots(const double* U, const double* rhs, int M, int j, int lane, int nl, double& s2, double& pr) {
  const double* u = U + (size_t)j * M;
  s2 = pr = 0.0;
  for (int r = lane; r < M; r += nl) {
    s2 += u[r] * u[r];
    pr += u[r] * rhs[r];
  }
}

// Squared cut: sigma_j counts when sigma_j^2 > cut2(M, max sigma^2).
PADE_HD double cut2(int M, double s2max) { return (kEps * M) * (kEps * M) * s2max; }

// Denominator entry b_{i+1} = sum_j V[i][j] w_j (w_j = (U_j . rhs) / sigma_j^2 or 0).
PADE_HD double denominator(const double* V, const double* w, int M2, int i) {
  double acc = 0.0;
  for (int j = 0; j < M2; ++j) acc += V[(size_t)j * M2 + i] * w[j];
  return acc;
}

// Numerator a_k = sum_{m<=k} b_m c_{k-m}.
PADE_HD double numerator(const double* b, const double* c, int k) {
  double acc = 0.0;
  for (int m = 0; m <= k; ++m) acc += b[m] * c[k - m];
  return acc;
}

// P(z) / Q(z) at z = (zr, zi) by Horner's rule (a, b: M + 1 coefficients each).
PADE_HD void ratio(const double* a, const double* b, int M, double zr, double zi, double& vr, double& vi) {
  double pr = a[M], pi = 0.0, qr = b[M], qi = 0.0;
  for (int k = M - 1; k >= 0; --k) {
    const double tr = pr * zr - pi * zi + a[k], ti = pr * zi + pi * zr;
    pr = tr;
    pi = ti;
    const double ur = qr * zr - qi * zi + b[k], ui = qr * zi + qi * zr;
    qr = ur;
    qi = ui;
  }
  const double den = qr * qr + qi * qi;
  vr = (pr * qr + pi * qi) / den;
  vi = (pi * qr - pr * qi) / den;
}

}  // namespace pade
}  // namespace rtcc
