// Host build of the Pade core (paper_2205_05175_gb300/csrc/pade_core.cuh) for the CPU tests:
// the same per-lane arithmetic the device kernels run, with the 32 lanes of a warp and the
// warp's shuffle-down reduction tree replayed in order.  Not part of the library.
//
// stdin:  "pairs n"                      -> every (round, p, q) of the tournament over n columns
//         "pade N c_0..c_{N-1} nz z..."  -> sweeps, then P/Q at each z = (re, im)
#include <cstdio>
#include <cstring>
#include <vector>

#include "pade_core.cuh"

using namespace rtcc::pade;

static double warp_sum(double* x) {
  for (int off = 16; off > 0; off >>= 1)
    for (int l = 0; l + off < 32; ++l) x[l] += x[l + off];
  return x[0];
}

int main() {
  char mode[16];
  if (scanf("%15s", mode) != 1) return 2;
  if (!strcmp(mode, "pairs")) {
    int n;
    if (scanf("%d", &n) != 1) return 2;
    for (int r = 0; r < n - 1; ++r)
      for (int k = 0; k < n / 2; ++k) {
        int p, q;
        pair_of(n, r, k, p, q);
        printf("%d %d %d\n", r, p, q);
      }
    return 0;
  }
  int N;
  if (scanf("%d", &N) != 1 || N < 3) return 2;
  std::vector<double> c(N);
  for (double& x : c)
    if (scanf("%lf", &x) != 1) return 2;
  int nz;
  if (scanf("%d", &nz) != 1) return 2;
  std::vector<double> zr(nz), zi(nz);
  for (int i = 0; i < nz; ++i)
    if (scanf("%lf %lf", &zr[i], &zi[i]) != 2) return 2;
  const int M = (N - 1) / 2, M2 = padded(M);
  std::vector<double> work(work_doubles(M));
  double* U = work.data();
  double* V = U + (size_t)M * M2;
  double* rhs = V + (size_t)M2 * M2;
  double* s2 = rhs + M2;
  double* w = s2 + M2;
  fill(c.data(), M, U, V, rhs, 0, 1);
  const double fl = floor2(fro2_partial(c.data(), M, 0, 1));
  int sweep = 0;
  for (; sweep < kMaxSweeps; ++sweep) {
    bool rotated = false;
    for (int r = 0; r < M2 - 1; ++r)
      for (int k = 0; k < M2 / 2; ++k) {
        int p, q;
        pair_of(M2, r, k, p, q);
        double A[32], B[32], G[32];
        for (int l = 0; l < 32; ++l) pair_dots(U, M, p, q, l, 32, A[l], B[l], G[l]);
        const double a = warp_sum(A), b = warp_sum(B), g = warp_sum(G);
        double cs, sn;
        if (rotation(a, b, g, fl, cs, sn)) {
          for (int l = 0; l < 32; ++l) pair_apply(U, V, M, M2, p, q, cs, sn, l, 32);
          rotated = true;
        }
      }
    if (!rotated) break;
  }
  double s2max = 0.0;
  for (int j = 0; j < M2; ++j) {
    double S[32], P[32];
    for (int l = 0; l < 32; ++l) col_dots(U, rhs, M, j, l, 32, S[l], P[l]);
    s2[j] = warp_sum(S);
    w[j] = warp_sum(P);
    if (s2[j] > s2max) s2max = s2[j];
  }
  const double cut = cut2(M, s2max);
  for (int j = 0; j < M2; ++j) w[j] = (s2[j] > cut) ? w[j] / s2[j] : 0.0;
  std::vector<double> a(M + 1), b(M + 1);
  b[0] = 1.0;
  for (int i = 0; i < M; ++i) b[i + 1] = denominator(V, w, M2, i);
  for (int k = 0; k <= M; ++k) a[k] = numerator(b.data(), c.data(), k);
  printf("%d\n", sweep);
  for (int i = 0; i < nz; ++i) {
    double vr, vi;
    ratio(a.data(), b.data(), M, zr[i], zi[i], vr, vi);
    printf("%.17g %.17g\n", vr, vi);
  }
  return 0;
}
