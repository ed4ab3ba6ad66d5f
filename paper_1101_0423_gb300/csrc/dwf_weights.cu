// dwf_weights.cu -- weights of the optimal domain-wall operator (host code only).
//
// With sigma = omega, Eq. 1 reduces in four dimensions to an operator built on
//   S(lam) = (1 - T(lam)) / (1 + T(lam)),  T(lam) = prod_s (1 - omega_s lam) / (1 + omega_s lam)
// over the spectrum [lmin, lmax] of |H_w|.  Sec. 2.1 wants the weights that give the best
// chiral symmetry Ns slices allow and takes them from a cited formula it does not print;
// the reading here is the best uniform approximation of sgn: omega minimizing max |1 - S| on
// [lmin, lmax].  The optimum is characterised by alternation (the error e = 1 - S reaches
// +-delta with alternating signs at Ns + 1 points), which the Remez exchange below solves:
//   1. with x_s = 1 / omega_s the zeros of T, solve e(lam_i) = (-1)^i delta at the
//      reference points lam_0 < ... < lam_Ns by Newton's method in (log x_s, delta);
//   2. move lam_i to the extremum of |e| between consecutive zeros (one per interval),
//      located by golden-section search in log lam;
//   3. repeat until the extrema agree.
#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/dwf.h"

namespace {

// T and e = 2 T / (1 + T) at lam for the zeros x
void error_at(const std::vector<double> &x, double lam, double *T, double *e) {
  double t = 1.0;
  for (double xs : x) t *= (xs - lam) / (xs + lam);
  *T = t;
  *e = 2.0 * t / (1.0 + t);
}

double abs_error(const std::vector<double> &x, double lam) {
  double T, e;
  error_at(x, lam, &T, &e);
  return fabs(e);
}

// dense solve of A y = b (n x n, row-major) by Gaussian elimination with partial pivoting
bool solve(std::vector<double> &A, std::vector<double> &b, int n) {
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(A[r * n + c]) > fabs(A[p * n + c])) p = r;
    if (A[p * n + c] == 0.0) return false;
    if (p != c) {
      for (int k = 0; k < n; ++k) std::swap(A[c * n + k], A[p * n + k]);
      std::swap(b[c], b[p]);
    }
    for (int r = c + 1; r < n; ++r) {
      const double f = A[r * n + c] / A[c * n + c];
      for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
      b[r] -= f * b[c];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = b[r];
    for (int k = r + 1; k < n; ++k) s -= A[r * n + k] * b[k];
    b[r] = s / A[r * n + r];
  }
  return true;
}

// residuals F_i = e(lam_i) - (-1)^i delta and, if A is given, their Jacobian in (log x, delta)
double residuals(const std::vector<double> &x, double delta, const std::vector<double> &lam,
                 std::vector<double> &F, std::vector<double> *A) {
  const int ns = (int)x.size(), n = ns + 1;
  double fmax = 0.0;
  for (int i = 0; i < n; ++i) {
    double T, e;
    error_at(x, lam[i], &T, &e);
    const double sg = (i & 1) ? -1.0 : 1.0;
    F[i] = e - sg * delta;
    fmax = std::max(fmax, fabs(F[i]));
    if (A) {
      const double dedT = 2.0 / ((1.0 + T) * (1.0 + T));
      for (int s = 0; s < ns; ++s)  // d e / d log x_s
        (*A)[(size_t)i * n + s] = dedT * T * 2.0 * lam[i] * x[s] / (x[s] * x[s] - lam[i] * lam[i]);
      (*A)[(size_t)i * n + ns] = -sg;
    }
  }
  return fmax;
}

// step 1: Newton on F = 0 in (log x, delta), every zero kept strictly between its two
// reference points, with backtracking on max |F|
bool levelled(std::vector<double> &x, double &delta, const std::vector<double> &lam) {
  const int ns = (int)x.size(), n = ns + 1;
  std::vector<double> A((size_t)n * n), F(n), G(n), xt(ns);
  double fmax = residuals(x, delta, lam, F, &A);
  for (int it = 0; it < 200; ++it) {
    // T is a product of Ns rounded ratios: its relative accuracy is a few Ns ulp
    if (fmax <= 1e-13 * std::max(fabs(delta), 1e-300)) return true;
    for (int i = 0; i < n; ++i) F[i] = -F[i];
    if (!solve(A, F, n)) return false;
    double scale = 1.0;  // at most half of the way to either neighbour, in log lam
    for (int s = 0; s < ns; ++s) {
      const double room = F[s] > 0 ? log(lam[s + 1] / x[s]) : log(lam[s] / x[s]);
      if (F[s] != 0.0) scale = std::min(scale, 0.5 * room / F[s]);
    }
    double step = fabs(F[ns]) / std::max(fabs(delta), 1e-300);
    for (int s = 0; s < ns; ++s) step = std::max(step, fabs(F[s]));
    bool moved = false;
    for (int k = 0; k < 40 && !moved; ++k, scale *= 0.5) {
      for (int s = 0; s < ns; ++s) xt[s] = x[s] * exp(scale * F[s]);
      const double dt = delta + scale * F[ns];
      const double ft = residuals(xt, dt, lam, G, nullptr);
      if (ft < fmax || (ft <= fmax && step * scale <= 1e-14)) {
        x = xt, delta = dt, moved = true;
      }
    }
    if (!moved) return fmax <= 1e-10 * std::max(fabs(delta), 1e-300);
    fmax = residuals(x, delta, lam, F, &A);
    if (step <= 1e-14) return true;
  }
  return false;
}

// step 2: the extremum of |e| on [a, b] (golden section in log lam)
double extremum(const std::vector<double> &x, double a, double b) {
  const double g = 0.5 * (sqrt(5.0) - 1.0);
  double lo = log(a), hi = log(b);
  double c = hi - g * (hi - lo), d = lo + g * (hi - lo);
  double fc = abs_error(x, exp(c)), fd = abs_error(x, exp(d));
  for (int it = 0; it < 200 && hi - lo > 1e-15 * (fabs(lo) + 1.0); ++it) {
    if (fc > fd) {
      hi = d, d = c, fd = fc;
      c = hi - g * (hi - lo), fc = abs_error(x, exp(c));
    } else {
      lo = c, c = d, fc = fd;
      d = lo + g * (hi - lo), fd = abs_error(x, exp(d));
    }
  }
  // an extremum at an end of the interval (the first and last intervals)
  double best = exp(0.5 * (lo + hi)), fb = abs_error(x, best);
  if (abs_error(x, a) >= fb) best = a, fb = abs_error(x, a);
  if (abs_error(x, b) > fb) best = b;
  return best;
}

}  // namespace

extern "C" dwf_status dwf_optimal_weights(int Ns, double lambda_min, double lambda_max, double *omega,
                                          double *delta_out) {
  if (Ns < 1 || Ns > 64 || !omega || !(lambda_min > 0.0) || !(lambda_max > lambda_min) || !std::isfinite(lambda_max))
    return DWF_EINVAL;
  const double r = lambda_max / lambda_min;
  std::vector<double> x(Ns), lam(Ns + 1);
  for (int s = 0; s < Ns; ++s) x[s] = lambda_min * pow(r, (s + 0.5) / Ns);
  for (int i = 0; i <= Ns; ++i) lam[i] = lambda_min * pow(r, (double)i / Ns);
  double delta = 0.0;
  for (int i = 0; i <= Ns; ++i) delta = std::max(delta, abs_error(x, lam[i]));
  bool settled = false;
  for (int round = 0; round < 100 && !settled; ++round) {
    if (!levelled(x, delta, lam)) return DWF_ENOCONV;
    double emin = 1e300, emax = 0.0;
    for (int i = 0; i <= Ns; ++i) {
      const double a = i == 0 ? lambda_min : x[i - 1], b = i == Ns ? lambda_max : x[i];
      lam[i] = extremum(x, a, b);
      const double v = abs_error(x, lam[i]);
      emin = std::min(emin, v), emax = std::max(emax, v);
    }
    settled = emax - emin <= 2e-14 * (Ns + 4) * emax;  // rounding of a product of Ns ratios
    delta = emax;
  }
  if (!settled) return DWF_ENOCONV;
  for (int s = 0; s < Ns; ++s) omega[s] = 1.0 / x[s];  // x ascending: omega decreasing
  if (delta_out) *delta_out = delta;
  return DWF_OK;
}
