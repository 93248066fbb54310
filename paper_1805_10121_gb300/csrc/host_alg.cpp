// Host-side pieces of the ChASE iteration: the degree rule (Alg. 5), the
// locking rule (Alg. 3), the symmetric tridiagonal eigensolve of the Lanczos
// matrices T_k (Alg. 6) and the density-of-states quantile (Eq. 10).  These
// act on O(nev + nex) or O(k^2) numbers and run between kernel launches.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "chase.h"
#include "common.cuh"
#include "context.hpp"

namespace chase {

// Alg. 5 for one Ritz pair.
static int degree_of(double tol, double res, double lam, double c, double e, int deg_extra,
                     int deg_max) {
  const double t = (lam - c) / e;
  // |rho| = max |t -+ sqrt(t^2 - 1)|: for |t| > 1 this is |t| + sqrt(t^2 - 1),
  // for |t| <= 1 both roots have modulus 1.
  const double rho = std::fabs(t) > 1.0 ? std::fabs(t) + std::sqrt(t * t - 1.0) : 1.0;
  int deg;
  double q = HUGE_VAL;
  if (rho > 1.0 + 1e-14 && res > 0.0) q = std::fabs(std::log(res / tol) / std::log(rho));
  if (!std::isfinite(q) || q > 1e6)
    deg = deg_max;
  else
    deg = static_cast<int>(std::ceil(q));
  deg = std::min(deg + deg_extra, deg_max);
  deg = deg + deg % 2;
  if (deg > deg_max) deg -= 2;
  return deg;
}

// Implicit symmetric QR sweeps with Wilkinson shifts on a dense copy of the
// tridiagonal matrix (k is the Lanczos length, a few dozen at most), with
// deflation of negligible sub-diagonal entries.
bool tridiag_eigh(int k, const double* diag, const double* off, double* w, double* z) {
  if (k <= 0) return true;
  std::vector<double> T(static_cast<size_t>(k) * k, 0.0);
  auto at = [&](int r, int c) -> double& { return T[static_cast<size_t>(c) * k + r]; };
  for (int i = 0; i < k; ++i) at(i, i) = diag[i];
  for (int i = 0; i + 1 < k; ++i) at(i + 1, i) = at(i, i + 1) = off[i];
  std::vector<double> Z(static_cast<size_t>(k) * k, 0.0);
  for (int i = 0; i < k; ++i) Z[static_cast<size_t>(i) * k + i] = 1.0;
  const double eps = 2.220446049250313e-16;
  auto negligible = [&](int i) {  // sub-diagonal entry (i, i-1)
    return std::fabs(at(i, i - 1)) <= eps * (std::fabs(at(i, i)) + std::fabs(at(i - 1, i - 1)));
  };
  // rotation in the (p, p+1) plane: T <- G^T T G, Z <- Z G, G = [[c, -s], [s, c]]
  auto rotate = [&](int p, double c, double s) {
    for (int j = 0; j < k; ++j) {
      const double x = at(p, j), y = at(p + 1, j);
      at(p, j) = c * x + s * y;
      at(p + 1, j) = -s * x + c * y;
    }
    for (int i = 0; i < k; ++i) {
      const double x = at(i, p), y = at(i, p + 1);
      at(i, p) = c * x + s * y;
      at(i, p + 1) = -s * x + c * y;
    }
    for (int i = 0; i < k; ++i) {
      double* zp = &Z[static_cast<size_t>(p) * k + i];
      double* zq = &Z[static_cast<size_t>(p + 1) * k + i];
      const double x = *zp, y = *zq;
      *zp = c * x + s * y;
      *zq = -s * x + c * y;
    }
  };
  int hi = k - 1;
  long iters = 0;
  while (hi > 0) {
    if (negligible(hi)) {
      at(hi, hi - 1) = at(hi - 1, hi) = 0.0;
      --hi;
      continue;
    }
    int lo = hi - 1;
    while (lo > 0 && !negligible(lo)) --lo;
    if (lo > 0) at(lo, lo - 1) = at(lo - 1, lo) = 0.0;
    if (++iters > 60L * k) return false;
    // Wilkinson shift: eigenvalue of the trailing 2 x 2 block closer to T(hi, hi)
    const double a = at(hi - 1, hi - 1), bb = at(hi, hi - 1), cc = at(hi, hi);
    const double dd = 0.5 * (a - cc);
    const double den = dd + std::copysign(std::hypot(dd, bb), dd == 0.0 ? 1.0 : dd);
    const double mu = den != 0.0 ? cc - bb * bb / den : cc;
    for (int p = lo; p < hi; ++p) {
      double x, y;
      if (p == lo) {
        x = at(lo, lo) - mu;
        y = at(lo + 1, lo);
      } else {
        x = at(p, p - 1);
        y = at(p + 1, p - 1);
      }
      const double r = std::hypot(x, y);
      if (r == 0.0) continue;
      rotate(p, x / r, y / r);
      if (p > lo) at(p + 1, p - 1) = at(p - 1, p + 1) = 0.0;  // bulge chased away
    }
  }
  std::vector<int> order(k);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return at(x, x) < at(y, y); });
  for (int j = 0; j < k; ++j) {
    w[j] = at(order[j], order[j]);
    for (int i = 0; i < k; ++i)
      z[static_cast<size_t>(j) * k + i] = Z[static_cast<size_t>(order[j]) * k + i];
  }
  return true;
}

// Alg. 6 line 11: the target quantile of the Eq. 10 density estimate, kept
// strictly inside (mu1, b_sup).  Run c contributes the nodes
// theta[off_c .. off_c + steps[c]) with weights w (|Z_1i|^2); the estimate
// is the average of the runs' Gaussian sums.  Sec. 4.2 leaves its
// safeguards unpublished; the width is halved (at most 40 times) until the
// quantile lies inside the interval by 1e-6 of its width, failing which the
// quantile of a uniform density on [mu1, b_sup] is taken (target clamped to
// [1e-3, 0.5]).
double dos_estimate(int nruns, const int* steps, const double* theta, const double* w,
                    double target, double mu1, double b_sup, double dos_sigma, int* halvings,
                    bool* fallback) {
  const double half = 0.5 * (b_sup - mu1);
  double sig = half > 1e-12 * std::max(1.0, std::max(std::fabs(b_sup), std::fabs(mu1)))
                   ? dos_sigma * half
                   : dos_sigma;
  double tmin = HUGE_VAL, tmax = -HUGE_VAL;
  int total = 0;
  for (int c = 0; c < nruns; ++c) total += steps[c];
  for (int i = 0; i < total; ++i) {
    tmin = std::min(tmin, theta[i]);
    tmax = std::max(tmax, theta[i]);
  }
  auto normal_cdf = [](double x) { return 0.5 * (1.0 + std::erf(x / std::sqrt(2.0))); };
  auto cdf = [&](double t, double s) {  // integral of Eq. 10 up to t
    double acc = 0.0;
    for (int i = 0; i < total; ++i) acc += w[i] * normal_cdf((t - theta[i]) / s);
    return acc / nruns;
  };
  auto quantile = [&](double s) {  // bisection on the monotone cdf
    double lo = tmin - 10.0 * s, hi = tmax + 10.0 * s;
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (cdf(mid, s) < target)
        lo = mid;
      else
        hi = mid;
    }
    return 0.5 * (lo + hi);
  };
  const double margin = 1e-6 * (b_sup - mu1);
  auto inside = [&](double m) { return mu1 + margin < m && m < b_sup - margin; };
  double mu = quantile(sig);
  int h = 0;
  while (!inside(mu) && h < 40) {
    sig *= 0.5;
    ++h;
    mu = quantile(sig);
  }
  if (halvings) *halvings = h;
  if (fallback) *fallback = !inside(mu);
  if (inside(mu)) return mu;
  return mu1 + (b_sup - mu1) * std::min(std::max(target, 1e-3), 0.5);
}

}  // namespace chase

extern "C" int chase_dos_estimate(int nruns, const int* steps, const double* theta,
                                  const double* weights, double target, double mu1, double b_sup,
                                  double dos_sigma, double* mu_out, int* halvings_out) {
  bool ok = nruns > 0 && steps && theta && weights && mu_out && std::isfinite(target) &&
            target > 0.0 && target < 1.0 && std::isfinite(mu1) && std::isfinite(b_sup) &&
            mu1 <= b_sup && dos_sigma > 0.0 && std::isfinite(dos_sigma);
  for (int c = 0; ok && c < nruns; ++c) ok = steps[c] > 0;
  if (!ok) {
    chase::set_error("chase_dos_estimate: invalid argument");
    return CHASE_INVALID_ARG;
  }
  int h = 0;
  bool fb = false;
  *mu_out = chase::dos_estimate(nruns, steps, theta, weights, target, mu1, b_sup, dos_sigma, &h,
                                &fb);
  // halvings_out: the number of halvings, or -1 when the uniform fallback was taken
  if (halvings_out) *halvings_out = fb ? -1 : h;
  return CHASE_OK;
}

extern "C" int chase_degrees(int b, const double* resid, const double* ritz, double c, double e,
                             double tol, int deg_extra, int deg_max, int* degrees_out) {
  if (b < 0 || (b > 0 && (!resid || !ritz || !degrees_out)) || !(e > 0.0) || !(tol > 0.0) ||
      deg_max < 2 || deg_extra < 0) {
    chase::set_error("chase_degrees: invalid argument");
    return CHASE_INVALID_ARG;
  }
  for (int a = 0; a < b; ++a)
    degrees_out[a] = chase::degree_of(tol, resid[a], ritz[a], c, e, deg_extra, deg_max);
  return CHASE_OK;
}

extern "C" int chase_lock(int b, const double* ritz, const double* resid, double tol,
                          int* order_out, int* n_lock) {
  if (b < 0 || (b > 0 && (!ritz || !resid || !order_out)) || !n_lock) {
    chase::set_error("chase_lock: invalid argument");
    return CHASE_INVALID_ARG;
  }
  std::vector<int> order(b);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return ritz[x] < ritz[y]; });
  int n = 0;
  while (n < b && !(resid[order[n]] > tol)) ++n;
  for (int a = 0; a < b; ++a) order_out[a] = order[a];
  *n_lock = n;
  return CHASE_OK;
}

extern "C" int chase_tridiag_eigh(int k, const double* diag, const double* off, double* w,
                                  double* z) {
  if (k < 0 || (k > 0 && (!diag || !w || !z)) || (k > 1 && !off)) {
    chase::set_error("chase_tridiag_eigh: invalid argument");
    return CHASE_INVALID_ARG;
  }
  if (!chase::tridiag_eigh(k, diag, off, w, z)) {
    chase::set_error("chase_tridiag_eigh: no convergence");
    return CHASE_EIGENSOLVER_ERROR;
  }
  return CHASE_OK;
}
