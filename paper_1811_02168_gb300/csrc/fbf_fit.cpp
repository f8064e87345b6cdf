// Host FP64 fitter for the cosine approximation of the range kernel.
//
// Section II of the paper: b(t) = phi(t) on Lambda = {-R..R}; A(t,k) = cos(nu t k),
// nu = 2 pi/(2T+1), k = 0..K-1; E(K,T) = min_c ||A c - b||^2 (eq. 5);
// e(K) = min_T E(K,T) (eq. 6); Algorithm 1 picks the smallest K with e(K) <= eps.
//
// Implementation (independent of the NumPy oracle): both the rows t and -t of A are
// identical, so for the even part b_e of b the squared residual folds onto t = 0..R with
// weights 1 (t = 0) and 2 (t > 0); the odd part b_o is orthogonal to every cosine and adds
// ||b_o||^2 to E.  The folded, row-scaled system (R+1) x K is reduced by Householder
// reflections one column at a time, which yields E(1,T), E(2,T), ... in one pass: after
// column j the residual energy is the squared tail of the transformed right-hand side.
// A column whose remaining norm is negligible (exact rank deficiency, K > T+1) is
// dropped; its coefficient is 0.  T is scanned over 1..T_max in parallel threads; each T
// is independent, so the result does not depend on the thread count.
//
// Readings where the paper is silent: T_max = 4R, doubled while the optimum is above
// T_max/2; errors below 1e-20 ||b||^2 count as equal and the smallest T among them wins.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <thread>

#include "fbf_internal.h"

namespace fbf {
namespace {

constexpr double kFloorRel = 1e-20;
constexpr double kDependentTol = 1e-12;

struct Folded {
  int R;
  std::vector<double> be;     // even part on t = 0..R
  double odd_energy;          // sum over Lambda of b_o(t)^2
  double bnorm2;              // ||b||^2 over Lambda
};

Folded fold(const double* b, int R) {
  Folded f;
  f.R = R;
  f.be.resize(R + 1);
  f.odd_energy = 0.0;
  f.bnorm2 = 0.0;
  for (int i = 0; i <= 2 * R; ++i) f.bnorm2 += b[i] * b[i];
  for (int t = 0; t <= R; ++t) {
    double bp = b[R + t], bm = b[R - t];
    f.be[t] = 0.5 * (bp + bm);
    double o = 0.5 * (bp - bm);
    f.odd_energy += (t == 0 ? 1.0 : 2.0) * o * o;
  }
  return f;
}

// Householder reduction of the folded system at one T, for columns 0..Kc-1.
// E_out[j] = E(j+1, T).  If c_out != nullptr, also solves for the coefficients of the
// first Kc columns (dropped columns get 0).
void reduce(const Folded& F, int T, int Kc, double* E_out, double* c_out) {
  const int n = F.R + 1;
  const int P = 2 * T + 1;
  std::vector<double> tab(P);
  for (int m = 0; m < P; ++m) tab[m] = std::cos(2.0 * M_PI * (double)m / (double)P);
  // column-major n x Kc, rows scaled by sqrt(weight)
  std::vector<double> A((size_t)n * Kc), y(n);
  for (int t = 0; t <= F.R; ++t) {
    double s = (t == 0) ? 1.0 : std::sqrt(2.0);
    y[t] = s * F.be[t];
    for (int k = 0; k < Kc; ++k) {
      long m = ((long)t * (long)k) % P;
      A[(size_t)k * n + t] = s * tab[m];
    }
  }
  std::vector<double> colnorm0(Kc);
  for (int k = 0; k < Kc; ++k) {
    double s = 0;
    for (int i = 0; i < n; ++i) s += A[(size_t)k * n + i] * A[(size_t)k * n + i];
    colnorm0[k] = std::sqrt(s);
  }
  std::vector<int> pivot_row(Kc, -1);
  std::vector<double> v(n);
  int p = 0;  // next pivot row
  for (int j = 0; j < Kc; ++j) {
    double* a = &A[(size_t)j * n];
    double s = 0;
    for (int i = p; i < n; ++i) s += a[i] * a[i];
    double nrm = std::sqrt(s);
    if (p < n && nrm > kDependentTol * colnorm0[j]) {
      // reflector H = I - 2 v v^T / (v^T v) mapping a[p..] to (-sign(a_p) nrm, 0, ...)
      double alpha = (a[p] >= 0) ? -nrm : nrm;
      for (int i = p; i < n; ++i) v[i] = a[i];
      v[p] -= alpha;
      double vv = 0;
      for (int i = p; i < n; ++i) vv += v[i] * v[i];
      if (vv > 0) {
        for (int jj = j; jj < Kc; ++jj) {
          double* col = &A[(size_t)jj * n];
          double d = 0;
          for (int i = p; i < n; ++i) d += v[i] * col[i];
          d = 2.0 * d / vv;
          for (int i = p; i < n; ++i) col[i] -= d * v[i];
        }
        double d = 0;
        for (int i = p; i < n; ++i) d += v[i] * y[i];
        d = 2.0 * d / vv;
        for (int i = p; i < n; ++i) y[i] -= d * v[i];
      }
      pivot_row[j] = p;
      ++p;
    }
    double e = 0;
    for (int i = p; i < n; ++i) e += y[i] * y[i];
    E_out[j] = e + F.odd_energy;
  }
  if (c_out) {
    for (int j = Kc - 1; j >= 0; --j) {
      if (pivot_row[j] < 0) { c_out[j] = 0.0; continue; }
      int pr = pivot_row[j];
      double s = y[pr];
      for (int jj = j + 1; jj < Kc; ++jj) s -= A[(size_t)jj * n + pr] * c_out[jj];
      c_out[j] = s / A[(size_t)j * n + pr];
    }
  }
}

// E[T-1][K-1] for T = 1..T_max, K = 1..Kc (row-major T x Kc).
std::vector<double> error_table(const Folded& F, int T_max, int Kc) {
  std::vector<double> tab((size_t)T_max * Kc);
  unsigned hw = std::thread::hardware_concurrency();
  int nth = (int)std::max(1u, std::min(hw ? hw : 1u, 16u));
  nth = std::min(nth, T_max);
  // stripe w takes T = 1 + w, 1 + w + nth, ...; an exception in a stripe (an allocation) is
  // recorded and rethrown here after every thread has joined
  std::atomic<bool> failed{false};
  auto stripe = [&](int w) {
    try {
      for (int T = 1 + w; T <= T_max; T += nth) reduce(F, T, Kc, &tab[(size_t)(T - 1) * Kc], nullptr);
    } catch (...) {
      failed = true;
    }
  };
  std::vector<std::thread> pool;
  pool.reserve(nth);
  int started = 1;
  for (; started < nth; ++started) {
    try {
      pool.emplace_back(stripe, started);
    } catch (...) {
      break;                                   // no more threads: this one takes the rest
    }
  }
  for (int w = started; w < nth; ++w) stripe(w);
  stripe(0);
  for (auto& th : pool) th.join();
  if (failed) throw std::bad_alloc();
  return tab;
}

// argmin over T of max(E(K,T), floor), smallest T on ties.
int argmin_T(const std::vector<double>& tab, int T_max, int Kc, int K, double floor_v) {
  int best = 1;
  double bv = std::max(tab[(size_t)0 * Kc + (K - 1)], floor_v);
  for (int T = 2; T <= T_max; ++T) {
    double v = std::max(tab[(size_t)(T - 1) * Kc + (K - 1)], floor_v);
    if (v < bv) { bv = v; best = T; }
  }
  return best;
}

}  // namespace

void kernel_error_curve(const double* b, int R, int T, int Kc, double* E_out) {
  Folded F = fold(b, R);
  reduce(F, T, Kc, E_out, nullptr);
}

int fit_range_kernel(const double* b, int R, int K, double eps, int T_fixed, FitResult* out,
                     std::string* msg) {
  if (R < 1 || !b || !out) { *msg = "fit: R < 1 or null pointer"; return FBF_EINVAL; }
  if (K < 0 || (K == 0 && !(eps > 0))) { *msg = "fit: need K >= 1 or eps > 0"; return FBF_EINVAL; }
  for (int i = 0; i <= 2 * R; ++i)
    if (!std::isfinite(b[i])) { *msg = "fit: non-finite kernel sample"; return FBF_EINVAL; }
  Folded F = fold(b, R);
  const double floor_v = kFloorRel * F.bnorm2;
  int T_star = 0, K_star = 0;

  if (T_fixed > 0) {
    if (K == 0) {  // smallest K at this fixed T with E <= eps
      int Kc = 8;
      while (true) {
        std::vector<double> E(Kc);
        reduce(F, T_fixed, Kc, E.data(), nullptr);
        for (int k = 1; k <= Kc; ++k)
          if (std::max(E[k - 1], floor_v) <= eps) { K_star = k; break; }
        if (K_star) break;
        if (Kc >= 2 * R + 1) { *msg = "fit: eps not reached"; return FBF_EUNSUPPORTED; }
        Kc = std::min(2 * Kc, 2 * R + 1);
      }
    } else {
      K_star = K;
    }
    T_star = T_fixed;
  } else {
    int T_max = 4 * R;
    int Kc = (K > 0) ? K : 8;
    for (int iter = 0; iter < 16; ++iter) {
      std::vector<double> tab = error_table(F, T_max, Kc);
      int Ksel = 0, Tsel = 0;
      if (K > 0) {
        Ksel = K;
        Tsel = argmin_T(tab, T_max, Kc, K, floor_v);
      } else {
        for (int k = 1; k <= Kc && !Ksel; ++k) {
          int t = argmin_T(tab, T_max, Kc, k, floor_v);
          if (std::max(tab[(size_t)(t - 1) * Kc + (k - 1)], floor_v) <= eps) { Ksel = k; Tsel = t; }
        }
        if (!Ksel) {
          if (Kc >= 2 * R + 1) { *msg = "fit: eps not reached"; return FBF_EUNSUPPORTED; }
          Kc = std::min(2 * Kc, 2 * R + 1);
          continue;
        }
      }
      if (Tsel > T_max / 2) { T_max *= 2; continue; }
      K_star = Ksel;
      T_star = Tsel;
      break;
    }
    if (!K_star) { *msg = "fit: period search did not settle"; return FBF_EUNSUPPORTED; }
  }

  out->K = K_star;
  out->T = T_star;
  out->c.assign(K_star, 0.0);
  std::vector<double> E(K_star);
  reduce(F, T_star, K_star, E.data(), out->c.data());
  out->E = E[K_star - 1];
  const int P = 2 * T_star + 1;
  double dmax = 0;
  for (int t = -R; t <= R; ++t) {
    double s = 0;
    for (int k = 0; k < K_star; ++k) {
      long m = (((long)t * k) % P + P) % P;
      s += out->c[k] * std::cos(2.0 * M_PI * (double)m / (double)P);
    }
    dmax = std::max(dmax, std::fabs(s - b[t + R]));
  }
  out->delta_max = dmax;
  return FBF_OK;
}

}  // namespace fbf
