// Lookup table of the optimal order K* and period parameter T* (Section II, after
// Algorithm 1): Algorithm 1 is run offline on a grid of (sigma, eps) for the Gaussian range
// kernel of eq. (2); at run time K and T for any (sigma, eps) inside the grid are estimated
// by bilinear interpolation in (sigma, log(1/eps)), and only the least squares of eq. (5)
// for the coefficients is solved.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <new>
#include <string>
#include <vector>

#include "fbf.h"
#include "fbf_internal.h"

struct fbf_lut_s {
  int R = 0;
  std::vector<double> sigma;   // increasing
  std::vector<double> u;       // log(1/eps), increasing
  std::vector<int> K, T;       // [i_sigma * n_u + j_u]
};

namespace {

int check_grid(const std::vector<double>& v, const char* what) {
  if (v.size() < 2) return fbf::set_error(FBF_EINVAL, std::string("fbf_lut: need at least two ") + what);
  for (size_t i = 0; i < v.size(); ++i) {
    if (!std::isfinite(v[i])) return fbf::set_error(FBF_EINVAL, std::string("fbf_lut: non-finite ") + what);
    if (i && !(v[i] > v[i - 1])) return fbf::set_error(FBF_EINVAL, std::string("fbf_lut: ") + what + " must be strictly monotone");
  }
  return FBF_OK;
}

// cell index and weight of x in the increasing grid g (x inside [g.front(), g.back()])
void locate(const std::vector<double>& g, double x, int* i, double* a) {
  int k = (int)(std::upper_bound(g.begin(), g.end(), x) - g.begin()) - 1;
  k = std::max(0, std::min(k, (int)g.size() - 2));
  *i = k;
  *a = (x - g[k]) / (g[k + 1] - g[k]);
}

bool inside(const std::vector<double>& g, double x) {
  const double tol = 1e-12 * std::max(1.0, std::fabs(x));
  return x >= g.front() - tol && x <= g.back() + tol;
}

}  // namespace

extern "C" {

int fbf_lut_build(fbf_lut_t* out, int R, const double* sigmas, int n_sigma, const double* eps, int n_eps) try {
  if (!out) return fbf::set_error(FBF_EINVAL, "fbf_lut_build: out is NULL");
  *out = nullptr;
  if (!sigmas || !eps) return fbf::set_error(FBF_EINVAL, "fbf_lut_build: NULL grid");
  if (R < 1 || R > (1 << 16)) return fbf::set_error(FBF_EINVAL, "fbf_lut_build: R out of range");
  if (n_sigma < 2 || n_eps < 2 || n_sigma > 4096 || n_eps > 4096)
    return fbf::set_error(FBF_EINVAL, "fbf_lut_build: grid sizes must be in [2, 4096]");
  std::vector<double> s(sigmas, sigmas + n_sigma), u(n_eps);
  for (int j = 0; j < n_eps; ++j) {
    if (!(eps[j] > 0) || !(eps[j] < 1)) return fbf::set_error(FBF_EINVAL, "fbf_lut_build: eps must be in (0, 1)");
    u[j] = std::log(1.0 / eps[j]);
  }
  for (double v : s)
    if (!(v > 0)) return fbf::set_error(FBF_EINVAL, "fbf_lut_build: sigma must be > 0");
  int rc = check_grid(s, "sigmas");
  if (rc != FBF_OK) return rc;
  rc = check_grid(u, "eps (decreasing)");
  if (rc != FBF_OK) return rc;
  fbf_lut_s* L = new (std::nothrow) fbf_lut_s();
  if (!L) return fbf::set_error(FBF_ENOMEM, "fbf_lut_build: out of host memory");
  L->R = R;
  L->sigma = s;
  L->u = u;
  L->K.resize((size_t)n_sigma * n_eps);
  L->T.resize((size_t)n_sigma * n_eps);
  std::vector<double> b(2 * R + 1);
  for (int i = 0; i < n_sigma; ++i) {
    for (int t = -R; t <= R; ++t) b[t + R] = std::exp(-(double)t * t / (2.0 * s[i] * s[i]));
    for (int j = 0; j < n_eps; ++j) {
      fbf::FitResult fr;
      std::string msg;
      rc = fbf::fit_range_kernel(b.data(), R, 0, eps[j], 0, &fr, &msg);
      if (rc != FBF_OK) { delete L; return fbf::set_error(rc, "fbf_lut_build: " + msg); }
      L->K[(size_t)i * n_eps + j] = fr.K;
      L->T[(size_t)i * n_eps + j] = fr.T;
    }
  }
  *out = L;
  fbf::clear_error();
  return FBF_OK;
} FBF_ABI_CATCH("fbf_lut_build")

int fbf_lut_entry(fbf_lut_t lut, int i_sigma, int j_eps, int* K, int* T) try {
  if (!lut || !K || !T) return fbf::set_error(FBF_EINVAL, "fbf_lut_entry: NULL argument");
  const int ns = (int)lut->sigma.size(), nu = (int)lut->u.size();
  if (i_sigma < 0 || i_sigma >= ns || j_eps < 0 || j_eps >= nu)
    return fbf::set_error(FBF_EINVAL, "fbf_lut_entry: index out of range");
  *K = lut->K[(size_t)i_sigma * nu + j_eps];
  *T = lut->T[(size_t)i_sigma * nu + j_eps];
  return FBF_OK;
} FBF_ABI_CATCH("fbf_lut_entry")

int fbf_lut_lookup(fbf_lut_t lut, double sigma, double eps, int* K, int* T) try {
  if (!lut || !K || !T) return fbf::set_error(FBF_EINVAL, "fbf_lut_lookup: NULL argument");
  if (!(sigma > 0) || !(eps > 0) || !(eps < 1)) return fbf::set_error(FBF_EINVAL, "fbf_lut_lookup: sigma > 0, 0 < eps < 1");
  const double u = std::log(1.0 / eps);
  if (!inside(lut->sigma, sigma) || !inside(lut->u, u))
    return fbf::set_error(FBF_EUNSUPPORTED, "fbf_lut_lookup: (sigma, eps) outside the table");
  int i, j;
  double a, c;
  locate(lut->sigma, sigma, &i, &a);
  locate(lut->u, u, &j, &c);
  a = std::min(1.0, std::max(0.0, a));
  c = std::min(1.0, std::max(0.0, c));
  const int nu = (int)lut->u.size();
  auto at = [&](const std::vector<int>& v, int ii, int jj) { return (double)v[(size_t)ii * nu + jj]; };
  auto bil = [&](const std::vector<int>& v) {
    return (1 - a) * (1 - c) * at(v, i, j) + a * (1 - c) * at(v, i + 1, j) + (1 - a) * c * at(v, i, j + 1) +
           a * c * at(v, i + 1, j + 1);
  };
  // reading: the interpolated values are rounded to the nearest integer
  *K = std::max(1, (int)std::lround(bil(lut->K)));
  *T = std::max(1, (int)std::lround(bil(lut->T)));
  return FBF_OK;
} FBF_ABI_CATCH("fbf_lut_lookup")

int fbf_plan_from_lut(fbf_plan_t* out, fbf_lut_t lut, double sigma, double eps, double theta, int precision) try {
  if (!out) return fbf::set_error(FBF_EINVAL, "fbf_plan_from_lut: out is NULL");
  *out = nullptr;
  int K = 0, T = 0;
  int rc = fbf_lut_lookup(lut, sigma, eps, &K, &T);
  if (rc != FBF_OK) return rc;
  const int R = lut->R;
  std::vector<double> b(2 * R + 1);
  for (int t = -R; t <= R; ++t) b[t + R] = std::exp(-(double)t * t / (2.0 * sigma * sigma));
  return fbf::build_plan(out, b.data(), R, theta, K, 0.0, precision, 0, sigma, T);
} FBF_ABI_CATCH("fbf_plan_from_lut")

int fbf_lut_save(fbf_lut_t lut, const char* path) try {
  if (!lut || !path) return fbf::set_error(FBF_EINVAL, "fbf_lut_save: NULL argument");
  FILE* f = std::fopen(path, "w");
  if (!f) return fbf::set_error(FBF_EINVAL, std::string("fbf_lut_save: cannot open ") + path);
  const int ns = (int)lut->sigma.size(), nu = (int)lut->u.size();
  std::fprintf(f, "fbf-lut 1\n%d %d %d\n", lut->R, ns, nu);
  for (double v : lut->sigma) std::fprintf(f, "%.17g\n", v);
  for (double v : lut->u) std::fprintf(f, "%.17g\n", std::exp(-v));
  for (int i = 0; i < ns * nu; ++i) std::fprintf(f, "%d %d\n", lut->K[i], lut->T[i]);
  const bool ok = std::fclose(f) == 0;
  return ok ? FBF_OK : fbf::set_error(FBF_EINVAL, "fbf_lut_save: write failed");
} FBF_ABI_CATCH("fbf_lut_save")

int fbf_lut_load(fbf_lut_t* out, const char* path) try {
  if (!out || !path) return fbf::set_error(FBF_EINVAL, "fbf_lut_load: NULL argument");
  *out = nullptr;
  FILE* f = std::fopen(path, "r");
  if (!f) return fbf::set_error(FBF_EINVAL, std::string("fbf_lut_load: cannot open ") + path);
  int ver = 0, R = 0, ns = 0, nu = 0;
  // the same bounds as fbf_lut_build: the file is input, and R sizes the samples of a plan
  bool ok = std::fscanf(f, "fbf-lut %d %d %d %d", &ver, &R, &ns, &nu) == 4 && ver == 1 && R >= 1 &&
            R <= (1 << 16) && ns >= 2 && nu >= 2 && ns <= 4096 && nu <= 4096;
  fbf_lut_s* L = ok ? new (std::nothrow) fbf_lut_s() : nullptr;
  if (ok && !L) { std::fclose(f); return fbf::set_error(FBF_ENOMEM, "fbf_lut_load: out of host memory"); }
  if (ok) {
    L->R = R;
    L->sigma.resize(ns);
    L->u.resize(nu);
    L->K.resize((size_t)ns * nu);
    L->T.resize((size_t)ns * nu);
    for (int i = 0; ok && i < ns; ++i) ok = std::fscanf(f, "%lf", &L->sigma[i]) == 1 && L->sigma[i] > 0;
    for (int j = 0; ok && j < nu; ++j) {
      double e = 0;
      ok = std::fscanf(f, "%lf", &e) == 1 && e > 0 && e < 1;
      if (ok) L->u[j] = std::log(1.0 / e);
    }
    for (int i = 0; ok && i < ns * nu; ++i) ok = std::fscanf(f, "%d %d", &L->K[i], &L->T[i]) == 2 && L->K[i] >= 1 && L->T[i] >= 1;
  }
  std::fclose(f);
  if (!ok || check_grid(L->sigma, "sigmas") != FBF_OK || check_grid(L->u, "eps (decreasing)") != FBF_OK) {
    delete L;
    return fbf::set_error(FBF_EINVAL, "fbf_lut_load: malformed table file");
  }
  *out = L;
  fbf::clear_error();
  return FBF_OK;
} FBF_ABI_CATCH("fbf_lut_load")

int fbf_lut_destroy(fbf_lut_t lut) try {
  delete lut;
  return FBF_OK;
} FBF_ABI_CATCH("fbf_lut_destroy")

}  // extern "C"
