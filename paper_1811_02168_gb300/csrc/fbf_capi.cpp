// C ABI: plans, parameter read-back, errors (host only; the launches live in the .cu files).
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "fbf_internal.h"

namespace fbf {

static thread_local std::string g_last_error;

int set_error(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}
void clear_error() { g_last_error.clear(); }

}  // namespace fbf

using fbf::Plan;

struct fbf_plan_s {
  Plan p;
};

namespace fbf {
const Plan* plan_of(fbf_plan_t h) { return &h->p; }
}  // namespace fbf

namespace {

int radius_of(double theta) { return (int)std::ceil(3.0 * theta - 1e-12); }

bool precision_known(int precision) {
  return precision == FBF_FP32 || precision == FBF_FP16_TC || precision == FBF_BF16_TC || precision == FBF_FAST;
}

}  // namespace

namespace fbf {

// A plan from kernel samples b(-R..R).  T_given > 0 fixes the period parameter (with K >= 1:
// only the least squares of eq. (5) for c runs, as with a lookup table); otherwise T follows
// FBF_FLAG_FIXED_PERIOD (T = R) or the optimisation of eq. (6) / Algorithm 1.
int build_plan(fbf_plan_t* out, const double* b, int R, double theta, int K, double eps,
               int precision, int flags, double sigma, int T_given) {
  if (!out) return fbf::set_error(FBF_EINVAL, "fbf_plan: out is NULL");
  *out = nullptr;
  if (R < 1) return fbf::set_error(FBF_EINVAL, "fbf_plan: R must be >= 1");
  if (!(theta > 0) || !std::isfinite(theta)) return fbf::set_error(FBF_EINVAL, "fbf_plan: theta must be > 0");
  if (K < 0) return fbf::set_error(FBF_EINVAL, "fbf_plan: K must be >= 0");
  if (K == 0 && !(eps > 0)) return fbf::set_error(FBF_EINVAL, "fbf_plan: K == 0 needs eps > 0");
  if (!precision_known(precision)) return fbf::set_error(FBF_EINVAL, "fbf_plan: unknown precision form");
  if (flags & ~FBF_FLAG_FIXED_PERIOD) return fbf::set_error(FBF_EINVAL, "fbf_plan: unknown flag");
  if (!(b[R] > 0)) return fbf::set_error(FBF_EINVAL, "fbf_plan: phi(0) must be > 0");
  const int r = radius_of(theta);
  if (r > FBF_MAX_RADIUS)
    return fbf::set_error(FBF_EUNSUPPORTED, "fbf_plan: radius ceil(3 theta) exceeds FBF_MAX_RADIUS");
  // FBF_FAST: the faster form at this radius (FP32 for short windows and beyond the
  // tensor-core limit, the compensated BF16 tensor-core form between)
  if (precision == FBF_FAST)
    precision = (r <= FBF_FAST_FP32_MAX_RADIUS || r > FBF_MAX_RADIUS_TC) ? FBF_FP32 : FBF_BF16_TC;
  if (precision != FBF_FP32 && r > FBF_MAX_RADIUS_TC)
    return fbf::set_error(FBF_EUNSUPPORTED, "fbf_plan: the tensor-core forms support r <= FBF_MAX_RADIUS_TC");
  if (K > FBF_MAX_K) return fbf::set_error(FBF_EUNSUPPORTED, "fbf_plan: K exceeds FBF_MAX_K");

  std::unique_ptr<fbf_plan_s> h(new (std::nothrow) fbf_plan_s());
  if (!h) return fbf::set_error(FBF_ENOMEM, "fbf_plan: out of host memory");
  Plan& p = h->p;
  p.sigma = sigma;
  p.theta = theta;
  p.R = R;
  p.r = r;
  p.precision = precision;
  p.flags = flags;
  std::string msg;
  int T_fixed = (flags & FBF_FLAG_FIXED_PERIOD) ? R : (T_given > 0 ? T_given : 0);
  int rc = fbf::fit_range_kernel(b, R, K, eps, T_fixed, &p.fit, &msg);
  if (rc != FBF_OK) return fbf::set_error(rc, "fbf_plan: " + msg);
  if (p.fit.K > FBF_MAX_K) return fbf::set_error(FBF_EUNSUPPORTED, "fbf_plan: fitted K exceeds FBF_MAX_K");
  if (2L * p.fit.T + 1 > FBF_MAX_PERIOD) return fbf::set_error(FBF_EUNSUPPORTED, "fbf_plan: period exceeds FBF_MAX_PERIOD");

  // device constants
  fbf::DeviceParams& d = p.dp;
  std::memset(&d, 0, sizeof(d));
  d.K = p.fit.K;
  d.P = 2 * p.fit.T + 1;
  d.r = r;
  d.nu = (float)(2.0 * M_PI / (double)d.P);
  d.invP = (float)(1.0 / (double)d.P);
  d.center = (float)(0.5 * (double)R);
  d.R = R;
  for (int a = 0; a * fbf::kTrigLo < d.P && a < fbf::kTrigHi; ++a) {
    const double ang = 2.0 * M_PI * (double)(a * fbf::kTrigLo) / (double)d.P;
    d.ta[2 * a] = (float)std::cos(ang);
    d.ta[2 * a + 1] = (float)std::sin(ang);
  }
  for (int b = 0; b < fbf::kTrigLo; ++b) {
    const double ang = 2.0 * M_PI * (double)b / (double)d.P;
    d.tb[2 * b] = (float)std::cos(ang);
    d.tb[2 * b + 1] = (float)std::sin(ang);
  }
  for (int k = 0; k < d.K; ++k) d.c[k] = (float)p.fit.c[k];
  double gs = 0;
  for (int i = -r; i <= r; ++i) gs += std::exp(-(double)i * i / (2.0 * theta * theta));
  for (int i = -r; i <= r; ++i) d.g[i + r] = (float)(std::exp(-(double)i * i / (2.0 * theta * theta)) / gs);
  *out = h.release();
  fbf::clear_error();
  return FBF_OK;
}

}  // namespace fbf

using fbf::build_plan;

extern "C" {

int fbf_plan(fbf_plan_t* out, double sigma, int R, double theta, int K, double eps,
             int precision, int flags) try {
  const fbf::NvtxRange tr("fbf_plan");
  if (!(sigma > 0) || !std::isfinite(sigma)) {
    if (out) *out = nullptr;
    return fbf::set_error(FBF_EINVAL, "fbf_plan: sigma must be > 0");
  }
  if (R < 1 || R > (1 << 20)) {
    if (out) *out = nullptr;
    return fbf::set_error(FBF_EINVAL, "fbf_plan: R out of range");
  }
  std::vector<double> b(2 * (size_t)R + 1);
  for (int t = -R; t <= R; ++t) b[t + R] = std::exp(-(double)t * t / (2.0 * sigma * sigma));
  return build_plan(out, b.data(), R, theta, K, eps, precision, flags, sigma, 0);
} FBF_ABI_CATCH("fbf_plan")

int fbf_plan_from_samples(fbf_plan_t* out, const double* b, int R, double theta, int K,
                          double eps, int precision, int flags) try {
  if (!b) {
    if (out) *out = nullptr;
    return fbf::set_error(FBF_EINVAL, "fbf_plan_from_samples: b is NULL");
  }
  if (R < 1 || R > (1 << 20)) {
    if (out) *out = nullptr;
    return fbf::set_error(FBF_EINVAL, "fbf_plan_from_samples: R out of range");
  }
  return build_plan(out, b, R, theta, K, eps, precision, flags, NAN, 0);
} FBF_ABI_CATCH("fbf_plan_from_samples")

int fbf_plan_info(fbf_plan_t plan, int* K, int* T, double* c, double* E, double* delta_max) try {
  if (!plan) return fbf::set_error(FBF_EINVAL, "fbf_plan_info: plan is NULL");
  const fbf::FitResult& f = plan->p.fit;
  if (K) *K = f.K;
  if (T) *T = f.T;
  if (c) for (int k = 0; k < f.K; ++k) c[k] = f.c[k];
  if (E) *E = f.E;
  if (delta_max) *delta_max = f.delta_max;
  return FBF_OK;
} FBF_ABI_CATCH("fbf_plan_info")

int fbf_plan_radius(fbf_plan_t plan, int* r) try {
  if (!plan || !r) return fbf::set_error(FBF_EINVAL, "fbf_plan_radius: NULL argument");
  *r = plan->p.r;
  return FBF_OK;
} FBF_ABI_CATCH("fbf_plan_radius")

int fbf_plan_destroy(fbf_plan_t plan) try {
  delete plan;
  return FBF_OK;
} FBF_ABI_CATCH("fbf_plan_destroy")

int fbf_filter(fbf_plan_t plan, const float* d_in, float* d_out, int H, int W,
               size_t pitch_elems, void* cuda_stream) try {
  const fbf::NvtxRange tr("fbf_filter");
  if (!plan) return fbf::set_error(FBF_EINVAL, "fbf_filter: plan is NULL");
  if (!d_in || !d_out) return fbf::set_error(FBF_EINVAL, "fbf_filter: NULL image pointer");
  if (H < 1 || W < 1) return fbf::set_error(FBF_EINVAL, "fbf_filter: H and W must be >= 1");
  if (pitch_elems < (size_t)W) return fbf::set_error(FBF_EINVAL, "fbf_filter: pitch < W");
  const size_t span = ((size_t)(H - 1) * pitch_elems + (size_t)W) * sizeof(float);
  const char* a = (const char*)d_in;
  const char* o = (const char*)d_out;
  if (a < o + span && o < a + span) return fbf::set_error(FBF_EINVAL, "fbf_filter: in and out overlap");
  switch (plan->p.precision) {
    case FBF_FP32:
      return fbf::launch_fp32(plan->p.dp, d_in, d_out, H, W, pitch_elems, cuda_stream);
    case FBF_FP16_TC:
    case FBF_BF16_TC:
      return fbf::launch_tc(plan->p.dp, d_in, d_out, H, W, pitch_elems, cuda_stream, plan->p.precision);
    default:
      return fbf::set_error(FBF_EINVAL, "fbf_filter: unknown precision form");
  }
} FBF_ABI_CATCH("fbf_filter")

int fbf_filter_noalloc(fbf_plan_t plan, const float* d_in, float* d_out, int H, int W,
                       size_t pitch_elems, void* cuda_stream) try {
  if (!plan) return fbf::set_error(FBF_EINVAL, "fbf_filter_noalloc: plan is NULL");
  if (!d_in || !d_out) return fbf::set_error(FBF_EINVAL, "fbf_filter_noalloc: NULL image pointer");
  if (H < 1 || W < 1) return fbf::set_error(FBF_EINVAL, "fbf_filter_noalloc: H and W must be >= 1");
  if (pitch_elems < (size_t)W) return fbf::set_error(FBF_EINVAL, "fbf_filter_noalloc: pitch < W");
  const size_t span = ((size_t)(H - 1) * pitch_elems + (size_t)W) * sizeof(float);
  const char* a = (const char*)d_in;
  const char* o = (const char*)d_out;
  if (a < o + span && o < a + span) return fbf::set_error(FBF_EINVAL, "fbf_filter_noalloc: in and out overlap");
  if (plan->p.precision != FBF_FP32)
    return fbf::set_error(FBF_EUNSUPPORTED, "fbf_filter_noalloc: only the FBF_FP32 form");
  return fbf::launch_fp32_noalloc(plan->p.dp, d_in, d_out, H, W, pitch_elems, cuda_stream);
} FBF_ABI_CATCH("fbf_filter_noalloc")

const char* fbf_last_error(void) { return fbf::g_last_error.c_str(); }

const char* fbf_version(void) { return "fbf-gb300 0.1"; }

int fbf_device_errors(int* flags, int clear) try {
  if (!flags) return fbf::set_error(FBF_EINVAL, "fbf_device_errors: flags is NULL");
  return fbf::device_errors(flags, clear);
} FBF_ABI_CATCH("fbf_device_errors")

// Test hook: E(K,T) for K = 1..Kc at one T from the C++ fitter (host only).
int fbf_debug_set_wait_limit(int polls) try {
  fbf::clear_error();
  if (polls < 0) return fbf::set_error(FBF_EINVAL, "fbf_debug_set_wait_limit: polls must be >= 0");
  int rc = fbf::fp32_set_wait_polls(polls);
  if (rc == FBF_OK) rc = fbf::tc_set_wait_polls(polls);
  return rc;
} FBF_ABI_CATCH("fbf_debug_set_wait_limit")

int fbf_debug_error_curve(const double* b, int R, int T, int Kc, double* E_out) try {
  if (!b || !E_out || R < 1 || T < 1 || Kc < 1) return fbf::set_error(FBF_EINVAL, "bad argument");
  fbf::kernel_error_curve(b, R, T, Kc, E_out);
  return FBF_OK;
} FBF_ABI_CATCH("fbf_debug_error_curve")

}  // extern "C"
