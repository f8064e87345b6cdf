// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <exception>
#include <new>
#include <string>
#include <vector>

#include "fbf.h"

#include <nvtx3/nvToolsExt.h>

struct CUstream_st;
using cudaStream_t_ = CUstream_st*;

namespace fbf {

// ---- host fitter (fbf_fit.cpp) --------------------------------------------------------
struct FitResult {
  int K = 0;                 // number of cosine terms
  int T = 0;                 // period parameter: phi_hat has period 2T+1 (eq. 3)
  std::vector<double> c;     // c_0..c_{K-1}
  double E = 0.0;            // E(K,T) of eq. (5), including the odd part of b
  double delta_max = 0.0;    // max over {-R..R} of |phi_hat - phi|
};

// b has 2R+1 samples phi(-R..R).  K >= 1: fixed order (T optimised unless T_fixed > 0).
// K == 0: Algorithm 1 with tolerance eps.  Returns FBF_OK or an error code; msg is set on
// error.
int fit_range_kernel(const double* b, int R, int K, double eps, int T_fixed,
                     FitResult* out, std::string* msg);

// Plan from kernel samples (fbf_capi.cpp); T_given > 0 fixes the period parameter.
int build_plan(struct fbf_plan_s** out, const double* b, int R, double theta, int K, double eps,
               int precision, int flags, double sigma, int T_given);

// E(K,T) for K = 1..Kc at one T (folded Householder QR); used by tests via the C ABI.
void kernel_error_curve(const double* b, int R, int T, int Kc, double* E_out);

// ---- device parameters ----------------------------------------------------------------
// Everything a filter kernel needs, passed by value at launch (constant bank), so plans
// own no device memory.
// Unit-circle tables: e(n) = exp(i 2 pi n / P) for integer n = 128 a + b is the product
// ta[a] * tb[b] of two tables rounded from double on the host (error ~2 ulp).
constexpr int kTrigLo = 128;                                        // tb entries
constexpr int kTrigHi = (FBF_MAX_PERIOD + kTrigLo - 1) / kTrigLo;  // ta entries

struct DeviceParams {
  int K;                        // cosine terms
  int P;                        // period 2T+1
  int r;                        // spatial radius
  int R;                        // intensity range [0, R]
  float nu;                     // 2 pi / P
  float invP;                   // 1 / P
  float center;                 // m: f-channels carry (f - m); m is added back at the end
  float pad_;
  float c[FBF_MAX_K];           // c_k (eq. 3)
  float g[2 * FBF_MAX_RADIUS + 1];  // g[d] = exp(-(d-r)^2/(2 theta^2)) / sum, d = 0..2r
  float ta[2 * kTrigHi];        // (cos, sin)(2 pi 128 a / P), a = 0..P/128
  float tb[2 * kTrigLo];        // (cos, sin)(2 pi b / P),     b = 0..127
};

struct Plan {
  double sigma = 0, theta = 0;
  int R = 0, r = 0, precision = 0, flags = 0;
  FitResult fit;
  DeviceParams dp{};
};

// the Plan behind a C handle (defined with the handle type in fbf_capi.cpp)
const Plan* plan_of(fbf_plan_t h);

// ---- tracing ----------------------------------------------------------------------------
// An NVTX range over a host-side stage (plan, launch, serving admission and completion), so
// that a timeline of a process using the library shows where the host time goes.  Without
// a tool attached, a push/pop costs a call to an empty function.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---- errors ---------------------------------------------------------------------------
int set_error(int code, const std::string& msg);

// Closes each entry point of the ABI, written as a function-try-block: a C++ exception from
// the host side (an allocation, a thread that cannot start) becomes FBF_ENOMEM with a
// message, so that no exception crosses the C ABI.
#define FBF_ABI_CATCH(fn)                                                                 \
  catch (const std::bad_alloc&) {                                                         \
    return fbf::set_error(FBF_ENOMEM, fn ": out of host memory");                         \
  }                                                                                       \
  catch (const std::exception& ex) {                                                      \
    return fbf::set_error(FBF_ENOMEM, std::string(fn ": host resources: ") + ex.what());  \
  }
void clear_error();

// ---- kernels --------------------------------------------------------------------------
// FP32 fused kernel launcher (fbf_fp32.cu).
// row0 / rows (rows = 0: all): filter only output rows [row0, row0 + rows) of the H x W
// image (a band; row0 a multiple of the configuration's tile height), reading halo rows
// from the whole image.
int launch_fp32(const DeviceParams& dp, const float* in, float* out, int H, int W,
                size_t pitch, void* stream, int row0 = 0, int rows = 0);
// tile height of the FP32 configuration serving radius r on a launch of `rows` rows of width W
int fp32_tile_rows(int r, int W, int rows);
// Per-(device, stream) scratch: `counters` zeroed ints (left at zero by every launch) and
// `partial_bytes` of partial sums; grown with cudaMalloc when too small.
int get_workspace(int dev, cudaStream_t_ st, size_t partial_bytes, size_t counters,
                  float** partial, int** counter);
// Tensor-core forms (fbf_tc.cu): precision FBF_FP16_TC or FBF_BF16_TC.
int launch_tc(const DeviceParams& dp, const float* in, float* out, int H, int W, size_t pitch,
              void* stream, int precision, int row0 = 0, int rows = 0);
// Device error word of the tensor-core kernels (bit 0: a bounded wait gave up).
int device_errors(int* flags, int clear);
// FP32 single-image kernels' error word (bit 1: a TMA wait gave up), and the reset of the
// cached split-tile counters that a launch which gave up part way leaves nonzero.
int fp32_device_errors(int* flags, int clear);
// Test hook: poll limit of the kernels' pipeline waits (0 = normal limits), per kernel family.
int fp32_set_wait_polls(int polls);
int tc_set_wait_polls(int polls);
int reset_workspace_counters();

// batched tensor-core launch of one radius class (6, 15 or 30) from a device work-list
namespace fp32 { struct Work; }
int launch_tc_batch(int rad, int precision, const DeviceParams* dparams, const fp32::Work* dwork, int n,
                    long long wtot, float* partial, int* counter, void* stream, int dev);
int tc_batch_partial_bytes(int dev, size_t* out);
int tc_tile_rows(int rad, int precision);   // output tile height of a tensor-core configuration
// Same kernel, scratch from a fixed device array instead of the per-stream workspace.
int launch_fp32_noalloc(const DeviceParams& dp, const float* in, float* out, int H, int W,
                        size_t pitch, void* stream);

}  // namespace fbf
