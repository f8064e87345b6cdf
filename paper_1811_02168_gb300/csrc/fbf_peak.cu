// FP32 multiply-add throughput probe: the measured denominator of the FP32 form's
// roofline.  The fused filter is bound by the FP32 FMA pipe (Section II's convolutions are
// 2r+1 multiply-adds per pixel, pass and convolved image), so its fraction of peak is taken
// against the rate this probe reaches on the same GPU: every thread runs 16 independent
// multiply-add chains (packed fma.rn.f32x2 pairs, or scalar fmaf) with values that settle
// at a fixed point (no overflow, no denormals).  Not part of the method.
#include <cuda_runtime.h>

#include <string>

#include "fbf_internal.h"

namespace fbf {
namespace {

constexpr int kChains = 16;

template <bool PAIRS>
__global__ void __launch_bounds__(256) fp32_fma_probe(float2 a, float2 b, long long iters, float* out) {
  float2 acc[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) acc[j] = make_float2(1e-3f * (float)threadIdx.x + (float)j, 0.5f * (float)j);
#pragma unroll 4
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
      if constexpr (PAIRS) {
        acc[j] = __ffma2_rn(a, acc[j], b);
      } else {
        acc[j].x = fmaf(a.x, acc[j].x, b.x);
        acc[j].y = fmaf(a.y, acc[j].y, b.y);
      }
    }
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += acc[j].x + acc[j].y;
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace fbf

extern "C" int fbf_debug_fp32_peak(int pairs, int blocks, int threads, long long iters, float* d_out,
                                   void* cuda_stream, double* flop) try {
  fbf::clear_error();
  if (blocks < 1 || threads < 32 || threads > 256 || threads % 32 != 0 || iters < 1 || !d_out || !flop)
    return fbf::set_error(FBF_EINVAL, "fbf_debug_fp32_peak: bad arguments");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  const float2 a = make_float2(0.9999f, 0.9999f), b = make_float2(1e-4f, 1e-4f);
  if (pairs)
    fbf::fp32_fma_probe<true><<<blocks, threads, 0, st>>>(a, b, iters, d_out);
  else
    fbf::fp32_fma_probe<false><<<blocks, threads, 0, st>>>(a, b, iters, d_out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fbf::set_error(FBF_ECUDA, std::string("fbf_debug_fp32_peak: launch: ") + cudaGetErrorString(e));
  // 16 chains x 2 lanes x 2 flop per multiply-add
  *flop = (double)blocks * threads * (double)iters * fbf::kChains * 4.0;
  return FBF_OK;
}
FBF_ABI_CATCH("fbf_debug_fp32_peak")
