// Direct evaluation of the bilateral filter, eq. (1), with the Gaussian range kernel of
// eq. (2): for every pixel i, the sums over the (2r+1)^2 window of
// w = g(j_x) g(j_y) phi(f(i - j) - f(i)) times f(i - j) (numerator) and times 1
// (denominator), r = ceil(3 theta).  Pixels i - j outside the image are absent from both
// sums.  This is the accuracy reference of the method (the paper's PSNR in Section III is
// measured against it) and the "brute force" of its cost model, 2 (6 theta + 1)^2 operations
// per pixel (Section I).
//
// A CTA filters a 32 x 32 tile: the tile and its r-pixel halo are staged in shared memory
// once; each thread owns one column of four pixels (rows y, y + 8, y + 16, y + 24).  When
// every pixel of the tile and halo is an integer in [0, L] (L = min(R, 1023)), the range
// kernel is read from a table of phi over the integer differences -L..L, built per CTA with
// expf (1 ulp); other tiles evaluate expf per neighbour.  FP32 throughout.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "fbf_internal.h"

namespace fbf {
namespace brute {

constexpr int BX = 32, BY = 32;          // output tile
constexpr int NT = 256;                  // threads: 32 columns x 8 row groups
constexpr int PY = BY / 8;               // pixels per thread
constexpr int kMaxLut = 1023;            // table range of integer differences

struct Params {
  const float* in;
  float* out;
  long long pitch;
  int H, W;
  int lut_r;                             // L: integer tiles use the table when values <= L
  float inv2s2;                          // 1 / (2 sigma^2)
  float g[2 * FBF_MAX_RADIUS + 1];       // g(x) = exp(-x^2 / (2 theta^2)), x = -r..r
};

template <int RAD>
struct BCfg {
  static constexpr int SW = BX + 2 * RAD;           // halo tile width (floats)
  static constexpr int SH = BY + 2 * RAD;
  static constexpr size_t bytes(int lut_r) { return (size_t)(SW * SH + 2 * lut_r + 1) * sizeof(float); }
};

template <int RAD>
__global__ void __launch_bounds__(NT) fbf_brute_kernel(const __grid_constant__ Params p) {
  using C = BCfg<RAD>;
  extern __shared__ float sm[];
  float* sf = sm;                                   // f over tile + halo; NaN outside the image
  float* lut = sm + C::SW * C::SH;                  // phi(t), t = -L..L, at lut[t + L]
  const int tid = threadIdx.x;
  const int tx0 = blockIdx.x * BX, ty0 = blockIdx.y * BY;
  const int L = p.lut_r;
  const float nan = __int_as_float(0x7fc00000);
  int ok = 1;
  for (int i = tid; i < C::SW * C::SH; i += NT) {
    const int hy = i / C::SW, hx = i - hy * C::SW;
    const int gy = ty0 - RAD + hy, gx = tx0 - RAD + hx;
    float v = nan;
    if (gy >= 0 && gy < p.H && gx >= 0 && gx < p.W) {
      v = __ldg(p.in + (long long)gy * p.pitch + gx);
      ok &= (v == rintf(v)) & (v >= 0.f) & (v <= (float)L);
    }
    sf[i] = v;
  }
  for (int t = tid; t <= 2 * L; t += NT) {
    const float d = (float)(t - L);
    lut[t] = expf(-d * d * p.inv2s2);
  }
  const bool tile_int = __syncthreads_and(ok) != 0;
  const bool interior = tx0 - RAD >= 0 && ty0 - RAD >= 0 && tx0 + BX + RAD <= p.W && ty0 + BY + RAD <= p.H;

  const int x = tid & 31, y0 = tid >> 5;
  float fi[PY], num[PY], den[PY];
#pragma unroll
  for (int k = 0; k < PY; ++k) {
    fi[k] = sf[(y0 + 8 * k + RAD) * C::SW + x + RAD];
    if (fi[k] != fi[k]) fi[k] = 0.f;   // pixel outside the image (not stored): keeps table indices in range
    num[k] = 0.f;
    den[k] = 0.f;
  }
  // integer differences t = f(j) - f(i) read the table at lut[t + L]: adding 1.5 * 2^23 gives
  // an exactly representable float whose bit pattern is 0x4B400000 + t (|t| < 2^22)
  const float kMagic = 12582912.0f;
  const int kBias = 0x4B400000 - L;
  if (tile_int && interior) {
    for (int dy = -RAD; dy <= RAD; ++dy) {
      const float wy = p.g[dy + RAD];
      const float* row = sf + (y0 + RAD + dy) * C::SW + x + RAD;
#pragma unroll 4
      for (int dx = -RAD; dx <= RAD; ++dx) {
        const float w0 = wy * p.g[dx + RAD];
#pragma unroll
        for (int k = 0; k < PY; ++k) {
          const float fj = row[8 * k * C::SW + dx];
          const float w = w0 * lut[__float_as_int((fj - fi[k]) + kMagic) - kBias];
          num[k] = fmaf(w, fj, num[k]);
          den[k] += w;
        }
      }
    }
  } else {
    for (int dy = -RAD; dy <= RAD; ++dy) {
      const float wy = p.g[dy + RAD];
      const float* row = sf + (y0 + RAD + dy) * C::SW + x + RAD;
      for (int dx = -RAD; dx <= RAD; ++dx) {
        const float w0 = wy * p.g[dx + RAD];
#pragma unroll
        for (int k = 0; k < PY; ++k) {
          const float fj = row[8 * k * C::SW + dx];
          if (fj == fj) {                           // inside the image
            const float t = fj - fi[k];
            const float ph = tile_int ? lut[__float_as_int(t + kMagic) - kBias] : expf(-t * t * p.inv2s2);
            const float w = w0 * ph;
            num[k] = fmaf(w, fj, num[k]);
            den[k] += w;
          }
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < PY; ++k) {
    const int gy = ty0 + y0 + 8 * k, gx = tx0 + x;
    if (gy < p.H && gx < p.W) p.out[(long long)gy * p.pitch + gx] = num[k] / den[k];
  }
}

template <int RAD>
int launch(const Params& p, cudaStream_t st) {
  using C = BCfg<RAD>;
  const size_t smem = C::bytes(p.lut_r);
  cudaError_t e = cudaFuncSetAttribute(fbf_brute_kernel<RAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_brute_filter: ") + cudaGetErrorString(e));
  Params q = p;
  const dim3 grid((unsigned)(((long long)p.W + BX - 1) / BX), (unsigned)(((long long)p.H + BY - 1) / BY));
  fbf_brute_kernel<RAD><<<grid, NT, smem, st>>>(q);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_brute_filter: launch: ") + cudaGetErrorString(e));
  return FBF_OK;
}

}  // namespace brute
}  // namespace fbf

extern "C" int fbf_brute_filter(const float* d_in, float* d_out, int H, int W, size_t pitch_elems,
                                double theta, double sigma, int R, void* cuda_stream) try {
  using namespace fbf;
  if (!d_in || !d_out) return set_error(FBF_EINVAL, "fbf_brute_filter: NULL image pointer");
  if (H < 1 || W < 1) return set_error(FBF_EINVAL, "fbf_brute_filter: H and W must be >= 1");
  if (pitch_elems < (size_t)W) return set_error(FBF_EINVAL, "fbf_brute_filter: pitch < W");
  if (!(theta > 0.0) || !(sigma > 0.0) || !std::isfinite(theta) || !std::isfinite(sigma))
    return set_error(FBF_EINVAL, "fbf_brute_filter: theta and sigma must be positive and finite");
  if (R < 1) return set_error(FBF_EINVAL, "fbf_brute_filter: R must be >= 1");
  // one launch covers the image with a 2-D grid of 32 x 32 tiles; grid y is at most 65535
  if (((long long)H + brute::BY - 1) / brute::BY > 65535)
    return set_error(FBF_EUNSUPPORTED, "fbf_brute_filter: H above " + std::to_string(65535LL * brute::BY) +
                                           " rows");
  const size_t span = ((size_t)(H - 1) * pitch_elems + (size_t)W) * sizeof(float);
  const char* a = (const char*)d_in;
  const char* o = (const char*)d_out;
  if (a < o + span && o < a + span) return set_error(FBF_EINVAL, "fbf_brute_filter: in and out overlap");
  const int r = (int)std::ceil(3.0 * theta - 1e-12);
  if (r > FBF_MAX_RADIUS) return set_error(FBF_EUNSUPPORTED, "fbf_brute_filter: r = ceil(3 theta) above FBF_MAX_RADIUS");
  brute::Params p{};
  p.in = d_in;
  p.out = d_out;
  p.pitch = (long long)pitch_elems;
  p.H = H;
  p.W = W;
  p.lut_r = R < brute::kMaxLut ? R : brute::kMaxLut;
  p.inv2s2 = (float)(1.0 / (2.0 * sigma * sigma));
  const int RADK = r <= 6 ? 6 : r <= 15 ? 15 : r <= 30 ? 30 : 48;
  for (int i = 0; i <= 2 * RADK; ++i) {   // the window's taps, zero beyond r
    const int x = i - RADK;
    p.g[i] = (x >= -r && x <= r) ? (float)std::exp(-(double)x * x / (2.0 * theta * theta)) : 0.f;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  switch (RADK) {
    case 6: return brute::launch<6>(p, st);
    case 15: return brute::launch<15>(p, st);
    case 30: return brute::launch<30>(p, st);
    default: return brute::launch<48>(p, st);
  }
} FBF_ABI_CATCH("fbf_brute_filter")
