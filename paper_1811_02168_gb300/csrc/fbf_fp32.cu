// FP32 fused Fourier bilateral filter on the CUDA cores (precision form FBF_FP32).
//
// One CTA owns an output tile of TX x TY pixels.  For each cosine term k it
//   1. generates, band by band, the images of the term over the tile plus an r-pixel
//      halo: cos(k nu f), sin(k nu f), (f-m) cos(k nu f), (f-m) sin(k nu f) for k >= 1 and
//      (f-m) for k = 0 (Section II: with phi_hat of eq. (3) the sums of eq. (1) become
//      convolutions of these images), zero outside the image;
//   2. convolves each band along x with the 2r+1 Gaussian taps (register-blocked, 8
//      outputs per thread, taps read from the constant bank) into a shared buffer that
//      covers TY + 2r rows;
//   3. convolves that buffer along y for the thread's own pixels and folds the result
//      straight into the per-pixel numerator and denominator:
//        den += c_k [cos(k nu f_i) B(cos) + sin(k nu f_i) B(sin)]
//        num += c_k [cos(k nu f_i) B((f-m)cos) + sin(k nu f_i) B((f-m)sin)]
//      with the k = 0 terms c_0 B(f-m) and c_0 B(1), B(1) from 1-D partial tap sums.
// At the end f_BF = m + num/den (num carries f - m, which leaves eq. (1) unchanged since
// its weights are normalised).  Only f is read from and only f_BF is written to HBM.
// The whole stack (4K-3 images) lives only in shared memory, one term at a time.
#include <cuda_runtime.h>

#include <cstdio>
#include <string>

#include "fbf_internal.h"

namespace fbf {
namespace {

constexpr int TX = 32;   // tile width (fixed: sets the shared-memory bank layout)
constexpr int NXH = 8;   // x outputs per thread in the horizontal pass
constexpr int NY = 8;    // y outputs per thread in the vertical pass

template <int RAD, int TY, int NT>
struct Cfg {
  static constexpr int HROWS = TY + 2 * RAD;                 // rows of the x-pass output
  static constexpr int SR = NT / (4 * (TX / NXH));           // rows per band: 4 ch * SR * (TX/8) == NT
  static constexpr int NQ4 = (NXH + 2 * RAD + 3) / 4;        // float4 loads per x-pass item
  static constexpr int SW0 = TX - NXH + 4 * NQ4;
  static constexpr int SW = (SW0 % 8 == 0) ? SW0 + 4 : SW0;   // stage row stride (== 4 mod 8)
  static constexpr int TXH = TX + 2 * RAD;                   // generated columns
  static constexpr int HS = TX + 4;                          // x-pass buffer row stride
  static constexpr int NXV = TX * TY / (NT * NY);            // x columns per thread (y pass)
  static constexpr int VCOLS = TX / NXV;                     // threads across a row (y pass)
  static constexpr int STAGE_FLOATS = 4 * SR * SW;
  static constexpr int HBUF_FLOATS = 4 * HROWS * HS;
  static constexpr int SMEM_BYTES = (STAGE_FLOATS + HBUF_FLOATS + TX + TY) * 4;
  static_assert(4 * SR * (TX / NXH) == NT, "x-pass mapping");
  static_assert(NXV >= 1 && NXV * NY * NT == TX * TY, "y-pass mapping");
  static_assert(NXV == 1 || NXV == 2, "y-pass vector width");
};

// phase reduction: n = (k*v) mod P mapped to (-P/2, P/2], then (sin, cos)(n * nu).
__device__ __forceinline__ void term_sincos(float kf, float v, const DeviceParams& p,
                                            float* s, float* c) {
  const float Pf = (float)p.P;
  float x = kf * v;
  float q = floorf(x * p.invP);
  float n = fmaf(-q, Pf, x);
  n = (n < 0.f) ? n + Pf : n;
  n = (n >= Pf) ? n - Pf : n;
  n = (n > 0.5f * Pf) ? n - Pf : n;
  __sincosf(n * p.nu, s, c);
}

template <int RAD, int TY, int NT>
__global__ void __launch_bounds__(NT, (NT <= 256) ? 2 : 1)
fbf_fp32_kernel(const __grid_constant__ DeviceParams p, const float* __restrict__ in,
                float* __restrict__ out, int H, int W, long pitch) {
  using C = Cfg<RAD, TY, NT>;
  extern __shared__ float4 smem_f4[];
  float* stage = reinterpret_cast<float*>(smem_f4);
  float* hbuf = stage + C::STAGE_FLOATS;
  float* sx = hbuf + C::HBUF_FLOATS;
  float* sy = sx + TX;

  const int tid = threadIdx.x;
  const int tx0 = blockIdx.x * TX;
  const int ty0 = blockIdx.y * TY;
  const float m = p.center;

  // B(1) = sx(x) * sy(y): the blur of the constant image under zero padding.
  for (int i = tid; i < TX + TY; i += NT) {
    const bool isx = i < TX;
    const int base = isx ? tx0 + i : ty0 + (i - TX);
    const int lim = isx ? W : H;
    float s = 0.f;
#pragma unroll
    for (int d = 0; d <= 2 * RAD; ++d) {
      int q = base - RAD + d;
      s += (q >= 0 && q < lim) ? p.g[d] : 0.f;
    }
    (isx ? sx : sy - TX)[i] = s;
  }

  // own pixels for the y pass and the recombination
  const int vcol = tid % C::VCOLS;
  const int vrow = tid / C::VCOLS;
  const int ox = vcol * C::NXV;   // within tile
  const int oy = vrow * NY;
  float fo[NY][C::NXV], num[NY][C::NXV], den[NY][C::NXV];
#pragma unroll
  for (int u = 0; u < NY; ++u)
#pragma unroll
    for (int c = 0; c < C::NXV; ++c) {
      int gy = ty0 + oy + u, gx = tx0 + ox + c;
      fo[u][c] = (gy < H && gx < W) ? __ldg(in + (long)gy * pitch + gx) : 0.f;
      num[u][c] = 0.f;
      den[u][c] = 0.f;
    }

  // x-pass item of this thread
  const int hx = tid % (TX / NXH);
  const int hrow = (tid / (TX / NXH)) % C::SR;
  const int hch = tid / (C::SR * (TX / NXH));

  for (int k = 0; k < p.K; ++k) {
    const float kf = (float)k;
    const int nch = (k == 0) ? 1 : 4;
    // ---- steps 1+2: generate + x-convolve, band by band --------------------------
    for (int b0 = 0; b0 < C::HROWS; b0 += C::SR) {
      for (int idx = tid; idx < C::SR * C::TXH; idx += NT) {
        const int row = idx / C::TXH;
        const int xx = idx - row * C::TXH;
        const int gy = ty0 - RAD + b0 + row;
        const int gx = tx0 - RAD + xx;
        float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
        if (b0 + row < C::HROWS && gy >= 0 && gy < H && gx >= 0 && gx < W) {
          const float v = __ldg(in + (long)gy * pitch + gx);
          if (k == 0) {
            c0 = v - m;
          } else {
            float s, c;
            term_sincos(kf, v, p, &s, &c);
            const float fm = v - m;
            c0 = c;
            c1 = s;
            c2 = fm * c;
            c3 = fm * s;
          }
        }
        float* st = stage + row * C::SW + xx;
        st[0] = c0;
        if (k != 0) {
          st[1 * C::SR * C::SW] = c1;
          st[2 * C::SR * C::SW] = c2;
          st[3 * C::SR * C::SW] = c3;
        }
      }
      __syncthreads();
      if (hch < nch && b0 + hrow < C::HROWS) {
        const float* srow = stage + (hch * C::SR + hrow) * C::SW + hx * NXH;
        float acc[NXH];
#pragma unroll
        for (int u = 0; u < NXH; ++u) acc[u] = 0.f;
#pragma unroll
        for (int q4 = 0; q4 < C::NQ4; ++q4) {
          const float4 v4 = *reinterpret_cast<const float4*>(srow + 4 * q4);
          const float vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int q = 4 * q4 + e;
#pragma unroll
            for (int u = 0; u < NXH; ++u) {
              const int d = q - u;
              if (d >= 0 && d <= 2 * RAD) acc[u] = fmaf(p.g[d], vv[e], acc[u]);
            }
          }
        }
        float* hd = hbuf + (hch * C::HROWS + b0 + hrow) * C::HS + hx * NXH;
        *reinterpret_cast<float4*>(hd) = make_float4(acc[0], acc[1], acc[2], acc[3]);
        *reinterpret_cast<float4*>(hd + 4) = make_float4(acc[4], acc[5], acc[6], acc[7]);
      }
      __syncthreads();
    }
    // ---- step 3: y-convolve own pixels and recombine ------------------------------
    float wc[NY][C::NXV], ws[NY][C::NXV];
    if (k == 0) {
#pragma unroll
      for (int u = 0; u < NY; ++u)
#pragma unroll
        for (int c = 0; c < C::NXV; ++c) {
          wc[u][c] = p.c[0];
          ws[u][c] = 0.f;
          den[u][c] = fmaf(p.c[0], sx[ox + c] * sy[oy + u], den[u][c]);
        }
    } else {
      const float ck = p.c[k];
#pragma unroll
      for (int u = 0; u < NY; ++u)
#pragma unroll
        for (int c = 0; c < C::NXV; ++c) {
          float s, cc;
          term_sincos(kf, fo[u][c], p, &s, &cc);
          wc[u][c] = ck * cc;
          ws[u][c] = ck * s;
        }
    }
    for (int ch = 0; ch < nch; ++ch) {
      float acc[NY][C::NXV];
#pragma unroll
      for (int u = 0; u < NY; ++u)
#pragma unroll
        for (int c = 0; c < C::NXV; ++c) acc[u][c] = 0.f;
      const float* hcol = hbuf + (ch * C::HROWS + oy) * C::HS + ox;
#pragma unroll
      for (int q = 0; q < NY + 2 * RAD; ++q) {
        float v[C::NXV];
        if constexpr (C::NXV == 2) {
          const float2 v2 = *reinterpret_cast<const float2*>(hcol + q * C::HS);
          v[0] = v2.x;
          v[1] = v2.y;
        } else {
          v[0] = hcol[q * C::HS];
        }
#pragma unroll
        for (int u = 0; u < NY; ++u) {
          const int d = q - u;
          if (d >= 0 && d <= 2 * RAD) {
#pragma unroll
            for (int c = 0; c < C::NXV; ++c) acc[u][c] = fmaf(p.g[d], v[c], acc[u][c]);
          }
        }
      }
      // channel order: k = 0: (f-m); k >= 1: cos, sin, (f-m)cos, (f-m)sin
#pragma unroll
      for (int u = 0; u < NY; ++u)
#pragma unroll
        for (int c = 0; c < C::NXV; ++c) {
          if (k == 0) {
            num[u][c] = fmaf(wc[u][c], acc[u][c], num[u][c]);
          } else if (ch == 0) {
            den[u][c] = fmaf(wc[u][c], acc[u][c], den[u][c]);
          } else if (ch == 1) {
            den[u][c] = fmaf(ws[u][c], acc[u][c], den[u][c]);
          } else if (ch == 2) {
            num[u][c] = fmaf(wc[u][c], acc[u][c], num[u][c]);
          } else {
            num[u][c] = fmaf(ws[u][c], acc[u][c], num[u][c]);
          }
        }
    }
    __syncthreads();   // hbuf is rewritten by the next term
  }

#pragma unroll
  for (int u = 0; u < NY; ++u)
#pragma unroll
    for (int c = 0; c < C::NXV; ++c) {
      const int gy = ty0 + oy + u, gx = tx0 + ox + c;
      if (gy < H && gx < W) {
        const float d = den[u][c];
        out[(long)gy * pitch + gx] = (d > 0.f) ? m + num[u][c] / d : fo[u][c];
      }
    }
}

template <int RAD, int TY, int NT>
int launch_cfg(const DeviceParams& dp, const float* in, float* out, int H, int W, size_t pitch,
               cudaStream_t st) {
  using C = Cfg<RAD, TY, NT>;
  static bool attr_set[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(fbf_fp32_kernel<RAD, TY, NT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES);
    if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_filter: ") + cudaGetErrorString(e));
    attr_set[dev] = true;
  }
  DeviceParams p = dp;
  // taps beyond the plan's radius are zero (a wider instantiation serves a smaller r)
  float g[2 * FBF_MAX_RADIUS + 1];
  for (int i = 0; i <= 2 * RAD; ++i) {
    int d = i - (RAD - dp.r);
    g[i] = (d >= 0 && d <= 2 * dp.r) ? dp.g[d] : 0.f;
  }
  for (int i = 0; i <= 2 * RAD; ++i) p.g[i] = g[i];
  p.r = RAD;
  dim3 grid((W + TX - 1) / TX, (H + TY - 1) / TY);
  if (grid.y > 65535) return set_error(FBF_EUNSUPPORTED, "fbf_filter: image too tall");
  fbf_fp32_kernel<RAD, TY, NT><<<grid, NT, C::SMEM_BYTES, st>>>(p, in, out, H, W, (long)pitch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_filter: launch: ") + cudaGetErrorString(e));
  return FBF_OK;
}

// Tile height: 128 rows unless that leaves fewer than two CTAs per SM on a 152-SM part.
template <int RAD, int NT_BIG>
int launch_rad(const DeviceParams& dp, const float* in, float* out, int H, int W, size_t pitch,
               cudaStream_t st) {
  const long tiles128 = (long)((W + TX - 1) / TX) * ((H + 127) / 128);
  if (tiles128 >= 2 * 152) return launch_cfg<RAD, 128, NT_BIG>(dp, in, out, H, W, pitch, st);
  return launch_cfg<RAD, 64, 256>(dp, in, out, H, W, pitch, st);
}

}  // namespace

int launch_fp32(const DeviceParams& dp, const float* in, float* out, int H, int W, size_t pitch,
                void* stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int r = dp.r;
  if (r <= 3) return launch_rad<3, 256>(dp, in, out, H, W, pitch, st);
  if (r <= 6) return launch_rad<6, 256>(dp, in, out, H, W, pitch, st);
  if (r <= 9) return launch_rad<9, 256>(dp, in, out, H, W, pitch, st);
  if (r <= 15) return launch_rad<15, 256>(dp, in, out, H, W, pitch, st);
  if (r <= 24) return launch_rad<24, 512>(dp, in, out, H, W, pitch, st);
  if (r <= 30) return launch_rad<30, 512>(dp, in, out, H, W, pitch, st);
  if (r <= 48) return launch_rad<48, 512>(dp, in, out, H, W, pitch, st);
  return set_error(FBF_EUNSUPPORTED, "fbf_filter: radius too large");
}

}  // namespace fbf
