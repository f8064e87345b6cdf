// FP32 fused Fourier bilateral filter on the CUDA cores (precision form FBF_FP32).
//
// What is computed (Section II of the paper): with phi_hat of eq. (3) as the range kernel,
// numerator and denominator of eq. (1) are, per pixel i,
//   num(i) = sum_k c_k [ C_k(i) B(f' C_k)(i) + S_k(i) B(f' S_k)(i) ]
//   den(i) = sum_k c_k [ C_k(i) B(C_k)(i)    + S_k(i) B(S_k)(i)    ]
// with C_k = cos(k nu f), S_k = sin(k nu f), nu = 2 pi/(2T+1), B the zero-padded Gaussian
// convolution with the weights of eq. (2), and f' = f - m (m = R/2; the weights of eq. (1)
// are normalised, so f_BF = m + num/den).  For k = 0 the terms are c_0 B(f') and c_0 B(1).
//
// Images are convolved in pairs, each pair held as a float2 so that every multiply-add is
// a packed two-lane FP32 FMA (fma.rn.f32x2): (C_k, S_k) and (f'C_k, f'S_k) for k >= 1, and
// (f', 1) for k = 0 (the constant image is convolved like the others, which gives its
// zero-padded blur exactly).  The Gaussian is symmetric, so only the r+1 distinct taps
// are kept in registers.
//
// Work decomposition.  The image is cut into TX x TY output tiles; each (tile, term k) is
// one unit of work of weight 2 (k >= 1: two pairs) or 1 (k = 0).  A persistent grid of
// G CTAs (G = SMs x resident CTAs) splits the weighted sequence of units tile-major into G
// equal contiguous ranges (stream-K), so every CTA does the same convolution work whatever
// the image size.  A tile whose terms span several CTAs is finished by the CTA that
// completes it last: each contributor stores its partial num/den in a per-CTA scratch
// slot and adds its weight to the tile's counter; the last one sums the partials in CTA
// order (ascending k, independent of timing) and divides.
//
// Per tile a CTA stages f of the tile plus an r-pixel halo in shared memory.  Per term,
//   1. each warp, four halo rows at a time, generates the term's image pairs into a
//      warp-private buffer and convolves them along x (8 outputs per lane) into a shared
//      buffer of TY + 2r rows; only __syncwarp separates the two;
//   2. after one CTA barrier each thread convolves that buffer along y for its own pixels
//      and folds the results into its num/den registers.
// Only f is read from and only f_BF (and split-tile partials) written to global memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <utility>

#include "fbf_internal.h"

namespace fbf {

namespace {

constexpr int TX = 32;                 // tile width
constexpr int NXH = 8;                 // x outputs per lane in the x pass
constexpr float kOutside = -3.0e38f;   // marks halo pixels outside the image
constexpr int TABN = 256;              // per-term (cos, sin) table over integer intensities

template <int RAD, int TY, int NT, int NY>
struct Cfg {
  static constexpr int NW = NT / 32;                       // warps
  static constexpr int HROWS = TY + 2 * RAD;               // rows of the x-pass output
  static constexpr int HROWS_P = (HROWS + 4 * NW - 1) / (4 * NW) * (4 * NW);  // whole rounds
  static constexpr int TXH = TX + 2 * RAD;                 // halo tile width
  static constexpr int FHS = TXH + 1;                      // f-halo row stride (floats)
  static constexpr int NQ2 = (NXH + 2 * RAD + 1) / 2;      // 16-byte loads per x-pass item
  static constexpr int SWP0 = 3 * NXH + 2 * NQ2;           // float2 slots read per stage row
  static constexpr int SWP = SWP0 + ((2 - SWP0 % 16) + 16) % 16;   // == 2 (mod 16)
  static constexpr int STAGE_F2 = 8 * SWP;                 // per warp: 4 rows x 2 pairs
  static constexpr int HS2 = TX + 2;                       // x-pass buffer row stride (float2)
  static constexpr int CPS0 = HROWS_P * HS2;
  static constexpr int CPS = CPS0 + ((4 - CPS0 % 16) + 16) % 16;  // pair stride, == 4 (mod 16)
  static constexpr size_t SMEM_BYTES =
      (size_t)(NW * STAGE_F2 + 2 * CPS + 2 * TABN) * 8 + (size_t)HROWS_P * FHS * 4 + 16;
  static_assert(TX * TY == NT * NY, "y-pass mapping: one column of NY pixels per thread");
  static_assert(TY % NY == 0 && (TY / NY) * 32 == NT, "y-pass mapping");
  static_assert(SMEM_BYTES <= 232448, "shared memory per CTA exceeds 227 KB");
};

struct Sched {
  int tiles_x, tiles_y, K, wtile;     // wtile = 2K - 1
  long long wtot;                     // tiles * wtile
  float* partial;                     // G * 2 slots * 2 * NY * NT floats
  int* counter;                       // one per tile, zero between launches
};

__device__ __forceinline__ long long ceil_div_ll(long long a, long long b) { return (a + b - 1) / b; }

// weighted start of term k within a tile (k = 0 weighs 1, k >= 1 weighs 2)
__device__ __forceinline__ int term_start(int k) { return k == 0 ? 0 : 2 * k - 1; }

// first term whose weighted start is >= s (global term index tile*K + k)
__device__ __forceinline__ long long first_term_at(long long s, int K, int wtile) {
  long long t = s / wtile;
  long long rem = s - t * wtile;
  int k = (rem == 0) ? 0 : (int)((rem + 2) / 2);   // smallest k >= 1 with 2k-1 >= rem
  if (k >= K) { ++t; k = 0; }
  return t * K + k;
}

// (cos, sin)(k nu v) for any v: reduce x = k v by the period (n = x - P rint(x/P) lies in
// [-P/2, P/2]), then the accurate sincospi.  Used for tiles whose values are not all
// integers in [0, min(R, TABN-1)].
__device__ __forceinline__ float2 term_cs_any(float kf, float v, const DeviceParams& p) {
  const float x = kf * v;
  const float n = fmaf(-rintf(x * p.invP), (float)p.P, x);
  float s, c;
  sincospif(n * (2.0f * p.invP), &s, &c);
  return make_float2(c, s);
}

// Table of (cos, sin)(k nu v) for integer v = 0..TABN-1: the phase index n = (k v) mod P
// is exact in integers and exp(i 2 pi n / P) is the product of the plan's two host-rounded
// tables (n = 128 a + b), so every entry is within a few ulp of the exact value.
template <int NT>
__device__ __forceinline__ void build_term_table(const DeviceParams& p, int k, float2* dst2) {
  float* dst = reinterpret_cast<float*>(dst2);   // [0, TABN): cos, [TABN, 2 TABN): sin
  for (int v = threadIdx.x; v < TABN; v += NT) {
    const int n = (k * v) % p.P;
    const int a = n >> 7, b = n & (kTrigLo - 1);
    const float ca = p.ta[2 * a], sa = p.ta[2 * a + 1];
    const float cb = p.tb[2 * b], sb = p.tb[2 * b + 1];
    dst[v] = fmaf(ca, cb, -sa * sb);
    dst[TABN + v] = fmaf(sa, cb, ca * sb);
  }
}

// table lookup for an integer value 0 <= v < TABN: the index is read from the float's
// mantissa (v + 2^23 has v in its low bits), which keeps the conversion off the XU pipe
__device__ __forceinline__ float2 tab_lookup(const float2* tab2, float v) {
  const float* tab = reinterpret_cast<const float*>(tab2);
  const unsigned i = __float_as_uint(v + 8388608.0f) & (TABN - 1);
  return make_float2(tab[i], tab[TABN + i]);
}

// tap d of 0..2*RAD, read through the symmetric half so only RAD+1 registers are live
template <int RAD>
__device__ __forceinline__ float2 tap2(const DeviceParams& p, int d) {
  const float g = p.g[d <= RAD ? d : 2 * RAD - d];
  return make_float2(g, g);
}

// x pass of one item: 8 consecutive outputs of one float2 image pair in one row.
template <int RAD>
__device__ __forceinline__ void xconv8(const float2* __restrict__ srow, const DeviceParams& p,
                                       float2* __restrict__ dst) {
  constexpr int NQ2 = (NXH + 2 * RAD + 1) / 2;
  float2 acc[NXH];
#pragma unroll
  for (int u = 0; u < NXH; ++u) acc[u] = make_float2(0.f, 0.f);
#pragma unroll
  for (int q2 = 0; q2 < NQ2; ++q2) {
    const float4 v4 = *reinterpret_cast<const float4*>(srow + 2 * q2);
    const float2 vv[2] = {make_float2(v4.x, v4.y), make_float2(v4.z, v4.w)};
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int q = 2 * q2 + e;
#pragma unroll
      for (int u = 0; u < NXH; ++u) {
        const int d = q - u;
        if (d >= 0 && d <= 2 * RAD) acc[u] = __ffma2_rn(tap2<RAD>(p, d), vv[e], acc[u]);
      }
    }
  }
#pragma unroll
  for (int u = 0; u < NXH; u += 2)
    *reinterpret_cast<float4*>(dst + u) = make_float4(acc[u].x, acc[u].y, acc[u + 1].x, acc[u + 1].y);
}

template <int RAD, int TY, int NT, int NY>
__global__ void __launch_bounds__(NT, 1)
fbf_fp32_kernel(const __grid_constant__ DeviceParams p, const float* __restrict__ in,
                float* __restrict__ out, int H, int W, long pitch, Sched sc) {
  using C = Cfg<RAD, TY, NT, NY>;
  extern __shared__ float4 smem_f4[];
  float2* smem2 = reinterpret_cast<float2*>(smem_f4);
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  float2* stage = smem2 + warp * C::STAGE_F2;
  float2* hbuf = smem2 + C::NW * C::STAGE_F2;
  float2* tabs = hbuf + 2 * C::CPS;                    // two term tables (double buffer)
  float* fh = reinterpret_cast<float*>(tabs + 2 * TABN);
  __shared__ int s_last;

  const int K = sc.K;
  const int G = gridDim.x;
  const int c = blockIdx.x;
  const long long Lc = ceil_div_ll((long long)c * sc.wtot, G);
  const long long Lc1 = ceil_div_ll((long long)(c + 1) * sc.wtot, G);
  long long u = first_term_at(Lc, K, sc.wtile);
  const long long uend = first_term_at(Lc1, K, sc.wtile);
  const float m = p.center;

  // own pixels: one column of NY rows
  const int ox = lane;
  const int oy = warp * NY;
  // x-pass lane roles (bank-conflict-free 16-byte accesses within each quarter warp)
  const int x_cp = lane & 1, x_rlo = (lane >> 1) & 1, x_xlo = (lane >> 2) & 1;
  const int x_rhi = (lane >> 3) & 1, x_xhi = (lane >> 4) & 1;
  const int x_row4 = x_rhi * 2 + x_rlo;        // 0..3 (k >= 1)
  const int x_xg = x_xhi * 2 + x_xlo;          // 0..3
  const int x_row8 = x_row4 * 2 + x_cp;        // 0..7 (k == 0: eight rows, one pair)

  while (u < uend) {
    const long long t = u / K;
    const int kb = (int)(u - t * K);
    const int ke = (int)((uend - t * K < K) ? uend - t * K : K);
    const int tx0 = (int)(t % sc.tiles_x) * TX;
    const int ty0 = (int)(t / sc.tiles_x) * TY;

    // f of the tile plus halo (rows padded to whole x-pass rounds); kOutside marks
    // pixels outside the image.  The tile uses the term tables when all its values are
    // integers in [0, min(R, TABN-1)] (8-bit images), else the sincospi path.
    const float vmax = (float)min(p.R, TABN - 1);
    int ok = 1;
    for (int i = tid; i < C::HROWS_P * C::TXH; i += NT) {
      const int row = i / C::TXH, xx = i - row * C::TXH;
      const int gy = ty0 - RAD + row, gx = tx0 - RAD + xx;
      float v = kOutside;
      if (row < C::HROWS && gy >= 0 && gy < H && gx >= 0 && gx < W) {
        v = __ldg(in + (long)gy * pitch + gx);
        ok &= (v == rintf(v)) & (v >= 0.f) & (v <= vmax);
      }
      fh[row * C::FHS + xx] = v;
    }
    // every halo pixel inside the image: generation needs no masking
    const bool interior = tx0 - RAD >= 0 && ty0 - RAD >= 0 && tx0 + TX + RAD <= W &&
                          ty0 + TY + RAD <= H;
    const bool tile_int = __syncthreads_and(ok) != 0;
    if (tile_int && kb >= 1) {
      build_term_table<NT>(p, kb, tabs + (kb & 1) * TABN);
      __syncthreads();
    }

    float2 num2[NY], den2[NY];
#pragma unroll
    for (int a = 0; a < NY; ++a) {
      num2[a] = make_float2(0.f, 0.f);
      den2[a] = make_float2(0.f, 0.f);
    }

    for (int k = kb; k < ke; ++k) {
      const float kf = (float)k;
      if (k == 0) {
        // ---- term 0: pair (f - m, 1); eight halo rows per warp iteration -------------
        for (int rb = warp * 8; rb < C::HROWS_P; rb += C::NW * 8) {
#pragma unroll
          for (int r8 = 0; r8 < 8; ++r8) {
#pragma unroll
            for (int xx = lane; xx < C::TXH; xx += 32) {
              const float v = fh[(rb + r8) * C::FHS + xx];
              stage[r8 * C::SWP + xx] = (v > kOutside) ? make_float2(v - m, 1.f) : make_float2(0.f, 0.f);
            }
          }
          __syncwarp();
          xconv8<RAD>(stage + x_row8 * C::SWP + x_xg * NXH, p,
                      hbuf + (rb + x_row8) * C::HS2 + x_xg * NXH);
          __syncwarp();
        }
      } else {
        // ---- term k >= 1: pairs (C, S) and (f'C, f'S); four halo rows per iteration --
        const float2* tab = tabs + (k & 1) * TABN;
        for (int rb = warp * 4; rb < C::HROWS_P; rb += C::NW * 4) {
          if (tile_int && interior) {
#pragma unroll
            for (int r4 = 0; r4 < 4; ++r4) {
#pragma unroll
              for (int xx = lane; xx < C::TXH; xx += 32) {
                const float v = fh[(rb + r4) * C::FHS + xx];
                const float2 cs = tab_lookup(tab, v);
                const float fm = v - m;
                stage[(r4 * 2) * C::SWP + xx] = cs;
                stage[(r4 * 2 + 1) * C::SWP + xx] = make_float2(fm * cs.x, fm * cs.y);
              }
            }
          } else if (tile_int) {
#pragma unroll
            for (int r4 = 0; r4 < 4; ++r4) {
#pragma unroll
              for (int xx = lane; xx < C::TXH; xx += 32) {
                const float v = fh[(rb + r4) * C::FHS + xx];
                const bool in_img = v > kOutside;
                float2 cs = tab_lookup(tab, in_img ? v : 0.f);
                cs.x = in_img ? cs.x : 0.f;
                cs.y = in_img ? cs.y : 0.f;
                const float fm = in_img ? v - m : 0.f;
                stage[(r4 * 2) * C::SWP + xx] = cs;
                stage[(r4 * 2 + 1) * C::SWP + xx] = make_float2(fm * cs.x, fm * cs.y);
              }
            }
          } else {
#pragma unroll
            for (int r4 = 0; r4 < 4; ++r4) {
#pragma unroll
              for (int xx = lane; xx < C::TXH; xx += 32) {
                const float v = fh[(rb + r4) * C::FHS + xx];
                const bool in_img = v > kOutside;
                float2 cs = term_cs_any(kf, in_img ? v : 0.f, p);
                cs.x = in_img ? cs.x : 0.f;
                cs.y = in_img ? cs.y : 0.f;
                const float fm = in_img ? v - m : 0.f;
                stage[(r4 * 2) * C::SWP + xx] = cs;
                stage[(r4 * 2 + 1) * C::SWP + xx] = make_float2(fm * cs.x, fm * cs.y);
              }
            }
          }
          __syncwarp();
          xconv8<RAD>(stage + (x_row4 * 2 + x_cp) * C::SWP + x_xg * NXH, p,
                      hbuf + x_cp * C::CPS + (rb + x_row4) * C::HS2 + x_xg * NXH);
          __syncwarp();
        }
      }
      __syncthreads();
      // the next term's table goes to the other buffer while this term's is still read
      if (tile_int && k + 1 < ke) build_term_table<NT>(p, k + 1, tabs + ((k + 1) & 1) * TABN);

      // ---- y pass for own pixels, folded into num/den ---------------------------------
      const int ncp = (k == 0) ? 1 : 2;
      float2 w[NY];
      if (k != 0) {
        const float ck = p.c[k];
        const float2* tab = tabs + (k & 1) * TABN;
#pragma unroll
        for (int a = 0; a < NY; ++a) {
          const float v = fh[(oy + a + RAD) * C::FHS + ox + RAD];
          const bool in_img = v > kOutside;   // false only for pixels past the image edge
          const float2 cs = tile_int ? tab_lookup(tab, in_img ? v : 0.f) : term_cs_any(kf, v, p);
          w[a] = make_float2(ck * cs.x, ck * cs.y);
        }
      }
      for (int cp = 0; cp < ncp; ++cp) {
        float2 acc[NY];
#pragma unroll
        for (int a = 0; a < NY; ++a) acc[a] = make_float2(0.f, 0.f);
        const float2* hcol = hbuf + cp * C::CPS + oy * C::HS2 + ox;
#pragma unroll
        for (int q = 0; q < NY + 2 * RAD; ++q) {
          const float2 v = hcol[q * C::HS2];
#pragma unroll
          for (int a = 0; a < NY; ++a) {
            const int d = q - a;
            if (d >= 0 && d <= 2 * RAD) acc[a] = __ffma2_rn(tap2<RAD>(p, d), v, acc[a]);
          }
        }
        if (k == 0) {
          const float c0 = p.c[0];
#pragma unroll
          for (int a = 0; a < NY; ++a) {
            num2[a].x = fmaf(c0, acc[a].x, num2[a].x);   // c_0 B(f - m)
            den2[a].x = fmaf(c0, acc[a].y, den2[a].x);   // c_0 B(1)
          }
        } else if (cp == 0) {
#pragma unroll
          for (int a = 0; a < NY; ++a) den2[a] = __ffma2_rn(w[a], acc[a], den2[a]);
        } else {
#pragma unroll
          for (int a = 0; a < NY; ++a) num2[a] = __ffma2_rn(w[a], acc[a], num2[a]);
        }
      }
      __syncthreads();   // hbuf and stage are rewritten by the next term
    }

    float num[NY], den[NY];
#pragma unroll
    for (int a = 0; a < NY; ++a) {
      num[a] = num2[a].x + num2[a].y;
      den[a] = den2[a].x + den2[a].y;
    }

    // ---- finish the tile --------------------------------------------------------------
    bool finish = true;
    if (!(kb == 0 && ke == K)) {
      const int wmine = term_start(ke) - term_start(kb);
      const int slot = (first_term_at(Lc, K, sc.wtile) / K == t) ? 0 : 1;
      float* pp = sc.partial + ((long long)(c * 2 + slot) * 2) * NY * NT;
#pragma unroll
      for (int a = 0; a < NY; ++a) {
        pp[a * NT + tid] = num[a];
        pp[(NY + a) * NT + tid] = den[a];
      }
      __threadfence();
      __syncthreads();
      if (tid == 0) {
        const int prev = atomicAdd(sc.counter + t, wmine);
        s_last = (prev + wmine == sc.wtile);
      }
      __syncthreads();
      finish = s_last != 0;
      if (finish) {
        __threadfence();
        // sum the partials of all contributing CTAs in CTA (= term) order
        const long long c0 = (t * sc.wtile) * G / sc.wtot;
        const long long c1 = (t * sc.wtile + term_start(K - 1)) * G / sc.wtot;
#pragma unroll
        for (int a = 0; a < NY; ++a) { num[a] = 0.f; den[a] = 0.f; }
        for (long long cc = c0; cc <= c1; ++cc) {
          const long long f0 = first_term_at(ceil_div_ll(cc * sc.wtot, G), K, sc.wtile);
          const long long f1 = first_term_at(ceil_div_ll((cc + 1) * sc.wtot, G), K, sc.wtile);
          if (f0 >= f1) continue;  // no term starts in this CTA's range
          const int sl = (f0 / K == t) ? 0 : 1;
          const float* qp = sc.partial + ((cc * 2 + sl) * 2) * NY * NT;
#pragma unroll
          for (int a = 0; a < NY; ++a) {
            num[a] += __ldcg(qp + a * NT + tid);
            den[a] += __ldcg(qp + (NY + a) * NT + tid);
          }
        }
        if (tid == 0) sc.counter[t] = 0;
      }
    }
    if (finish) {
#pragma unroll
      for (int a = 0; a < NY; ++a) {
        const int gy = ty0 + oy + a, gx = tx0 + ox;
        if (gy < H && gx < W) {
          const float d = den[a];
          const float f = fh[(oy + a + RAD) * C::FHS + ox + RAD];
          out[(long)gy * pitch + gx] = (d > 0.f) ? m + num[a] / d : f;
        }
      }
    }
    u = t * K + ke;
    __syncthreads();   // the f halo is rewritten by the next tile
  }
}

// ---- per-(device, stream) scratch: tile counters and partial sums ----------------------
// Layout: [counter_cap ints, zero between launches][partial sums].  Each launch leaves the
// counters it used at zero, so they are cleared only when the buffer is (re)allocated.
struct Workspace {
  void* base = nullptr;
  size_t counter_cap = 0;
  size_t partial_cap = 0;
};
std::mutex g_ws_mu;
std::map<std::pair<int, uintptr_t>, Workspace> g_ws;

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

int get_workspace(int dev, cudaStream_t st, size_t partial_bytes, size_t counters,
                  float** partial, int** counter) {
  std::lock_guard<std::mutex> lk(g_ws_mu);
  Workspace& w = g_ws[{dev, (uintptr_t)st}];
  if (w.counter_cap < counters || w.partial_cap < partial_bytes) {
    if (w.base) {
      cudaError_t e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_filter: ") + cudaGetErrorString(e));
      cudaFree(w.base);
      w.base = nullptr;
      w.counter_cap = w.partial_cap = 0;
    }
    const size_t cc = std::max(counters + counters / 2, (size_t)1024);
    const size_t pc = partial_bytes + partial_bytes / 2;
    const size_t total = align256(cc * sizeof(int)) + pc;
    cudaError_t e = cudaMalloc(&w.base, total);
    if (e != cudaSuccess) {
      w.base = nullptr;
      return set_error(FBF_ENOMEM, std::string("fbf_filter: workspace: ") + cudaGetErrorString(e));
    }
    e = cudaMemsetAsync(w.base, 0, align256(cc * sizeof(int)), st);
    if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_filter: ") + cudaGetErrorString(e));
    w.counter_cap = cc;
    w.partial_cap = pc;
  }
  *counter = reinterpret_cast<int*>(w.base);
  *partial = reinterpret_cast<float*>(static_cast<char*>(w.base) + align256(w.counter_cap * sizeof(int)));
  return FBF_OK;
}

template <int RAD, int TY, int NT, int NY>
int launch_cfg(const DeviceParams& dp, const float* in, float* out, int H, int W, size_t pitch,
               cudaStream_t st) {
  using C = Cfg<RAD, TY, NT, NY>;
  static int occ[64] = {0};
  static int sms[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_filter: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= 64) return set_error(FBF_EUNSUPPORTED, "fbf_filter: device index >= 64");
  if (!occ[dev]) {
    e = cudaFuncSetAttribute(fbf_fp32_kernel<RAD, TY, NT, NY>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM_BYTES);
    if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_filter: ") + cudaGetErrorString(e));
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fbf_fp32_kernel<RAD, TY, NT, NY>, NT,
                                                      C::SMEM_BYTES);
    if (e != cudaSuccess || n < 1) return set_error(FBF_ECUDA, "fbf_filter: kernel does not fit on an SM");
    int s = 0;
    cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
    sms[dev] = s;
    occ[dev] = n;
  }
  DeviceParams p = dp;
  // taps beyond the plan's radius are zero (a wider instantiation serves a smaller r)
  float g[2 * FBF_MAX_RADIUS + 1];
  for (int i = 0; i <= 2 * RAD; ++i) {
    const int d = i - (RAD - dp.r);
    g[i] = (d >= 0 && d <= 2 * dp.r) ? dp.g[d] : 0.f;
  }
  for (int i = 0; i <= 2 * RAD; ++i) p.g[i] = g[i];
  p.r = RAD;

  Sched sc{};
  sc.tiles_x = (W + TX - 1) / TX;
  sc.tiles_y = (H + TY - 1) / TY;
  sc.K = dp.K;
  sc.wtile = 2 * dp.K - 1;
  const long long tiles = (long long)sc.tiles_x * sc.tiles_y;
  if (tiles > (1LL << 30)) return set_error(FBF_EUNSUPPORTED, "fbf_filter: image too large");
  sc.wtot = tiles * sc.wtile;
  long long G = (long long)sms[dev] * occ[dev];
  if (G > sc.wtot) G = sc.wtot;
  const size_t partial_bytes = (size_t)G * 2 * 2 * NY * NT * sizeof(float);
  int rc = get_workspace(dev, st, partial_bytes, (size_t)tiles, &sc.partial, &sc.counter);
  if (rc != FBF_OK) return rc;
  fbf_fp32_kernel<RAD, TY, NT, NY><<<(unsigned)G, NT, C::SMEM_BYTES, st>>>(p, in, out, H, W, (long)pitch, sc);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_filter: launch: ") + cudaGetErrorString(e));
  return FBF_OK;
}

}  // namespace

int launch_fp32(const DeviceParams& dp, const float* in, float* out, int H, int W, size_t pitch,
                void* stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int r = dp.r;
  // Tile heights keep TY + 2r just under a whole number of x-pass rounds (4 rows per
  // warp); radii above 15 need more registers for their taps and use 256 threads.
  if (r <= 3) return launch_cfg<3, 112, 512, 7>(dp, in, out, H, W, pitch, st);
  if (r <= 6) return launch_cfg<6, 112, 512, 7>(dp, in, out, H, W, pitch, st);
  if (r <= 9) return launch_cfg<9, 96, 512, 6>(dp, in, out, H, W, pitch, st);
  if (r <= 15) return launch_cfg<15, 96, 512, 6>(dp, in, out, H, W, pitch, st);
  if (r <= 24) return launch_cfg<24, 128, 256, 16>(dp, in, out, H, W, pitch, st);
  if (r <= 30) return launch_cfg<30, 128, 256, 16>(dp, in, out, H, W, pitch, st);
  if (r <= 48) return launch_cfg<48, 64, 128, 16>(dp, in, out, H, W, pitch, st);
  return set_error(FBF_EUNSUPPORTED, "fbf_filter: radius too large");
}

// ---- allocation-free variant --------------------------------------------------------------
// Some callers cannot allocate device memory while they filter: a framework whose caching
// allocator already owns (nearly) all of the GPU's memory, or a latency-bound serving loop
// in which a cudaMalloc/cudaFree -- which may synchronise the whole device -- is not
// acceptable.  For them the FP32 kernel can take its scratch (tile counters and split-tile
// partial sums) from this fixed, file-scope device array instead of the per-stream
// workspace.  Every GPU that loads the library holds the array until the process exits.
// Its address is looked up once per device (cudaGetSymbolAddress, with that device
// current) by the first call on that device.  All calls share the array: calls whose
// work overlaps on the GPU race on it.
namespace {

constexpr size_t kNoAllocCounterBytes = size_t(1) << 20;              // 262144 tile counters
constexpr size_t kNoAllocPartialBytes = size_t(FBF_NOALLOC_SCRATCH_BYTES) - kNoAllocCounterBytes;
static_assert(FBF_NOALLOC_SCRATCH_BYTES > (1 << 20), "scratch must hold the counters");

static __device__ __align__(256) unsigned char g_noalloc_scratch[FBF_NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64] = {nullptr};

// Host code must not use g_noalloc_scratch directly: in host code it names a host-side
// stand-in, not device memory.  This returns the device address for the current device.
int noalloc_scratch(int dev, void** out) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || ptr == nullptr)
      return set_error(FBF_ECUDA, std::string("fbf_filter_noalloc: cudaGetSymbolAddress: ") +
                                      cudaGetErrorString(e));
    g_noalloc_ptr[dev] = ptr;
  }
  *out = g_noalloc_ptr[dev];
  return FBF_OK;
}

template <int RAD, int TY, int NT, int NY>
int launch_cfg_noalloc(const DeviceParams& dp, const float* in, float* out, int H, int W,
                       size_t pitch, cudaStream_t st) {
  using C = Cfg<RAD, TY, NT, NY>;
  static int occ[64] = {0};
  static int sms[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_filter_noalloc: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= 64) return set_error(FBF_EUNSUPPORTED, "fbf_filter_noalloc: device index >= 64");
  Sched sc{};
  sc.tiles_x = (W + TX - 1) / TX;
  sc.tiles_y = (H + TY - 1) / TY;
  sc.K = dp.K;
  sc.wtile = 2 * dp.K - 1;
  const long long tiles = (long long)sc.tiles_x * sc.tiles_y;
  if ((size_t)tiles * sizeof(int) > kNoAllocCounterBytes)
    return set_error(FBF_EUNSUPPORTED,
                     "fbf_filter_noalloc: image needs " + std::to_string(tiles) + " tiles; the fixed "
                     "scratch holds counters for " + std::to_string(kNoAllocCounterBytes / sizeof(int)));
  void* base = nullptr;
  int rc = noalloc_scratch(dev, &base);
  if (rc != FBF_OK) return rc;
  if (!occ[dev]) {
    e = cudaFuncSetAttribute(fbf_fp32_kernel<RAD, TY, NT, NY>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM_BYTES);
    if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_filter_noalloc: ") + cudaGetErrorString(e));
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fbf_fp32_kernel<RAD, TY, NT, NY>, NT,
                                                      C::SMEM_BYTES);
    if (e != cudaSuccess || n < 1) return set_error(FBF_ECUDA, "fbf_filter_noalloc: kernel does not fit on an SM");
    int s = 0;
    cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
    sms[dev] = s;
    occ[dev] = n;
  }
  DeviceParams p = dp;
  float g[2 * FBF_MAX_RADIUS + 1];
  for (int i = 0; i <= 2 * RAD; ++i) {
    const int d = i - (RAD - dp.r);
    g[i] = (d >= 0 && d <= 2 * dp.r) ? dp.g[d] : 0.f;
  }
  for (int i = 0; i <= 2 * RAD; ++i) p.g[i] = g[i];
  p.r = RAD;
  sc.wtot = tiles * sc.wtile;
  long long G = (long long)sms[dev] * occ[dev];
  const long long per_cta = 2LL * 2 * NY * NT * (long long)sizeof(float);
  if (G > (long long)(kNoAllocPartialBytes / per_cta)) G = (long long)(kNoAllocPartialBytes / per_cta);
  if (G > sc.wtot) G = sc.wtot;
  sc.counter = reinterpret_cast<int*>(base);
  sc.partial = reinterpret_cast<float*>(static_cast<unsigned char*>(base) + kNoAllocCounterBytes);
  // counters must start at zero; the array keeps whatever the previous call left
  e = cudaMemsetAsync(sc.counter, 0, (size_t)tiles * sizeof(int), st);
  if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_filter_noalloc: ") + cudaGetErrorString(e));
  fbf_fp32_kernel<RAD, TY, NT, NY><<<(unsigned)G, NT, C::SMEM_BYTES, st>>>(p, in, out, H, W, (long)pitch, sc);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_filter_noalloc: launch: ") + cudaGetErrorString(e));
  return FBF_OK;
}

}  // namespace

int launch_fp32_noalloc(const DeviceParams& dp, const float* in, float* out, int H, int W,
                        size_t pitch, void* stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int r = dp.r;
  if (r <= 3) return launch_cfg_noalloc<3, 112, 512, 7>(dp, in, out, H, W, pitch, st);
  if (r <= 6) return launch_cfg_noalloc<6, 112, 512, 7>(dp, in, out, H, W, pitch, st);
  if (r <= 9) return launch_cfg_noalloc<9, 96, 512, 6>(dp, in, out, H, W, pitch, st);
  if (r <= 15) return launch_cfg_noalloc<15, 96, 512, 6>(dp, in, out, H, W, pitch, st);
  if (r <= 24) return launch_cfg_noalloc<24, 128, 256, 16>(dp, in, out, H, W, pitch, st);
  if (r <= 30) return launch_cfg_noalloc<30, 128, 256, 16>(dp, in, out, H, W, pitch, st);
  if (r <= 48) return launch_cfg_noalloc<48, 64, 128, 16>(dp, in, out, H, W, pitch, st);
  return set_error(FBF_EUNSUPPORTED, "fbf_filter_noalloc: radius too large");
}

}  // namespace fbf
