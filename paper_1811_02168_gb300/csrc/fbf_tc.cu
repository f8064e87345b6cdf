// Tensor-core forms of the fused Fourier bilateral filter (FBF_FP16_TC, FBF_BF16_TC).
//
// Same method and schedule as the FP32 kernel (see fbf_fp32.cu): eq. (1) with phi_hat of
// eq. (3) through Gaussian convolutions of cos(k nu f), sin(k nu f), (f-m)cos, (f-m)sin
// (Section II), stream-K over weighted (tile, term) units, partial sums finished by the
// last contributing CTA.  Here each separable Gaussian pass is a dense contraction on the
// 5th-generation tensor cores: with a 128 x 128 output tile, an r-pixel halo and
// KP = 128 + 2r rounded up to 16,
//   x pass:  D1[x', hy] = sum_hx G[x', hx] B_h[hy, hx]    (M = 128, N = KP, K = KP)
//   y pass:  D2[y', x'] = sum_hy G[y', hy] D1[x', hy]     (M = 128, N = 128, K = KP)
// where G[o, i] = g(i - o - r) is the banded Toeplitz matrix of the 2r+1 Gaussian taps (one
// copy serves both passes) and B_h holds one convolved image over the tile plus halo.  The
// operands are FP16 or BF16 in shared memory (K-major, no swizzle: 8-row x 16-byte core
// matrices), the accumulators FP32 in tensor memory (TMEM).  One thread issues the
// tcgen05.mma instructions; completion is signalled through mbarriers.  After the x pass the
// warps copy D1 from TMEM into shared memory as the y pass's B operand (TMEM lane = output
// column = B row, so no transpose is needed), rounding it to the operand type.  After the
// y pass each thread folds its 32 pixels of D2 into num/den registers with the per-pixel
// weights c_k cos(k nu f_i), c_k sin(k nu f_i) (or c_0), two images at a time:
// (cos, (f-m)cos), (sin, (f-m)sin), and for k = 0 ((f-m), 1).
//
// Every wait is bounded; a wait that gives up sets the device error word (read with
// fbf_device_errors), makes every thread leave the tile loop, and the CTA still frees its
// TMEM before returning.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <type_traits>

#include "fbf_fp32_body.cuh"
#include "fbf_internal.h"

namespace fbf {
namespace tc {

using namespace fp32;

__device__ int g_tc_error;   // bit 0: an mbarrier wait gave up

constexpr int TT = 128;            // tile edge = MMA M
constexpr int NTHREADS = 512;      // 16 warps: 4 TMEM lane quarters x 4 column groups
constexpr int kWaitLimit = 1 << 22;

template <int RAD>
struct TcCfg {
  static constexpr int HW = TT + 2 * RAD;                 // halo extent
  static constexpr int KP = (HW + 15) / 16 * 16;          // padded contraction length
  static constexpr int NH = KP;                           // x-pass N (halo rows, padded)
  static constexpr int OPB = TT * KP * 2;                 // bytes of G or B_v
  static constexpr int BHB = NH * KP * 2;                 // bytes of one B_h
  static constexpr int FHS = KP + 8;                      // f-halo row stride (bytes), == 8 (mod 16)
  static constexpr int FHB = ((NH * FHS) + 127) / 128 * 128;   // rows up to NH (padding is finite)
  static constexpr int TABB = 3 * 4 * 256 * 4;            // 3 term-table slots (cos, sin, (f-m)cos, (f-m)sin)
  static constexpr int FIXED = 2 * OPB + FHB + TABB + 128;
  static constexpr int NBH = (FIXED + 2 * BHB + 1024 <= 232448) ? 2 : 1;
  static constexpr int SMEM = FIXED + NBH * BHB + 1024;   // + alignment slack
  static constexpr int L = NBH;                           // x-pass MMAs issued ahead
  static_assert(L * 192 + 128 <= 512, "TMEM columns");
  static_assert(SMEM <= 232448, "tensor-core tile does not fit in shared memory");
  static_assert(NH <= 256, "x-pass N exceeds one MMA");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of element (row, k) in a K-major no-swizzle operand with KP columns
template <int KP>
__device__ __forceinline__ int core_off(int row, int k) {
  return ((row >> 3) * (KP >> 3) + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// shared-memory matrix descriptor: K-major, no swizzle; LBO = 128 B (next core matrix
// along K), SBO = 16 KP B (next 8-row group), version 1
template <int KP>
__device__ __forceinline__ uint64_t op_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)(((uint32_t)(KP / 8 * 128) >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor: D FP32, A and B FP16 (fmt 0) or BF16 (fmt 1), both K-major
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt, int M, int N) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <typename T>
__device__ __forceinline__ uint32_t pack2(float a, float b);
template <>
__device__ __forceinline__ uint32_t pack2<__half>(float a, float b) {
  const __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}
template <>
__device__ __forceinline__ uint32_t pack2<__nv_bfloat16>(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t da, uint64_t db, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
      :: "r"(dtmem), "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :: "r"(smem_u32(mbar)) : "memory");
}

// bounded wait for phase `parity` of an mbarrier; false if it gave up
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity) {
  uint32_t done = 0;
  for (int it = 0; it < kWaitLimit; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done) : "r"(smem_u32(mbar)), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                 "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// kind of convolved image
enum Chan { CH_FM = 0, CH_ONE = 1, CH_C = 2, CH_FC = 3, CH_S = 4, CH_FS = 5 };

// The tile's images in processing order: k = 0 gives ((f-m), 1), k >= 1 gives
// (cos, (f-m)cos, sin, (f-m)sin).  Image c of a tile whose first term is kb:
__device__ __forceinline__ void chan_of(int kb, int c, int* k, int* kind) {
  if (kb == 0) {
    if (c < 2) { *k = 0; *kind = c; return; }
    c -= 2;
    *k = 1 + (c >> 2);
  } else {
    *k = kb + (c >> 2);
  }
  *kind = CH_C + (c & 3);
}

// Term table slot (three slots: generation runs ahead of the fold by up to two images):
// [cos | sin | (v-m) cos | (v-m) sin], 256 entries each, built from the exact phase index.
__device__ __forceinline__ void build_tables(const DeviceParams& p, int k, float* t) {
  const float m = p.center;
  for (int v = threadIdx.x; v < 256; v += NTHREADS) {
    const int n = (k * v) % p.P;
    const int a = n >> 7, b = n & (kTrigLo - 1);
    const float ca = p.ta[2 * a], sa = p.ta[2 * a + 1];
    const float cb = p.tb[2 * b], sb = p.tb[2 * b + 1];
    const float c = fmaf(ca, cb, -sa * sb), s = fmaf(sa, cb, ca * sb);
    const float fm = (float)v - m;
    t[v] = c;
    t[256 + v] = s;
    t[512 + v] = fm * c;
    t[768 + v] = fm * s;
  }
}

// Generate image `KIND` of term k over the halo tile into a K-major operand (rows = halo
// rows, K = halo columns).  Eight consecutive threads fill the eight rows of one core matrix,
// so the 16-byte stores are conflict-free.  Rows and columns past the halo need only be
// finite: the matching entries of G are zero.  Pixels outside the image are zero (only
// tiles at the image border test for them, with a column bit mask per 8-pixel group).
template <int RAD, typename T, int KIND>
__device__ __forceinline__ void generate(unsigned char* dst, const unsigned char* fh, const float* tab,
                                         bool tile_int, bool interior, int tx0, int ty0, int H, int W,
                                         const float* __restrict__ in, long long pitch, int k,
                                         const DeviceParams& p) {
  using C = TcCfg<RAD>;
  constexpr int KP = C::KP;
  constexpr int KG = KP / 8;
  const float m = p.center;
  const int col_lo = max(0, RAD - tx0), col_hi = min(C::HW, W - tx0 + RAD);   // inside: [lo, hi)
  for (int i = threadIdx.x; i < C::NH * KG; i += NTHREADS) {
    const int hy = ((i >> 3) / KG) * 8 + (i & 7);
    const int hx0 = ((i >> 3) % KG) * 8;
    float v8[8];
    if (tile_int) {
      const uint2 bytes = *reinterpret_cast<const uint2*>(fh + hy * C::FHS + hx0);
      unsigned mask = 0xFFu;
      if (!interior) {
        const int gy = ty0 - RAD + hy;
        const bool row_in = hy < C::HW && gy >= 0 && gy < H;
        const int a = min(8, max(0, col_lo - hx0)), b = min(8, max(0, col_hi - hx0));
        mask = row_in && b > a ? (((1u << b) - 1u) & ~((1u << a) - 1u)) : 0u;
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const unsigned bv = ((j < 4 ? bytes.x : bytes.y) >> (8 * (j & 3))) & 0xFFu;
        float val;
        if (KIND == CH_FM) val = (float)bv - m;
        else if (KIND == CH_ONE) val = 1.f;
        else val = tab[(KIND == CH_C ? 0 : KIND == CH_S ? 256 : KIND == CH_FC ? 512 : 768) + bv];
        v8[j] = ((mask >> j) & 1u) ? val : 0.f;
      }
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int hx = hx0 + j, gy = ty0 - RAD + hy, gx = tx0 - RAD + hx;
        const bool inside = hy < C::HW && hx < C::HW && gy >= 0 && gy < H && gx >= 0 && gx < W;
        float val = 0.f;
        if (inside) {
          const float fv = __ldg(in + (long long)gy * pitch + gx);
          if (KIND == CH_FM) val = fv - m;
          else if (KIND == CH_ONE) val = 1.f;
          else {
            const float2 cs = term_cs_any((float)k, fv, p);
            const float tr = (KIND == CH_C || KIND == CH_FC) ? cs.x : cs.y;
            val = (KIND == CH_C || KIND == CH_S) ? tr : (fv - m) * tr;
          }
        }
        v8[j] = val;
      }
    }
    *reinterpret_cast<uint4*>(dst + core_off<KP>(hy, hx0)) =
        make_uint4(pack2<T>(v8[0], v8[1]), pack2<T>(v8[2], v8[3]), pack2<T>(v8[4], v8[5]),
                   pack2<T>(v8[6], v8[7]));
  }
}

template <int RAD, typename T>
__device__ __forceinline__ void generate_kind(int kind, unsigned char* dst, const unsigned char* fh,
                                              const float* tab, bool tile_int, bool interior, int tx0,
                                              int ty0, int H, int W, const float* __restrict__ in,
                                              long long pitch, int k, const DeviceParams& p) {
  switch (kind) {
    case CH_FM: generate<RAD, T, CH_FM>(dst, fh, tab, tile_int, interior, tx0, ty0, H, W, in, pitch, k, p); break;
    case CH_ONE: generate<RAD, T, CH_ONE>(dst, fh, tab, tile_int, interior, tx0, ty0, H, W, in, pitch, k, p); break;
    case CH_C: generate<RAD, T, CH_C>(dst, fh, tab, tile_int, interior, tx0, ty0, H, W, in, pitch, k, p); break;
    case CH_FC: generate<RAD, T, CH_FC>(dst, fh, tab, tile_int, interior, tx0, ty0, H, W, in, pitch, k, p); break;
    case CH_S: generate<RAD, T, CH_S>(dst, fh, tab, tile_int, interior, tx0, ty0, H, W, in, pitch, k, p); break;
    default: generate<RAD, T, CH_FS>(dst, fh, tab, tile_int, interior, tx0, ty0, H, W, in, pitch, k, p); break;
  }
}

template <int RAD, typename T>
__global__ void __launch_bounds__(NTHREADS, 1)
fbf_tc_kernel(const __grid_constant__ DeviceParams p, const Work w, const Scratch sc) {
  using C = TcCfg<RAD>;
  constexpr int KP = C::KP;
  constexpr int L = C::L;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned base, kept as an offset into the shared array (shared address space)
  unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* sG = base;                        // G (A operand of both passes)
  unsigned char* sBv = sG + C::OPB;                // y-pass B operand
  unsigned char* sFh = sBv + C::OPB;               // f of the halo tile (uint8)
  float* sTab = reinterpret_cast<float*>(sFh + C::FHB);   // 3 slots x 1024 floats
  uint64_t* mbH = reinterpret_cast<uint64_t*>(reinterpret_cast<unsigned char*>(sTab) + C::TABB);  // [2]
  uint64_t* mbV = mbH + 2;
  uint32_t* sTmem = reinterpret_cast<uint32_t*>(mbH + 3);
  int* sFlags = reinterpret_cast<int*>(sTmem + 1);
  unsigned char* sBh = reinterpret_cast<unsigned char*>(mbH) + 128;   // NBH x B_h

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q = warp & 3;            // TMEM lane quarter
  const int cg = warp >> 2;          // column group
  const uint32_t fmt = std::is_same<T, __nv_bfloat16>::value ? 1u : 0u;
  const uint32_t idH = instr_desc(fmt, TT, C::NH);
  const uint32_t idV = instr_desc(fmt, TT, TT);

  // ---- set-up: G, barriers, TMEM ---------------------------------------------------------
  for (int i = tid; i < TT * (KP / 8); i += NTHREADS) {
    const int o = i / (KP / 8), k8 = (i - o * (KP / 8)) * 8;
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int d = k8 + j - o;   // tap index 0..2r
      v[j] = (d >= 0 && d <= 2 * RAD) ? p.g[d] : 0.f;
    }
    *reinterpret_cast<uint4*>(sG + core_off<KP>(o, k8)) =
        make_uint4(pack2<T>(v[0], v[1]), pack2<T>(v[2], v[3]), pack2<T>(v[4], v[5]), pack2<T>(v[6], v[7]));
  }
  if (tid == 0) {
    for (int j = 0; j < 3; ++j) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(mbH + j)));
  }
  proxy_fence();
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" :: "r"(smem_u32(sTmem)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *sTmem;
  const uint32_t tD2 = tmem + 384;           // y-pass accumulator, 128 columns
  uint32_t phH[2] = {0, 0}, phV = 0;

  const SingleSrc src{&p, w};
  const int G = gridDim.x;
  const int cta = blockIdx.x;
  const long long Lc = ceil_div_ll((long long)cta * sc.wtot, G);
  const long long Lc1 = ceil_div_ll((long long)(cta + 1) * sc.wtot, G);
  int img, img_end;
  long long u, u_end;
  locate(src, Lc, sc.wtot, img, u);
  locate(src, Lc1, sc.wtot, img_end, u_end);
  const long long u_first = u;
  const int K = w.K, H = w.H, W = w.W;
  const long long pitch = w.pitch;
  const float m = p.center;
  const int oy = 32 * q + lane;      // own pixels: row oy, columns ox0 .. ox0 + 31
  const int ox0 = 32 * cg;
  bool abort = false;

  auto issue_x = [&](int c, int tc_slot) {   // x pass of image c: D1[c % L] = G x B_h[c % NBH]^T
    if (tid == 0) {
      const uint32_t aG = smem_u32(sG), aB = smem_u32(sBh + (c % C::NBH) * C::BHB);
      const uint32_t d1 = tmem + 192u * (uint32_t)(c % L);
#pragma unroll 1
      for (int ks = 0; ks < KP / 16; ++ks)
        mma_f16(d1, op_desc<KP>(aG + ks * 256), op_desc<KP>(aB + ks * 256), idH, ks > 0);
      mma_commit(mbH + (c % L));
    }
    (void)tc_slot;
  };

  while (!abort && (img < img_end || (img == img_end && u < u_end))) {
    const long long t = u / K;
    const int kb = (int)(u - t * K);
    const int ke = (img == img_end && t == u_end / K) ? (int)(u_end - t * K) : K;
    const int tx0 = (int)(t % w.tiles_x) * TT;
    const int ty0 = (int)(t / w.tiles_x) * TT;
    const int nchan = (kb == 0 ? 2 + 4 * (ke - 1) : 4 * (ke - kb));

    // f of the tile + halo as bytes; the tile takes the table path when every pixel in the
    // image is an integer in [0, min(R, 255)], else values are read from global memory
    const float vmax = (float)min(p.R, 255);
    int ok = 1;
    for (int i = tid; i < C::NH * C::FHS; i += NTHREADS) {
      const int hy = i / C::FHS, hx = i - hy * C::FHS;
      const int gy = ty0 - RAD + hy, gx = tx0 - RAD + hx;
      unsigned char b = 0;
      if (hy < C::HW && hx < C::HW && gy >= 0 && gy < H && gx >= 0 && gx < W) {
        const float v = __ldg(w.in + (long long)gy * pitch + gx);
        ok &= (v == rintf(v)) & (v >= 0.f) & (v <= vmax);
        b = (unsigned char)(int)fminf(fmaxf(v, 0.f), 255.f);
      }
      sFh[hy * C::FHS + hx] = b;
    }
    const bool interior = tx0 - RAD >= 0 && ty0 - RAD >= 0 && tx0 + TT + RAD <= W && ty0 + TT + RAD <= H;
    // tables of the terms of the first L images
    {
      int k0, kd0, k1, kd1;
      chan_of(kb, 0, &k0, &kd0);
      chan_of(kb, min(L, nchan) - 1, &k1, &kd1);
      if (k0 >= 1) build_tables(p, k0, sTab + (k0 % 3) * 1024);
      if (k1 != k0 && k1 >= 1) build_tables(p, k1, sTab + (k1 % 3) * 1024);
    }
    const bool tile_int = __syncthreads_and(ok) != 0;

    const unsigned char* own = sFh + (oy + RAD) * C::FHS + ox0 + RAD;   // own pixels' intensities
    float nm[32], dn[32];   // num / den of the thread's 32 pixels
#pragma unroll
    for (int i = 0; i < 32; ++i) { nm[i] = 0.f; dn[i] = 0.f; }

    // ---- prologue: generate and issue the x pass of the first L images ---------------------
    for (int j = 0; j < L && j < nchan; ++j) {
      int k, kind;
      chan_of(kb, j, &k, &kind);
      generate_kind<RAD, T>(kind, sBh + (j % C::NBH) * C::BHB, sFh, sTab + (k % 3) * 1024, tile_int,
                            interior, tx0, ty0, H, W, w.in, pitch, k, p);
    }
    proxy_fence();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    for (int j = 0; j < L && j < nchan; ++j) issue_x(j, 0);

    for (int c = 0; c < nchan; ++c) {
      int k, kind;
      chan_of(kb, c, &k, &kind);
      if (!mbar_wait(mbH + (c % L), phH[c % L])) abort = true;
      phH[c % L] ^= 1;
      if (c >= 1) {
        if (!mbar_wait(mbV, phV)) abort = true;
        phV ^= 1;
      }
      tc_fence_after();
      if (__syncthreads_or(abort)) { abort = true; break; }
      // ---- fold image c-1 (in D2) into num/den ------------------------------------------
      if (c >= 1) {
        int kp, kindp;
        chan_of(kb, c - 1, &kp, &kindp);
        const float* tab = sTab + (kp % 3) * 1024;
        const float ck = p.c[kp];
        const bool to_num = (kindp == CH_FM || kindp == CH_FC || kindp == CH_FS);
        const int woff = (kindp == CH_S || kindp == CH_FS) ? 256 : 0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          uint32_t a[16];
          tmem_ld16(tD2 + ((uint32_t)(32 * q) << 16) + (uint32_t)(ox0 + 16 * h), a);
          tmem_wait_ld();
#pragma unroll
          for (int ii = 0; ii < 16; ++ii) {
            const int i = 16 * h + ii;
            float wgt = ck;
            if (kindp >= CH_C) {
              if (tile_int) {
                wgt = ck * tab[woff + own[i]];
              } else {
                const int gy = ty0 + oy, gx = tx0 + ox0 + i;
                const float fv = (gy < H && gx < W) ? __ldg(w.in + (long long)gy * pitch + gx) : 0.f;
                const float2 cs = term_cs_any((float)kp, fv, p);
                wgt = ck * (woff ? cs.y : cs.x);
              }
            }
            const float v = __uint_as_float(a[ii]);
            if (to_num) nm[i] = fmaf(wgt, v, nm[i]);
            else dn[i] = fmaf(wgt, v, dn[i]);
          }
        }
      }
      // ---- D1 -> B_v (rounded to the operand type) ------------------------------------
      {
        const uint32_t d1 = tmem + 192u * (uint32_t)(c % L) + ((uint32_t)(32 * q) << 16);
        constexpr int NJ = (C::NH / 8 + 3) / 4;   // chunks of 8 columns per warp
#pragma unroll
        for (int j0 = 0; j0 < NJ; j0 += 2) {      // two chunks per batch of TMEM loads
          uint32_t r[2][8];
#pragma unroll
          for (int jj = 0; jj < 2; ++jj) {
            const int j = cg + 4 * (j0 + jj);
            if (j0 + jj < NJ && j < C::NH / 8) tmem_ld8(d1 + 8 * j, r[jj]);
          }
          tmem_wait_ld();
#pragma unroll
          for (int jj = 0; jj < 2; ++jj) {
            const int j = cg + 4 * (j0 + jj);
            if (j0 + jj < NJ && j < C::NH / 8)
              *reinterpret_cast<uint4*>(sBv + core_off<KP>(32 * q + lane, 8 * j)) =
                  make_uint4(pack2<T>(__uint_as_float(r[jj][0]), __uint_as_float(r[jj][1])),
                             pack2<T>(__uint_as_float(r[jj][2]), __uint_as_float(r[jj][3])),
                             pack2<T>(__uint_as_float(r[jj][4]), __uint_as_float(r[jj][5])),
                             pack2<T>(__uint_as_float(r[jj][6]), __uint_as_float(r[jj][7])));
          }
        }
      }
      // table for the term of image c + L if it starts one
      if (c + L < nchan) {
        int kn, kindn, kl, kindl;
        chan_of(kb, c + L, &kn, &kindn);
        chan_of(kb, c + L - 1, &kl, &kindl);
        if (kn != kl && kn >= 1) build_tables(p, kn, sTab + (kn % 3) * 1024);
      }
      proxy_fence();
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      // ---- y pass of image c: D2 = G x B_v^T -----------------------------------------
      if (tid == 0) {
        const uint32_t aG = smem_u32(sG), aB = smem_u32(sBv);
#pragma unroll 1
        for (int ks = 0; ks < KP / 16; ++ks)
          mma_f16(tD2, op_desc<KP>(aG + ks * 256), op_desc<KP>(aB + ks * 256), idV, ks > 0);
        mma_commit(mbV);
      }
      // ---- generate image c + L while the tensor cores work ------------------------------
      if (c + L < nchan) {
        int kn, kindn;
        chan_of(kb, c + L, &kn, &kindn);
        generate_kind<RAD, T>(kindn, sBh + ((c + L) % C::NBH) * C::BHB, sFh, sTab + (kn % 3) * 1024,
                              tile_int, interior, tx0, ty0, H, W, w.in, pitch, kn, p);
        proxy_fence();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        issue_x(c + L, 0);
      }
    }
    // ---- fold the last image ---------------------------------------------------------------
    if (!abort) {
      if (!mbar_wait(mbV, phV)) abort = true;
      phV ^= 1;
      tc_fence_after();
    }
    if (__syncthreads_or(abort)) { abort = true; break; }
    {
      int kp, kindp;
      chan_of(kb, nchan - 1, &kp, &kindp);
      const float* tab = sTab + (kp % 3) * 1024;
      const float ck = p.c[kp];
      const bool to_num = (kindp == CH_FM || kindp == CH_FC || kindp == CH_FS);
      const int woff = (kindp == CH_S || kindp == CH_FS) ? 256 : 0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          uint32_t a[16];
          tmem_ld16(tD2 + ((uint32_t)(32 * q) << 16) + (uint32_t)(ox0 + 16 * h), a);
          tmem_wait_ld();
#pragma unroll
          for (int ii = 0; ii < 16; ++ii) {
            const int i = 16 * h + ii;
            float wgt = ck;
            if (kindp >= CH_C) {
              if (tile_int) {
                wgt = ck * tab[woff + own[i]];
              } else {
                const int gy = ty0 + oy, gx = tx0 + ox0 + i;
                const float fv = (gy < H && gx < W) ? __ldg(w.in + (long long)gy * pitch + gx) : 0.f;
                const float2 cs = term_cs_any((float)kp, fv, p);
                wgt = ck * (woff ? cs.y : cs.x);
              }
            }
            const float v = __uint_as_float(a[ii]);
            if (to_num) nm[i] = fmaf(wgt, v, nm[i]);
            else dn[i] = fmaf(wgt, v, dn[i]);
          }
        }
    }
    tc_fence_before();

    // ---- finish the tile (as in the FP32 kernel) --------------------------------------------
    bool finish = true;
    constexpr int PX = 32;
    if (!(kb == 0 && ke == K)) {
      const int wmine = term_start(ke) - term_start(kb);
      const int slot = (u_first / K == t) ? 0 : 1;
      float* pp = sc.partial + ((long long)(cta * 2 + slot) * 2) * PX * NTHREADS;
#pragma unroll
      for (int a = 0; a < PX; ++a) {
        pp[a * NTHREADS + tid] = nm[a];
        pp[(PX + a) * NTHREADS + tid] = dn[a];
      }
      __threadfence();
      __syncthreads();
      if (tid == 0) {
        const int prev = atomicAdd(sc.counter + t, wmine);
        sFlags[1] = (prev + wmine == w.wtile);
      }
      __syncthreads();
      finish = sFlags[1] != 0;
      if (finish) {
        __threadfence();
        const long long g0 = t * w.wtile;
        const long long c0 = g0 * G / sc.wtot;
        const long long c1 = (g0 + term_start(K - 1)) * G / sc.wtot;
#pragma unroll
        for (int a = 0; a < PX; ++a) { nm[a] = 0.f; dn[a] = 0.f; }
        for (long long cc = c0; cc <= c1; ++cc) {
          int fi, gi;
          long long fu, gu;
          locate(src, ceil_div_ll(cc * sc.wtot, G), sc.wtot, fi, fu);
          locate(src, ceil_div_ll((cc + 1) * sc.wtot, G), sc.wtot, gi, gu);
          if (!(fi < gi || (fi == gi && fu < gu))) continue;
          const int sl = (fu / K == t) ? 0 : 1;
          const float* qp = sc.partial + ((cc * 2 + sl) * 2) * PX * NTHREADS;
#pragma unroll
          for (int a = 0; a < PX; ++a) {
            nm[a] += __ldcg(qp + a * NTHREADS + tid);
            dn[a] += __ldcg(qp + (PX + a) * NTHREADS + tid);
          }
        }
        if (tid == 0) sc.counter[t] = 0;
      }
    }
    if (finish) {
      const int gy = ty0 + oy;
      if (gy < H) {
#pragma unroll
        for (int a = 0; a < PX; ++a) {
          const int gx = tx0 + ox0 + a;
          if (gx < W) {
            const float d = dn[a];
            const float f = __ldg(w.in + (long long)gy * pitch + gx);
            w.out[(long long)gy * pitch + gx] = (d > 0.f) ? m + nm[a] / d : f;
          }
        }
      }
    }
    u = t * K + ke;
    if (u >= w.tiles * K) { ++img; u = 0; }
    __syncthreads();
  }

  if (abort && lane == 0) atomicOr(&g_tc_error, 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" :: "r"(tmem));
}

template <int RAD, typename T>
int launch_rad(const DeviceParams& dp, const float* in, float* out, int H, int W, size_t pitch,
               cudaStream_t st) {
  using C = TcCfg<RAD>;
  static int occ[64] = {0};
  static int sms[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_filter: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= 64) return set_error(FBF_EUNSUPPORTED, "fbf_filter: device index >= 64");
  if (!occ[dev]) {
    e = cudaFuncSetAttribute(fbf_tc_kernel<RAD, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_filter: ") + cudaGetErrorString(e));
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fbf_tc_kernel<RAD, T>, NTHREADS, C::SMEM);
    if (e != cudaSuccess || n != 1)
      return set_error(FBF_ECUDA, "fbf_filter: tensor-core kernel needs exactly one CTA per SM");
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
  Work w{};
  w.in = in;
  w.out = out;
  w.pitch = (long long)pitch;
  w.H = H;
  w.W = W;
  w.tiles_x = (W + TT - 1) / TT;
  w.tiles_y = (H + TT - 1) / TT;
  w.K = dp.K;
  w.wtile = 2 * dp.K - 1;
  w.tiles = (long long)w.tiles_x * w.tiles_y;
  Scratch sc{};
  sc.wtot = w.tiles * w.wtile;
  long long G = sms[dev];
  if (G > sc.wtot) G = sc.wtot;
  const size_t partial_bytes = (size_t)G * 2 * 2 * 32 * NTHREADS * sizeof(float);
  int rc = get_workspace(dev, st, partial_bytes, (size_t)w.tiles, &sc.partial, &sc.counter);
  if (rc != FBF_OK) return rc;
  fbf_tc_kernel<RAD, T><<<(unsigned)G, NTHREADS, C::SMEM, st>>>(p, w, sc);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_filter: launch: ") + cudaGetErrorString(e));
  return FBF_OK;
}

template <typename T>
int launch_type(const DeviceParams& dp, const float* in, float* out, int H, int W, size_t pitch,
                cudaStream_t st) {
  const int r = dp.r;
  if (r <= 6) return launch_rad<6, T>(dp, in, out, H, W, pitch, st);
  if (r <= 15) return launch_rad<15, T>(dp, in, out, H, W, pitch, st);
  if (r <= 30) return launch_rad<30, T>(dp, in, out, H, W, pitch, st);
  return set_error(FBF_EUNSUPPORTED, "fbf_filter: the tensor-core forms support r = ceil(3 theta) <= 30");
}

}  // namespace tc

int launch_tc(const DeviceParams& dp, const float* in, float* out, int H, int W, size_t pitch,
              void* stream, int precision) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (precision == FBF_BF16_TC) return tc::launch_type<__nv_bfloat16>(dp, in, out, H, W, pitch, st);
  return tc::launch_type<__half>(dp, in, out, H, W, pitch, st);
}

int device_errors(int* flags, int clear) {
  int v = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, tc::g_tc_error, sizeof(int));
  if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_device_errors: ") + cudaGetErrorString(e));
  if (clear) {
    const int z = 0;
    e = cudaMemcpyToSymbol(tc::g_tc_error, &z, sizeof(int));
    if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_device_errors: ") + cudaGetErrorString(e));
  }
  *flags = v;
  return FBF_OK;
}

}  // namespace fbf
