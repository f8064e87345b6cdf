// Shared by the single-image and batched launchers: the FP32 fused Fourier bilateral
// filter kernel body (see fbf_fp32.cu for the description of the method and schedule).
#pragma once
#include <cuda.h>   // CUtensorMap (the type only; maps are encoded on the host)
#include <cuda_runtime.h>

#include "fbf_internal.h"

namespace fbf {
namespace fp32 {

constexpr int TX = 32;                 // tile width
constexpr int NXH = 8;                 // x outputs per lane in the x pass
constexpr float kOutside = -3.0e38f;   // marks halo pixels outside the image
constexpr int TABN = 256;              // per-term (cos, sin) table over integer intensities

// Split-tile hand-off: every thread of the block has stored its partial sums and passed a
// block barrier; one thread then adds the block's weight to the tile counter with a
// GPU-scope acquire-release atomic.  Release (cumulative through the barrier) publishes the
// whole block's partials; acquire makes every earlier contributor's partials visible to the
// block once the following barrier is passed.  Returns the counter's previous value.
__device__ __forceinline__ int counter_add_acq_rel(int* counter, int v) {
  int old;
  asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(counter), "r"(v) : "memory");
  return old;
}

// ---- TMA helpers (f-halo staging) ----------------------------------------------------------
// Bounded wait: each poll may suspend the thread for up to kTmaSuspendNs (woken early when the
// phase completes); gives up (false) after kTmaWaitLimit polls or kTmaWaitNs of wall time.
constexpr uint32_t kTmaSuspendNs = 1000000;
constexpr unsigned long long kTmaWaitNs = 2000000000ull;
constexpr int kTmaWaitLimit = 1 << 22;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void tma_bar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(bar)) : "memory");
}
// Load the box at (x, y) of `map` into dst and have it complete phase of `bar` (bytes = box size,
// elements outside the image included: they arrive as NaN).
__device__ __forceinline__ void tma_load_box(float* dst, const CUtensorMap* map, int x, int y,
                                             unsigned long long* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
               :: "r"(smem_addr(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
               " [%0], [%1, {%2, %3}], [%4];"
               :: "r"(smem_addr(dst)), "l"(map), "r"(x), "r"(y), "r"(smem_addr(bar)) : "memory");
}
// L2 policies for the carried rows: a slot is rewritten one tile later, so its lines are
// kept in L2 ahead of streaming data (evict_last); a slot read for the last time is marked
// evict_first and its lines discarded (dead data is not written back to DRAM).
__device__ __forceinline__ unsigned long long l2_policy_keep() {
  unsigned long long pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ unsigned long long l2_policy_drop() {
  unsigned long long pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
// 16-byte asynchronous copy global -> shared with an L2 policy (completed by cp.async.wait_all)
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc, unsigned long long pol) {
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;"
               :: "r"(smem_addr(smem_dst)), "l"(gsrc), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_global_v4(void* p, float4 v, unsigned long long pol) {
  asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;"
               :: "l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "l"(pol) : "memory");
}
// invalidate the 128-byte L2 line at p (its contents become undefined; nothing is written back)
__device__ __forceinline__ void l2_discard_line(const void* p) {
  asm volatile("discard.global.L2 [%0], 128;" :: "l"(p) : "memory");
}
__device__ __forceinline__ bool tma_bar_wait(unsigned long long* bar, uint32_t parity, int polls = 0) {
  const uint32_t a = smem_addr(bar);
  if (polls > 0) {   // test hook: that many non-blocking polls
    for (int it = 0; it < polls; ++it) {
      uint32_t done;
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
          " selp.u32 %0, 1, 0, p;\n}"
          : "=r"(done) : "r"(a), "r"(parity) : "memory");
      if (done) return true;
    }
    return false;
  }
  unsigned long long t0 = 0;
  for (int it = 0; it < kTmaWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done) : "r"(a), "r"(parity), "r"(kTmaSuspendNs) : "memory");
    if (done) return true;
    if ((it & 15) == 0) {
      unsigned long long now;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
      if (it == 0) t0 = now;
      else if (now - t0 > kTmaWaitNs) return false;
    }
  }
  return false;
}

// Device error word of the FP32 kernels (bit 1: a TMA wait gave up; that launch's output is
// incomplete).  Each translation unit has its own copy; the single-image launcher reads its own.
static __device__ int g_fp32_error;
// Test hook (fbf_debug_set_wait_limit): > 0 makes the wait for a tile's TMA box give up after
// that many non-blocking polls (the wait for the copy in flight before leaving keeps its full
// limit); 0 = normal limits.  Per translation unit, like the error word.
static __device__ int g_fp32_wait_polls;

// largest divisor of rows_per_warp whose group keeps at most 24 loads per lane in flight
__host__ __device__ constexpr int stage_group(int rows_per_warp, int cols_per_lane) {
  int g = 24 / cols_per_lane;
  if (g < 1) g = 1;
  while (g > 1 && rows_per_warp % g != 0) --g;
  return g;
}

template <int RAD, int TY, int NT, int NY>
struct Cfg {
  static constexpr int NW = NT / 32;                       // warps
  static constexpr int HROWS = TY + 2 * RAD;               // rows of the x-pass output
  // x-pass buffer rows: HROWS in whole 8-row groups (the k = 0 term convolves 8 rows per
  // warp step; the last round of either term may leave warps idle); staged f rows: that, in
  // whole rows per warp
  static constexpr int XB = (HROWS + 7) / 8 * 8;
  static constexpr int HROWS_P = (XB + NW - 1) / NW * NW;
  static constexpr int TXH = TX + 2 * RAD;                 // halo tile width
  static constexpr int FHS = TXH + 1;                      // f-halo row stride (floats)
  static constexpr int NQ2 = (NXH + 2 * RAD + 1) / 2;      // 16-byte loads per x-pass item
  static constexpr int SWP0 = 3 * NXH + 2 * NQ2;           // float2 slots read per stage row
  static constexpr int SWP = SWP0 + ((2 - SWP0 % 16) + 16) % 16;   // == 2 (mod 16)
  static constexpr int STAGE_F2 = 8 * SWP;                 // per warp: 4 rows x 2 pairs
  static constexpr int HS2 = TX + 2;                       // x-pass buffer row stride (float2)
  static constexpr int CPS0 = XB * HS2;
  static constexpr int CPS = CPS0 + ((4 - CPS0 % 16) + 16) % 16;  // pair stride, == 4 (mod 16)
  // f-halo staging: rows per warp, columns per lane, rows per group of loads in flight
  static constexpr int STAGE_RPW = HROWS_P / NW;
  static constexpr int STAGE_CPL = (TXH + 31) / 32;
  static constexpr int STAGE_RG = stage_group(STAGE_RPW, STAGE_CPL);
  static constexpr size_t SMEM_BYTES =
      (size_t)(NW * STAGE_F2 + 2 * CPS + 2 * TABN) * 8 + (size_t)HROWS_P * FHS * 4 + 16;
  // TMA staging of the f halo (single-image launches): a box of TMA_BW x HROWS_P floats whose
  // first column, tx0 - TMA_RX, is 16-byte aligned (tx0 is a multiple of 32); two buffers
  // (the next tile's box is loaded during the current tile), 128-byte aligned.
  static constexpr int TMA_RX = (RAD + 3) / 4 * 4;
  static constexpr int TMA_OFF = TMA_RX - RAD;                     // halo column 0 in the box
  static constexpr int TMA_BW = (TXH + TMA_OFF + 3) / 4 * 4;       // box width = row stride
  static constexpr int TMA_FH = HROWS_P * TMA_BW;                  // floats per buffer
  static constexpr size_t TMA_SMEM_BYTES =
      128 + (size_t)2 * TMA_FH * 4 + (size_t)(NW * STAGE_F2 + 2 * CPS + 2 * TABN) * 8 + 16;
  static constexpr bool TMA_OK = RAD <= 15 && TMA_BW <= 256 && HROWS_P <= 256 && TMA_SMEM_BYTES <= 232448;
  static_assert(TX * TY == NT * NY, "y-pass mapping: one column of NY pixels per thread");
  static_assert(HROWS_P % NW == 0, "f-halo staging: whole rows per warp");
  static_assert(TY % NY == 0 && (TY / NY) * 32 == NT, "y-pass mapping");
  static_assert(SMEM_BYTES <= 232448, "shared memory per CTA exceeds 227 KB");
};

// One image of a launch.  Units of work are (tile, term) pairs of weight 2 (k >= 1) or
// 1 (k = 0); the images of a launch form one weighted sequence, image after image.
struct Work {
  const float* in;
  float* out;
  long long pitch;                    // row stride in elements (in and out)
  int H, W, tiles_x, tiles_y;
  int K, wtile;                       // wtile = 2K - 1
  long long tiles;
  long long wstart;                   // weighted offset of the image's first unit
  int counter_base;                   // index of the image's first tile counter
  int param_idx;                      // index of the image's DeviceParams (work-lists)
  int row0;                           // image row of the first tile row (a band of rows)
  int row1;                           // image row past the last output row (<= H): a band's
                                      // last tile row may reach beyond it, writing nothing there
};

struct Scratch {
  long long wtot;                     // total weight of the launch
  float* partial;                     // G * 2 slots * 2 * NY * NT floats
  int* counter;                       // one per tile of every image, zero between launches
  float2* carry;                      // carried x-pass rows (carry sources): G * kmax slots
  int kmax;                           // largest K of the launch's images (carry slots per CTA)
};

// The spatial taps of a batched launch, in the constant bank (kernel parameter): all images
// of one launch share their Gaussian, so the multiply-adds of both passes take their taps
// from the constant bank as the single-image kernels do, not from per-image loads.
struct SpatialTaps {
  float g[2 * FBF_MAX_RADIUS + 1];
};

// A single image whose parameters sit in the constant bank (kernel parameter).
struct SingleSrc {
  static constexpr bool kTma = false;
  static constexpr bool kCarry = false;
  const DeviceParams* p;
  Work w;
  __device__ __forceinline__ int count() const { return 1; }
  __device__ __forceinline__ Work work(int) const { return w; }
  __device__ __forceinline__ const DeviceParams& params(int) const { return *p; }
  __device__ __forceinline__ const DeviceParams& taps(const DeviceParams& q) const { return q; }
  __device__ __forceinline__ int find(long long) const { return 0; }
};

// A single image whose f halo tiles are fetched by TMA through `map` (a kernel parameter
// encoded on the host: FP32, dims {W, H}, row stride pitch, box {TMA_BW, HROWS_P}, NaN for
// elements outside the image).
struct SingleSrcTma {
  static constexpr bool kTma = true;
  static constexpr bool kCarry = false;
  const DeviceParams* p;
  Work w;
  const CUtensorMap* map;
  __device__ __forceinline__ int count() const { return 1; }
  __device__ __forceinline__ Work work(int) const { return w; }
  __device__ __forceinline__ const DeviceParams& params(int) const { return *p; }
  __device__ __forceinline__ const DeviceParams& taps(const DeviceParams& q) const { return q; }
  __device__ __forceinline__ int find(long long) const { return 0; }
};

// A single image filtered strip by strip with the x-pass halo carried down each strip.
// Tiles are numbered column-major (tile t is row t % tiles_y of strip t / tiles_y), so the
// tiles of a CTA's range walk down a strip.  The y pass of a tile needs the x-pass rows
// [0, 2r) of its buffer, which are rows [TY, TY + 2r) of the tile above: when the CTA
// filtered term k of the tile above, it left those rows in its carry slot (sc.carry) and the
// tile reloads them instead of convolving them again, so the x pass covers TY new rows per
// tile instead of TY + 2r.  A tile at the top of a strip or at the start of the CTA's range
// (or a term the CTA did not filter for the tile above) convolves all its rows.
struct SingleSrcCarry {
  static constexpr bool kTma = false;
  static constexpr bool kCarry = true;
  const DeviceParams* p;
  Work w;
  __device__ __forceinline__ int count() const { return 1; }
  __device__ __forceinline__ Work work(int) const { return w; }
  __device__ __forceinline__ const DeviceParams& params(int) const { return *p; }
  __device__ __forceinline__ const DeviceParams& taps(const DeviceParams& q) const { return q; }
  __device__ __forceinline__ int find(long long) const { return 0; }
};

// rows of the x-pass buffer a tile can take over from the tile above: the largest multiple
// of the row-group height (4 rows for k >= 1, 8 for k = 0) not above 2r
__host__ __device__ constexpr int carry_rows(int rad, int group) { return (2 * rad) / group * group; }

// whether carrying rows saves a whole x-pass round of a tile (4 rows per warp and round for
// k >= 1): the configurations for which the carried-row kernels are instantiated
__host__ __device__ constexpr bool carry_saves_round(int rad, int ty, int nt) {
  return ((ty + 2 * rad + 3) / 4 * 4 - carry_rows(rad, 4) + 4 * (nt / 32) - 1) / (4 * (nt / 32)) <
         ((ty + 2 * rad + 3) / 4 * 4 + 4 * (nt / 32) - 1) / (4 * (nt / 32));
}

// A device work-list of images (batched launch); with CARRY, each image's tiles are numbered
// down its strips and x-pass rows are carried as for SingleSrcCarry, within one image.
template <bool CARRY = false>
struct ListSrcT {
  static constexpr bool kTma = false;
  static constexpr bool kCarry = CARRY;
  const DeviceParams* __restrict__ prm;
  const Work* __restrict__ wl;
  int n;
  const SpatialTaps* tp;   // the launch's taps (every image of the list has them)
  __device__ __forceinline__ int count() const { return n; }
  __device__ __forceinline__ Work work(int i) const { return wl[i]; }
  __device__ __forceinline__ const DeviceParams& params(int i) const { return prm[wl[i].param_idx]; }
  __device__ __forceinline__ const SpatialTaps& taps(const DeviceParams&) const { return *tp; }
  // last image whose weighted start is <= s
  __device__ __forceinline__ int find(long long s) const {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (wl[mid].wstart <= s) lo = mid; else hi = mid - 1;
    }
    return lo;
  }
};
using ListSrc = ListSrcT<false>;

__device__ __forceinline__ long long ceil_div_ll(long long a, long long b) { return (a + b - 1) / b; }

// weighted start of term k within a tile (k = 0 weighs 1, k >= 1 weighs 2)
__device__ __forceinline__ int term_start(int k) { return k == 0 ? 0 : 2 * k - 1; }

// first term of an image whose weighted start is >= s (image-local index tile*K + k)
__device__ __forceinline__ long long first_term_at(long long s, int K, int wtile) {
  long long t = s / wtile;
  long long rem = s - t * wtile;
  int k = (rem == 0) ? 0 : (int)((rem + 2) / 2);   // smallest k >= 1 with 2k-1 >= rem
  if (k >= K) { ++t; k = 0; }
  return t * K + k;
}

// first unit of the launch whose weighted start is >= s: image i, image-local unit u
// (i == src.count() past the end)
template <class Src>
__device__ __forceinline__ void locate(const Src& src, long long s, long long wtot, int& i,
                                       long long& u) {
  if (s >= wtot) { i = src.count(); u = 0; return; }
  i = src.find(s);
  const Work w = src.work(i);
  u = first_term_at(s - w.wstart, w.K, w.wtile);
  if (u >= w.tiles * w.K) { ++i; u = 0; }
}

// The partial-sum slot that CTA cc (of G, weighted range [ceil(cc wtot / G),
// ceil((cc + 1) wtot / G))) wrote for tile t of image img: 0 when t is the first tile its
// range reaches, 1 when t is its last, -1 when no unit of t starts in its range.  cc is one
// of the CTAs whose range meets the tile's units (c0 <= cc <= c1 of the finisher).  The
// tensor-core kernel's finisher evaluates it one contributor per lane.
template <class Src>
__device__ __forceinline__ int contributor_slot(const Src& src, long long cc, long long G, long long wtot,
                                                int img, long long t, int K) {
  int fi, gi;
  long long fu, gu;
  locate(src, ceil_div_ll(cc * wtot, G), wtot, fi, fu);
  locate(src, ceil_div_ll((cc + 1) * wtot, G), wtot, gi, gu);
  if (!(fi < gi || (fi == gi && fu < gu))) return -1;
  return (fi == img && fu / K == t) ? 0 : 1;
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
template <int RAD, class TP>
__device__ __forceinline__ float2 tap2(const TP& p, int d) {
  const float g = p.g[d <= RAD ? d : 2 * RAD - d];
  return make_float2(g, g);
}

// x pass of one item: 8 consecutive outputs of one float2 image pair in one row.
template <int RAD, class TP>
__device__ __forceinline__ void xconv8(const float2* __restrict__ srow, const TP& p,
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

template <int RAD, int TY, int NT, int NY, class Src>
__device__ __forceinline__ void fbf_body(const Src& src, const Scratch& sc) {
  using C = Cfg<RAD, TY, NT, NY>;
  constexpr bool TMA = Src::kTma;
  static_assert(!TMA || C::TMA_OK, "TMA staging does not fit this configuration");
  // carried x-pass rows (SingleSrcCarry): rows [0, CS) of a term's buffer come from the tile
  // above, rows [CS, XR) are convolved; CSLOT float2 per (CTA, term) slot
  constexpr bool CARRY = Src::kCarry;
  static_assert(!(TMA && CARRY), "carried tiles take the plain f staging");
  constexpr int CS1 = carry_rows(RAD, 4), CS0 = carry_rows(RAD, 8);
  constexpr int XR4 = (C::HROWS + 3) / 4 * 4, XR8 = (C::HROWS + 7) / 8 * 8;
  constexpr int CSLOT = 2 * CS1 * TX;
  static_assert(XR8 == C::XB && XR8 <= C::HROWS_P && TY + CS1 <= C::HROWS, "carried rows must lie inside the buffer");
  constexpr int FS = TMA ? C::TMA_BW : C::FHS;        // f-halo row stride (floats)
  extern __shared__ float4 smem_f4[];
  // TMA: two f buffers first (128-byte aligned), then the plain path's layout without its f.
  // The alignment is a byte offset added to the shared array itself, so every pointer below
  // stays a known shared-memory pointer (shared loads and stores, not generic ones).
  float* fhb = reinterpret_cast<float*>(reinterpret_cast<char*>(smem_f4) +
                                        ((128u - (smem_addr(smem_f4) & 127u)) & 127u));
  float2* smem2 = TMA ? reinterpret_cast<float2*>(fhb + 2 * C::TMA_FH) : reinterpret_cast<float2*>(smem_f4);
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  float2* stage = smem2 + warp * C::STAGE_F2;
  float2* hbuf = smem2 + C::NW * C::STAGE_F2;
  float2* tabs = hbuf + 2 * C::CPS;                    // two term tables (double buffer)
  float* fh = reinterpret_cast<float*>(tabs + 2 * TABN);     // TMA: set per tile
  unsigned long long* fbar = reinterpret_cast<unsigned long long*>(tabs + 2 * TABN);   // TMA
  __shared__ int s_last;

  const int G = gridDim.x;
  const int c = blockIdx.x;
  const long long Lc = ceil_div_ll((long long)c * sc.wtot, G);
  const long long Lc1 = ceil_div_ll((long long)(c + 1) * sc.wtot, G);
  int img, img_end, img_first;
  long long u, u_end, u_first;
  locate(src, Lc, sc.wtot, img, u);
  locate(src, Lc1, sc.wtot, img_end, u_end);
  img_first = img;
  u_first = u;

  // TMA: one mbarrier per f buffer; the first tile's box is requested at once, each later
  // one while the tile before it is filtered
  uint32_t fph = 0;   // phase parity to wait for, per buffer
  int fb = 0;         // buffer of the current tile
  const int wait_polls = TMA ? g_fp32_wait_polls : 0;
  if constexpr (TMA) {
    if (tid == 0) {
      tma_bar_init(fbar);
      tma_bar_init(fbar + 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0 && (img < img_end || (img == img_end && u < u_end))) {
      const Work w0 = src.work(img);
      const long long t0 = u / w0.K;
      tma_load_box(fhb, src.map, (int)(t0 % w0.tiles_x) * TX - C::TMA_RX, w0.row0 + (int)(t0 / w0.tiles_x) * TY - RAD,
                   fbar, C::TMA_FH * 4);
    }
  }

  // own pixels: one column of NY rows
  const int ox = lane;
  const int oy = warp * NY;
  // x-pass lane roles (bank-conflict-free 16-byte accesses within each quarter warp)
  const int x_cp = lane & 1, x_rlo = (lane >> 1) & 1, x_xlo = (lane >> 2) & 1;
  const int x_rhi = (lane >> 3) & 1, x_xhi = (lane >> 4) & 1;
  const int x_row4 = x_rhi * 2 + x_rlo;        // 0..3 (k >= 1)
  const int x_xg = x_xhi * 2 + x_xlo;          // 0..3
  const int x_row8 = x_row4 * 2 + x_cp;        // 0..7 (k == 0: eight rows, one pair)

  while (img < img_end || (img == img_end && u < u_end)) {
    const Work wk = src.work(img);
    const DeviceParams& p = src.params(img);
    const auto& pt = src.taps(p);   // the taps, in the constant bank
    const int K = wk.K;
    const int H = wk.H, W = wk.W;
    const long long pitch = wk.pitch;
    const float* __restrict__ in = wk.in;
    float* __restrict__ out = wk.out;
    const float m = p.center;
    const long long t = u / K;
    const int kb = (int)(u - t * K);
    const int ke = (img == img_end && t == u_end / K) ? (int)(u_end - t * K) : K;
    // tile coordinates: row-major, or column-major (strips) when rows are carried
    const int tyi = CARRY ? (int)(t % wk.tiles_y) : (int)(t / wk.tiles_x);
    const int tx0 = (int)(CARRY ? t / wk.tiles_y : t % wk.tiles_x) * TX;
    const int ty0 = wk.row0 + tyi * TY;

    // f of the tile plus halo (rows padded to whole x-pass rounds); kOutside marks
    // pixels outside the image.  The tile uses the term tables when all its values are
    // integers in [0, min(R, TABN-1)] (8-bit images), else the sincospi path.  Each warp
    // copies whole rows (coalesced); every load of a group of rows is issued before the
    // first store, so a tile costs one or two memory round trips, not one per row.
    const float vmax = (float)min(p.R, TABN - 1);
    int ok = 1;
    if constexpr (TMA) {
      // this tile's box was requested by the previous tile (or above); NaN marks outside pixels
      const uint32_t par = (fph >> fb) & 1u;
      const bool got = tma_bar_wait(fbar + fb, par, wait_polls);
      fph ^= 1u << fb;
      if (__syncthreads_or(!got)) {
        // gave up: record it, let the copy in flight land (bounded), and leave
        if (tid == 0) {
          atomicOr(&g_fp32_error, 2);
          tma_bar_wait(fbar + fb, par);
        }
        return;
      }
      fh = fhb + fb * C::TMA_FH + C::TMA_OFF;
      for (int row = warp; row < C::HROWS; row += C::NW) {
#pragma unroll
        for (int xx = lane; xx < C::TXH; xx += 32) {
          const float x = fh[row * FS + xx];
          if (x > kOutside) ok &= (x == rintf(x)) & (x >= 0.f) & (x <= vmax);
        }
      }
    } else {
      constexpr int CPL = C::STAGE_CPL, RPW = C::STAGE_RPW, RG = C::STAGE_RG;
      for (int g0 = 0; g0 < RPW; g0 += RG) {
        float v[RG][CPL];
#pragma unroll
        for (int a = 0; a < RG; ++a) {
          const int row = (g0 + a) * C::NW + warp;
          const int gy = ty0 - RAD + row;
          const bool rin = row < C::HROWS && gy >= 0 && gy < H;
          const float* __restrict__ src_row = in + (long long)(rin ? gy : 0) * pitch;
#pragma unroll
          for (int b = 0; b < CPL; ++b) {
            const int xx = lane + 32 * b;
            const int gx = tx0 - RAD + xx;
            v[a][b] = (rin && xx < C::TXH && gx >= 0 && gx < W) ? __ldg(src_row + gx) : kOutside;
          }
        }
#pragma unroll
        for (int a = 0; a < RG; ++a) {
          const int row = (g0 + a) * C::NW + warp;
#pragma unroll
          for (int b = 0; b < CPL; ++b) {
            const int xx = lane + 32 * b;
            if (xx < C::TXH) {
              const float x = v[a][b];
              if (x > kOutside) ok &= (x == rintf(x)) & (x >= 0.f) & (x <= vmax);
              fh[row * C::FHS + xx] = x;
            }
          }
        }
      }
    }
    // every halo pixel inside the image: generation needs no masking
    const bool interior = tx0 - RAD >= 0 && ty0 - RAD >= 0 && tx0 + TX + RAD <= W &&
                          ty0 + TY + RAD <= H;
    const bool tile_int = __syncthreads_and(ok) != 0;
    if constexpr (TMA) {
      // request the next tile's box into the other buffer, last read by the previous tile
      // (before the barrier that closed it)
      const long long un = t * K + ke;
      if (tid == 0 && un < wk.tiles * K && (img < img_end || un < u_end)) {
        const long long tn = un / K;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tma_load_box(fhb + (fb ^ 1) * C::TMA_FH, src.map, (int)(tn % wk.tiles_x) * TX - C::TMA_RX,
                     wk.row0 + (int)(tn / wk.tiles_x) * TY - RAD, fbar + (fb ^ 1), C::TMA_FH * 4);
      }
      fb ^= 1;
    }
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
      // carried rows: this CTA filtered term k of the tile above, whose buffer rows
      // [TY, TY + cs) are this tile's rows [0, cs); they are copied in while the new rows
      // are generated and convolved
      const int cs = (k == 0) ? CS0 : CS1;
      const int ncs = ((k == 0) ? 1 : 2) * cs * (TX / 2);   // 16-byte chunks
      const bool carried = CARRY && tyi > 0 && (img != img_first || (t - 1) * K + k >= u_first);
      // the tile below takes rows from this one when this CTA filters its term k too
      const bool keeps = CARRY && tyi + 1 < wk.tiles_y && (img < img_end || (t + 1) * K + k < u_end);
      float2* const slot = CARRY ? sc.carry + ((long long)c * sc.kmax + k) * CSLOT : nullptr;
      if (CARRY && carried) {
        const unsigned long long pol = keeps ? l2_policy_keep() : l2_policy_drop();
        for (int i = tid; i < ncs; i += NT) {
          const int cp = i / (cs * (TX / 2)), rem = i - cp * cs * (TX / 2);
          const int row = rem / (TX / 2), col = (rem - row * (TX / 2)) * 2;
          cp_async16(hbuf + cp * C::CPS + row * C::HS2 + col, slot + (cp * CS1 + row) * TX + col, pol);
        }
      }
      const int xr0 = carried ? cs : 0;
      if (k == 0) {
        // ---- term 0: pair (f - m, 1); eight halo rows per warp iteration -------------
        for (int rb = xr0 + warp * 8; rb < XR8; rb += C::NW * 8) {
#pragma unroll
          for (int r8 = 0; r8 < 8; ++r8) {
#pragma unroll
            for (int xx = lane; xx < C::TXH; xx += 32) {
              const float v = fh[(rb + r8) * FS + xx];
              stage[r8 * C::SWP + xx] = (v > kOutside) ? make_float2(v - m, 1.f) : make_float2(0.f, 0.f);
            }
          }
          __syncwarp();
          xconv8<RAD>(stage + x_row8 * C::SWP + x_xg * NXH, pt,
                      hbuf + (rb + x_row8) * C::HS2 + x_xg * NXH);
          __syncwarp();
        }
      } else {
        // ---- term k >= 1: pairs (C, S) and (f'C, f'S); four halo rows per iteration --
        const float2* tab = tabs + (k & 1) * TABN;
        for (int rb = xr0 + warp * 4; rb < XR4; rb += C::NW * 4) {
          if (tile_int && interior) {
#pragma unroll
            for (int r4 = 0; r4 < 4; ++r4) {
#pragma unroll
              for (int xx = lane; xx < C::TXH; xx += 32) {
                const float v = fh[(rb + r4) * FS + xx];
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
                const float v = fh[(rb + r4) * FS + xx];
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
                const float v = fh[(rb + r4) * FS + xx];
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
          xconv8<RAD>(stage + (x_row4 * 2 + x_cp) * C::SWP + x_xg * NXH, pt,
                      hbuf + x_cp * C::CPS + (rb + x_row4) * C::HS2 + x_xg * NXH);
          __syncwarp();
        }
      }
      if (CARRY && carried) asm volatile("cp.async.wait_all;" ::: "memory");
      __syncthreads();
      // rows [TY, TY + cs) are rows [0, cs) of the next tile of the strip: keep them for it
      // when this CTA filters its term k (same chunk per thread as the load above, so each
      // thread rereads only what it wrote itself)
      if (CARRY && keeps) {
        const unsigned long long pol = l2_policy_keep();
        for (int i = tid; i < ncs; i += NT) {
          const int cp = i / (cs * (TX / 2)), rem = i - cp * cs * (TX / 2);
          const int row = rem / (TX / 2), col = (rem - row * (TX / 2)) * 2;
          st_global_v4(slot + (cp * CS1 + row) * TX + col,
                       *reinterpret_cast<const float4*>(hbuf + cp * C::CPS + (TY + row) * C::HS2 + col), pol);
        }
      } else if (CARRY && carried) {
        // read for the last time (every thread's copies completed before the barrier above)
        for (int i = tid * 8; i < ncs; i += NT * 8) {
          const int cp = i / (cs * (TX / 2)), rem = i - cp * cs * (TX / 2);
          const int row = rem / (TX / 2), col = (rem - row * (TX / 2)) * 2;
          l2_discard_line(slot + (cp * CS1 + row) * TX + col);
        }
      }
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
          const float v = fh[(oy + a + RAD) * FS + ox + RAD];
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
            if (d >= 0 && d <= 2 * RAD) acc[a] = __ffma2_rn(tap2<RAD>(pt, d), v, acc[a]);
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
      const int slot = (img_first == img && u_first / K == t) ? 0 : 1;
      float* pp = sc.partial + ((long long)(c * 2 + slot) * 2) * NY * NT;
#pragma unroll
      for (int a = 0; a < NY; ++a) {
        pp[a * NT + tid] = num[a];
        pp[(NY + a) * NT + tid] = den[a];
      }
      __syncthreads();
      if (tid == 0) {
        const int prev = counter_add_acq_rel(sc.counter + wk.counter_base + t, wmine);
        s_last = (prev + wmine == wk.wtile);
      }
      __syncthreads();
      finish = s_last != 0;
      if (finish) {
        // sum the partials of all contributing CTAs in CTA (= term) order
        const long long g0 = wk.wstart + t * wk.wtile;
        const long long c0 = g0 * G / sc.wtot;
        const long long c1 = (g0 + term_start(K - 1)) * G / sc.wtot;
#pragma unroll
        for (int a = 0; a < NY; ++a) { num[a] = 0.f; den[a] = 0.f; }
        for (long long cc = c0; cc <= c1; ++cc) {
          int fi, gi;
          long long fu, gu;
          locate(src, ceil_div_ll(cc * sc.wtot, G), sc.wtot, fi, fu);
          locate(src, ceil_div_ll((cc + 1) * sc.wtot, G), sc.wtot, gi, gu);
          if (!(fi < gi || (fi == gi && fu < gu))) continue;  // no unit starts in this CTA's range
          const int sl = (fi == img && fu / K == t) ? 0 : 1;
          const float* qp = sc.partial + ((cc * 2 + sl) * 2) * NY * NT;
#pragma unroll
          for (int a = 0; a < NY; ++a) {
            num[a] += __ldcg(qp + a * NT + tid);
            den[a] += __ldcg(qp + (NY + a) * NT + tid);
          }
        }
        if (tid == 0) sc.counter[wk.counter_base + t] = 0;
      }
    }
    if (finish) {
#pragma unroll
      for (int a = 0; a < NY; ++a) {
        const int gy = ty0 + oy + a, gx = tx0 + ox;
        if (gy < wk.row1 && gx < W) {
          const float d = den[a];
          const float f = fh[(oy + a + RAD) * FS + ox + RAD];
          __stcs(out + (long)gy * pitch + gx, (d > 0.f) ? m + num[a] / d : f);   // streamed
        }
      }
    }
    u = t * K + ke;
    if (u >= wk.tiles * K) { ++img; u = 0; }
    __syncthreads();   // the f halo is rewritten by the next tile
  }
}

// One image, parameters in the constant bank.
template <int RAD, int TY, int NT, int NY>
__global__ void __launch_bounds__(NT, 1)
fbf_fp32_kernel(const __grid_constant__ DeviceParams p, const Work w, const Scratch sc) {
  const SingleSrc src{&p, w};
  fbf_body<RAD, TY, NT, NY>(src, sc);
}

// One image, parameters in the constant bank, f-halo tiles by TMA through `map`.
template <int RAD, int TY, int NT, int NY>
__global__ void __launch_bounds__(NT, 1)
fbf_fp32_tma_kernel(const __grid_constant__ DeviceParams p, const Work w, const Scratch sc,
                    const __grid_constant__ CUtensorMap map) {
  const SingleSrcTma src{&p, w, &map};
  fbf_body<RAD, TY, NT, NY>(src, sc);
}

// One image, parameters in the constant bank, x-pass halo rows carried down each strip.
template <int RAD, int TY, int NT, int NY>
__global__ void __launch_bounds__(NT, 1)
fbf_fp32_carry_kernel(const __grid_constant__ DeviceParams p, const Work w, const Scratch sc) {
  const SingleSrcCarry src{&p, w};
  fbf_body<RAD, TY, NT, NY>(src, sc);
}

// A device work-list of images sharing one radius class and one spatial kernel (batched
// launch).
template <int RAD, int TY, int NT, int NY>
__global__ void __launch_bounds__(NT, 1)
fbf_fp32_batch_kernel(const DeviceParams* __restrict__ params, const Work* __restrict__ work,
                      int n, const Scratch sc, const __grid_constant__ SpatialTaps taps) {
  const ListSrc src{params, work, n, &taps};
  fbf_body<RAD, TY, NT, NY>(src, sc);
}


// A device work-list of images sharing one radius class and one spatial kernel, x-pass rows
// carried down each strip.
template <int RAD, int TY, int NT, int NY>
__global__ void __launch_bounds__(NT, 1)
fbf_fp32_batch_carry_kernel(const DeviceParams* __restrict__ params, const Work* __restrict__ work,
                            int n, const Scratch sc, const __grid_constant__ SpatialTaps taps) {
  const ListSrcT<true> src{params, work, n, &taps};
  fbf_body<RAD, TY, NT, NY>(src, sc);
}

// padded copy of a plan's parameters for the RAD instantiation (taps beyond the plan's
// radius are zero, so a wider instantiation serves a smaller r)
template <int RAD>
inline DeviceParams pad_params(const DeviceParams& dp) {
  DeviceParams p = dp;
  float g[2 * FBF_MAX_RADIUS + 1];
  for (int i = 0; i <= 2 * RAD; ++i) {
    const int d = i - (RAD - dp.r);
    g[i] = (d >= 0 && d <= 2 * dp.r) ? dp.g[d] : 0.f;
  }
  for (int i = 0; i <= 2 * RAD; ++i) p.g[i] = g[i];
  p.r = RAD;
  return p;
}

}  // namespace fp32
}  // namespace fbf
