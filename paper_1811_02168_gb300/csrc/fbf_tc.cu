// Tensor-core forms of the fused Fourier bilateral filter (FBF_FP16_TC, FBF_BF16_TC).
//
// Same method and schedule as the FP32 kernel (see fbf_fp32.cu): eq. (1) with phi_hat of
// eq. (3) through Gaussian convolutions of cos(k nu f), sin(k nu f), (f-m)cos, (f-m)sin
// (Section II), stream-K over weighted (tile, term) units, partial sums finished by the
// last contributing CTA.  Here each separable Gaussian pass is a dense contraction on the
// 5th-generation tensor cores.  With a 128 (x) by 64 (y) output tile, an r-pixel halo,
// KX = 128 + 2r and KY = 64 + 2r, both rounded up to 16:
//   x pass:  D1[x', hy] = sum_hx Gx[x', hx] B_h[hy, hx]   M = 128, N = KY, K = KX   (FP16/BF16)
//   y pass:  D2[x', y'] = sum_hy D1[x', hy] Gy[y', hy]    M = 128, N = 64, K = KY   (TF32)
// where Gx[o, i] = Gy[o, i] = g(i - o - r) hold the 2r+1 Gaussian taps as banded Toeplitz
// matrices and B_h holds one convolved image over the tile plus halo.  Gx and B_h are FP16
// or BF16 in shared memory; the x-pass accumulator D1 stays in tensor memory (TMEM) in FP32
// and is read there, as TF32, by the y pass (TMEM lane = output column x' = the y pass's M
// row), so nothing is copied between the passes.  Gy is TF32 in shared memory.
//
// The eight images of a term come in pairs that share a table entry and a fold weight:
// (1, f-m) for k = 0, (cos, (f-m)cos) and (sin, (f-m)sin) for k >= 1.  A pair is generated in
// one sweep (one packed table entry gives both operand values of a pixel) into two B_h
// buffers, convolved into two D1 and two D2 accumulators, and folded with one weight per
// pixel: den += w D2[first], num += w D2[second], w = c_0, c_k cos(k nu f_i) or
// c_k sin(k nu f_i).
//
// Roles: 16 compute warps build tables, generate pairs and fold; one more warp issues the
// tcgen05.mma instructions from a single thread.  They hand buffers over with mbarriers:
//   full   (16 warp arrivals)   pair P generated           -> x pass may start
//   xdone  (tcgen05.commit)     x pass of P complete        -> B_h reusable, y pass may start
//   ydone  (tcgen05.commit)     y pass of P complete        -> D2 readable, D1 reusable
//   fdone  (16 warp arrivals)   D2 of P folded              -> D2 reusable
// Every wait is bounded; a wait that gives up raises the CTA's abort flag, every role leaves
// its loop, the issuing thread drains its MMAs, and the CTA frees its TMEM before returning.
// The device error word (read with fbf_device_errors) records the abort.
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

using fp32::Work;
using fp32::Scratch;
using fp32::SingleSrc;
using fp32::ListSrc;
using fp32::ceil_div_ll;
using fp32::term_start;
using fp32::locate;
using fp32::term_cs_any;

__device__ int g_tc_error;   // bit 0: an mbarrier wait gave up
// Test hook (fbf_debug_set_wait_limit): > 0 makes the role waits give up after that many
// non-blocking polls (the final drain of the MMAs keeps its full limit); 0 = normal limits.
__device__ int g_tc_wait_polls;

constexpr int TILE_X = 128;             // output tile width  = TMEM lanes = MMA M
constexpr int TILE_Y_MAX = 64;          // output tile height = y-pass N (per configuration: TcCfg::TY)
constexpr int NCW = 16;                 // compute warps: 4 TMEM lane quarters x 4 row groups
constexpr int NCT = NCW * 32;           // compute threads
constexpr int NTHREADS = NCT + 32;      // + the MMA-issuing warp
constexpr int PX_MAX = TILE_Y_MAX / 4;  // output pixels per compute thread (one column)
constexpr int kWaitLimit = 1 << 22;

// FBF_BF16_TC stores every operand value and every x-pass tap as a compensated pair of BF16
// numbers (hi + lo, lo = the rounding error of hi); the x pass accumulates Gx_hi B_hi +
// Gx_hi B_lo + Gx_lo B_hi (the lo x lo product is below the FP32 accumulation error),
// which keeps about 16 significant bits.  FBF_FP16_TC stores one FP16 value per operand.
template <typename T>
struct Parts { static constexpr int value = std::is_same<T, __nv_bfloat16>::value ? 2 : 1; };

template <int RAD, int NPART>
struct TcCfg {
  static constexpr int HX = TILE_X + 2 * RAD;             // halo columns
  static constexpr int KX = (HX + 15) / 16 * 16;          // x-pass K
  static constexpr int TY = TILE_Y_MAX;
  // the compensated form at r > 15 keeps Gx in shared memory (the split x-pass result takes
  // its tensor-memory columns); its x pass then reads both operands from shared memory
  static constexpr bool GX_SMEM = NPART == 2 && RAD > 15;
  static constexpr int PX = TY / 4;                       // output pixels per compute thread
  static constexpr int HY = TY + 2 * RAD;                 // halo rows
  static constexpr int KY = (HY + 15) / 16 * 16;          // x-pass N = y-pass K
  static constexpr int GYB = TY * KY * 4;                 // Gy, TF32 (shared memory)
  static constexpr int GY16B = NPART == 2 ? TY * KY * 2 : 0;   // Gy, FP16: the lo part's y pass
  // Gx in shared memory is kept as one tall band: the x pass's A block of K-step s,
  // Gx[x', 16 s + j] = g(16 s + j - x'), is rows [16 (KS - 1 - s), +128) of
  // U[y, j] = g(j - y + 16 (KS - 1)), y < GXU rows (a banded Toeplitz matrix repeats itself
  // shifted by 16 rows per K-step), so the descriptor of step s starts 2 (KS - 1 - s) row
  // groups into U instead of a TILE_X x KX copy
  static constexpr int GXU = TILE_X + 16 * (KX / 16 - 1);          // rows of the band U
  static constexpr int GLB = NPART == 2 ? GXU * 16 * 2 : 0;       // Gx_lo band (shared memory)
  static constexpr int GXHB = GX_SMEM ? GXU * 16 * 2 : 0;         // Gx (hi) band in shared memory
  static constexpr int FHS = KX + 8;                      // f-halo row stride (bytes)
  static constexpr int FHB = (KY * FHS + 127) / 128 * 128;
  static constexpr int GENW = 256 * NPART;                // words of one pair's operand table
  static constexpr int TABW = 2 * GENW + 512;             // words per term-table slot
  static constexpr int TABB = 2 * TABW * 4;               // 2 slots (terms k even / odd)
  static constexpr int BARB = 256;
  static constexpr int FIXED = GYB + GY16B + GLB + GXHB + FHB + TABB + BARB + 1024;
  // B_h is produced as NC column chunks of CK x-pass K-steps (16 columns each) into a ring of
  // NSLOT chunk slots, each holding the chunk of both images of a pair (and of both parts of
  // the compensated form), with its own full / empty barriers: generation runs ahead of the
  // x pass by up to NSLOT chunks.  CK is the largest divisor of the K-step count that leaves
  // room for two slots: every chunk hand-off costs a round trip between the roles (the
  // compensated form at r = 30 at 4096^2: 1-, 2- and 3-K-step chunks with 7, 3 and 2 slots
  // took 3.89, 3.21 and 3.13 ms).
  static constexpr int KS = KX / 16;
  static constexpr int slot_bytes(int ck) { return 2 * NPART * KY * 16 * ck * 2; }
  static constexpr int pick_ck() {
    for (int ck = KS; ck > 1; --ck)
      if (KS % ck == 0 && (232448 - FIXED) / slot_bytes(ck) >= 2) return ck;
    return 1;
  }
  static constexpr int CK = pick_ck();
  static constexpr int NC = KS / CK;
  static constexpr int CW = 16 * CK;                      // chunk columns
  static constexpr int CB = KY * CW * 2;                  // bytes of one image part's chunk (16-bit)
  static constexpr int SLOTB = 2 * NPART * CB;            // a chunk slot: [a, b] per part
  static constexpr int NSLOT0 = (232448 - FIXED) / SLOTB;
  static constexpr int NSLOT = NSLOT0 < 2 * NC ? NSLOT0 : 2 * NC;
  static constexpr int SMEM = FIXED + NSLOT * SLOTB;
  // tensor memory: Gx (16-bit pairs, one column per two K elements), two x-pass and two
  // y-pass accumulators
  static constexpr int GXC = 0;
  static constexpr int GXS = GX_SMEM ? 0 : (KX / 2 + 31) / 32 * 32;
  static constexpr int D1S = (KY + 31) / 32 * 32;
  static constexpr int D1C = GXS;
  // compensated form: the x-pass result splits into hi (TF32, in place) + lo (FP16 pairs,
  // KY/2 columns per image) so that the y pass carries ~21 significant bits
  static constexpr int D1LS = NPART == 2 ? (KY / 2 + 15) / 16 * 16 : 0;
  static constexpr int D1LC = D1C + 2 * D1S;
  static constexpr int D2C = D1LC + 2 * D1LS;
  static_assert(D2C + 2 * TY <= 512, "TMEM columns");
  static_assert(NSLOT >= 1, "chunk ring");
  static_assert(SMEM <= 232448, "tensor-core tile does not fit in shared memory");
  static_assert(KY <= 256, "x-pass N exceeds one MMA");
  static_assert(NC * CK == KS, "chunking");
  static_assert(2 * NSLOT + 8 <= BARB / 8 - 2, "barrier space (then four ints: TMEM base, abort, finish, polls)");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of element (row, k) in a K-major no-swizzle operand of 16-bit elements with
// KP columns: 8-row x 16-byte core matrices, K-adjacent core matrices 128 bytes apart
template <int KP>
__device__ __forceinline__ int off16(int row, int k) {
  return ((row >> 3) * (KP >> 3) + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2;
}
// the same for 32-bit (TF32) elements: a core matrix row holds 4 elements
template <int KP>
__device__ __forceinline__ int off32(int row, int k) {
  return ((row >> 3) * (KP >> 2) + (k >> 2)) * 128 + (row & 7) * 16 + (k & 3) * 4;
}

// shared-memory matrix descriptor: K-major, no swizzle; LBO = 128 B (next core matrix
// along K), SBO = next 8-row group, version 1
__device__ __forceinline__ uint64_t op_desc(uint32_t saddr, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor: D FP32; A and B FP16 (0), BF16 (1) or TF32 (2); both K-major
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

template <typename T>
__device__ __forceinline__ float round16(float x);
template <>
__device__ __forceinline__ float round16<__half>(float x) { return __half2float(__float2half_rn(x)); }
template <>
__device__ __forceinline__ float round16<__nv_bfloat16>(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// operand words of one pixel of a pair (values a, b): the packed pair, and for the
// compensated form the packed pair of rounding errors
template <typename T, int NPART>
__device__ __forceinline__ uint2 pair_words(float a, float b) {
  uint2 r;
  r.x = pack2<T>(a, b);
  r.y = NPART == 2 ? pack2<T>(a - round16<T>(a), b - round16<T>(b)) : 0u;
  return r;
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// A and B from shared memory (x pass)
__device__ __forceinline__ void mma_ss(uint32_t dtmem, uint64_t da, uint64_t db, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
      :: "r"(dtmem), "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}
// The issuing warp runs converged (operands stay warp-uniform); one elected lane issues.
// A from tensor memory, B from shared memory, FP16/BF16 (x pass)
__device__ __forceinline__ void mma_ts_f16(uint32_t dtmem, uint32_t atmem, uint64_t db, uint32_t idesc,
                                           uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p, e;\n setp.ne.b32 p, %4, 0;\n elect.sync _|e, 0xffffffff;\n"
      " @e tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}"
      :: "r"(dtmem), "r"(atmem), "l"(db), "r"(idesc), "r"(accumulate));
}
// A from tensor memory, B from shared memory, TF32 (y pass)
__device__ __forceinline__ void mma_ts_tf32(uint32_t dtmem, uint32_t atmem, uint64_t db, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p, e;\n setp.ne.b32 p, %4, 0;\n elect.sync _|e, 0xffffffff;\n"
      " @e tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}"
      :: "r"(dtmem), "r"(atmem), "l"(db), "r"(idesc), "r"(accumulate));
}
// A and B from shared memory, FP16/BF16 (the Gx_lo term of the compensated x pass)
__device__ __forceinline__ void mma_ss_el(uint32_t dtmem, uint64_t da, uint64_t db, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p, e;\n setp.ne.b32 p, %4, 0;\n elect.sync _|e, 0xffffffff;\n"
      " @e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
      :: "r"(dtmem), "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit_el(uint64_t* mbar) {
  asm volatile("{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n"
               " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}"
               :: "r"(smem_u32(mbar)) : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :: "r"(smem_u32(mbar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}"
               :: "r"(smem_u32(mbar)) : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait for phase `parity` of an mbarrier.  Each poll is a try_wait without a
// suspend-time hint (the hardware's own short limit; measured 3% faster on 4096^2 than
// polls that may suspend the thread for up to 1 ms).  Gives up (false) after kWaitLimit
// polls or kWaitNs of wall time, or early once the CTA's abort flag is raised (when `flag`
// is given: flag[0] the abort flag, flag[2] the test hook's poll limit, which turns the wait
// into that many non-blocking polls).
constexpr uint64_t kWaitNs = 2000000000ull;
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, const volatile int* flag) {
  const uint32_t a = smem_u32(mbar);
  if (flag && flag[2] > 0) {
    for (int it = 0; it < flag[2]; ++it) {
      uint32_t done;
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
          " selp.u32 %0, 1, 0, p;\n}"
          : "=r"(done) : "r"(a), "r"(parity) : "memory");
      if (done) return true;
    }
    return false;
  }
  uint64_t t0 = 0;
  for (int it = 0; it < kWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done) : "r"(a), "r"(parity) : "memory");
    if (done) return true;
    if ((it & 7) == 7 && flag && *flag) return false;
    if ((it & 15) == 0) {
      const uint64_t now = global_ns();
      if (it == 0) t0 = now;
      else if (now - t0 > kWaitNs) return false;
    }
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
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
               :: "r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]),
                  "r"(r[7]) : "memory");
}
__device__ __forceinline__ void tmem_st4(uint32_t taddr, const uint32_t (&r)[4]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};"
               :: "r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]) : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// barrier 1 over the compute warps only (the MMA warp never takes part)
__device__ __forceinline__ void sync_compute() { asm volatile("bar.sync 1, %0;" :: "n"(NCT) : "memory"); }
__device__ __forceinline__ bool sync_compute_or(bool v) {
  int r;
  asm volatile("{\n .reg .pred p, q;\n setp.ne.b32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n"
               " selp.s32 %0, 1, 0, q;\n}" : "=r"(r) : "r"((int)v), "n"(NCT) : "memory");
  return r != 0;
}
__device__ __forceinline__ bool sync_compute_and(bool v) {
  int r;
  asm volatile("{\n .reg .pred p, q;\n setp.ne.b32 p, %1, 0;\n bar.red.and.pred q, 1, %2, p;\n"
               " selp.s32 %0, 1, 0, q;\n}" : "=r"(r) : "r"((int)v), "n"(NCT) : "memory");
  return r != 0;
}

// Pairs of a tile in processing order: tile pair index gp = 0 is k = 0 (1, f-m); then per
// term k >= 1 the cos pair (gp = 2k - 1) and the sin pair (gp = 2k).  A (tile, term)
// fragment [kb, ke) has 2 ke - 1 pairs when kb = 0, else 2 (ke - kb).
__device__ __forceinline__ int frag_pairs(int kb, int ke) { return kb == 0 ? 2 * ke - 1 : 2 * (ke - kb); }
__device__ __forceinline__ void pair_of(int kb, int j, int* k, int* kind) {
  const int gp = (kb == 0) ? j : 2 * kb - 1 + j;
  *k = (gp + 1) >> 1;
  *kind = gp == 0 ? 0 : 1 + ((gp - 1) & 1);   // 0: (1, f-m), 1: cos, 2: sin
}

// Term-table slot over integer intensities v = 0..255: [0, GENW) the cos pair's operand
// words (the two values packed, first in the low half; for the compensated form followed
// by the packed rounding errors), [GENW, 2 GENW) the sin pair's, then the two fold weight
// tables (FP32 bits).  For k = 0 only the cos parts are used, holding the pair (1, f - m)
// and the weight c_0.  One sincospif per entry serves both pairs.
template <typename T, int NPART>
__device__ __forceinline__ void build_term_table(const DeviceParams& p, int k, uint32_t* slot, int ctid) {
  constexpr int GENW = 256 * NPART;
  const int v = ctid & 255;
  const float fm = (float)v - p.center;
  float cs = 1.f, sn = 0.f;
  if (k != 0) {
    // phase index n = (k v) mod P, exact: k v < 2^24 and the float quotient is corrected
    const int x = k * v;
    int n = x - (int)floorf((float)x * p.invP) * p.P;
    n += n < 0 ? p.P : 0;
    n -= n >= p.P ? p.P : 0;
    sincospif(2.0f * (float)n * p.invP, &sn, &cs);   // 2 n / P within one ulp
  }
  if (ctid < 256) {
    const uint2 wc = pair_words<T, NPART>(cs, fm * cs), ws = pair_words<T, NPART>(sn, fm * sn);
    if (NPART == 1) {
      slot[v] = wc.x;
      slot[GENW + v] = ws.x;
    } else {
      reinterpret_cast<uint2*>(slot)[v] = wc;
      reinterpret_cast<uint2*>(slot + GENW)[v] = ws;
    }
  } else {
    const float ck = p.c[k];
    slot[2 * GENW + v] = __float_as_uint(ck * cs);
    slot[2 * GENW + 256 + v] = __float_as_uint(ck * sn);
  }
}

// General (non-integer or out-of-table) values, one pixel at a time.  Kept out of line so
// the table paths stay small in the instruction cache.
template <typename T, int NPART>
__device__ __noinline__ void gen_item_slow(unsigned char* dst, int cb, int off, int hy, int hx0, int HY, int HX,
                                           int gy0, int gx0, int H, int W, const float* __restrict__ in,
                                           long long pitch, int k, int kind, const DeviceParams& p) {
  const int gy = gy0 + hy;
  for (int j = 0; j < 8; ++j) {
    const int hx = hx0 + j, gx = gx0 + hx;
    float a = 0.f, fm = 0.f;
    if (hy < HY && hx < HX && gy >= 0 && gy < H && gx >= 0 && gx < W) {
      const float fv = __ldg(in + (long long)gy * pitch + gx);
      fm = fv - p.center;
      a = 1.f;
      if (kind != 0) {
        const float2 cs = term_cs_any((float)k, fv, p);
        a = kind == 1 ? cs.x : cs.y;
      }
    }
    const uint2 e = pair_words<T, NPART>(a, fm * a);
    *reinterpret_cast<unsigned short*>(dst + off + 2 * j) = (unsigned short)(e.x & 0xFFFFu);
    *reinterpret_cast<unsigned short*>(dst + cb + off + 2 * j) = (unsigned short)(e.x >> 16);
    if (NPART == 2) {
      *reinterpret_cast<unsigned short*>(dst + 2 * cb + off + 2 * j) = (unsigned short)(e.y & 0xFFFFu);
      *reinterpret_cast<unsigned short*>(dst + 3 * cb + off + 2 * j) = (unsigned short)(e.y >> 16);
    }
  }
}

__device__ __noinline__ float fold_weight_slow(const DeviceParams& p, int k, int kind, const float* __restrict__ in,
                                               long long pitch, int H, int W, int gy, int gx) {
  float wgt = p.c[k];
  if (kind != 0) {
    const float fv = (gy < H && gx < W) ? __ldg(in + (long long)gy * pitch + gx) : 0.f;
    const float2 cs = term_cs_any((float)k, fv, p);
    wgt *= kind == 1 ? cs.x : cs.y;
  }
  return wgt;
}

// Generate chunk c (halo columns [c CW, (c+1) CW)) of one pair into the chunk slot (rows =
// halo rows hy, K = halo columns; image a at `dst`, image b at dst + CB).  Eight consecutive
// threads fill the eight rows of one core matrix, so the 16-byte stores are conflict-free.
// Rows and columns past the halo need only be finite (the matching entries of Gx and Gy are
// zero); pixels outside the image are zero, tested only on border tiles, with a column bit
// mask per 8-pixel group.
template <int RAD, typename T>
__device__ __forceinline__ void gen_chunk(unsigned char* dst, int c, const unsigned char* fh, const uint32_t* tab,
                                          bool tile_int, bool interior, int tx0, int ty0, int H, int W,
                                          const float* __restrict__ in, long long pitch, int k, int kind,
                                          const DeviceParams& p, int ctid) {
  constexpr int NPART = Parts<T>::value;
  using C = TcCfg<RAD, NPART>;
  constexpr int KG = C::CW / 8;                  // 8-column groups per chunk row
  const int col_lo = max(0, RAD - tx0), col_hi = min(C::HX, W - tx0 + RAD);   // inside: [lo, hi)
  // item i = 8 g + r7: core-matrix group g = (row block) KG + (column group), row r7 of the
  // block; its 16-byte store lands at 16 i
  constexpr int GSTEP = NCT / 8;                 // groups advanced per sweep
  const int r7 = ctid & 7;
  int rb = (ctid >> 3) / KG, cx = (ctid >> 3) % KG;
#pragma unroll 1
  for (int i = ctid; i < C::KY * KG; i += NCT) {
    const int hy = rb * 8 + r7;
    const int hx0 = (c * KG + cx) * 8;
    const int off = 16 * i;
    cx += GSTEP % KG;
    rb += GSTEP / KG;
    if (cx >= KG) { cx -= KG; ++rb; }
    if (!tile_int) {
      gen_item_slow<T, NPART>(dst, C::CB, off, hy, hx0, C::HY, C::HX, ty0 - RAD, tx0 - RAD, H, W, in, pitch, k,
                              kind, p);
      continue;
    }
    unsigned mask = 0xFFu;
    if (!interior) {
      const int gy = ty0 - RAD + hy;
      const bool row_in = hy < C::HY && gy >= 0 && gy < H;
      const int a = min(8, max(0, col_lo - hx0)), b = min(8, max(0, col_hi - hx0));
      mask = row_in && b > a ? (((1u << b) - 1u) & ~((1u << a) - 1u)) : 0u;
    }
    const uint2 bytes = *reinterpret_cast<const uint2*>(fh + hy * C::FHS + hx0);
    // the value words, then (compensated form) the error words; the compensated form reads a
    // pixel's two words with one 64-bit load (two 32-bit loads of words 2v and 2v + 1 would
    // each reach only half of the banks)
    uint32_t e[NPART][8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint32_t v = __byte_perm(j < 4 ? bytes.x : bytes.y, 0u, 0x4440u | (j & 3));
      if (NPART == 2) {
        const uint2 w = reinterpret_cast<const uint2*>(tab)[v];
        e[0][j] = w.x;
        e[NPART - 1][j] = w.y;
      } else {
        e[0][j] = tab[v];
      }
      if (!interior) {
#pragma unroll
        for (int h = 0; h < NPART; ++h) e[h][j] = ((mask >> j) & 1u) ? e[h][j] : 0u;
      }
    }
#pragma unroll
    for (int h = 0; h < NPART; ++h) {
      *reinterpret_cast<uint4*>(dst + 2 * h * C::CB + off) =
          make_uint4(__byte_perm(e[h][0], e[h][1], 0x5410), __byte_perm(e[h][2], e[h][3], 0x5410),
                     __byte_perm(e[h][4], e[h][5], 0x5410), __byte_perm(e[h][6], e[h][7], 0x5410));
      *reinterpret_cast<uint4*>(dst + (2 * h + 1) * C::CB + off) =
          make_uint4(__byte_perm(e[h][0], e[h][1], 0x7632), __byte_perm(e[h][2], e[h][3], 0x7632),
                     __byte_perm(e[h][4], e[h][5], 0x7632), __byte_perm(e[h][6], e[h][7], 0x7632));
    }
  }
}

// Taps of an image's radius class into the operand layouts: Gy (TF32, shared memory), Gx_lo
// (compensated form, shared memory) by all compute threads; Gx (tensor memory, lanes
// x' = 32 warp + lane, two K elements per column) by compute warps 0-3.
template <int RAD, typename T>
__device__ __forceinline__ void load_taps(const DeviceParams& p, unsigned char* sGy, unsigned char* sGl,
                                          uint32_t tmem, int tid) {
  constexpr int NPART = Parts<T>::value;
  using C = TcCfg<RAD, NPART>;
  for (int i = tid; i < C::TY * (C::KY / 4); i += NCT) {
    const int o = i / (C::KY / 4), k4 = (i - o * (C::KY / 4)) * 4;
    uint32_t v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int d = k4 + j - o;   // tap index 0..2r
      v[j] = to_tf32((d >= 0 && d <= 2 * RAD) ? p.g[d] : 0.f);
    }
    *reinterpret_cast<uint4*>(sGy + off32<C::KY>(o, k4)) = make_uint4(v[0], v[1], v[2], v[3]);
  }
  if (NPART == 2) {   // FP16 copy of Gy for the y pass of the x-pass result's lo part
    unsigned char* sGy16 = sGy + C::GYB;
    for (int i = tid; i < C::TY * (C::KY / 8); i += NCT) {
      const int o = i / (C::KY / 8), k8 = (i - o * (C::KY / 8)) * 8;
      float v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int d = k8 + j - o;
        v[j] = (d >= 0 && d <= 2 * RAD) ? p.g[d] : 0.f;
      }
      *reinterpret_cast<uint4*>(sGy16 + off16<C::KY>(o, k8)) =
          make_uint4(pack2<__half>(v[0], v[1]), pack2<__half>(v[2], v[3]), pack2<__half>(v[4], v[5]),
                     pack2<__half>(v[6], v[7]));
    }
  }
  // the Gx bands U[y, j] = g(j - y + 16 (KS - 1)) (see TcCfg::GXU): lo parts (compensated
  // form) and, at r > 15, hi parts
  constexpr int SH = C::KX - 16;   // 16 (KS - 1)
  if (NPART == 2) {
    for (int i = tid; i < C::GXU * 2; i += NCT) {
      const int y = i >> 1, k8 = (i & 1) * 8;
      float v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int d = k8 + j - y + SH;
        const float gv = (d >= 0 && d <= 2 * RAD) ? p.g[d] : 0.f;
        v[j] = gv - round16<T>(gv);
      }
      *reinterpret_cast<uint4*>(sGl + off16<16>(y, k8)) =
          make_uint4(pack2<T>(v[0], v[1]), pack2<T>(v[2], v[3]), pack2<T>(v[4], v[5]), pack2<T>(v[6], v[7]));
    }
  }
  if (C::GX_SMEM) {
    unsigned char* sGxh = sGl + C::GLB;
    for (int i = tid; i < C::GXU * 2; i += NCT) {
      const int y = i >> 1, k8 = (i & 1) * 8;
      float v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int d = k8 + j - y + SH;
        v[j] = (d >= 0 && d <= 2 * RAD) ? p.g[d] : 0.f;
      }
      *reinterpret_cast<uint4*>(sGxh + off16<16>(y, k8)) =
          make_uint4(pack2<T>(v[0], v[1]), pack2<T>(v[2], v[3]), pack2<T>(v[4], v[5]), pack2<T>(v[6], v[7]));
    }
  }
  const int warp = tid >> 5, lane = tid & 31;
  if (warp < 4 && !C::GX_SMEM) {
    const int o = 32 * warp + lane;
    for (int j0 = 0; j0 < C::KX / 2; j0 += 8) {
      uint32_t v[8];
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        const int d0 = 2 * (j0 + jj) - o, d1 = d0 + 1;
        v[jj] = pack2<T>((d0 >= 0 && d0 <= 2 * RAD) ? p.g[d0] : 0.f, (d1 >= 0 && d1 <= 2 * RAD) ? p.g[d1] : 0.f);
      }
      tmem_st8(tmem + ((uint32_t)(32 * warp) << 16) + C::GXC + j0, v);
    }
    tmem_wait_st();
  }
  proxy_fence();
  tc_fence_before();
}

// The kernel body over a source of images (one image, or a device work-list of images of the
// same radius class whose parameters may differ).
template <int RAD, typename T, class Src>
__device__ __forceinline__ void tc_body(const Src& src, const Scratch& sc) {
  constexpr int NPART = Parts<T>::value;
  using C = TcCfg<RAD, NPART>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned base, kept as an offset into the shared array (shared address space)
  unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* sGy = base;                        // y-pass B operand
  unsigned char* sGl = sGy + C::GYB + C::GY16B;     // Gx_lo (compensated form; Gy16 before it)
  unsigned char* sBh = sGl + C::GLB + C::GXHB;      // chunk ring (Gx hi before it when in smem)
  unsigned char* sFh = sBh + C::NSLOT * C::SLOTB;   // f of the halo tile (uint8)
  uint32_t* sTab = reinterpret_cast<uint32_t*>(sFh + C::FHB);   // 2 term-table slots
  uint64_t* bars = reinterpret_cast<uint64_t*>(sTab + 2 * C::TABW);
  uint64_t* bXa = bars + 0;            // x pass of the pair's first image complete
  uint64_t* bXb = bars + 1;            // ... second image
  uint64_t* bYa = bars + 2;            // y pass of the first image complete
  uint64_t* bYb = bars + 3;            // ... second image (and so the whole pair)
  uint64_t* bFd = bars + 4;            // the pair's D2 folded (16 warp arrivals)
  uint64_t* bDrain = bars + 5;
  uint64_t* bRa = bars + 6;            // D1 of the first image rounded to TF32 (16 warp arrivals)
  uint64_t* bRb = bars + 7;            // ... second image
  uint64_t* bFull = bars + 8;                  // [NSLOT] chunk generated (16 warp arrivals)
  uint64_t* bEmpty = bars + 8 + C::NSLOT;      // [NSLOT] chunk consumed (tcgen05.commit)
  uint32_t* sTmem = reinterpret_cast<uint32_t*>(bars + 8 + 2 * C::NSLOT);
  volatile int* sAbort = reinterpret_cast<volatile int*>(sTmem + 1);
  volatile int* sFin = sAbort + 1;
  volatile int* sPolls = sAbort + 2;   // test hook's poll limit (see mbar_wait)

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // ---- set-up: barriers, TMEM (the taps are loaded per image by the compute warps) ----------
  if (tid == 0) {
    for (int i = 0; i < C::NSLOT; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(bFull + i)), "r"(NCW));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(bEmpty + i)));
    }
    for (int i = 0; i < 4; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(bXa + i)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(bFd)), "r"(NCW));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(bRa)), "r"(NCW));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(bRb)), "r"(NCW));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(bDrain)));
    *sAbort = 0;
    *sPolls = g_tc_wait_polls;
  }
  proxy_fence();
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (warp == NCW) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" :: "r"(smem_u32(sTmem)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *sTmem;

  // ---- this CTA's share of the weighted (tile, term) sequence --------------------------------
  const int G = gridDim.x;
  const int cta = blockIdx.x;
  int img0, img_end;
  long long u0, u_end;
  locate(src, ceil_div_ll((long long)cta * sc.wtot, G), sc.wtot, img0, u0);
  locate(src, ceil_div_ll((long long)(cta + 1) * sc.wtot, G), sc.wtot, img_end, u_end);

  if (warp == NCW) {
    // ===================== MMA issuer ======================================================
    // Issue order per pair: the x passes of both images chunk by chunk, then y(a), y(b).  The
    // y pass of an image waits for its D1 to be rounded by the compute warps.
    {
      // every lane waits; a wait counts as given up when any lane gave up
      auto wait_all = [&](uint64_t* bar, uint32_t par) { return __all_sync(0xffffffffu, mbar_wait(bar, par, sAbort)); };
      const uint32_t fmt = std::is_same<T, __nv_bfloat16>::value ? 1u : 0u;
      const uint32_t idX = instr_desc(fmt, TILE_X, C::KY);
      const uint32_t idY = instr_desc(2u, TILE_X, C::TY);
      const uint32_t idY16 = instr_desc(0u, TILE_X, C::TY);   // lo part: FP16 operands
      const uint64_t dGy = op_desc(smem_u32(sGy), 32 * C::KY);
      const uint64_t dGy16 = op_desc(smem_u32(sGy + C::GYB), 16 * C::KY);
      const uint64_t dBh = op_desc(smem_u32(sBh), 16 * C::CW);
      // Gx bands: K-step ks starts 2 (KS - 1 - ks) row groups (512 bytes each step) into U
      const uint64_t dGl = op_desc(smem_u32(sGl), 256);
      const uint64_t dGxh = op_desc(smem_u32(sGl + C::GLB), 256);
      constexpr int KSL = C::KX / 16 - 1;
      uint32_t P = 0;
      int slot0 = 0, ring0 = 0;        // ring slot and use count of the next chunk
      bool ab = false;
      int img = img0;
      long long u = u0;
      while (!ab && (img < img_end || (img == img_end && u < u_end))) {
        const Work wk = src.work(img);
        const int K = wk.K;
        const long long t = u / K;
        const int kb = (int)(u - t * K);
        const int ke = (img == img_end && t == u_end / K) ? (int)(u_end - t * K) : K;
        const int np = frag_pairs(kb, ke);
        for (int j = 0; j < np; ++j, ++P) {
          // D1 is free once the previous pair's y passes have completed
          if (P > 0 && (!wait_all(bYa, (P - 1) & 1) || !wait_all(bYb, (P - 1) & 1))) { ab = true; break; }
          // x passes of both images, chunk by chunk (each chunk slot is released as soon as
          // both images have consumed it)
          for (int c = 0; c < C::NC; ++c) {
            if (!wait_all(bFull + slot0, ring0 & 1)) { ab = true; break; }
            tc_fence_after();
#pragma unroll
            for (int s = 0; s < 2; ++s) {
#pragma unroll
              for (int kk = 0; kk < C::CK; ++kk) {
                const int ks = c * C::CK + kk;
                const uint64_t bhi = dBh + (uint64_t)((slot0 * C::SLOTB + s * C::CB + kk * 256) >> 4);
                const uint64_t blo = bhi + (uint64_t)((2 * C::CB) >> 4);
                if (C::GX_SMEM) {
                  mma_ss_el(tmem + C::D1C + s * C::D1S, dGxh + (uint64_t)(32 * (KSL - ks)), bhi, idX, ks > 0 ? 1u : 0u);
                  mma_ss_el(tmem + C::D1C + s * C::D1S, dGxh + (uint64_t)(32 * (KSL - ks)), blo, idX, 1u);
                } else {
                  mma_ts_f16(tmem + C::D1C + s * C::D1S, tmem + C::GXC + 8 * ks, bhi, idX, ks > 0 ? 1u : 0u);
                  if (NPART == 2) mma_ts_f16(tmem + C::D1C + s * C::D1S, tmem + C::GXC + 8 * ks, blo, idX, 1u);
                }
                if (NPART == 2) mma_ss_el(tmem + C::D1C + s * C::D1S, dGl + (uint64_t)(32 * (KSL - ks)), bhi, idX, 1u);
              }
              if (c == C::NC - 1) mma_commit_el(s ? bXb : bXa);
            }
            mma_commit_el(bEmpty + slot0);
            if (++slot0 == C::NSLOT) { slot0 = 0; ++ring0; }
          }
          if (ab) break;
#pragma unroll
          for (int s = 0; s < 2; ++s) {
            // the compute warps round D1 to nearest TF32 once the x pass is complete
            if (!wait_all(s ? bRb : bRa, P & 1)) { ab = true; break; }
            // D2 is free once the previous pair has been folded
            if (s == 0 && P > 0 && !wait_all(bFd, (P - 1) & 1)) { ab = true; break; }
            tc_fence_after();
#pragma unroll
            for (int ks = 0; ks < C::KY / 8; ++ks)
              mma_ts_tf32(tmem + C::D2C + s * C::TY, tmem + C::D1C + s * C::D1S + 8 * ks,
                          dGy + (uint64_t)(16 * ks), idY, ks > 0);
            if (NPART == 2) {   // + Gy x lo (FP16 pairs, 16 K elements per 8 columns)
#pragma unroll
              for (int ks = 0; ks < C::KY / 16; ++ks)
                mma_ts_f16(tmem + C::D2C + s * C::TY, tmem + C::D1LC + s * C::D1LS + 8 * ks,
                           dGy16 + (uint64_t)(16 * ks), idY16, 1u);
            }
            mma_commit_el(s ? bYb : bYa);
          }
        }
        u = t * K + ke;
        if (u >= wk.tiles * K) { ++img; u = 0; }
      }
      if (ab && lane == 0) *sAbort = 1;
      // every MMA this thread issued has completed before TMEM is released
      mma_commit_el(bDrain);
      mbar_wait(bDrain, 0, nullptr);
    }
    __syncwarp();
  } else {
    // ===================== compute warps ==================================================
    const int q = warp & 3;              // TMEM lane quarter: output columns x' = 32 q + lane
    const int rg = warp >> 2;            // output rows y' = 16 rg .. 16 rg + 15
    constexpr int PX = C::PX;
    const int ox = 32 * q + lane, oy0 = PX * rg;
    const uint32_t tq = tmem + ((uint32_t)(32 * q) << 16) + C::D2C + PX * rg;
    uint32_t P = 0;
    int slot = 0, ring = 0;              // ring slot and use count of the next chunk
    bool ab = false;
    int img = img0;
    long long u = u0;
    float nm[PX], dn[PX];
    const DeviceParams* cp = nullptr;    // the current fragment's image parameters and record
    Work cw{};
    int cur_pidx = -1;                   // parameters whose taps are loaded

    // D1 of image s rounded to nearest TF32 in place: the y pass reads its A operand from
    // tensor memory as TF32, which drops the low mantissa bits (truncation); rounding first
    // keeps the error unbiased.  Warp (q, rg) takes the 8-column chunks rg, rg + 4, ...
    auto round_d1 = [&](uint32_t Pr, int s) {
      if (!mbar_wait(s ? bXb : bXa, Pr & 1, sAbort)) { ab = true; *sAbort = 1; }
      tc_fence_after();
      const uint32_t d1 = tmem + ((uint32_t)(32 * q) << 16) + C::D1C + s * C::D1S;
      const uint32_t d1lo = tmem + ((uint32_t)(32 * q) << 16) + C::D1LC + s * C::D1LS;
      constexpr int NCH = C::KY / 8;
#pragma unroll
      for (int c0 = 0; c0 < NCH; c0 += 8) {   // two chunks per warp at a time
        uint32_t v[2][8];
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
          const int c = c0 + rg + 4 * jj;
          if (c < NCH) tmem_ld8(d1 + 8 * c, v[jj]);
        }
        tmem_wait_ld();
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
          const int c = c0 + rg + 4 * jj;
          if (c < NCH) {
            uint32_t lo[4];
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
              const float x0 = __uint_as_float(v[jj][e]), x1 = __uint_as_float(v[jj][e + 1]);
              if (NPART == 2) {
                // compensated form: hi stays in place as the FP32 value, which the y pass
                // reads as TF32 by dropping the low 13 mantissa bits; lo is what that drops
                // (exact in FP32), as FP16
                const float h0 = __uint_as_float(v[jj][e] & 0xFFFFE000u);
                const float h1 = __uint_as_float(v[jj][e + 1] & 0xFFFFE000u);
                lo[e / 2] = pack2<__half>(x0 - h0, x1 - h1);
              } else {
                v[jj][e] = to_tf32(x0);
                v[jj][e + 1] = to_tf32(x1);
              }
            }
            if (NPART == 2) tmem_st4(d1lo + 4 * c, lo);
            else tmem_st8(d1 + 8 * c, v[jj]);
          }
        }
      }
      tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(s ? bRb : bRa);
    };
    auto wtab = [&](int k, int kind) { return sTab + (k & 1) * C::TABW + 2 * C::GENW + (kind == 2 ? 256 : 0); };
    // own pixels' weights for rows h .. h + 7 (table path: the pair's weight table)
    auto weights8 = [&](int h, int k, int kind, bool tile_int, int tx0, int ty0, const uint32_t* wt, float (&wv)[8]) {
      const unsigned char* own = sFh + (oy0 + RAD + h) * C::FHS + ox + RAD;
#pragma unroll
      for (int ii = 0; ii < 8; ++ii)
        wv[ii] = tile_int ? __uint_as_float(wt[own[ii * C::FHS]])
                          : fold_weight_slow(*cp, k, kind, cw.in, cw.pitch, cw.H, cw.W, ty0 + oy0 + h + ii, tx0 + ox);
    };
    auto fold = [&](uint32_t Pf, int k, int kind, bool tile_int, int tx0, int ty0, const uint32_t* wt) {
      float wv[8];
      weights8(0, k, kind, tile_int, tx0, ty0, wt, wv);   // before the wait: off the critical path
      if (!mbar_wait(bYb, Pf & 1, sAbort)) { ab = true; *sAbort = 1; }
      tc_fence_after();
#pragma unroll
      for (int h = 0; h < PX; h += 8) {   // 8 rows at a time keeps the live registers low
        uint32_t a[8], b[8];
        tmem_ld8(tq + h, a);
        tmem_ld8(tq + C::TY + h, b);
        if (h > 0) weights8(h, k, kind, tile_int, tx0, ty0, wt, wv);
        tmem_wait_ld();
#pragma unroll
        for (int ii = 0; ii < 8; ++ii) {
          dn[h + ii] = fmaf(wv[ii], __uint_as_float(a[ii]), dn[h + ii]);
          nm[h + ii] = fmaf(wv[ii], __uint_as_float(b[ii]), nm[h + ii]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bFd);
    };

    while (img < img_end || (img == img_end && u < u_end)) {
      cw = src.work(img);
      cp = &src.params(img);
      const int K = cw.K, H = cw.H, W = cw.W;
      const long long pitch = cw.pitch;
      const float m = cp->center;
      const float vmax = (float)min(cp->R, 255);
      if (cw.param_idx != cur_pidx) {   // this image's taps (the previous fragment's MMAs are complete)
        load_taps<RAD, T>(*cp, sGy, sGl, tmem, tid);
        cur_pidx = cw.param_idx;
      }
      const long long t = u / K;
      const int kb = (int)(u - t * K);
      const int ke = (img == img_end && t == u_end / K) ? (int)(u_end - t * K) : K;
      const int np = frag_pairs(kb, ke);
      const int tx0 = (int)(t % cw.tiles_x) * TILE_X;
      const int ty0 = cw.row0 + (int)(t / cw.tiles_x) * C::TY;

      // f of the tile + halo as bytes (zero outside the image and in the padding); the tile
      // takes the table path when every pixel is an integer in [0, min(R, 255)]
      int ok = 1;
#pragma unroll 4
      for (int i = tid; i < C::KY * C::FHS / 4; i += NCT) {
        const int hy = (4 * i) / C::FHS, hx = 4 * i - hy * C::FHS;
        const int gy = ty0 - RAD + hy;
        uint32_t word = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int gx = tx0 - RAD + hx + j;
          if (hy < C::HY && hx + j < C::HX && gy >= 0 && gy < H && gx >= 0 && gx < W) {
            const float v = __ldg(cw.in + (long long)gy * pitch + gx);
            ok &= (v == rintf(v)) & (v >= 0.f) & (v <= vmax);
            word |= (uint32_t)(int)fminf(fmaxf(v, 0.f), 255.f) << (8 * j);
          }
        }
        *reinterpret_cast<uint32_t*>(sFh + 4 * i) = word;
      }
      const bool tile_int = sync_compute_and(ok != 0);
      const bool interior = tx0 - RAD >= 0 && ty0 - RAD >= 0 && tx0 + TILE_X + RAD <= W && ty0 + C::TY + RAD <= H;
#pragma unroll
      for (int i = 0; i < PX; ++i) { nm[i] = 0.f; dn[i] = 0.f; }

      int kprev = 0, kindprev = 0;
      for (int j = 0; j < np; ++j, ++P) {
        int k, kind;
        pair_of(kb, j, &k, &kind);
        // the term's tables are built at its first pair; slot k & 1 is free by then (its
        // previous term was last read by a fold before the previous pair's barrier)
        uint32_t* tslot = sTab + (k & 1) * C::TABW + (kind == 2 ? C::GENW : 0);
        if (tile_int && kind != 2) build_term_table<T, NPART>(*cp, k, sTab + (k & 1) * C::TABW, tid);
        ab = sync_compute_or(ab || *sAbort);   // also publishes the table
        if (ab) break;
        // a ring slot is free once the x pass has consumed the chunk it held NSLOT chunks ago
        for (int c = 0; c < C::NC; ++c) {
          if (ring > 0 && !mbar_wait(bEmpty + slot, (ring - 1) & 1, sAbort)) { ab = true; *sAbort = 1; }
          gen_chunk<RAD, T>(sBh + slot * C::SLOTB, c, sFh, tslot, tile_int, interior, tx0, ty0, H, W, cw.in,
                            pitch, k, kind, *cp, tid);
          proxy_fence();
          __syncwarp();
          if (lane == 0) mbar_arrive(bFull + slot);
          if (++slot == C::NSLOT) { slot = 0; ++ring; }
        }
        if (j > 0) fold(P - 1, kprev, kindprev, tile_int, tx0, ty0, wtab(kprev, kindprev));
        round_d1(P, 0);
        round_d1(P, 1);
        kprev = k;
        kindprev = kind;
      }
      // last pair (also on abort, where its bounded wait returns at once: every lane of a warp
      // must reach the fold's __syncwarp)
      fold(P - 1, kprev, kindprev, tile_int, tx0, ty0, wtab(kprev, kindprev));
      ab = sync_compute_or(ab || *sAbort);
      if (ab) break;

      // ---- finish the tile (as in the FP32 kernel) ------------------------------------------
      bool finish = true;
      if (!(kb == 0 && ke == K)) {
        const int wmine = term_start(ke) - term_start(kb);
        const int pslot = (img == img0 && u0 / K == t) ? 0 : 1;
        float* pp = sc.partial + ((long long)(cta * 2 + pslot) * 2) * PX * NCT;
#pragma unroll
        for (int a = 0; a < PX; ++a) {
          pp[a * NCT + tid] = nm[a];
          pp[(PX + a) * NCT + tid] = dn[a];
        }
        sync_compute();
        if (tid == 0) {
          const int prev = fp32::counter_add_acq_rel(sc.counter + cw.counter_base + t, wmine);
          *sFin = (prev + wmine == cw.wtile);
        }
        sync_compute();
        finish = *sFin != 0;
        if (finish) {
          const long long g0 = cw.wstart + t * cw.wtile;
          const long long c0 = g0 * G / sc.wtot;
          const long long c1 = (g0 + term_start(K - 1)) * G / sc.wtot;
#pragma unroll
          for (int a = 0; a < PX; ++a) { nm[a] = 0.f; dn[a] = 0.f; }
          // each lane finds the slot of one contributor (the divisions run side by side),
          // then every thread adds the slots in CTA order
          for (long long base = c0; base <= c1; base += 32) {
            const int my_sl = base + lane <= c1 ? fp32::contributor_slot(src, base + lane, G, sc.wtot, img, t, K) : -1;
            const int n = (int)min(32LL, c1 - base + 1);
            for (int q = 0; q < n; ++q) {
              const int sl = __shfl_sync(0xffffffffu, my_sl, q);
              if (sl < 0) continue;
              const float* qp = sc.partial + (((base + q) * 2 + sl) * 2) * PX * NCT;
#pragma unroll
              for (int a = 0; a < PX; ++a) {
                nm[a] += __ldcg(qp + a * NCT + tid);
                dn[a] += __ldcg(qp + (PX + a) * NCT + tid);
              }
            }
          }
          if (tid == 0) sc.counter[cw.counter_base + t] = 0;
        }
      }
      if (finish) {
        const int gx = tx0 + ox;
        if (gx < W) {
#pragma unroll
          for (int a = 0; a < PX; ++a) {
            const int gy = ty0 + oy0 + a;
            if (gy < cw.row1) {
              const float d = dn[a];
              const float f = __ldg(cw.in + (long long)gy * pitch + gx);
              cw.out[(long long)gy * pitch + gx] = (d > 0.f) ? m + nm[a] / d : f;
            }
          }
        }
      }
      u = t * K + ke;
      if (u >= cw.tiles * K) { ++img; u = 0; }
      sync_compute();   // sFh and the finish flag are rewritten by the next fragment
    }
    if (ab) *sAbort = 1;
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid == 0 && *sAbort) atomicOr(&g_tc_error, 1);
  if (warp == NCW) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" :: "r"(tmem));
}

template <int RAD, typename T>
__global__ void __launch_bounds__(NTHREADS, 1)
fbf_tc_kernel(const __grid_constant__ DeviceParams p, const Work w, const Scratch sc) {
  const SingleSrc src{&p, w};
  tc_body<RAD, T>(src, sc);
}

// Batched form: the images of one radius class from a device work-list (parameters per plan
// de-duplicated), one persistent stream-K launch over all of them.
template <int RAD, typename T>
__global__ void __launch_bounds__(NTHREADS, 1)
fbf_tc_batch_kernel(const DeviceParams* __restrict__ prm, const Work* __restrict__ wl, int n, const Scratch sc) {
  const ListSrc src{prm, wl, n, nullptr};   // taps come from prm (staged per image)
  tc_body<RAD, T>(src, sc);
}

template <int RAD, typename T>
int launch_rad(const DeviceParams& dp, const float* in, float* out, int H, int W, size_t pitch,
               cudaStream_t st, int row0, int rows) {
  using C = TcCfg<RAD, Parts<T>::value>;
  if (rows <= 0) rows = H - row0;
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
  w.tiles_x = (W + TILE_X - 1) / TILE_X;
  w.tiles_y = (rows + C::TY - 1) / C::TY;
  w.row0 = row0;
  w.row1 = row0 + rows;
  w.K = dp.K;
  w.wtile = 2 * dp.K - 1;
  w.tiles = (long long)w.tiles_x * w.tiles_y;
  Scratch sc{};
  sc.wtot = w.tiles * w.wtile;
  long long G = sms[dev];
  if (G > sc.wtot) G = sc.wtot;
  const size_t partial_bytes = (size_t)G * 2 * 2 * C::PX * NCT * sizeof(float);
  int rc = get_workspace(dev, st, partial_bytes, (size_t)w.tiles, &sc.partial, &sc.counter);
  if (rc != FBF_OK) return rc;
  fbf_tc_kernel<RAD, T><<<(unsigned)G, NTHREADS, C::SMEM, st>>>(p, w, sc);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_filter: launch: ") + cudaGetErrorString(e));
  return FBF_OK;
}
// Batched launch of one radius class (work-list already on the device).
template <int RAD, typename T>
int launch_batch_rad(const DeviceParams* dparams, const Work* dwork, int n, long long wtot, float* partial,
                     int* counter, cudaStream_t st, int dev) {
  using C = TcCfg<RAD, Parts<T>::value>;
  static int sms[64] = {0};
  if (dev < 0 || dev >= 64) return set_error(FBF_EUNSUPPORTED, "fbf_launch: device index >= 64");
  if (!sms[dev]) {
    cudaError_t e = cudaFuncSetAttribute(fbf_tc_batch_kernel<RAD, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_launch: ") + cudaGetErrorString(e));
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fbf_tc_batch_kernel<RAD, T>, NTHREADS, C::SMEM);
    if (e != cudaSuccess || occ != 1)
      return set_error(FBF_ECUDA, "fbf_launch: tensor-core kernel needs exactly one CTA per SM");
    int s = 0;
    cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
    sms[dev] = s;
  }
  long long G = sms[dev];
  if (G > wtot) G = wtot;
  if (G < 1) return FBF_OK;
  Scratch sc{};
  sc.wtot = wtot;
  sc.partial = partial;
  sc.counter = counter;
  fbf_tc_batch_kernel<RAD, T><<<(unsigned)G, NTHREADS, C::SMEM, st>>>(dparams, dwork, n, sc);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_launch: ") + cudaGetErrorString(e));
  return FBF_OK;
}

template <typename T>
int launch_type(const DeviceParams& dp, const float* in, float* out, int H, int W, size_t pitch,
                cudaStream_t st, int row0, int rows) {
  const int r = dp.r;
  if (r <= 6) return launch_rad<6, T>(dp, in, out, H, W, pitch, st, row0, rows);
  if (r <= 15) return launch_rad<15, T>(dp, in, out, H, W, pitch, st, row0, rows);
  if (r <= 30) return launch_rad<30, T>(dp, in, out, H, W, pitch, st, row0, rows);
  return set_error(FBF_EUNSUPPORTED, "fbf_filter: the tensor-core forms support r = ceil(3 theta) <= 30");
}

}  // namespace tc

int launch_tc(const DeviceParams& dp, const float* in, float* out, int H, int W, size_t pitch,
              void* stream, int precision, int row0, int rows) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (precision == FBF_BF16_TC) return tc::launch_type<__nv_bfloat16>(dp, in, out, H, W, pitch, st, row0, rows);
  return tc::launch_type<__half>(dp, in, out, H, W, pitch, st, row0, rows);
}

int launch_tc_batch(int rad, int precision, const DeviceParams* dparams, const fp32::Work* dwork, int n, long long wtot,
                    float* partial, int* counter, void* stream, int dev) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const bool bf = precision == FBF_BF16_TC;
  switch (rad) {
    case 6: return bf ? tc::launch_batch_rad<6, __nv_bfloat16>(dparams, dwork, n, wtot, partial, counter, st, dev)
                      : tc::launch_batch_rad<6, __half>(dparams, dwork, n, wtot, partial, counter, st, dev);
    case 15: return bf ? tc::launch_batch_rad<15, __nv_bfloat16>(dparams, dwork, n, wtot, partial, counter, st, dev)
                       : tc::launch_batch_rad<15, __half>(dparams, dwork, n, wtot, partial, counter, st, dev);
    case 30: return bf ? tc::launch_batch_rad<30, __nv_bfloat16>(dparams, dwork, n, wtot, partial, counter, st, dev)
                       : tc::launch_batch_rad<30, __half>(dparams, dwork, n, wtot, partial, counter, st, dev);
    default: return set_error(FBF_EUNSUPPORTED, "fbf_launch: no tensor-core radius class");
  }
}

int tc_tile_rows(int rad, int precision) {
  const bool bf = precision == FBF_BF16_TC;
  switch (rad) {
    case 6: return bf ? tc::TcCfg<6, 2>::TY : tc::TcCfg<6, 1>::TY;
    case 15: return bf ? tc::TcCfg<15, 2>::TY : tc::TcCfg<15, 1>::TY;
    default: return bf ? tc::TcCfg<30, 2>::TY : tc::TcCfg<30, 1>::TY;
  }
}

int tc_batch_partial_bytes(int dev, size_t* out) {
  int s = 0;
  cudaError_t e = cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_launch: ") + cudaGetErrorString(e));
  *out = (size_t)s * 2 * 2 * tc::PX_MAX * tc::NCT * sizeof(float);
  return FBF_OK;
}

int tc_set_wait_polls(int polls) {
  const cudaError_t e = cudaMemcpyToSymbol(tc::g_tc_wait_polls, &polls, sizeof(int));
  if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_debug_set_wait_limit: ") + cudaGetErrorString(e));
  return FBF_OK;
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
  int v32 = 0;
  int rc = fp32_device_errors(&v32, clear);
  if (rc != FBF_OK) return rc;
  v |= v32;
  // a launch that gave up left some split-tile counters nonzero: clear them for the next one
  if (clear && v) {
    rc = reset_workspace_counters();
    if (rc != FBF_OK) return rc;
  }
  *flags = v;
  return FBF_OK;
}

}  // namespace fbf
