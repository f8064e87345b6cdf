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
// Per tile a CTA stages f of the tile plus an r-pixel halo in shared memory: for single
// images at r <= 15 whose base and row stride are 16-byte aligned, by TMA (a 2-D tensor map
// of the image; the next tile's box is loaded into a second buffer while the current tile is
// filtered; elements outside the image arrive as NaN, which marks them as absent), otherwise
// by plain loads (whole rows per warp; outside pixels marked by a sentinel).  Per term,
//   1. each warp, four halo rows at a time, generates the term's image pairs into a
//      warp-private buffer and convolves them along x (8 outputs per lane) into a shared
//      buffer of TY + 2r rows; only __syncwarp separates the two;
//   2. after one CTA barrier each thread convolves that buffer along y for its own pixels
//      and folds the results into its num/den registers.
// Only f is read from and only f_BF (and split-tile partials) written to global memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <utility>

#include "fbf_fp32_body.cuh"
#include "fbf_internal.h"

namespace fbf {

// ---- per-(device, stream) scratch: tile counters and partial sums ----------------------
// Layout: [counter_cap ints, zero between launches][partial sums].  Each launch leaves the
// counters it used at zero, so they are cleared only when the buffer is (re)allocated.
namespace {
struct Workspace {
  void* base = nullptr;
  size_t counter_cap = 0;
  size_t partial_cap = 0;
};
std::mutex g_ws_mu;
std::map<std::pair<int, uintptr_t>, Workspace> g_ws;

size_t align256(size_t x) { return (x + 255) / 256 * 256; }
}  // namespace

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


// Zero the tile counters of every cached workspace (after a launch that gave up part way
// left some of them nonzero).  Synchronises each device that has a workspace.
int reset_workspace_counters() {
  std::lock_guard<std::mutex> lk(g_ws_mu);
  int cur = 0;
  cudaGetDevice(&cur);
  for (auto& kv : g_ws) {
    Workspace& w = kv.second;
    if (!w.base) continue;
    cudaSetDevice(kv.first.first);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemset(w.base, 0, align256(w.counter_cap * sizeof(int)));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
      cudaSetDevice(cur);
      return set_error(FBF_ECUDA, std::string("fbf_device_errors: ") + cudaGetErrorString(e));
    }
  }
  cudaSetDevice(cur);
  return FBF_OK;
}

// Test hook of the single-image FP32 kernels' TMA wait (fbf_debug_set_wait_limit).
int fp32_set_wait_polls(int polls) {
  const cudaError_t e = cudaMemcpyToSymbol(fp32::g_fp32_wait_polls, &polls, sizeof(int));
  if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_debug_set_wait_limit: ") + cudaGetErrorString(e));
  return FBF_OK;
}

// The FP32 device error word of this translation unit's kernels (the single-image ones).
int fp32_device_errors(int* flags, int clear) {
  int v = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, fp32::g_fp32_error, sizeof(int));
  if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_device_errors: ") + cudaGetErrorString(e));
  if (clear && v) {
    const int z = 0;
    e = cudaMemcpyToSymbol(fp32::g_fp32_error, &z, sizeof(int));
    if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_device_errors: ") + cudaGetErrorString(e));
  }
  *flags = v;
  return FBF_OK;
}

namespace {

using namespace fp32;

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime (no link
// dependence on the driver library)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }();
  return fn;
}

// Tensor map of the image for the TMA staging of the f halo: FP32, dims {W, H}, row stride
// pitch, box {box_w, box_h}, NaN for elements outside the image.  False when the image does
// not allow one (base not 16-byte aligned, row stride not a multiple of 16 bytes, not in
// device memory) or the driver has no encoder; the caller then stages with plain loads.
bool encode_f_map(CUtensorMap* map, const float* in, int H, int W, size_t pitch, int box_w, int box_h) {
  if ((reinterpret_cast<uintptr_t>(in) & 15) != 0 || (pitch * sizeof(float)) % 16 != 0) return false;
  // device memory only: images the kernel reads from host memory (mapped, page-locked) take
  // the plain loads
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, in) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return false;
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)H};
  const cuuint64_t strides[1] = {(cuuint64_t)(pitch * sizeof(float))};
  const cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(in), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NAN_REQUEST_ZERO_FMA) == CUDA_SUCCESS;
}

// SMs and resident CTAs of one instantiation on one device (set once per device, under a
// lock: several host threads may launch at once)
std::mutex g_slots_mu;
template <class KernelFn>
int kernel_slots(KernelFn fn, int nt, size_t smem, int dev, int* sms_out, int* occ_out,
                 int* cache_sms, int* cache_occ, const char* who) {
  std::lock_guard<std::mutex> lk(g_slots_mu);
  if (!cache_occ[dev]) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string(who) + ": " + cudaGetErrorString(e));
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, nt, smem);
    if (e != cudaSuccess || n < 1) return set_error(FBF_ECUDA, std::string(who) + ": kernel does not fit on an SM");
    int s = 0;
    cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
    cache_sms[dev] = s;
    cache_occ[dev] = n;
  }
  *sms_out = cache_sms[dev];
  *occ_out = cache_occ[dev];
  return FBF_OK;
}

// Carried rows are used when the image has at least this many tiles per CTA.
constexpr long long kCarryMinTilesPerCta = 3;

// SM count of the current device (cached per device)
int device_sms() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1 << 20;
  int n = cache[dev].load(std::memory_order_relaxed);
  if (n == 0) {
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) return 1 << 20;
    cache[dev].store(n, std::memory_order_relaxed);
  }
  return n;
}

Work single_work(const float* in, float* out, int H, int W, size_t pitch, int K, int TY, int row0 = 0,
                 int rows = 0) {
  if (rows <= 0) rows = H - row0;
  Work w{};
  w.row0 = row0;
  w.row1 = row0 + rows;
  w.in = in;
  w.out = out;
  w.pitch = (long long)pitch;
  w.H = H;
  w.W = W;
  w.tiles_x = (W + TX - 1) / TX;
  w.tiles_y = (rows + TY - 1) / TY;
  w.K = K;
  w.wtile = 2 * K - 1;
  w.tiles = (long long)w.tiles_x * w.tiles_y;
  w.wstart = 0;
  w.counter_base = 0;
  w.param_idx = 0;
  return w;
}

template <int RAD, int TY, int NT, int NY>
int launch_cfg(const DeviceParams& dp, const float* in, float* out, int H, int W, size_t pitch,
               cudaStream_t st, int row0, int rows) {
  using C = Cfg<RAD, TY, NT, NY>;
  static int occ[64] = {0};
  static int sms[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_filter: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= 64) return set_error(FBF_EUNSUPPORTED, "fbf_filter: device index >= 64");
  int nsm = 0, nocc = 0;
  int rc = FBF_OK;
  CUtensorMap map;
  bool tma = false;
  // Carried x-pass rows pay when each CTA's range covers several tiles of a strip (the
  // first tile of a range convolves all its rows) and carrying saves a whole x-pass round
  // per tile; carried tiles stage f with plain loads (the TMA staging is not combined)
  constexpr int CSLOT = 2 * carry_rows(RAD, 4) * TX;
  constexpr bool kCarryCfg = carry_saves_round(RAD, TY, NT);
  bool want_carry = false;
  if constexpr (kCarryCfg) {
    const long long tiles = (long long)((W + TX - 1) / TX) * (((rows > 0 ? rows : H - row0) + TY - 1) / TY);
    want_carry = tiles >= kCarryMinTilesPerCta * device_sms();
  }
  if constexpr (C::TMA_OK) {
    if (!want_carry) tma = encode_f_map(&map, in, H, W, pitch, C::TMA_BW, C::HROWS_P);
    if (tma) {
      static int occ_t[64] = {0};
      static int sms_t[64] = {0};
      rc = kernel_slots(fbf_fp32_tma_kernel<RAD, TY, NT, NY>, NT, C::TMA_SMEM_BYTES, dev, &nsm, &nocc, sms_t,
                        occ_t, "fbf_filter");
    }
  }
  if (!tma)
    rc = kernel_slots(fbf_fp32_kernel<RAD, TY, NT, NY>, NT, C::SMEM_BYTES, dev, &nsm, &nocc, sms, occ,
                      "fbf_filter");
  if (rc != FBF_OK) return rc;
  const DeviceParams p = pad_params<RAD>(dp);
  const Work w = single_work(in, out, H, W, pitch, dp.K, TY, row0, rows);
  if (w.tiles > (1LL << 30)) return set_error(FBF_EUNSUPPORTED, "fbf_filter: image too large");
  Scratch sc{};
  sc.wtot = w.tiles * w.wtile;
  long long G = (long long)nsm * nocc;
  if (G > sc.wtot) G = sc.wtot;
  const bool carry = want_carry && !tma && w.tiles >= kCarryMinTilesPerCta * G;
  if constexpr (kCarryCfg) {
    if (carry) {
      static int occ_c[64] = {0};
      static int sms_c[64] = {0};
      int nsm_c = 0, nocc_c = 0;
      rc = kernel_slots(fbf_fp32_carry_kernel<RAD, TY, NT, NY>, NT, C::SMEM_BYTES, dev, &nsm_c, &nocc_c,
                        sms_c, occ_c, "fbf_filter");
      if (rc != FBF_OK) return rc;
      if ((long long)nsm_c * nocc_c != G)
        return set_error(FBF_ECUDA, "fbf_filter: carried-row kernel occupancy differs");
    }
  }
  const size_t partial_bytes = (size_t)G * 2 * 2 * NY * NT * sizeof(float);
  const size_t carry_bytes = carry ? (size_t)G * dp.K * CSLOT * sizeof(float2) : 0;
  rc = get_workspace(dev, st, align256(partial_bytes) + carry_bytes, (size_t)w.tiles, &sc.partial, &sc.counter);
  if (rc != FBF_OK) return rc;
  if (carry) {
    sc.carry = reinterpret_cast<float2*>(reinterpret_cast<char*>(sc.partial) + align256(partial_bytes));
    sc.kmax = dp.K;
  }
  bool launched = false;
  if constexpr (C::TMA_OK) {
    if (tma) {
      fbf_fp32_tma_kernel<RAD, TY, NT, NY><<<(unsigned)G, NT, C::TMA_SMEM_BYTES, st>>>(p, w, sc, map);
      launched = true;
    }
  }
  if constexpr (kCarryCfg) {
    if (!launched && carry) {
      fbf_fp32_carry_kernel<RAD, TY, NT, NY><<<(unsigned)G, NT, C::SMEM_BYTES, st>>>(p, w, sc);
      launched = true;
    }
  }
  if (!launched) fbf_fp32_kernel<RAD, TY, NT, NY><<<(unsigned)G, NT, C::SMEM_BYTES, st>>>(p, w, sc);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_filter: launch: ") + cudaGetErrorString(e));
  return FBF_OK;
}

}  // namespace

int fp32_tile_rows(int r, int W, int rows) {
  const long long strips = (W + TX - 1) / TX, many = kCarryMinTilesPerCta * device_sms();
  if (r <= 6) return 112;
  if (r <= 9) return 96;
  if (r <= 15) return 96;
  if (r <= 30) return strips * ((rows + 95) / 96) >= many ? 96 : 128;
  return 64;
}

int launch_fp32(const DeviceParams& dp, const float* in, float* out, int H, int W, size_t pitch,
                void* stream, int row0, int rows) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int r = dp.r;
  // Tile heights keep TY + 2r just under a whole number of x-pass rounds (4 rows per
  // warp); radii above 15 need more registers for their taps and use 256 threads.
  if (r <= 3) return launch_cfg<3, 112, 512, 7>(dp, in, out, H, W, pitch, st, row0, rows);
  if (r <= 6) return launch_cfg<6, 112, 512, 7>(dp, in, out, H, W, pitch, st, row0, rows);
  if (r <= 9) return launch_cfg<9, 96, 512, 6>(dp, in, out, H, W, pitch, st, row0, rows);
  // (a 112-row configuration carrying rows at r <= 15, 2 instead of 3 x-pass rounds per
  // tile, measured slower than these 96-row tiles with TMA staging: 2.59-2.62 against
  // 2.54 ms at 4096^2, theta 5, K 12)
  if (r <= 15) return launch_cfg<15, 96, 512, 6>(dp, in, out, H, W, pitch, st, row0, rows);
  // 15 < r <= 30: images with at least three 96-row tiles per SM carry their x-pass rows
  // down the strips in a 96-row, 12-warp configuration; others take 128-row tiles, 8 warps
  const long long tiles96 = (long long)((W + TX - 1) / TX) * (((rows > 0 ? rows : H - row0) + 95) / 96);
  const bool carry96 = tiles96 >= kCarryMinTilesPerCta * device_sms();
  if (r <= 24) {
    if (carry96) return launch_cfg<24, 96, 384, 8>(dp, in, out, H, W, pitch, st, row0, rows);
    return launch_cfg<24, 128, 256, 16>(dp, in, out, H, W, pitch, st, row0, rows);
  }
  if (r <= 30) {
    if (carry96) return launch_cfg<30, 96, 384, 8>(dp, in, out, H, W, pitch, st, row0, rows);
    return launch_cfg<30, 128, 256, 16>(dp, in, out, H, W, pitch, st, row0, rows);
  }
  if (r <= 48) return launch_cfg<48, 64, 128, 16>(dp, in, out, H, W, pitch, st, row0, rows);
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

using namespace fp32;

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
  const Work w = single_work(in, out, H, W, pitch, dp.K, TY);
  if ((size_t)w.tiles * sizeof(int) > kNoAllocCounterBytes)
    return set_error(FBF_EUNSUPPORTED,
                     "fbf_filter_noalloc: image needs " + std::to_string(w.tiles) + " tiles; the fixed "
                     "scratch holds counters for " + std::to_string(kNoAllocCounterBytes / sizeof(int)));
  void* base = nullptr;
  int rc = noalloc_scratch(dev, &base);
  if (rc != FBF_OK) return rc;
  int nsm = 0, nocc = 0;
  rc = kernel_slots(fbf_fp32_kernel<RAD, TY, NT, NY>, NT, C::SMEM_BYTES, dev, &nsm, &nocc, sms, occ,
                    "fbf_filter_noalloc");
  if (rc != FBF_OK) return rc;
  const DeviceParams p = pad_params<RAD>(dp);
  Scratch sc{};
  sc.wtot = w.tiles * w.wtile;
  long long G = (long long)nsm * nocc;
  const long long per_cta = 2LL * 2 * NY * NT * (long long)sizeof(float);
  if (G > (long long)(kNoAllocPartialBytes / per_cta)) G = (long long)(kNoAllocPartialBytes / per_cta);
  if (G > sc.wtot) G = sc.wtot;
  sc.counter = reinterpret_cast<int*>(base);
  sc.partial = reinterpret_cast<float*>(static_cast<unsigned char*>(base) + kNoAllocCounterBytes);
  // counters must start at zero; the array keeps whatever the previous call left
  e = cudaMemsetAsync(sc.counter, 0, (size_t)w.tiles * sizeof(int), st);
  if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_filter_noalloc: ") + cudaGetErrorString(e));
  fbf_fp32_kernel<RAD, TY, NT, NY><<<(unsigned)G, NT, C::SMEM_BYTES, st>>>(p, w, sc);
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
