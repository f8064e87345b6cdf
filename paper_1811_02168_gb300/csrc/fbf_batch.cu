// Batched Fourier bilateral filtering: many images in one persistent launch.
//
// Images are queued with fbf_batch_submit (host only), then fbf_launch groups them by radius
// class (the kernel instantiation that serves their r = ceil(3 theta)) and, for the FP32
// form, by spatial kernel within the class (the launch's taps are a kernel parameter, read
// from the constant bank by the multiply-adds), uploads one device work-list per group
// (per-image Work records and per-plan DeviceParams, one copy from a pinned staging buffer)
// and starts one stream-K persistent kernel per group over the concatenated (image, tile,
// term) sequence of the group.  An event recorded after the
// launches marks the generation; tickets name a generation and fbf_batch_poll / fbf_batch_wait query
// it.  fbf_batch_capture records the same work as a CUDA graph (copy + kernels) that
// fbf_batch_replay relaunches with the same pointers and sizes.
//
// Autotuning (FBF_BATCH_AUTOTUNE): the first launch of each (radius class, total pixels
// rounded to a power of two, longest K) key times every candidate tile configuration of the
// class on the real work-list with CUDA events and keeps the fastest; the choice is cached
// per device and, if FBF_TUNE_CACHE names a file, persisted there as "key config" lines.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <map>
#include <new>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "fbf_fp32_body.cuh"
#include "fbf_internal.h"

namespace fbf {
namespace {

using namespace fp32;

// ---- kernel configurations per radius class --------------------------------------------
struct ClassLaunch {
  // launches the batched kernel of one configuration; returns FBF_OK or an error code.
  // carry / kmax: the carried-row slots (configurations with carry_bytes_per_term) and the
  // largest K of the work-list; taps: the spatial taps every image of the list shares (FP32)
  int (*launch)(const DeviceParams* dparams, const Work* dwork, int n, long long wtot,
                float* partial, int* counter, float2* carry, int kmax, const SpatialTaps& taps,
                cudaStream_t st, int dev);
  // partial-sum bytes one launch of this configuration needs (per CTA slots) on dev
  int (*partial_bytes)(int dev, size_t* out);
  // carried-row bytes per cosine term of the longest image (0: rows are not carried)
  int (*carry_bytes_per_term)(int dev, size_t* out);
  int TY;
  const char* name;
  int TX = fp32::TX;   // tile width of the kernel's schedule
};

int no_carry(int, size_t* out) {
  *out = 0;
  return FBF_OK;
}

template <int RAD, int TY, int NT, int NY, bool CARRY>
struct BatchCfg {
  using C = Cfg<RAD, TY, NT, NY>;
  static constexpr auto kernel() {
    if constexpr (CARRY) return &fbf_fp32_batch_carry_kernel<RAD, TY, NT, NY>;
    else return &fbf_fp32_batch_kernel<RAD, TY, NT, NY>;
  }
  static int sms[64], occ[64];
  static std::mutex mu;
  static int slots(int dev, int* G) {
    std::lock_guard<std::mutex> lk(mu);
    if (!occ[dev]) {
      cudaError_t e = cudaFuncSetAttribute(kernel(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM_BYTES);
      if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_batch: ") + cudaGetErrorString(e));
      int n = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel(), NT, C::SMEM_BYTES);
      if (e != cudaSuccess || n < 1) return set_error(FBF_ECUDA, "fbf_batch: kernel does not fit on an SM");
      int s = 0;
      cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
      sms[dev] = s;
      occ[dev] = n;
    }
    *G = sms[dev] * occ[dev];
    return FBF_OK;
  }
  static int partial_bytes(int dev, size_t* out) {
    int G = 0;
    int rc = slots(dev, &G);
    if (rc != FBF_OK) return rc;
    *out = (size_t)G * 2 * 2 * NY * NT * sizeof(float);
    return FBF_OK;
  }
  static int carry_bytes_per_term(int dev, size_t* out) {
    int G = 0;
    int rc = slots(dev, &G);
    if (rc != FBF_OK) return rc;
    *out = CARRY ? (size_t)G * 2 * carry_rows(RAD, 4) * TX * sizeof(float2) : 0;
    return FBF_OK;
  }
  static int launch(const DeviceParams* dparams, const Work* dwork, int n, long long wtot,
                    float* partial, int* counter, float2* carry, int kmax, const SpatialTaps& taps,
                    cudaStream_t st, int dev) {
    int G = 0;
    int rc = slots(dev, &G);
    if (rc != FBF_OK) return rc;
    long long g = G;
    if (g > wtot) g = wtot;
    Scratch sc{};
    sc.wtot = wtot;
    sc.partial = partial;
    sc.counter = counter;
    sc.carry = carry;
    sc.kmax = kmax;
    kernel()<<<(unsigned)g, NT, C::SMEM_BYTES, st>>>(dparams, dwork, n, sc, taps);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_batch: ") + cudaGetErrorString(e));
    return FBF_OK;
  }
};
template <int RAD, int TY, int NT, int NY, bool CARRY> int BatchCfg<RAD, TY, NT, NY, CARRY>::sms[64] = {0};
template <int RAD, int TY, int NT, int NY, bool CARRY> int BatchCfg<RAD, TY, NT, NY, CARRY>::occ[64] = {0};
template <int RAD, int TY, int NT, int NY, bool CARRY> std::mutex BatchCfg<RAD, TY, NT, NY, CARRY>::mu;

template <int RAD, int TY, int NT, int NY, bool CARRY = false>
ClassLaunch cfg_entry(const char* name) {
  using B = BatchCfg<RAD, TY, NT, NY, CARRY>;
  return ClassLaunch{&B::launch, &B::partial_bytes, &B::carry_bytes_per_term, TY, name};
}

struct RadClass {
  int rad;
  std::vector<ClassLaunch> cands;   // first = default
  int precision = FBF_FP32;
};

// tensor-core forms: one configuration per (radius class, precision), 128 x 64 tiles
template <int RAD, int PREC>
int tc_launch(const DeviceParams* dparams, const Work* dwork, int n, long long wtot, float* partial, int* counter,
              float2*, int, const SpatialTaps&, cudaStream_t st, int dev) {
  return launch_tc_batch(RAD, PREC, dparams, dwork, n, wtot, partial, counter, st, dev);
}
template <int RAD, int PREC>
ClassLaunch tc_entry(const char* name) {
  ClassLaunch c{&tc_launch<RAD, PREC>, &tc_batch_partial_bytes, &no_carry, tc_tile_rows(RAD, PREC), name};
  c.TX = 128;
  return c;
}

const std::vector<RadClass>& classes() {
  static const std::vector<RadClass> cls = {
      {3, {cfg_entry<3, 112, 512, 7>("r3_ty112_nt512")}},
      {6, {cfg_entry<6, 112, 512, 7>("r6_ty112_nt512"), cfg_entry<6, 128, 256, 16>("r6_ty128_nt256")}},
      {9, {cfg_entry<9, 96, 512, 6>("r9_ty96_nt512")}},
      {15, {cfg_entry<15, 96, 512, 6>("r15_ty96_nt512"), cfg_entry<15, 128, 256, 16>("r15_ty128_nt256")}},
      {24, {cfg_entry<24, 96, 384, 8, true>("r24_ty96_nt384_carry"), cfg_entry<24, 128, 256, 16, true>("r24_ty128_nt256_carry"),
            cfg_entry<24, 128, 256, 16>("r24_ty128_nt256")}},
      {30, {cfg_entry<30, 96, 384, 8, true>("r30_ty96_nt384_carry"), cfg_entry<30, 128, 256, 16, true>("r30_ty128_nt256_carry"),
            cfg_entry<30, 128, 256, 16>("r30_ty128_nt256"), cfg_entry<30, 96, 256, 12>("r30_ty96_nt256")}},
      {48, {cfg_entry<48, 64, 128, 16, true>("r48_ty64_nt128_carry"), cfg_entry<48, 64, 128, 16>("r48_ty64_nt128")}},
      {6, {tc_entry<6, FBF_FP16_TC>("tc_fp16_r6")}, FBF_FP16_TC},
      {15, {tc_entry<15, FBF_FP16_TC>("tc_fp16_r15")}, FBF_FP16_TC},
      {30, {tc_entry<30, FBF_FP16_TC>("tc_fp16_r30")}, FBF_FP16_TC},
      {6, {tc_entry<6, FBF_BF16_TC>("tc_bf16_r6")}, FBF_BF16_TC},
      {15, {tc_entry<15, FBF_BF16_TC>("tc_bf16_r15")}, FBF_BF16_TC},
      {30, {tc_entry<30, FBF_BF16_TC>("tc_bf16_r30")}, FBF_BF16_TC},
  };
  return cls;
}

// the narrowest class of the plan's precision form that holds radius r
int class_of(int r, int precision) {
  const auto& cls = classes();
  for (size_t i = 0; i < cls.size(); ++i)
    if (cls[i].precision == precision && r <= cls[i].rad) return (int)i;
  return -1;
}

DeviceParams padded(const DeviceParams& dp, int rad) {
  DeviceParams p = dp;
  float g[2 * FBF_MAX_RADIUS + 1];
  for (int i = 0; i <= 2 * rad; ++i) {
    const int d = i - (rad - dp.r);
    g[i] = (d >= 0 && d <= 2 * dp.r) ? dp.g[d] : 0.f;
  }
  for (int i = 0; i <= 2 * rad; ++i) p.g[i] = g[i];
  p.r = rad;
  return p;
}

// ---- autotuner cache ----------------------------------------------------------------------
std::mutex g_tune_mu;
std::map<std::string, std::string> g_tune;   // key -> candidate name
bool g_tune_loaded = false;

std::string tune_key(int dev, int cls, long long pixels, int kmax) {
  cudaDeviceProp prop{};
  cudaGetDeviceProperties(&prop, dev);
  int lg = 0;
  while ((1LL << (lg + 1)) <= pixels) ++lg;
  std::string name(prop.name);
  for (auto& ch : name)
    if (ch == ' ') ch = '_';
  return name + "/r" + std::to_string(classes()[cls].rad) + "/px2^" + std::to_string(lg) + "/K" +
         std::to_string(kmax);
}

void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = std::getenv("FBF_TUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  // one "key name" pair per line; other lines are ignored, later lines win, and a name is
  // resolved within the key's own class when it is used
  char line[512], key[256], cfg[128], extra[2];
  while (std::fgets(line, sizeof(line), f))
    if (std::sscanf(line, "%255s %127s %1s", key, cfg, extra) == 2) g_tune[key] = cfg;
  std::fclose(f);
}

void tune_store_locked(const std::string& key, const char* cfg) {
  const char* path = std::getenv("FBF_TUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s %s\n", key.c_str(), cfg);
  std::fclose(f);
}

}  // namespace

// ---- the batch object ------------------------------------------------------------------------
struct Pending {
  DeviceParams dp;                       // the plan's constants, copied at submit
  int r, precision;
  const float* in;
  float* out;
  int H, W;
  size_t pitch;
};

struct Generation {
  unsigned long long id;
  cudaEvent_t ev;
};

struct Batch {
  int max_images = 0;
  int flags = 0;
  int dev = -1;
  std::vector<Pending> pending;
  unsigned long long next_gen = 1;       // generation the pending images will belong to
  std::vector<Generation> gens;          // launched, not yet known complete
  unsigned long long done_below = 1;     // every generation < done_below is complete
  // work-list buffers: a ring for fbf_launch (a slot is rewritten only after the copy that
  // read it has run) and one slot owned by the captured graph
  static constexpr int kRing = 4;
  struct ListBuf {
    void* h = nullptr;                   // pinned staging
    void* d = nullptr;
    size_t cap = 0;
    cudaEvent_t copied = nullptr;        // recorded after the copy out of h
    bool pending = false;
  };
  ListBuf ring[kRing + 1];               // [kRing] belongs to the graph
  int slot = 0;                          // slot in use by the current prepare/launch
  unsigned long long launches = 0;
  // split-tile scratch (tile counters, then partial sums): [0] for fbf_launch, [1] owned by
  // the captured graph, whose kernels have its addresses baked in
  struct ScratchBuf {
    void* d = nullptr;
    size_t counter_cap = 0, partial_cap = 0;
  };
  ScratchBuf scratch[2];
  // graph
  cudaGraphExec_t graph = nullptr;
  cudaStream_t capture_stream = nullptr;
  std::vector<cudaEvent_t> free_events;
  std::mutex mu;
};

namespace {

int ensure_device(Batch* b) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_batch: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= 64) return set_error(FBF_EUNSUPPORTED, "fbf_batch: device index >= 64");
  if (b->dev >= 0 && b->dev != dev) return set_error(FBF_EINVAL, "fbf_batch: batch used on another device");
  b->dev = dev;
  return FBF_OK;
}

// One launch: the images of one radius class (FP32: and one spatial kernel, whose taps the
// kernel takes from its parameters)
struct ClassPlan {
  int cls = -1;
  int cand = 0;
  SpatialTaps taps{};
  std::vector<Work> works;
  std::vector<DeviceParams> params;
  long long wtot = 0, tiles = 0, pixels = 0;
  int kmax = 0;
  size_t params_off = 0, work_off = 0;    // offsets in the lists buffer
};

// group the pending images by radius class and lay out the device lists
int build_lists(Batch* b, std::vector<ClassPlan>* out, size_t* bytes) {
  // FP32 classes: one launch per distinct spatial kernel (padded taps) within the class, in
  // order of first appearance; tensor-core classes stage each image's taps themselves
  std::map<std::pair<int, int>, ClassPlan> by;
  std::map<int, std::vector<SpatialTaps>> tapsets;
  for (const Pending& pd : b->pending) {
    const int cls = class_of(pd.r, pd.precision);
    if (cls < 0) return set_error(FBF_EUNSUPPORTED, "fbf_batch: radius too large");
    const int rad = classes()[cls].rad;
    const DeviceParams q = padded(pd.dp, rad);
    SpatialTaps tq{};
    for (int i = 0; i <= 2 * rad; ++i) tq.g[i] = q.g[i];
    int ts = 0;
    if (classes()[cls].precision == FBF_FP32) {
      std::vector<SpatialTaps>& seen = tapsets[cls];
      ts = -1;
      for (size_t i = 0; i < seen.size() && ts < 0; ++i)
        if (std::memcmp(seen[i].g, tq.g, sizeof(tq.g)) == 0) ts = (int)i;
      if (ts < 0) {
        seen.push_back(tq);
        ts = (int)seen.size() - 1;
      }
    }
    ClassPlan& cp = by[{cls, ts}];
    cp.cls = cls;
    cp.taps = tq;
    // one DeviceParams per distinct plan in the launch
    int pidx = -1;
    for (size_t i = 0; i < cp.params.size() && pidx < 0; ++i)
      if (std::memcmp(&q, &cp.params[i], sizeof(DeviceParams)) == 0) pidx = (int)i;
    if (pidx < 0) {
      cp.params.push_back(q);
      pidx = (int)cp.params.size() - 1;
    }
    Work w{};
    w.in = pd.in;
    w.out = pd.out;
    w.pitch = (long long)pd.pitch;
    w.H = pd.H;
    w.row1 = pd.H;
    w.W = pd.W;
    w.K = pd.dp.K;
    w.wtile = 2 * w.K - 1;
    w.param_idx = pidx;
    cp.works.push_back(w);
    cp.pixels += (long long)pd.H * pd.W;
    cp.kmax = std::max(cp.kmax, w.K);
  }
  size_t off = 0;
  for (auto& kv : by) {
    ClassPlan cp = kv.second;
    cp.params_off = off;
    off += ((cp.params.size() * sizeof(DeviceParams) + 255) / 256) * 256;
    cp.work_off = off;
    off += ((cp.works.size() * sizeof(Work) + 255) / 256) * 256;
    out->push_back(cp);
  }
  *bytes = off;
  return FBF_OK;
}

// tile geometry of a class plan for candidate `cand`
void layout(ClassPlan& cp, int cand) {
  const int TY = classes()[cp.cls].cands[cand].TY;
  const int TXc = classes()[cp.cls].cands[cand].TX;
  long long wst = 0, tiles = 0;
  for (Work& w : cp.works) {
    w.tiles_x = (w.W + TXc - 1) / TXc;
    w.tiles_y = (w.H + TY - 1) / TY;
    w.tiles = (long long)w.tiles_x * w.tiles_y;
    w.wstart = wst;
    w.counter_base = (int)tiles;
    wst += w.tiles * w.wtile;
    tiles += w.tiles;
  }
  cp.wtot = wst;
  cp.tiles = tiles;
  cp.cand = cand;
}

// The scratch set of the current prepare: the graph's when capturing (slot kRing).
Batch::ScratchBuf& cur_scratch(Batch* b) { return b->scratch[b->slot == Batch::kRing ? 1 : 0]; }

// Drop the captured graph before a buffer it reads is freed (a later replay is refused on
// the host instead of touching freed memory).
void drop_graph_if_owned(Batch* b) {
  if (b->slot == Batch::kRing && b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
}

int ensure_buffers(Batch* b, size_t list_bytes, size_t counters, size_t partial, cudaStream_t st) {
  cudaError_t e;
  Batch::ListBuf& lb = b->ring[b->slot];
  if (lb.pending) {   // the copy that last read this slot must have run
    e = cudaEventSynchronize(lb.copied);
    if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_batch: ") + cudaGetErrorString(e));
    lb.pending = false;
  }
  if (!lb.copied) {
    e = cudaEventCreateWithFlags(&lb.copied, cudaEventDisableTiming);
    if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_batch: ") + cudaGetErrorString(e));
  }
  // Buffers grow rarely (at least 1 MiB of work-lists, then doubling): a regrowth waits for
  // the work that may still read the old buffer -- the graph's replays may run on any stream
  // (the device), a launch's on its own stream (launches of a batch are ordered).
  const bool graph_slot = b->slot == Batch::kRing;
  auto drain_old = [&]() { return graph_slot ? cudaDeviceSynchronize() : cudaStreamSynchronize(st); };
  if (lb.cap < list_bytes) {
    drop_graph_if_owned(b);
    if (lb.d) {
      e = drain_old();
      if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_batch: ") + cudaGetErrorString(e));
      cudaFree(lb.d);
    }
    if (lb.h) cudaFreeHost(lb.h);
    lb.h = lb.d = nullptr;
    const size_t cap = std::max(2 * list_bytes, (size_t)1 << 20);
    lb.cap = 0;
    e = cudaMallocHost(&lb.h, cap);
    if (e != cudaSuccess) {
      lb.h = nullptr;
      return set_error(FBF_ENOMEM, std::string("fbf_batch: ") + cudaGetErrorString(e));
    }
    e = cudaMalloc(&lb.d, cap);
    if (e != cudaSuccess) {
      lb.d = nullptr;
      return set_error(FBF_ENOMEM, std::string("fbf_batch: ") + cudaGetErrorString(e));
    }
    lb.cap = cap;
  }
  Batch::ScratchBuf& sb = cur_scratch(b);
  if (sb.counter_cap < counters || sb.partial_cap < partial) {
    drop_graph_if_owned(b);
    if (sb.d) {
      e = drain_old();
      if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_batch: ") + cudaGetErrorString(e));
      cudaFree(sb.d);
    }
    sb.d = nullptr;
    sb.counter_cap = sb.partial_cap = 0;
    const size_t cc = std::max(2 * counters, (size_t)1 << 16);
    const size_t pc = partial + partial / 2;
    const size_t cbytes = ((cc * sizeof(int) + 255) / 256) * 256;
    e = cudaMalloc(&sb.d, cbytes + pc);
    if (e != cudaSuccess) {
      sb.d = nullptr;
      return set_error(FBF_ENOMEM, std::string("fbf_batch: ") + cudaGetErrorString(e));
    }
    // counters start at zero (launches leave them at zero), cleared in the order of the
    // stream that launches next, which may be a non-blocking one
    e = cudaMemsetAsync(sb.d, 0, cbytes, st);
    if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_batch: ") + cudaGetErrorString(e));
    sb.counter_cap = cc;
    sb.partial_cap = pc;
  }
  return FBF_OK;
}

int* scratch_counters(Batch* b) { return reinterpret_cast<int*>(cur_scratch(b).d); }
float* scratch_partials(Batch* b) {
  const Batch::ScratchBuf& sb = cur_scratch(b);
  const size_t cbytes = ((sb.counter_cap * sizeof(int) + 255) / 256) * 256;
  return reinterpret_cast<float*>(static_cast<char*>(sb.d) + cbytes);
}

void write_lists(Batch* b, const std::vector<ClassPlan>& cps) {
  char* h = static_cast<char*>(b->ring[b->slot].h);
  for (const ClassPlan& cp : cps) {
    std::memcpy(h + cp.params_off, cp.params.data(), cp.params.size() * sizeof(DeviceParams));
    std::memcpy(h + cp.work_off, cp.works.data(), cp.works.size() * sizeof(Work));
  }
}

// scratch bytes of one class launch: its partial sums (256-byte aligned, `part`) and, for a
// configuration that carries x-pass rows, the slots for kmax terms after them (`total`)
int class_scratch_bytes(const ClassLaunch& cl, int dev, int kmax, size_t* part, size_t* total) {
  size_t pb = 0, cb = 0;
  int rc = cl.partial_bytes(dev, &pb);
  if (rc == FBF_OK) rc = cl.carry_bytes_per_term(dev, &cb);
  if (rc != FBF_OK) return rc;
  *part = (pb + 255) / 256 * 256;
  *total = *part + cb * (size_t)kmax;
  return FBF_OK;
}

int launch_classes(Batch* b, const std::vector<ClassPlan>& cps, size_t list_bytes, cudaStream_t st,
                   bool capturing) {
  Batch::ListBuf& lb = b->ring[b->slot];
  cudaError_t e = cudaMemcpyAsync(lb.d, lb.h, list_bytes, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_batch: ") + cudaGetErrorString(e));
  if (!capturing) {
    e = cudaEventRecord(lb.copied, st);
    if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_batch: ") + cudaGetErrorString(e));
    lb.pending = true;
  }
  char* d = static_cast<char*>(lb.d);
  for (const ClassPlan& cp : cps) {
    const ClassLaunch& cl = classes()[cp.cls].cands[cp.cand];
    size_t part = 0, total = 0;
    int rc = class_scratch_bytes(cl, b->dev, cp.kmax, &part, &total);
    if (rc != FBF_OK) return rc;
    // the class's carried-row slots follow its partial sums (classes run one after another)
    float2* carry = total > part ? reinterpret_cast<float2*>(reinterpret_cast<char*>(scratch_partials(b)) + part)
                                 : nullptr;
    rc = cl.launch(reinterpret_cast<const DeviceParams*>(d + cp.params_off),
                   reinterpret_cast<const Work*>(d + cp.work_off), (int)cp.works.size(), cp.wtot,
                   scratch_partials(b), scratch_counters(b), carry, cp.kmax, cp.taps, st, b->dev);
    if (rc != FBF_OK) return rc;
  }
  return FBF_OK;
}

// choose a candidate per class (autotuned or default) and size the buffers
int prepare(Batch* b, std::vector<ClassPlan>* cps, size_t* list_bytes, cudaStream_t st, bool allow_tune) {
  int rc = build_lists(b, cps, list_bytes);
  if (rc != FBF_OK) return rc;
  size_t counters = 0, partial = 0;
  for (ClassPlan& cp : *cps) {
    const auto& cands = classes()[cp.cls].cands;
    int choice = 0;
    if ((b->flags & FBF_BATCH_AUTOTUNE) && cands.size() > 1) {
      const std::string key = tune_key(b->dev, cp.cls, cp.pixels, cp.kmax);
      int cached = -1;
      {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_load_locked();
        auto it = g_tune.find(key);
        for (size_t j = 0; it != g_tune.end() && j < cands.size(); ++j)
          if (it->second == cands[j].name) cached = (int)j;
      }
      if (cached >= 0) {
        choice = cached;
      } else if (allow_tune) {
        // time every candidate on this class's real work-list (outputs are rewritten later)
        float best = 1e30f;
        for (size_t j = 0; j < cands.size(); ++j) {
          ClassPlan one = cp;
          layout(one, (int)j);
          size_t part = 0, pb = 0;
          rc = class_scratch_bytes(cands[j], b->dev, one.kmax, &part, &pb);
          if (rc != FBF_OK) return rc;
          rc = ensure_buffers(b, *list_bytes, (size_t)one.tiles, pb, st);
          if (rc != FBF_OK) return rc;
          std::vector<ClassPlan> v{one};
          write_lists(b, v);
          cudaEvent_t e0 = nullptr, e1 = nullptr;
          cudaError_t ee = cudaEventCreate(&e0);
          if (ee == cudaSuccess) ee = cudaEventCreate(&e1);
          if (ee != cudaSuccess) {
            if (e0) cudaEventDestroy(e0);
            return set_error(FBF_ECUDA, std::string("fbf_batch: autotune: ") + cudaGetErrorString(ee));
          }
          float ms_best = 1e30f;
          for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, st);
            rc = launch_classes(b, v, *list_bytes, st, false);
            cudaEventRecord(e1, st);
            if (rc != FBF_OK) break;
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) ms_best = std::min(ms_best, ms);
          }
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          if (rc != FBF_OK) return rc;
          if (ms_best < best) { best = ms_best; choice = (int)j; }
        }
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = cands[choice].name;
        tune_store_locked(key, cands[choice].name);
      }
    }
    layout(cp, choice);
    size_t part = 0, pb = 0;
    rc = class_scratch_bytes(cands[choice], b->dev, cp.kmax, &part, &pb);
    if (rc != FBF_OK) return rc;
    counters = std::max(counters, (size_t)cp.tiles);
    partial = std::max(partial, pb);
  }
  rc = ensure_buffers(b, *list_bytes, counters, partial, st);
  if (rc != FBF_OK) return rc;
  write_lists(b, *cps);
  return FBF_OK;
}

int record_generation(Batch* b, cudaStream_t st, unsigned long long* gen_out) {
  cudaEvent_t ev;
  if (!b->free_events.empty()) {
    ev = b->free_events.back();
    b->free_events.pop_back();
  } else {
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_batch: ") + cudaGetErrorString(e));
  }
  cudaError_t e = cudaEventRecord(ev, st);
  if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_batch: ") + cudaGetErrorString(e));
  const unsigned long long g = b->next_gen++;
  b->gens.push_back({g, ev});
  *gen_out = g;
  // keep the outstanding list bounded: the oldest generations are waited for
  while (b->gens.size() > 1024) {
    cudaEventSynchronize(b->gens.front().ev);
    b->free_events.push_back(b->gens.front().ev);
    b->done_below = b->gens.front().id + 1;
    b->gens.erase(b->gens.begin());
  }
  return FBF_OK;
}

// status of a generation: FBF_DONE, FBF_PENDING, or an error code
int gen_status(Batch* b, unsigned long long g) {
  if (g >= b->next_gen) return FBF_PENDING;   // not launched yet
  if (g < b->done_below) return FBF_DONE;
  // complete generations at the front are retired in order
  while (!b->gens.empty()) {
    cudaError_t e = cudaEventQuery(b->gens.front().ev);
    if (e == cudaErrorNotReady) break;
    if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string("fbf_batch_poll: ") + cudaGetErrorString(e));
    b->done_below = b->gens.front().id + 1;
    b->free_events.push_back(b->gens.front().ev);
    b->gens.erase(b->gens.begin());
  }
  if (g < b->done_below) return FBF_DONE;
  for (const Generation& gen : b->gens) {
    if (gen.id == g) {
      cudaError_t e = cudaEventQuery(gen.ev);
      if (e == cudaSuccess) return FBF_DONE;
      if (e == cudaErrorNotReady) return FBF_PENDING;
      return set_error(FBF_ECUDA, std::string("fbf_batch_poll: ") + cudaGetErrorString(e));
    }
  }
  return FBF_DONE;
}

}  // namespace
}  // namespace fbf

struct fbf_batch_s {
  fbf::Batch b;
};

extern "C" {

int fbf_batch_create(fbf_batch_t* out, int max_images, int flags) try {
  if (!out) return fbf::set_error(FBF_EINVAL, "fbf_batch_create: out is NULL");
  *out = nullptr;
  if (max_images < 1) return fbf::set_error(FBF_EINVAL, "fbf_batch_create: max_images must be >= 1");
  if (flags & ~FBF_BATCH_AUTOTUNE) return fbf::set_error(FBF_EINVAL, "fbf_batch_create: unknown flag");
  fbf_batch_s* h = new (std::nothrow) fbf_batch_s();
  if (!h) return fbf::set_error(FBF_ENOMEM, "fbf_batch_create: out of host memory");
  h->b.max_images = max_images;
  h->b.flags = flags;
  *out = h;
  return FBF_OK;
} FBF_ABI_CATCH("fbf_batch_create")

int fbf_batch_submit(fbf_batch_t batch, fbf_plan_t plan, const float* d_in, float* d_out, int H, int W,
                     size_t pitch_elems, fbf_ticket_t* ticket) try {
  if (!batch || !plan) return fbf::set_error(FBF_EINVAL, "fbf_batch_submit: NULL batch or plan");
  if (!d_in || !d_out) return fbf::set_error(FBF_EINVAL, "fbf_batch_submit: NULL image pointer");
  if (H < 1 || W < 1) return fbf::set_error(FBF_EINVAL, "fbf_batch_submit: H and W must be >= 1");
  if (pitch_elems < (size_t)W) return fbf::set_error(FBF_EINVAL, "fbf_batch_submit: pitch < W");
  const fbf::Plan* p = fbf::plan_of(plan);
  if (fbf::class_of(p->r, p->precision) < 0)
    return fbf::set_error(FBF_EUNSUPPORTED, "fbf_batch_submit: radius too large for the plan's form");
  const size_t span = ((size_t)(H - 1) * pitch_elems + (size_t)W) * sizeof(float);
  const char* a = (const char*)d_in;
  const char* o = (const char*)d_out;
  if (a < o + span && o < a + span) return fbf::set_error(FBF_EINVAL, "fbf_batch_submit: in and out overlap");
  fbf::Batch& b = batch->b;
  std::lock_guard<std::mutex> lk(b.mu);
  if ((int)b.pending.size() >= b.max_images) return fbf::set_error(FBF_EBUSY, "fbf_batch_submit: batch is full");
  b.pending.push_back({p->dp, p->r, p->precision, d_in, d_out, H, W, pitch_elems});
  if (ticket) *ticket = (fbf_ticket_t)b.next_gen;
  return FBF_OK;
} FBF_ABI_CATCH("fbf_batch_submit")

// Empties a batch's queue when the call that took its images returns, whether or not the
// launch or capture succeeded: after an error the caller may free the images' buffers, so
// they must not stay queued for the next launch.
struct EmptyQueueOnExit {
  fbf::Batch& b;
  ~EmptyQueueOnExit() { b.pending.clear(); }
};

int fbf_launch(fbf_batch_t batch, void* cuda_stream) try {
  const fbf::NvtxRange tr("fbf_launch");
  if (!batch) return fbf::set_error(FBF_EINVAL, "fbf_launch: batch is NULL");
  fbf::Batch& b = batch->b;
  std::lock_guard<std::mutex> lk(b.mu);
  if (b.pending.empty()) return FBF_OK;
  EmptyQueueOnExit empty_on_exit{b};
  int rc = fbf::ensure_device(&b);
  if (rc != FBF_OK) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  b.slot = (int)(b.launches % fbf::Batch::kRing);
  std::vector<fbf::ClassPlan> cps;
  size_t list_bytes = 0;
  rc = fbf::prepare(&b, &cps, &list_bytes, st, true);
  if (rc != FBF_OK) return rc;
  rc = fbf::launch_classes(&b, cps, list_bytes, st, false);
  if (rc != FBF_OK) return rc;
  unsigned long long g = 0;
  rc = fbf::record_generation(&b, st, &g);
  if (rc != FBF_OK) return rc;
  ++b.launches;
  return FBF_OK;
} FBF_ABI_CATCH("fbf_launch")

int fbf_batch_capture(fbf_batch_t batch, void* cuda_stream) try {
  const fbf::NvtxRange tr("fbf_batch_capture");
  if (!batch) return fbf::set_error(FBF_EINVAL, "fbf_batch_capture: batch is NULL");
  fbf::Batch& b = batch->b;
  std::lock_guard<std::mutex> lk(b.mu);
  if (b.pending.empty()) return fbf::set_error(FBF_EINVAL, "fbf_batch_capture: no submitted images");
  EmptyQueueOnExit empty_on_exit{b};
  int rc = fbf::ensure_device(&b);
  if (rc != FBF_OK) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  b.slot = fbf::Batch::kRing;   // the graph owns this slot's staging and device lists
  std::vector<fbf::ClassPlan> cps;
  size_t list_bytes = 0;
  rc = fbf::prepare(&b, &cps, &list_bytes, st, true);   // tuning and allocation happen here
  if (rc != FBF_OK) return rc;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fbf::set_error(FBF_ECUDA, std::string("fbf_batch_capture: ") + cudaGetErrorString(e));
  // capture on the batch's own stream: the caller's may be the legacy default stream,
  // which cannot be captured; the graph is later launched on any stream
  if (!b.capture_stream) {
    e = cudaStreamCreateWithFlags(&b.capture_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fbf::set_error(FBF_ECUDA, std::string("fbf_batch_capture: ") + cudaGetErrorString(e));
  }
  cudaGraph_t graph = nullptr;
  e = cudaStreamBeginCapture(b.capture_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return fbf::set_error(FBF_ECUDA, std::string("fbf_batch_capture: ") + cudaGetErrorString(e));
  rc = fbf::launch_classes(&b, cps, list_bytes, b.capture_stream, true);
  e = cudaStreamEndCapture(b.capture_stream, &graph);
  if (rc != FBF_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return fbf::set_error(FBF_ECUDA, std::string("fbf_batch_capture: ") + cudaGetErrorString(e));
  if (b.graph) cudaGraphExecDestroy(b.graph);
  b.graph = nullptr;
  e = cudaGraphInstantiate(&b.graph, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fbf::set_error(FBF_ECUDA, std::string("fbf_batch_capture: ") + cudaGetErrorString(e));
  return FBF_OK;
} FBF_ABI_CATCH("fbf_batch_capture")

int fbf_batch_replay(fbf_batch_t batch, void* cuda_stream, fbf_ticket_t* ticket) try {
  const fbf::NvtxRange tr("fbf_batch_replay");
  if (!batch) return fbf::set_error(FBF_EINVAL, "fbf_batch_replay: batch is NULL");
  fbf::Batch& b = batch->b;
  std::lock_guard<std::mutex> lk(b.mu);
  if (!b.graph) return fbf::set_error(FBF_EINVAL, "fbf_batch_replay: nothing captured");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaGraphLaunch(b.graph, st);
  if (e != cudaSuccess) return fbf::set_error(FBF_ECUDA, std::string("fbf_batch_replay: ") + cudaGetErrorString(e));
  unsigned long long g = 0;
  int rc = fbf::record_generation(&b, st, &g);
  if (rc != FBF_OK) return rc;
  if (ticket) *ticket = (fbf_ticket_t)g;
  return FBF_OK;
} FBF_ABI_CATCH("fbf_batch_replay")

int fbf_batch_poll(fbf_batch_t batch, fbf_ticket_t ticket, int* status) try {
  if (!batch || !status) return fbf::set_error(FBF_EINVAL, "fbf_batch_poll: NULL argument");
  fbf::Batch& b = batch->b;
  std::lock_guard<std::mutex> lk(b.mu);
  const int s = fbf::gen_status(&b, (unsigned long long)ticket);
  if (s != FBF_DONE && s != FBF_PENDING) return s;
  *status = s;
  return FBF_OK;
} FBF_ABI_CATCH("fbf_batch_poll")

int fbf_batch_wait(fbf_batch_t batch, fbf_ticket_t ticket, double timeout_s) try {
  if (!batch) return fbf::set_error(FBF_EINVAL, "fbf_batch_wait: batch is NULL");
  if (!(timeout_s >= 0)) return fbf::set_error(FBF_EINVAL, "fbf_batch_wait: timeout must be >= 0");
  const auto t0 = std::chrono::steady_clock::now();
  while (true) {
    int s;
    {
      std::lock_guard<std::mutex> lk(batch->b.mu);
      s = fbf::gen_status(&batch->b, (unsigned long long)ticket);
    }
    if (s == FBF_DONE) return FBF_OK;
    if (s != FBF_PENDING) return s;
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (el >= timeout_s) return fbf::set_error(FBF_ETIMEDOUT, "fbf_batch_wait: timed out");
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
} FBF_ABI_CATCH("fbf_batch_wait")

int fbf_batch_pending(fbf_batch_t batch, int* n) try {
  if (!batch || !n) return fbf::set_error(FBF_EINVAL, "fbf_batch_pending: NULL argument");
  std::lock_guard<std::mutex> lk(batch->b.mu);
  *n = (int)batch->b.pending.size();
  return FBF_OK;
} FBF_ABI_CATCH("fbf_batch_pending")

int fbf_batch_destroy(fbf_batch_t batch) try {
  if (!batch) return FBF_OK;
  fbf::Batch& b = batch->b;
  for (auto& g : b.gens) {
    cudaEventSynchronize(g.ev);
    cudaEventDestroy(g.ev);
  }
  for (auto ev : b.free_events) cudaEventDestroy(ev);
  if (b.graph) cudaGraphExecDestroy(b.graph);
  if (b.capture_stream) cudaStreamDestroy(b.capture_stream);
  for (auto& lb : b.ring) {
    if (lb.copied) { cudaEventSynchronize(lb.copied); cudaEventDestroy(lb.copied); }
    if (lb.d) cudaFree(lb.d);
    if (lb.h) cudaFreeHost(lb.h);
  }
  for (auto& sb : b.scratch)
    if (sb.d) cudaFree(sb.d);
  delete batch;
  return FBF_OK;
} FBF_ABI_CATCH("fbf_batch_destroy")

}  // extern "C"

// ---- implicit per-device queue (fbf_submit / fbf_poll / fbf_wait) -----------------------------
// One batch and one non-blocking stream per device, created on first use and kept until the
// process exits.  A ticket carries its device: bits 48..55 hold device + 1, the low 48 bits
// the batch generation.
namespace fbf {
namespace {

constexpr int kImplicitMax = 4096;        // images per implicit launch
constexpr int kTicketShift = 48;

struct Implicit {
  fbf_batch_s* batch = nullptr;
  cudaStream_t st = nullptr;
};
std::mutex g_impl_mu;
Implicit g_impl[64];

// the implicit queue of device `dev` (created when `create`); nullptr with the error set
Implicit* implicit_of(int dev, bool create, const char* who) {
  if (dev < 0 || dev >= 64) {
    set_error(FBF_EINVAL, std::string(who) + ": unknown ticket");
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_impl_mu);
  Implicit& q = g_impl[dev];
  if (!q.batch) {
    if (!create) {
      set_error(FBF_EINVAL, std::string(who) + ": unknown ticket");
      return nullptr;
    }
    cudaStream_t st = nullptr;
    const cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      set_error(FBF_ECUDA, std::string(who) + ": " + cudaGetErrorString(e));
      return nullptr;
    }
    fbf_batch_t b = nullptr;
    if (fbf_batch_create(&b, kImplicitMax, 0) != FBF_OK) {
      cudaStreamDestroy(st);
      return nullptr;
    }
    q.batch = b;
    q.st = st;
  }
  return &q;
}

// launch the device's queue if the ticket's generation is still queued (on the device's
// own stream, with that device current)
int flush_for(Implicit* q, int dev, unsigned long long gen, const char* who) {
  int cur = 0;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return set_error(FBF_ECUDA, std::string(who) + ": " + cudaGetErrorString(e));
  int rc = FBF_OK;
  bool queued;
  {
    std::lock_guard<std::mutex> lk(q->batch->b.mu);
    queued = gen >= q->batch->b.next_gen;
  }
  if (queued) {
    if (cur != dev && (e = cudaSetDevice(dev)) != cudaSuccess)
      return set_error(FBF_ECUDA, std::string(who) + ": " + cudaGetErrorString(e));
    rc = fbf_launch(q->batch, q->st);
    if (cur != dev) cudaSetDevice(cur);
  }
  return rc;
}

}  // namespace
}  // namespace fbf

extern "C" {

int fbf_submit(fbf_plan_t plan, const float* d_in, float* d_out, int H, int W, size_t pitch_elems,
               fbf_ticket_t* ticket) try {
  int dev = 0;
  const cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fbf::set_error(FBF_ECUDA, std::string("fbf_submit: ") + cudaGetErrorString(e));
  fbf::Implicit* q = fbf::implicit_of(dev, true, "fbf_submit");
  if (!q) return FBF_ECUDA;
  fbf_ticket_t t = 0;
  int rc = fbf_batch_submit(q->batch, plan, d_in, d_out, H, W, pitch_elems, &t);
  if (rc == FBF_EBUSY) {   // a full queue is launched and the image starts the next one
    rc = fbf_launch(q->batch, q->st);
    if (rc == FBF_OK) rc = fbf_batch_submit(q->batch, plan, d_in, d_out, H, W, pitch_elems, &t);
  }
  if (rc != FBF_OK) return rc;
  if (ticket) *ticket = ((fbf_ticket_t)(dev + 1) << fbf::kTicketShift) | t;
  return FBF_OK;
} FBF_ABI_CATCH("fbf_submit")

int fbf_poll(fbf_ticket_t ticket, int* status) try {
  if (!status) return fbf::set_error(FBF_EINVAL, "fbf_poll: status is NULL");
  const int dev = (int)(ticket >> fbf::kTicketShift) - 1;
  const unsigned long long gen = ticket & ((1ull << fbf::kTicketShift) - 1);
  fbf::Implicit* q = fbf::implicit_of(dev, false, "fbf_poll");
  if (!q) return FBF_EINVAL;
  int rc = fbf::flush_for(q, dev, gen, "fbf_poll");
  if (rc != FBF_OK) return rc;
  return fbf_batch_poll(q->batch, gen, status);
} FBF_ABI_CATCH("fbf_poll")

int fbf_wait(fbf_ticket_t ticket, double timeout_s) try {
  if (!(timeout_s >= 0)) return fbf::set_error(FBF_EINVAL, "fbf_wait: timeout must be >= 0");
  const int dev = (int)(ticket >> fbf::kTicketShift) - 1;
  const unsigned long long gen = ticket & ((1ull << fbf::kTicketShift) - 1);
  fbf::Implicit* q = fbf::implicit_of(dev, false, "fbf_wait");
  if (!q) return FBF_EINVAL;
  int rc = fbf::flush_for(q, dev, gen, "fbf_wait");
  if (rc != FBF_OK) return rc;
  return fbf_batch_wait(q->batch, gen, timeout_s);
} FBF_ABI_CATCH("fbf_wait")

}  // extern "C"
