// fbf_filter_host: one image from host memory to host memory.
//
// Page-locked buffers (mapped into the device's address space, distinct): the kernel reads
// the image and writes the result through the host link directly, with no staging copies;
// the transfers spread over the launch instead of preceding and following it.  Otherwise
// (pageable memory, or in place) the image is staged through device memory, with the
// copies overlapped with the filter as follows.
//
// The image is cut into B bands of whole tile rows (1 to 4 bands, each with at least two tiles
// per SM; small images are one band).  On an upload stream each
// band's rows are copied into a device image in two pieces, its first r rows and then the
// rest, with an event after each; the filter of band b (the kernels' row-band launch:
// output rows of the band only, halo rows read from the whole device image) waits for all
// of band b and for the first r rows of band b + 1, so the uploads of later bands overlap
// the kernels of earlier ones; band b's result is copied back on a download stream as soon
// as its launch has run, overlapping the later launches.  The call returns once the result
// is on the host.  Device images and the two copy streams are kept per (device, stream) and
// reused; rows of the device image are padded to 16 bytes (the kernels' TMA staging needs
// 16-byte-aligned rows).
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <utility>

#include "fbf.h"
#include "fbf_internal.h"

namespace {

constexpr int kMaxBands = 4;

struct HostCtx {
  std::mutex mu;                       // one call on the context at a time
  float* d_in = nullptr;
  float* d_out = nullptr;
  size_t cap = 0;                      // floats per device image
  cudaStream_t up = nullptr, down = nullptr;
  cudaEvent_t ev_head[kMaxBands] = {}; // first r rows of band b on the device
  cudaEvent_t ev_in[kMaxBands] = {};   // all of band b on the device
  cudaEvent_t ev_k[kMaxBands] = {};    // band b filtered
  cudaEvent_t ev_start = nullptr;      // the caller's stream reached this call
};

std::mutex g_ctx_mu;                   // guards the map only
std::map<std::pair<int, uintptr_t>, std::unique_ptr<HostCtx>> g_ctx;

int fail(const char* what, cudaError_t e) {
  return fbf::set_error(FBF_ECUDA, std::string("fbf_filter_host: ") + what + ": " + cudaGetErrorString(e));
}

// The context of (device, stream), created on first use.
HostCtx* context_of(int dev, cudaStream_t st) {
  std::lock_guard<std::mutex> g(g_ctx_mu);
  std::unique_ptr<HostCtx>& c = g_ctx[{dev, (uintptr_t)st}];
  if (!c) c.reset(new HostCtx());
  return c.get();
}

// Streams, events and device images of at least n floats (context lock held).
int prepare(HostCtx& c, size_t n) {
  cudaError_t e = cudaSuccess;
  if (!c.up) {
    e = cudaStreamCreateWithFlags(&c.up, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c.down, cudaStreamNonBlocking);
    for (int b = 0; b < kMaxBands && e == cudaSuccess; ++b) {
      e = cudaEventCreateWithFlags(&c.ev_head[b], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.ev_in[b], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.ev_k[b], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.ev_start, cudaEventDisableTiming);
    if (e != cudaSuccess) return fail("setup", e);
  }
  if (c.cap < n) {
    // every earlier call on this context has returned, so nothing still uses the old images
    if (c.d_in) cudaFree(c.d_in);
    if (c.d_out) cudaFree(c.d_out);
    c.d_in = c.d_out = nullptr;
    c.cap = 0;
    e = cudaMalloc(&c.d_in, n * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&c.d_out, n * sizeof(float));
    if (e != cudaSuccess) {
      if (c.d_in) cudaFree(c.d_in);
      c.d_in = nullptr;
      return fbf::set_error(FBF_ENOMEM, std::string("fbf_filter_host: device images: ") + cudaGetErrorString(e));
    }
    c.cap = n;
  }
  return FBF_OK;
}

}  // namespace

extern "C" int fbf_filter_host(fbf_plan_t plan, const float* host_in, float* host_out, int H, int W,
                               size_t pitch_elems, void* cuda_stream) try {
  const fbf::NvtxRange tr("fbf_filter_host");
  if (!plan) return fbf::set_error(FBF_EINVAL, "fbf_filter_host: plan is NULL");
  if (!host_in || !host_out) return fbf::set_error(FBF_EINVAL, "fbf_filter_host: NULL image pointer");
  if (H < 1 || W < 1) return fbf::set_error(FBF_EINVAL, "fbf_filter_host: H and W must be >= 1");
  if (pitch_elems < (size_t)W) return fbf::set_error(FBF_EINVAL, "fbf_filter_host: pitch < W");
  {
    // in place (the same buffer) is fine: every row is uploaded before its band is written
    // back; a partial overlap is not
    const size_t span = ((size_t)(H - 1) * pitch_elems + (size_t)W) * sizeof(float);
    const char* a = (const char*)host_in;
    const char* o = (const char*)host_out;
    if (a != o && a < o + span && o < a + span)
      return fbf::set_error(FBF_EINVAL, "fbf_filter_host: in and out partially overlap");
  }
  const fbf::Plan* p = fbf::plan_of(plan);
  const int prec = p->precision;
  if (prec != FBF_FP32 && prec != FBF_FP16_TC && prec != FBF_BF16_TC)
    return fbf::set_error(FBF_EINVAL, "fbf_filter_host: unknown precision form");
  const int r = p->r;
  if (prec != FBF_FP32 && r > FBF_MAX_RADIUS_TC)
    return fbf::set_error(FBF_EUNSUPPORTED, "fbf_filter_host: the tensor-core forms support r <= 30");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail("device", e);

  // bands of whole tile rows (so each at least r rows), at most kMaxBands, and each with at
  // least two tiles per SM: a band launch with fewer tiles per CTA splits more of them and
  // stages f more often, which costs more than the copies its band hides
  const int ty = (prec == FBF_FP32) ? fbf::fp32_tile_rows(r, W, H / kMaxBands)
                                    : fbf::tc_tile_rows(r <= 6 ? 6 : r <= 15 ? 15 : 30, prec);
  const int tx = (prec == FBF_FP32) ? 32 : 128;
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail("device", e);
  const int tile_rows = (H + ty - 1) / ty;
  const int per_row = (W + tx - 1) / tx;
  const int min_rows = std::max(1, (2 * sms + per_row - 1) / per_row);   // tile rows per band
  const int nb = std::max(1, std::min(kMaxBands, tile_rows / min_rows));
  const int per = (tile_rows + nb - 1) / nb;        // tile rows per band (the last may be short)
  int b0[kMaxBands + 1];
  int nbands = 0;
  for (int t = 0; t < tile_rows && nbands < kMaxBands; t += per) b0[nbands++] = t * ty;
  b0[nbands] = H;

  // page-locked, mapped and distinct buffers: the kernel works on host memory directly
  if (host_in != host_out) {
    cudaPointerAttributes ai, ao;
    const bool known = cudaPointerGetAttributes(&ai, host_in) == cudaSuccess &&
                       cudaPointerGetAttributes(&ao, host_out) == cudaSuccess;
    if (!known) cudaGetLastError();
    if (known && ai.type == cudaMemoryTypeHost && ao.type == cudaMemoryTypeHost && ai.devicePointer &&
        ao.devicePointer) {
      const float* din = static_cast<const float*>(ai.devicePointer);
      float* dout = static_cast<float*>(ao.devicePointer);
      int rc0 = (prec == FBF_FP32) ? fbf::launch_fp32(p->dp, din, dout, H, W, pitch_elems, st)
                                   : fbf::launch_tc(p->dp, din, dout, H, W, pitch_elems, st, prec);
      if (rc0 != FBF_OK) return rc0;
      e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return fail("synchronise", e);
      return FBF_OK;
    }
  }

  const size_t dp = ((size_t)W + 3) / 4 * 4;        // device row stride: 16-byte rows
  HostCtx* c = context_of(dev, st);
  std::lock_guard<std::mutex> lk(c->mu);
  int rc = prepare(*c, dp * (size_t)H);
  if (rc != FBF_OK) return rc;

  const size_t hp = pitch_elems * sizeof(float), dpb = dp * sizeof(float), wb = (size_t)W * sizeof(float);
  // rows [y0, y0 + n) between host and device: one linear copy when both are packed alike
  auto copy_rows = [&](float* dst, size_t dst_pitch, const float* src, size_t src_pitch, int n,
                       cudaMemcpyKind kind, cudaStream_t s) {
    if (dst_pitch == src_pitch && dst_pitch == wb)
      return cudaMemcpyAsync(dst, src, wb * (size_t)n, kind, s);
    return cudaMemcpy2DAsync(dst, dst_pitch, src, src_pitch, wb, n, kind, s);
  };
  // on an error after copies were queued, wait for them (best effort) before returning, so
  // that no copy still reads or writes the caller's buffers once the call has returned
  auto drain = [&](int code) {
    cudaStreamSynchronize(st);
    cudaStreamSynchronize(c->up);
    cudaStreamSynchronize(c->down);
    return code;
  };
  if (nbands == 1) {
    // one band: nothing to overlap, so everything stays on the caller's stream
    e = copy_rows(c->d_in, dpb, host_in, hp, H, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return drain(fail("upload", e));
    rc = (prec == FBF_FP32) ? fbf::launch_fp32(p->dp, c->d_in, c->d_out, H, W, dp, st)
                            : fbf::launch_tc(p->dp, c->d_in, c->d_out, H, W, dp, st, prec);
    if (rc != FBF_OK) return drain(rc);
    e = copy_rows(host_out, hp, c->d_out, dpb, H, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return drain(fail("download", e));
    return FBF_OK;
  }
  // uploads start once the caller's stream has reached this call
  e = cudaEventRecord(c->ev_start, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->up, c->ev_start, 0);
  for (int b = 0; b < nbands && e == cudaSuccess; ++b) {
    const int head = std::min(b0[b + 1] - b0[b], std::max(r, 1));
    e = copy_rows(c->d_in + (size_t)b0[b] * dp, dpb, host_in + (size_t)b0[b] * pitch_elems, hp, head,
                  cudaMemcpyHostToDevice, c->up);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_head[b], c->up);
    if (e == cudaSuccess && b0[b + 1] - b0[b] > head)
      e = copy_rows(c->d_in + ((size_t)b0[b] + head) * dp, dpb, host_in + ((size_t)b0[b] + head) * pitch_elems,
                    hp, b0[b + 1] - b0[b] - head, cudaMemcpyHostToDevice, c->up);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_in[b], c->up);
  }
  if (e != cudaSuccess) return drain(fail("upload", e));
  for (int b = 0; b < nbands; ++b) {
    // rows [b0 - r, b1 + r) must be on the device: band b and the head of band b + 1 (the
    // upload stream is in order, so band b's event also covers the bands above it)
    e = cudaStreamWaitEvent(st, c->ev_in[b], 0);
    if (e == cudaSuccess && b + 1 < nbands) e = cudaStreamWaitEvent(st, c->ev_head[b + 1], 0);
    if (e != cudaSuccess) return drain(fail("order", e));
    rc = (prec == FBF_FP32)
             ? fbf::launch_fp32(p->dp, c->d_in, c->d_out, H, W, dp, st, b0[b], b0[b + 1] - b0[b])
             : fbf::launch_tc(p->dp, c->d_in, c->d_out, H, W, dp, st, prec, b0[b], b0[b + 1] - b0[b]);
    if (rc != FBF_OK) return drain(rc);
    e = cudaEventRecord(c->ev_k[b], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->down, c->ev_k[b], 0);
    if (e == cudaSuccess)
      e = copy_rows(host_out + (size_t)b0[b] * pitch_elems, hp, c->d_out + (size_t)b0[b] * dp, dpb,
                    b0[b + 1] - b0[b], cudaMemcpyDeviceToHost, c->down);
    if (e != cudaSuccess) return drain(fail("download", e));
  }
  e = cudaStreamSynchronize(c->down);
  if (e != cudaSuccess) return drain(fail("synchronise", e));
  return FBF_OK;
} FBF_ABI_CATCH("fbf_filter_host")
