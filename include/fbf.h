/*
 * fbf.h -- C ABI of the GB300 (sm_103a) Fourier bilateral filter.
 *
 * Method: Optimized Fourier Bilateral Filtering (Ghosh, Nair, Chaudhury, IEEE Signal
 * Processing Letters 25(10), 2018).  The bilateral filter of eq. (1), with the Gaussian
 * kernels of eq. (2), is computed with the range kernel replaced by the K-term cosine
 * series of eq. (3), phi_hat(t) = sum_{k<K} c_k cos(2 pi k t / (2T+1)).  The period T and
 * the coefficients c are fitted on the host in FP64 by least squares on the integer
 * differences t in {-R..R} (eqs. (4)-(6), Algorithm 1).  On the device, numerator and
 * denominator of eq. (1) become Gaussian convolutions of the images cos(k nu f),
 * sin(k nu f), f cos(k nu f), f sin(k nu f) (Section II, the remark after eq. (3)); the
 * kernels generate those images per tile, blur them and recombine them in one pass, so
 * only f is read from and only f_BF is written to device memory.
 *
 * Conventions for every entry point:
 *   - Return value: FBF_OK (0) or one of the FBF_E* codes below.  No C++ exception
 *     crosses this boundary: a host allocation or a thread that cannot start inside a call
 *     returns FBF_ENOMEM.  fbf_last_error() gives a message for the calling thread.
 *   - Images are single-channel float32, row-major, values in [0, R].  Integer values
 *     (8-bit images converted to float) are the case the paper treats (Lambda holds only
 *     integers, Section II); other values are filtered with the same formula.
 *   - Device pointers are owned by the caller, who keeps them alive until the work that
 *     uses them has completed (stream order, or fbf_poll reporting FBF_DONE).
 *   - Neighbours outside the image are absent from both sums of eq. (1) (zero padding of
 *     every convolved image, including the constant one).
 *   - A pixel whose denominator comes out <= 0 keeps its input value.
 */
#ifndef FBF_H
#define FBF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------------- */
#define FBF_OK         0
#define FBF_EINVAL     1   /* bad argument (see each function)                       */
#define FBF_ENOMEM     2   /* host or device allocation failed                       */
#define FBF_ECUDA      3   /* a CUDA runtime call failed (message in fbf_last_error)  */
#define FBF_ETIMEDOUT  4   /* a bounded wait gave up                                 */
#define FBF_EBUSY      5   /* admission refused: no free slot or over the budget     */
#define FBF_PENDING    6   /* fbf_poll status: submitted work not finished yet        */
#define FBF_DONE       7   /* fbf_poll status: finished                              */
#define FBF_EUNSUPPORTED 8 /* valid request outside what the kernels are built for   */

/* ---- precision forms (fbf_plan's `precision`) --------------------------------- */
#define FBF_FP32       0   /* FP32 channel stack and FP32 FIR on the CUDA cores       */
/* Tensor-core forms: both Gaussian passes of Section II run as banded Toeplitz
   contractions on the tensor cores (tcgen05) with FP32 accumulation.  The x pass takes
   the channel stack and its taps as 16-bit operands; its result is rounded to nearest
   TF32 and contracted with TF32 taps in the y pass.  Recombination and divide are FP32.
   Errors against the FP64 oracle grow where the bilateral denominator is small (a pixel
   unlike its whole window, so that the denominator is little more than the centre tap):
   absolute errors of numerator and denominator are divided by it.                       */
#define FBF_FP16_TC    1   /* FP16 stack and taps (fastest; 0.03-0.28 max error on typical
                              8-bit images, up to ~4 at small denominators)            */
#define FBF_BF16_TC    2   /* compensated BF16 stack: every operand value and x-pass tap
                              is a hi + lo BF16 pair (three x-pass products) and the
                              x-pass result is TF32 hi + FP16 lo (max error ~0.004 on
                              8-bit images, 0.08 at small denominators, against 0.003
                              for FBF_FP32)                                             */

/* Names of the precision forms in the problem statement's terms: the BF16 channel stack with
   FP32 accumulation is the compensated form, whose y pass is a TF32 banded-Toeplitz
   contraction on the tensor cores.  (A TF32-operand x pass would carry FP16's 10-bit
   mantissa, the precision that misses the 0.5 bound at small denominators, so no separate
   form is built for it.) */
#define FBF_BF16       FBF_BF16_TC
#define FBF_TF32_TC    FBF_BF16_TC

/* FBF_FAST: whichever of FBF_FP32 and FBF_BF16_TC filters faster at the plan's radius
   r = ceil(3 theta), chosen when the plan is made: FBF_FP32 for r <= FBF_FAST_FP32_MAX_RADIUS
   (there the short FIR costs less than the tensor-core form's operand generation: on a
   GB300, work-lists of 256^2-2048^2 images at r = 6 took 0.87 ms in FP32 against 1.30 ms in
   FBF_BF16_TC, at r = 15 1.13 against 0.88 ms), FBF_BF16_TC for larger r up to
   FBF_MAX_RADIUS_TC, FBF_FP32 above it.  Its error is that of the chosen form, so within
   FBF_BF16_TC's bound (0.5 gray levels).  Not in the paper (a scheduling choice).       */
#define FBF_FAST       3
#define FBF_FAST_FP32_MAX_RADIUS 6

/* ---- flags (fbf_plan's `flags`) ----------------------------------------------- */
#define FBF_FLAG_FIXED_PERIOD 1  /* T = R (fixed period, the FBF model the paper
                                    compares against, Section III); least squares only */

/* Limits of the device kernels. */
#define FBF_MAX_K       64  /* cosine terms                                       */
#define FBF_MAX_RADIUS  48  /* spatial radius r = ceil(3 theta)                   */
#define FBF_MAX_PERIOD  65535 /* 2T+1                                             */
#define FBF_MAX_RADIUS_TC 30  /* radius limit of the tensor-core forms            */

typedef struct fbf_plan_s* fbf_plan_t;

/*
 * fbf_plan -- fit (K, T, c) for one (sigma, R, theta) and precompute the device constants.
 *
 * Section II: b(t) = exp(-t^2/(2 sigma^2)) on t in {-R..R} (eq. 2);
 * A(t,k) = cos(nu t k), nu = 2 pi/(2T+1); E(K,T) = min_c ||A c - b||^2 (eq. 5).
 *   K >= 1            : fixed order; T = argmin over T of E(K,T) (eq. 6, the Fig. 1 setting).
 *   K == 0, eps > 0   : Algorithm 1 -- the smallest K with min_T E(K,T) <= eps.
 * T is searched over 1..T_max, T_max = 4R, doubled while the optimum lies above T_max/2.
 * Among T whose error is at FP64 round-off (below 1e-20 ||b||^2) the smallest is taken.
 * Rank-deficient systems (K > T+1) are solved with dependent columns dropped; phi_hat on
 * {-R..R} is the same for every least-squares solution.
 *
 * sigma > 0, R >= 1, theta > 0 (spatial std; window radius r = ceil(3 theta), the
 * (6 theta + 1)^2 window of Section I), precision one of FBF_FP32, FBF_FP16_TC,
 * FBF_BF16_TC or FBF_FAST (resolved here to FBF_FP32 or FBF_BF16_TC), flags a bitwise OR
 * of FBF_FLAG_*.  Runs on the host only; needs no GPU.  *out receives a handle owned by
 * the caller and released with fbf_plan_destroy.
 * Errors: FBF_EINVAL for bad arguments or a NULL out; FBF_EUNSUPPORTED when the fitted
 * K exceeds FBF_MAX_K, r exceeds FBF_MAX_RADIUS or 2T+1 exceeds FBF_MAX_PERIOD;
 * FBF_ENOMEM.
 */
int fbf_plan(fbf_plan_t* out, double sigma, int R, double theta, int K, double eps,
             int precision, int flags);

/*
 * fbf_plan_from_samples -- as fbf_plan, for an arbitrary range kernel given by its
 * samples b[0..2R] = phi(-R..R) (host pointer, read during the call only).  The paper
 * notes the least-squares fit applies to non-Gaussian kernels (Sections I and IV).  Only
 * the even part of b can be represented by the cosine series; E includes the odd part's
 * energy.  phi(0) = b[R] must be > 0.
 */
int fbf_plan_from_samples(fbf_plan_t* out, const double* b, int R, double theta, int K,
                          double eps, int precision, int flags);

/*
 * fbf_plan_info -- read back the fitted parameters.  Any output pointer may be NULL.
 * c receives K doubles (c_0..c_{K-1} of eq. 3); E = E(K,T) of eq. (5);
 * delta_max = max over t in {-R..R} of |phi_hat(t) - phi(t)|.
 */
int fbf_plan_info(fbf_plan_t plan, int* K, int* T, double* c, double* E, double* delta_max);

/* fbf_plan_radius -- spatial radius r = ceil(3 theta) used by the kernels. */
int fbf_plan_radius(fbf_plan_t plan, int* r);

/* fbf_plan_destroy -- release a plan (NULL is accepted).  The caller makes sure no
 * launched work still uses it (plans hold no device memory; kernels receive their
 * constants by value at launch, so a plan may be destroyed right after a launch). */
int fbf_plan_destroy(fbf_plan_t plan);

/*
 * fbf_filter -- f_BF of eq. (1) with phi_hat, for one H x W image, asynchronously on
 * `cuda_stream` (a cudaStream_t; NULL means the legacy default stream).
 *
 * d_in, d_out: device pointers to H x W float32 images with a row stride of pitch_elems
 * elements (pitch_elems >= W); in and out must not overlap.  H, W >= 1; H*W may be
 * anything the device memory holds.  Launch errors are reported as FBF_ECUDA; errors of
 * the asynchronous work surface at the caller's next synchronisation.
 */
int fbf_filter(fbf_plan_t plan, const float* d_in, float* d_out, int H, int W,
               size_t pitch_elems, void* cuda_stream);

/*
 * fbf_filter_noalloc -- fbf_filter for callers that cannot allocate device memory while
 * they filter (the paper has no counterpart; this is a deployment aid).  Examples: a
 * framework whose caching allocator already holds nearly all of the GPU's memory, or a
 * latency-bound serving loop in which cudaMalloc/cudaFree, which may synchronise the
 * whole device, are not acceptable.  fbf_filter keeps a per-stream scratch workspace
 * that it grows with cudaMalloc; this entry point instead takes its scratch (tile
 * counters and partial sums) from one fixed device array of FBF_NOALLOC_SCRATCH_BYTES
 * compiled into the library, which every GPU that loads the library holds until exit.
 * It calls no cudaMalloc, cudaFree or allocating library routine.
 *
 * Arguments, layout and results are those of fbf_filter (FBF_FP32 plans only, among them
 * FBF_FAST plans that took the FP32 form; else FBF_EUNSUPPORTED).  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before any
 * stream capture.  The address is kept for the life of the process: after a
 * cudaDeviceReset no entry point may be called again in that process (this address and the
 * other calls' cached workspaces would no longer be mapped).  Each call clears the counters it uses on `cuda_stream` before the
 * kernel runs.  All calls share the one array: calls whose work overlaps on the GPU
 * (different streams, or several host threads) race and must be serialised by the caller.
 * Limit: the image may need at most 262144 tiles of 32 columns by 64 to 128 rows
 * (about 2^28 pixels, e.g. 16384 x 16384); larger images are rejected with
 * FBF_EUNSUPPORTED before any device work.
 */
#define FBF_NOALLOC_SCRATCH_BYTES (16u << 20)
int fbf_filter_noalloc(fbf_plan_t plan, const float* d_in, float* d_out, int H, int W,
                       size_t pitch_elems, void* cuda_stream);

/*
 * fbf_filter_host -- f_BF of one image from host memory to host memory: the end-to-end
 * call (eq. (1) with phi_hat, as fbf_filter).  host_in / host_out: H x W floats, row stride
 * pitch_elems (>= W); host_out may be host_in (in place), but not partly overlap it.  When
 * both are distinct page-locked buffers mapped into the device's address space (e.g. from
 * cudaHostAlloc under unified addressing), the kernel reads the image and writes the result
 * through the host link directly, with no staging copies.  Otherwise the image is staged
 * through device memory (pageable memory works, with copies staged by the driver) in up to
 * four bands of whole tile rows, each with at least two tiles per SM (smaller images are one
 * band): band b's rows are
 * uploaded, its filter runs as soon as its rows and the first r rows of band b + 1 are on
 * the device (reading halo rows from the whole image), and its result is copied back while
 * later bands compute.  Runs on `cuda_stream` (plus two internal copy streams per stream)
 * and returns when the result is on the host.  Device images, copy streams and events are
 * kept per (device, stream), grown as needed and held until the process exits (a caller
 * that cycles through many streams holds one set per stream).  Errors: as fbf_filter,
 * FBF_ENOMEM when the device images cannot be allocated; on an error the call returns only
 * after the copies it queued have finished.
 */
int fbf_filter_host(fbf_plan_t plan, const float* host_in, float* host_out, int H, int W,
                    size_t pitch_elems, void* cuda_stream);

/* ---- batched form (many images in one persistent launch) ------------------------- */
typedef struct fbf_batch_s* fbf_batch_t;
typedef uint64_t fbf_ticket_t;
#define FBF_BATCH_AUTOTUNE 1   /* time each candidate tile configuration on first use */

/*
 * fbf_batch_create -- a batch context.  Images are queued with fbf_batch_submit and filtered
 * together by fbf_launch: per precision form and radius class (the kernel instantiation
 * serving their r = ceil(3 theta)), and for FBF_FP32 per spatial kernel (theta) within the
 * class, one persistent stream-K launch runs over a device work-list of all
 * (image, tile, cosine term) units, so small and large images share the GPU evenly.  Not
 * in the paper (Section III filters one image at a time); the arithmetic per image is
 * exactly fbf_filter's.  max_images (>= 1) bounds one launch; flags: FBF_BATCH_AUTOTUNE,
 * under which the first launch of each (radius class, size bucket, K) times the candidate
 * tile configurations and keeps the fastest (cached per process; appended to the file
 * named by the environment variable FBF_TUNE_CACHE, read back by later processes).
 * Host memory only until the first launch; device buffers are allocated at fbf_launch /
 * fbf_batch_capture (never during fbf_batch_replay).  A batch's launches must be ordered
 * (one stream, or caller-synchronised streams): they share the batch's scratch.
 */
int fbf_batch_create(fbf_batch_t* out, int max_images, int flags);

/*
 * fbf_batch_submit -- queue one image (host-side only; nothing runs until fbf_launch).
 * Arguments as fbf_filter, any precision form.  The plan's parameters are copied, so the
 * plan may be destroyed right after the call.  *ticket (may be NULL) identifies the launch
 * the image will belong to.
 * Errors: FBF_EINVAL (bad arguments), FBF_EBUSY (max_images already queued),
 * FBF_EUNSUPPORTED (radius beyond the form's limit: FBF_MAX_RADIUS, FBF_MAX_RADIUS_TC).
 */
int fbf_batch_submit(fbf_batch_t batch, fbf_plan_t plan, const float* d_in, float* d_out, int H, int W,
                     size_t pitch_elems, fbf_ticket_t* ticket);

/* fbf_launch -- upload the work-list of the queued images and launch them on `cuda_stream`
 * (asynchronous); the queue is emptied, also when the call fails (the queued images'
 * outputs are then undefined; submit them again).  A no-op when nothing is queued. */
int fbf_launch(fbf_batch_t batch, void* cuda_stream);

/* fbf_batch_capture -- instead of launching, record the queued images' launch (work-list
 * copy + kernels) as a CUDA graph owned by the batch, replacing any earlier one; the queue
 * is emptied, also when the call fails.  Tuning and allocation happen before the capture.
 * The graph has its own work-list and split-tile scratch buffers, which later fbf_launch
 * calls never resize, so launches and replays may be mixed in any order.  A failed capture
 * that had to grow those buffers leaves no graph (fbf_batch_replay then returns
 * FBF_EINVAL). */
int fbf_batch_capture(fbf_batch_t batch, void* cuda_stream);

/* fbf_batch_replay -- launch the captured graph on `cuda_stream` (same pointers and sizes,
 * current image contents); *ticket (may be NULL) names this replay. */
int fbf_batch_replay(fbf_batch_t batch, void* cuda_stream, fbf_ticket_t* ticket);

/* fbf_batch_poll -- non-blocking: *status = FBF_DONE when the ticket's launch has completed
 * on the device, FBF_PENDING while it runs or is not launched yet.  A device error of the
 * launch is returned as FBF_ECUDA. */
int fbf_batch_poll(fbf_batch_t batch, fbf_ticket_t ticket, int* status);

/* fbf_batch_wait -- block until the ticket's launch completes or timeout_s seconds pass
 * (FBF_ETIMEDOUT; a ticket whose launch never happens times out). */
int fbf_batch_wait(fbf_batch_t batch, fbf_ticket_t ticket, double timeout_s);

/*
 * fbf_submit -- queue one image on the calling thread's current device without a batch
 * handle: each device has one implicit queue and one library stream (non-blocking, created
 * on first use, kept until the process exits).  Arguments as fbf_filter (device pointers,
 * any precision form; the plan's parameters are copied, so the plan may be destroyed after
 * the call).  The queue is launched -- all its images in one batched launch, as fbf_launch --
 * at the first fbf_poll or fbf_wait of one of its tickets, or when it already holds 4096
 * images.  The library stream is not ordered after the caller's streams: d_in must hold the
 * image (its producer synchronised) when fbf_submit is called, and d_out holds the result
 * once fbf_poll has reported FBF_DONE.  The caller keeps both alive until then.
 * *ticket (may be NULL) names the image's launch.  Errors: as fbf_batch_submit, FBF_ECUDA
 * when the device's queue cannot be set up.
 */
int fbf_submit(fbf_plan_t plan, const float* d_in, float* d_out, int H, int W, size_t pitch_elems,
               fbf_ticket_t* ticket);

/* fbf_poll -- non-blocking state of a ticket from fbf_submit: launches the ticket's queue if
 * it has not been launched yet, then *status = FBF_DONE when the launch has completed on the
 * device, FBF_PENDING otherwise.  FBF_EINVAL for a ticket no fbf_submit returned (its
 * device has no queue); a device error of the launch is returned as FBF_ECUDA. */
int fbf_poll(fbf_ticket_t ticket, int* status);

/* fbf_wait -- as fbf_poll, then block until the launch completes or timeout_s seconds
 * pass (FBF_ETIMEDOUT). */
int fbf_wait(fbf_ticket_t ticket, double timeout_s);

/* fbf_batch_pending -- number of queued, not yet launched images. */
int fbf_batch_pending(fbf_batch_t batch, int* n);

/* fbf_batch_destroy -- wait for the batch's launches, release its buffers (NULL ok). */
int fbf_batch_destroy(fbf_batch_t batch);

/* ---- serving: continuous batching under an HBM budget --------------------------------
 * Not in the paper (Section III filters one image at a time); the arithmetic per request is
 * exactly fbf_filter's.  A server owns a worker thread, three streams (upload, compute,
 * download), a stream-ordered device memory pool and a batch.  Requests are admitted in
 * arrival order while their device buffers (input and output, 8 bytes per pixel) fit the
 * HBM budget and the next launch has room (max_batch); the image is copied in at once; all
 * admitted requests go into one batched launch whenever fewer than max_inflight launches
 * are in flight (requests that arrive meanwhile join the next launch); results are copied
 * back on the download stream and the device buffers released.  Latency is measured from
 * fbf_server_submit to the result being on the host.
 */
typedef struct fbf_server_s* fbf_server_t;

typedef struct {
  uint64_t requests;          /* finished with their result on the host                 */
  uint64_t pixels;            /* their pixels                                           */
  uint64_t launches;          /* batched launches                                       */
  uint64_t failed;            /* requests that ended with an error                      */
  uint64_t hbm_high_water;    /* most device bytes held by admitted requests at once    */
  uint64_t waited_for_budget; /* requests whose admission the budget deferred           */
  uint32_t max_inflight_seen; /* most launches in flight at once                        */
  double wall_s;              /* first submit to last completion                        */
  double p50_ms, p99_ms;      /* latency percentiles                                    */
  double tail_requests;       /* requests at or above p99, and the means of their parts: */
  double tail_queued_ms;      /*   submit -> admitted                                   */
  double tail_wait_for_launch_ms; /* admitted -> launched                               */
  double tail_launch_to_result_ms; /* launched -> result on the host                    */
  double tail_mpix;           /*   size (megapixels)                                    */
  double tail_batch;          /*   requests in their launch                             */
} fbf_server_stats_t;

/* fbf_server_create -- a server on CUDA device `device` filtering in precision form
 * `precision` (FBF_FP32, FBF_FP16_TC, FBF_BF16_TC, FBF_FAST: each request's plan takes
 * the faster form for its radius).  hbm_budget_bytes >= 1, max_batch >= 1
 * (requests per launch; 1 = one request per launch), max_inflight >= 1.  The caller's
 * current device is left unchanged.  Errors: FBF_EINVAL, FBF_ENOMEM, FBF_ECUDA. */
int fbf_server_create(fbf_server_t* out, int device, int precision, uint64_t hbm_budget_bytes,
                      int max_batch, int max_inflight);

/* fbf_server_submit -- queue one request (any thread).  host_in / host_out: H x W float
 * images, row-major, packed; page-locked host memory (for asynchronous copies), owned by
 * the caller and untouched by it until the request's status is FBF_DONE or an error.
 * theta, sigma, R, K, eps: as fbf_plan (plans are created once per distinct set and kept).
 * *ticket (may be NULL) names the request for fbf_server_poll.  Errors: FBF_EINVAL (bad
 * arguments, an image larger than the budget), FBF_EUNSUPPORTED (radius beyond the form's
 * limit), fbf_plan's errors. */
int fbf_server_submit(fbf_server_t s, const float* host_in, float* host_out, int H, int W, double theta,
                      double sigma, int R, int K, double eps, fbf_ticket_t* ticket);

/* fbf_server_replay -- submit n requests at arrival_s[i] seconds after the call (arrivals
 * sorted), from the calling thread, sleeping until each arrival: an open-loop load
 * generator for benchmarks.  Plans are created before the clock starts.  Array arguments
 * as fbf_server_submit's, one entry per request; tickets may be NULL. */
int fbf_server_replay(fbf_server_t s, int n, const double* arrival_s, const float* const* host_in,
                      float* const* host_out, const int* H, const int* W, const double* theta,
                      const double* sigma, const int* R, const int* K, const double* eps,
                      fbf_ticket_t* tickets);

/* fbf_server_poll -- non-blocking: *status = FBF_PENDING, FBF_DONE or the error code the
 * request ended with.  FBF_EINVAL for an unknown ticket. */
int fbf_server_poll(fbf_server_t s, fbf_ticket_t ticket, int* status);

/* fbf_server_drain -- wait until every submitted request has finished, at most timeout_s
 * seconds (FBF_ETIMEDOUT). */
int fbf_server_drain(fbf_server_t s, double timeout_s);

/* fbf_server_stats -- counters and latency statistics of the finished requests. */
int fbf_server_stats(fbf_server_t s, fbf_server_stats_t* out);

/* fbf_server_reset_stats -- clear the counters and latencies (after a warm-up); FBF_EBUSY
 * while requests are pending. */
int fbf_server_reset_stats(fbf_server_t s);

/* fbf_server_destroy -- finish the queued requests, stop the worker, release everything
 * (NULL ok). */
int fbf_server_destroy(fbf_server_t s);

/* fbf_debug_server_inject -- test aid, not part of the method: the server's next `count`
 * uploads (stage 1) or batched launches (stage 2) fail on the host with FBF_ECUDA before
 * any CUDA work of that step (a launch fails with its requests' images already queued in
 * the server's batch), so that a test drives the loop's failure handling -- the failed
 * requests end with the error, their buffers and budget are released, later requests are
 * served -- without a device fault.  count 0 clears.  FBF_EINVAL for a bad stage or count. */
int fbf_debug_server_inject(fbf_server_t s, int stage, int count);

/* fbf_last_error -- message for the last failing call on this thread ("" if none). */
/*
 * fbf_brute_filter -- eq. (1) evaluated directly with the Gaussian range kernel of eq. (2)
 * (no cosine series): for every pixel, weights g(j_x) g(j_y) exp(-(f(i-j) - f(i))^2 /
 * (2 sigma^2)) over the (2r+1)^2 window, r = ceil(3 theta), g(x) = exp(-x^2/(2 theta^2));
 * pixels outside the image are absent from both sums.  The accuracy reference against
 * which the paper measures PSNR (Section III); cost 2(6 theta + 1)^2 per pixel (Section I).
 *
 * d_in, d_out: device pointers to H x W float32 images, row stride pitch_elems elements
 * (>= W), not overlapping.  theta, sigma > 0, R >= 1 (the intensity range [0, R]; integer
 * tiles with values <= min(R, 1023) use a table of the range kernel).  r > FBF_MAX_RADIUS
 * returns FBF_EUNSUPPORTED.  Asynchronous on cuda_stream (NULL = legacy default stream);
 * FP32 arithmetic.  No plan and no scratch memory.
 */
int fbf_brute_filter(const float* d_in, float* d_out, int H, int W, size_t pitch_elems,
                     double theta, double sigma, int R, void* cuda_stream);

/* ---- lookup table of K* and T* (Section II, after Algorithm 1; Fig. 2) ------------
 * The paper runs Algorithm 1 offline on a grid of (sigma, eps), stores K* and T*, and at run
 * time reads them (bilinear interpolation in sigma and log(1/eps) off the grid) and solves
 * only the least squares of eq. (5) for the coefficients.  Gaussian range kernel of eq. (2)
 * on the intensity range [0, R].  Host only; a table owns host memory only. */
typedef struct fbf_lut_s* fbf_lut_t;

/* Run Algorithm 1 at every grid point.  sigmas: n_sigma >= 2 values, strictly increasing,
 * > 0; eps: n_eps >= 2 values in (0, 1), strictly decreasing (so log(1/eps) increases).
 * Errors: FBF_EINVAL for bad grids, or the fitter's code when a point cannot be fitted. */
int fbf_lut_build(fbf_lut_t* out, int R, const double* sigmas, int n_sigma, const double* eps, int n_eps);

/* K* and T* stored at grid point (i_sigma, j_eps). */
int fbf_lut_entry(fbf_lut_t lut, int i_sigma, int j_eps, int* K, int* T);

/* Bilinear interpolation of K* and T* in (sigma, log(1/eps)), each rounded to the nearest
 * integer.  (sigma, eps) outside the grid: FBF_EUNSUPPORTED. */
int fbf_lut_lookup(fbf_lut_t lut, double sigma, double eps, int* K, int* T);

/* A plan (as fbf_plan) whose K and T come from fbf_lut_lookup; only c is fitted (eq. 5). */
int fbf_plan_from_lut(fbf_plan_t* out, fbf_lut_t lut, double sigma, double eps, double theta, int precision);

/* Text file: "fbf-lut 1", R n_sigma n_eps, the sigmas, the eps values, then K T per grid
 * point (sigma-major).  fbf_lut_load checks the format (FBF_EINVAL when malformed). */
int fbf_lut_save(fbf_lut_t lut, const char* path);
int fbf_lut_load(fbf_lut_t* out, const char* path);
int fbf_lut_destroy(fbf_lut_t lut);

const char* fbf_last_error(void);

/* fbf_device_errors -- read (and with clear != 0 reset) the device error word of the
 * kernels: bit 0 set means a bounded mbarrier wait of a tensor-core kernel gave up, bit 1
 * that a bounded wait for a TMA copy of the f halo in the FP32 kernel gave up; in either
 * case that launch's output is incomplete.  Read it after synchronising the stream of the
 * launches in question.  Clearing a nonzero word also resets the library's cached
 * split-tile counters (synchronising the devices that hold them); a batch (fbf_batch_t) one
 * of whose launches gave up keeps its own counters and is to be destroyed and made anew. */
int fbf_device_errors(int* flags, int clear);

/* fbf_debug_fp32_peak -- measurement aid, not part of the method: launch a probe of the
 * FP32 multiply-add rate (blocks x threads threads, each running 16 independent chains of
 * `iters` packed fma.rn.f32x2 pairs when pairs != 0, else scalar fmaf pairs) on
 * cuda_stream, and return in *flop the floating-point operations the launch performs
 * (2 per multiply-add).  Timing the launch with events gives the FP32 peak the fused
 * filter's roofline is measured against.  d_out: device buffer of blocks x threads floats
 * (written, to keep the chains live).  threads a multiple of 32 in [32, 256], blocks >= 1,
 * iters >= 1, else FBF_EINVAL; launch errors FBF_ECUDA. */
int fbf_debug_fp32_peak(int pairs, int blocks, int threads, long long iters, float* d_out,
                        void* cuda_stream, double* flop);

/* fbf_debug_set_wait_limit -- test aid, not part of the method: with polls > 0, the bounded
 * waits inside the kernels' own pipelines on the current device (the FP32 single-image
 * kernel's wait for a TMA box of the f halo; the tensor-core kernels' mbarrier waits between
 * their roles) become `polls` non-blocking polls, so that a test can make them give up and
 * exercise the abort path: the launch leaves its output incomplete, reports the bit in
 * fbf_device_errors, and first lets every copy and MMA it started complete (those final
 * waits keep their full limits) and frees its tensor memory.  polls = 0 restores the
 * normal limits.  Affects launches made after the call.  Errors: FBF_EINVAL (polls < 0),
 * FBF_ECUDA. */
int fbf_debug_set_wait_limit(int polls);

/* fbf_version -- library version string. */
const char* fbf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FBF_H */
