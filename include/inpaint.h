/*
 * libinpaint: exemplar-based object removal on one GB300 GPU (sm_103a).
 *
 * The method is the exemplar-based inpainting loop of Sec. 3 of Wang, Xiong,
 * Yun, Cavallaro, "Computer Vision Accelerators for Mobile Systems based on
 * OpenCL GPGPU Co-Processing" (J. Sign. Process. Syst., 2014): repeat until
 * the target region Omega is empty -- compute priorities P(p) = C(p) D(p) on
 * the fill front (Eq. 1-2), take the highest-priority target patch, find the
 * source patch with the smallest masked sum of squared RGB differences
 * (Eq. 3-4, "findBestPatch", 97 % of the run time in Table 2), copy it into
 * the unknown part of the target patch and update the confidences.
 *
 * Every step runs in this library's CUDA kernels; there is no CPU fallback.
 *
 * Conventions for all entry points:
 *   - Images are W x H, row-major, linear index idx(x, y) = y * W + x.
 *     RGB is 3 interleaved bytes per pixel; rows may be padded (stride).
 *     A mask byte that is nonzero marks a pixel of Omega (to be removed).
 *   - The caller owns every host buffer; the library copies inputs when a
 *     context is created or reset and writes only caller-provided outputs.
 *   - A return value >= 0 is success, < 0 is an error (inpaint_status).
 *     No C++ exception crosses this interface.
 *   - One context is used by one host thread at a time.  Contexts are
 *     independent; each owns its device memory and uses one CUDA stream.
 *   - Results are deterministic and bit-identical to the algorithm as stated
 *     (ties: highest priority, then lowest linear index, is selected; lowest
 *     SSD, then lowest linear index, is copied).
 */
#ifndef INPAINT_H
#define INPAINT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct inpaint_ctx inpaint_ctx; /* opaque; owns its device memory */

typedef enum {
  INPAINT_OK = 0,
  INPAINT_DONE = 1,              /* Omega is already empty; nothing was done */
  INPAINT_ERR_ARG = -1,          /* invalid argument (sizes, radius, pointers, no known pixel) */
  INPAINT_ERR_NOMEM = -2,        /* a device or pinned-host allocation failed */
  INPAINT_ERR_CUDA = -3,         /* a CUDA runtime call failed */
  INPAINT_ERR_NO_SOURCE = -4,    /* no admissible source patch (fully known; with the partial-
                                    overlap search: known under every pixel to fill); state
                                    unchanged */
  INPAINT_ERR_TIMEOUT = -5,      /* a bounded device-side wait gave up */
  INPAINT_ERR_UNSUPPORTED = -6,  /* valid request this library or device cannot serve */
  INPAINT_ERR_INTERNAL = -7      /* a self-check (debug_checks) found inconsistent state */
} inpaint_status;

/* Search forms (both give identical results). */
#define INPAINT_FORM_PLAIN 0 /* CUDA-core integer SSD (byte-SIMD abs-diff + dot) */
#define INPAINT_FORM_TC 1    /* exact tensor-core correlation form (tcgen05, BF16 operands
                                holding small integers, FP32 accumulation exact below 2^24);
                                patch_radius <= 8.  In the persistent engine (single image,
                                teams of two or more CTAs) the image's candidates are cut
                                into tiles of 16 rows x 512 or 1024 columns searched from
                                five BF16 planes of the image (about 10 bytes per pixel of
                                extra device memory); where those tiles do not fit a CTA
                                the engine searches with the plain form.  inpaint_step
                                always runs the graph-loop kernels. */

/* Device allocator hooks: lets a host framework (e.g. PyTorch's caching
 * allocator) own device memory.  Both NULL: cudaMallocAsync/cudaFreeAsync on
 * the context's stream.  alloc returns NULL on failure, else a block aligned
 * to 256 bytes like cudaMalloc's (the kernels copy 16-byte units with
 * asynchronous copies); a context whose allocator returns a less aligned
 * block fails to build with INPAINT_ERR_NOMEM. */
typedef void* (*inpaint_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*inpaint_free_fn)(void* ptr, size_t bytes, void* stream, void* user);

typedef struct {
  int form;              /* INPAINT_FORM_PLAIN (default) or INPAINT_FORM_TC */
  void* cuda_stream;     /* cudaStream_t for all work; NULL = a non-blocking stream the
                            context creates and owns */
  int debug_checks;      /* nonzero: recount the candidate-validity map from scratch
                            after every iteration and fail with INPAINT_ERR_INTERNAL
                            on any difference (slow; for tests) */
  double search_alpha;   /* < 0: exhaustive search over every interior centre (default).
                            >= 0: search factor alpha of Sec. 5.3 / Eq. 6: candidate
                            centres are limited to the bounding box of the initial
                            Omega expanded by floor(alpha*w) columns left and right and
                            floor(alpha*h) rows up and down (w x h = box size). */
  inpaint_alloc_fn dev_alloc;
  inpaint_free_fn dev_free;
  void* alloc_user;
  int loop_mode;         /* how inpaint_run drives the iterations:
                            INPAINT_LOOP_AUTO (default): the persistent engine when
                            patch_radius <= 8, else the graph loop;
                            INPAINT_LOOP_ENGINE: one cooperative persistent kernel for
                            the whole loop (patch_radius <= 8 only);
                            INPAINT_LOOP_GRAPH: a CUDA graph with a conditional while
                            node around [search kernel, update kernel] */
  int tile_rows;         /* engine search, streaming mode (small images or small
                            teams): a search batch is 32 candidate rows (one per lane)
                            x 16 warps x 4 * tile_rows candidate columns per lane,
                            i.e. 64 (tile_rows = 1) or 128 (tile_rows = 2) columns;
                            0 = chosen by the library.  Large images on large teams
                            use the resident mode (units of 32 rows x 16 columns,
                            source tiles kept in shared memory), whatever this is */
  const char* tuning_file; /* NULL, or a text table written by the autotuner: one line
                            "radius max_pixels tile_rows" per bucket; the first line
                            with the image's radius and max_pixels >= the image's
                            pixels per CTA of its team (W*H / CTAs working on it)
                            gives tile_rows when tile_rows is 0 */
  int search_variant;    /* INPAINT_SEARCH_FULL (default): candidate patches lie inside
                            the image and inside the known region (Eq. 3-4);
                            INPAINT_SEARCH_OVERLAP: the partial-overlap variant of
                            Algorithm 1 / Sec. 5.4: every centre of the search rectangle
                            (clamped to the image, not to the interior) is a candidate,
                            its SSD runs over the offsets whose target and source pixels
                            are both known and in the image, and it is admissible when a
                            known in-image source pixel lies under every unknown in-image
                            target pixel.  Plain form, patch_radius <= 8, graph loop
                            (INPAINT_LOOP_AUTO picks it); not in batches or the server. */
} inpaint_options;

#define INPAINT_SEARCH_FULL 0
#define INPAINT_SEARCH_OVERLAP 1

#define INPAINT_LOOP_AUTO 0
#define INPAINT_LOOP_ENGINE 1
#define INPAINT_LOOP_GRAPH 2

/* One record per fill iteration. */
typedef struct {
  int32_t iter;        /* 0-based iteration number */
  int32_t px, py;      /* target centre p^: highest priority on the fill front */
  int32_t qx, qy;      /* source centre q~: lowest SSD among valid candidates */
  uint32_t ssd;        /* SSD of q~ (Eq. 4) over the known pixels of Psi_p^ */
  double priority;     /* P(p^) = C(p^) * D(p^) (Eq. 1) */
  double confidence;   /* C(p^) (Eq. 2); the filled pixels receive this value */
  int32_t filled;      /* pixels of Omega copied this iteration */
  int32_t remaining;   /* |Omega| after this iteration */
  int32_t n_known;     /* |K|: known in-image pixels of Psi_p^ */
  int32_t n_cand;      /* valid candidate centres searched this iteration */
} inpaint_step_info;

/* Fills *opt with the defaults (plain form, default stream, exhaustive search). */
void inpaint_options_default(inpaint_options* opt);

/* Creates a context from host RGB + mask and runs the initialisation stage
 * (Sec. 4.2: grey level, confidence C = 1 on Phi and 0 on Omega, fill front,
 * priorities, validity map of candidate centres).
 *   rgb: host, H rows of rgb_stride_bytes (>= 3*W), 3 bytes per pixel.
 *   mask: host, H rows of mask_stride_bytes (>= W), nonzero = remove.
 *   patch_radius r: 1..32 (patch side P = 2r+1); W, H >= P.
 *   opt: NULL for defaults.  *out receives the context.
 * Errors: INPAINT_ERR_ARG (bad sizes/pointers, mask covering every pixel),
 * INPAINT_ERR_NOMEM, INPAINT_ERR_CUDA, INPAINT_ERR_UNSUPPORTED (TC form with
 * patch_radius > 8). On error *out is NULL and nothing leaks. */
int inpaint_create(const uint8_t* rgb, int width, int height, int rgb_stride_bytes,
                   const uint8_t* mask, int mask_stride_bytes, int patch_radius,
                   const inpaint_options* opt, inpaint_ctx** out);

/* Re-initialises an existing context with a new image + mask of the same
 * size, reusing its device memory.  input_on_device = 0: rgb/mask are host
 * pointers (copied host->device on the context's stream); 1: device pointers
 * (densely packed or strided as given), read on the context's stream.
 * Same errors as inpaint_create. */
int inpaint_reset(inpaint_ctx* ctx, const uint8_t* rgb, int rgb_stride_bytes,
                  const uint8_t* mask, int mask_stride_bytes, int input_on_device);

/* One fill iteration (front priorities -> findBestPatch -> copy/update).
 * Returns INPAINT_OK, INPAINT_DONE (Omega already empty), or an error;
 * INPAINT_ERR_NO_SOURCE leaves the state unchanged.  info (nullable)
 * receives the iteration's record.  Synchronises the context's stream. */
int inpaint_step(inpaint_ctx* ctx, inpaint_step_info* info);

/* One fill iteration split over candidate rows, for a removal sharded over
 * several GPUs (each holding an identical replica of the context): every
 * shard searches its rows, the packed keys are reduced to their minimum,
 * and every replica applies that one key.  findBestPatch (Sec. 3, Eq. 3-4)
 * is a minimum over candidate centres, so the minimum of the rows' minima is
 * the full search's result (ties: lowest linear index, as the packed key
 * orders them), and replicas that apply the same keys stay identical.  Plain
 * form, exhaustive or alpha-limited search (not the tensor-core form or the
 * partial-overlap variant: INPAINT_ERR_UNSUPPORTED).
 *
 * inpaint_search_rows: searches the candidate centres of image rows
 * [y0, y1) (clipped to the search rectangle) for the current target p^ and
 * writes the smallest packed key (SSD << 32 | y * W + x) to *key_out (host
 * pointer), or INPAINT_KEY_NONE when those rows hold no candidate.  The state
 * does not change.  Returns INPAINT_OK, INPAINT_DONE (Omega empty) or an
 * error (INPAINT_ERR_ARG: null pointers or y0 > y1).  Synchronises the
 * context's stream.
 *
 * inpaint_apply_key: completes the iteration with `key` (the minimum over
 * all row ranges of the whole search rectangle): copy, confidence, mask,
 * validity counts, priorities, next p^, exactly as inpaint_step does, and
 * info (nullable) receives its record.  INPAINT_KEY_NONE means no source was
 * found anywhere: INPAINT_ERR_NO_SOURCE, state unchanged.  A key whose centre
 * is not an interior pixel (patch inside the image) is rejected with
 * INPAINT_ERR_ARG; any other key must come from inpaint_search_rows on a
 * replica in the same state.  Synchronises the context's stream. */
#define INPAINT_KEY_NONE 0xffffffffffffffffull
int inpaint_search_rows(inpaint_ctx* ctx, int y0, int y1, unsigned long long* key_out);
int inpaint_apply_key(inpaint_ctx* ctx, unsigned long long key, inpaint_step_info* info);

/* Runs iterations on the device until Omega is empty, an error occurs, or
 * max_iters iterations (<= 0: no limit) have run, with no host round trip
 * per iteration.  *iters_done (nullable) receives the number of iterations
 * run by this call; trace (nullable) receives the first min(trace_cap,
 * iterations) records of this call.  Returns INPAINT_OK when Omega became
 * empty or max_iters was reached, INPAINT_DONE if Omega was already empty,
 * or an error. Synchronises the context's stream. */
int inpaint_run(inpaint_ctx* ctx, int max_iters, int* iters_done,
                inpaint_step_info* trace, int trace_cap);

/* Copies the current image (RGB, 3 bytes per pixel, rows of stride_bytes)
 * and optionally the current Omega mask (1 = still unknown, rows of W bytes)
 * to host memory.  Synchronises the context's stream. */
int inpaint_result(const inpaint_ctx* ctx, uint8_t* rgb_out, int stride_bytes,
                   uint8_t* mask_out);

/* Checkpoint of the loop state: image (RGB), Omega (1 byte per pixel) and
 * confidence C (double per pixel), each dense W x H, any pointer nullable.
 * With inpaint_import_state it lets a removal stop and resume (the paper's
 * demo allows iterative editing, Sec. 6). */
int inpaint_export_state(const inpaint_ctx* ctx, uint8_t* rgb, uint8_t* omega, double* conf);

/* Replaces the loop state of a context by (rgb, omega, conf) from host
 * memory, as produced by inpaint_export_state, and recomputes everything
 * derived from it (grey level, front, priorities, validity map).  The
 * search rectangle of the context is kept. */
int inpaint_import_state(inpaint_ctx* ctx, const uint8_t* rgb, const uint8_t* omega,
                         const double* conf);

/* Image geometry and progress. */
int inpaint_info(const inpaint_ctx* ctx, int* width, int* height, int* patch_radius,
                 int* remaining, uint64_t* evals);

/* Phase clocks of the persistent engine since the last create/reset, from
 * the GPU's global timer: *search_ns sums, per iteration, the time from the
 * publication of the previous iteration to the last search CTA's arrival
 * (target staging, findBestPatch over all candidates, reduction, arrival);
 * *update_ns sums the copy/update/selection phases; *iters counts the
 * iterations timed.  The graph loop is not timed (all zero). */
int inpaint_loop_timing(const inpaint_ctx* ctx, uint64_t* search_ns, uint64_t* update_ns,
                        int* iters);

/* Iterations since the last create/reset whose search the persistent engine
 * ran in the tensor-core form (INPAINT_FORM_TC; the others, if any, ran the
 * plain form, with identical results). */
int inpaint_search_form_rounds(const inpaint_ctx* ctx, int* tc_rounds);

/* Candidate-centre rectangle [x0,x1] x [y0,y1] the context searches. */
int inpaint_search_rect(const inpaint_ctx* ctx, int* x0, int* x1, int* y0, int* y1);

/* findBestPatch for a single target patch, allocating no device memory.
 * The paper has no counterpart: this is for callers that cannot call
 * cudaMalloc -- a serving process whose device memory is reserved up front
 * by another framework's allocator, work issued while a stream is being
 * captured into a graph with a fixed memory plan, or a real-time loop that
 * forbids allocation after start-up.  The caller passes its own device
 * buffers; the only scratch the search needs (one partial result per CTA and
 * a ticket counter) is a fixed array inside the library, which every GPU
 * that loads the library holds until the process exits.
 *   d_rgb:  device, dense W x H x 3 bytes (RGB); d_mask: device, dense W x H
 *           bytes, nonzero = unknown (Omega).
 *   patch_radius 1..8; (px, py): target centre, inside the image.
 *   d_best_key: device uint64, receives (SSD << 32) | (qy * W + qx) of the
 *           fully-known in-image candidate patch with the lowest SSD over the
 *           known in-image pixels of the target patch (lowest index on ties),
 *           or UINT64_MAX if there is none.
 *   cuda_stream: cudaStream_t of the work (NULL = legacy default stream).
 * Limit: the interior (W - 2r) x (H - 2r) must fit in 4096 tiles of 8 rows x
 * 128 columns of candidates (e.g. 4096 x 1024 or 2048 x 2048 pixels); larger
 * images are rejected with INPAINT_ERR_ARG and a message in
 * inpaint_last_error().  The first call on a device looks up the scratch's
 * device address (cudaGetSymbolAddress); make that first call before any
 * stream capture.  Every call on a device shares the same scratch, which
 * keeps the last call's contents (the ticket is cleared at the start of each
 * call): calls that overlap on the GPU race and must be serialised by the
 * caller (one stream, or events).  Asynchronous: returns once the work is
 * enqueued. */
int inpaint_best_patch_noalloc(const uint8_t* d_rgb, const uint8_t* d_mask, int width, int height,
                               int patch_radius, int px, int py, uint64_t* d_best_key,
                               void* cuda_stream);

/* ---- Batched form: many independent images in one persistent launch ----
 * Every image runs the same fill loop as inpaint_run, bit for bit; the CTAs
 * of one cooperative launch are split into teams, each team running the loop
 * of its images one after the other (team sizes chosen to even out each image's
 * estimated work per CTA; images of any radius 1..8 mix in one launch).  Search
 * batch heights come from the tuning table (written by the autotune module
 * of the Python package) when opt->tuning_file names one, else from a rule
 * on the batches per CTA. */
typedef struct {
  const uint8_t* rgb;   /* host, H rows of rgb_stride_bytes, 3 bytes per pixel */
  int width, height, rgb_stride_bytes;
  const uint8_t* mask;  /* host, H rows of mask_stride_bytes, nonzero = remove */
  int mask_stride_bytes;
  int patch_radius;     /* 1..8 */
} inpaint_image;

typedef struct inpaint_batch inpaint_batch;

/* Allocates and initialises the device state of n images (inputs are copied;
 * a device copy of each input is kept for inpaint_batch_reset) and plans the
 * teams.  opt may be NULL; opt->cuda_stream is used for all work.  Errors as
 * inpaint_create (INPAINT_ERR_ARG names the first bad image in
 * inpaint_last_error()). */
int inpaint_batch_create(const inpaint_image* images, int n, const inpaint_options* opt,
                         inpaint_batch** out);

/* Re-initialises every image from its kept input (device to device). */
int inpaint_batch_reset(inpaint_batch* b);

/* Runs every image until its Omega is empty or an error stops it, in one
 * cooperative kernel launch (iterations limited to max_iters per image when
 * max_iters > 0).  status_out (nullable, n entries) receives each image's
 * status (INPAINT_OK, INPAINT_DONE or an error).  Returns INPAINT_OK when
 * the launch ran (even if some images failed), else an error.
 * Synchronises the batch's stream. */
int inpaint_batch_run_ctx(inpaint_batch* b, int max_iters, int* status_out);

/* Current image i (RGB, rows of stride_bytes) and its counters; any output
 * pointer may be NULL. */
int inpaint_batch_result(const inpaint_batch* b, int i, uint8_t* rgb_out, int stride_bytes,
                         int* iterations, uint64_t* evals);

/* The launch plan: grid size, number of teams, and per image its team, the
 * team's size and the search rows per warp.  Arrays may be NULL. */
int inpaint_batch_plan(const inpaint_batch* b, int* grid, int* n_teams, int* team_of_image,
                       int* team_size_of_image, int* rows_per_warp);

/* Releases everything (after synchronising the batch's stream). */
void inpaint_batch_destroy(inpaint_batch* b);

/* One-shot batched removal: n independent images, each W[i] x H[i] with
 * patch radius r[i] (1..8), run to completion in one persistent launch
 * (create, run, results, destroy of a batch object).  The fill loop of every
 * image is the one of Sec. 3 (Eq. 1-4), bit for bit as inpaint_run on that
 * image alone.
 *   rgb[i]: host, dense W x H x 3 bytes; mask[i]: host, dense W x H bytes,
 *           nonzero = remove.  Both are read only.
 *   opt: NULL for defaults (opt->cuda_stream carries the work).
 *   rgb_out[i]: host, dense W x H x 3 bytes, receives image i after its
 *           removal (or the state where its loop stopped, see status_out).
 *   status_out: nullable, n entries: INPAINT_OK, INPAINT_DONE (nothing to
 *           remove) or the error that stopped image i (INPAINT_ERR_NO_SOURCE
 *           for an image without an admissible source; the others still
 *           finish).
 * Returns INPAINT_OK when the launch ran, else the first error (a bad
 * argument: INPAINT_ERR_ARG, with the index in inpaint_last_error()).
 * Synchronous. */
int inpaint_batch_run(int n, const uint8_t* const* rgb, const uint8_t* const* mask, const int* w,
                      const int* h, const int* r, const inpaint_options* opt, uint8_t* const* rgb_out,
                      int* status_out);

/* ---- Serving loop: continuous batching of object-removal requests ----
 * A server owns a worker thread and a CUDA stream.  Submitted requests wait
 * in a FIFO queue; between scheduler ticks the worker admits queued requests
 * while slots are free and the estimated device memory of the admitted ones
 * stays within the budget (their state stays on the device until they
 * finish); each tick is one persistent engine launch over every active slot
 * that runs until about 20 ms of device time have passed (teams stop between
 * iterations and resume in the next tick) or each slot has done
 * iters_per_tick iterations, after which finished requests release their
 * memory and their result waits for inpaint_server_poll.
 * A request's result does not depend on what else is in flight: it equals
 * inpaint_run on that image alone. */
#define INPAINT_PENDING 2   /* inpaint_server_poll: request not finished yet */

typedef struct inpaint_server inpaint_server;

typedef struct {
  double t_submit, t_admit, t_done;  /* seconds on the server's clock */
  int status;                        /* inpaint_status of the removal */
  int iterations;
  uint64_t evals;
  int width, height;
} inpaint_request_info;

typedef struct {
  uint64_t submitted, admitted, completed, failed, ticks;
  int queued, active;
  size_t hbm_used, hbm_budget;
  double busy_s;                     /* worker time spent admitting and in ticks */
} inpaint_server_stats;

/* hbm_budget_bytes: limit on the estimated device memory of active requests;
 * max_slots: limit on simultaneously active requests; iters_per_tick: at most
 * this many engine iterations per slot per tick (<= 0: no limit besides the
 * tick's time budget).  opt as for inpaint_create
 * (cuda_stream ignored: the server makes its own). */
int inpaint_server_create(size_t hbm_budget_bytes, int max_slots, int iters_per_tick,
                          const inpaint_options* opt, inpaint_server** out);

/* Queues a request (inputs are copied; radius 1..8).  *id identifies it. */
int inpaint_server_submit(inpaint_server* s, const inpaint_image* img, uint64_t* id);

/* INPAINT_PENDING while request id runs; once done, copies its result (RGB,
 * rows of stride_bytes, nullable) and info (nullable), forgets the request
 * and returns INPAINT_OK (INPAINT_ERR_ARG for an unknown id). */
int inpaint_server_poll(inpaint_server* s, uint64_t id, uint8_t* rgb_out, int stride_bytes,
                        inpaint_request_info* info);

/* Blocks until nothing is queued or active, or timeout_s passed
 * (INPAINT_ERR_TIMEOUT). */
int inpaint_server_wait_idle(inpaint_server* s, double timeout_s);

int inpaint_server_stats_get(inpaint_server* s, inpaint_server_stats* st);

/* Seconds on the server's clock (the clock of inpaint_request_info). */
double inpaint_server_clock(const inpaint_server* s);

/* Stops the worker (after the current tick) and releases everything. */
void inpaint_server_destroy(inpaint_server* s);

/* Releases the context and all its device memory (after synchronising its
 * stream).  NULL is a no-op. */
void inpaint_destroy(inpaint_ctx* ctx);

/* Human-readable text for a status code (static storage). */
const char* inpaint_status_str(int status);

/* Last CUDA error text seen by this thread's most recent failing call. */
const char* inpaint_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
