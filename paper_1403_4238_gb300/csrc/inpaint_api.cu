// C-ABI of libinpaint: context lifetime, the iteration loop and host I/O.
//
// The three stages of Sec. 4.2 (initialisation, iterative computation,
// finalisation) map to inpaint_create/inpaint_reset, inpaint_step/inpaint_run
// and inpaint_result.  inpaint_run drives the whole iterative stage from the
// device: one CUDA graph whose conditional while-node repeats
// [findBestPatch search -> copy/update + next selection] until the update
// kernel reports an empty Omega, so no host round trip happens per iteration.
#include <algorithm>
#include <chrono>
#include <climits>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <queue>
#include <string>
#include <vector>

#include "inpaint_engine.h"
#include "inpaint_internal.cuh"

using namespace inp;

namespace {

thread_local std::string g_last_error;

int cuda_fail(cudaError_t e, const char* what) {
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  g_last_error = buf;
  return e == cudaErrorMemoryAllocation ? INPAINT_ERR_NOMEM : INPAINT_ERR_CUDA;
}

#define CK(call)                                     \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

}  // namespace

struct inpaint_ctx {
  int W = 0, H = 0, r = 0;
  inpaint_options opt{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  ImgState st{};
  int32_t* sat = nullptr;
  uint8_t* rgb_stage = nullptr;   // 3*W*H
  uint8_t* mask_stage = nullptr;  // W*H
  double* conf_stage = nullptr;   // W*H (import only)
  uint8_t* orig_rgb = nullptr;    // 3*W*H, batch members only: input kept for reset
  uint8_t* orig_mask = nullptr;   // W*H
  Ctrl* h_ctrl = nullptr;         // pinned mirror of the control block
  int* h_limit = nullptr;         // pinned staging for iter_limit
  std::vector<std::pair<void*, size_t>> allocs;
  cudaGraph_t run_graph = nullptr;
  cudaGraphExec_t run_exec = nullptr;
  unsigned long long cond = 0;
  TcPlan tc{};  // tensor-core search plan (form INPAINT_FORM_TC)
  // persistent engine (one team of every CTA)
  bool eng_ready = false;
  int eng_grid = 0, eng_sr = 0;
  size_t eng_smem = 0;
  EngineArgs ea{};
  ImgState* d_img = nullptr;
  CUtensorMap* d_tmap = nullptr;
  int* d_ints = nullptr;     // cta_team[grid], team_first[2], team_img_off[2], team_img[1]
  TeamCtl* d_team = nullptr;
  unsigned long long* d_epart = nullptr;
  int* d_err = nullptr;
  int* h_err = nullptr;
  unsigned long long* d_key = nullptr;  // key applied by inpaint_apply_key

  void* dalloc(size_t bytes) {
    void* p = nullptr;
    if (opt.dev_alloc) {
      p = opt.dev_alloc(bytes, (void*)stream, opt.alloc_user);
      if (p && (reinterpret_cast<uintptr_t>(p) & 255u) != 0) {
        // the kernels' 16-byte asynchronous copies need aligned blocks
        if (opt.dev_free) opt.dev_free(p, bytes, (void*)stream, opt.alloc_user);
        p = nullptr;
      }
    } else if (cudaMallocAsync(&p, bytes, stream) != cudaSuccess) {
      p = nullptr;
    }
    if (p) allocs.emplace_back(p, bytes);
    return p;
  }
  void release() {
    if (stream) cudaStreamSynchronize(stream);
    if (run_exec) cudaGraphExecDestroy(run_exec);
    if (run_graph) cudaGraphDestroy(run_graph);
    run_exec = nullptr;
    run_graph = nullptr;
    for (auto& a : allocs) {
      if (opt.dev_free)
        opt.dev_free(a.first, a.second, (void*)stream, opt.alloc_user);
      else
        cudaFreeAsync(a.first, stream);
    }
    allocs.clear();
    if (stream) cudaStreamSynchronize(stream);
    if (h_ctrl) cudaFreeHost(h_ctrl);
    if (h_limit) cudaFreeHost(h_limit);
    if (h_err) cudaFreeHost(h_err);
    h_ctrl = nullptr;
    h_limit = nullptr;
    h_err = nullptr;
    if (own_stream && stream) cudaStreamDestroy(stream);
    stream = nullptr;
  }
};

namespace {

template <class T>
bool alloc_n(inpaint_ctx* c, T*& p, size_t n) {
  p = static_cast<T*>(c->dalloc(n * sizeof(T)));
  return p != nullptr;
}

void search_rect(const uint8_t* mask, int mstride, int W, int H, int r, double alpha, bool overlap,
                 int* x0o, int* x1o, int* y0o, int* y1o) {
  // every interior centre; the partial-overlap variant admits border centres too
  int lo_x = overlap ? 0 : r, hi_x = overlap ? W - 1 : W - 1 - r;
  int lo_y = overlap ? 0 : r, hi_y = overlap ? H - 1 : H - 1 - r;
  if (alpha >= 0.0 && mask) {
    int bx0 = W, bx1 = -1, by0 = H, by1 = -1;
    for (int y = 0; y < H; ++y)
      for (int x = 0; x < W; ++x)
        if (mask[(size_t)y * mstride + x]) {
          bx0 = x < bx0 ? x : bx0;
          bx1 = x > bx1 ? x : bx1;
          by0 = y < by0 ? y : by0;
          by1 = y > by1 ? y : by1;
        }
    if (bx1 >= 0) {
      const int ex = (int)(alpha * (double)(bx1 - bx0 + 1));
      const int ey = (int)(alpha * (double)(by1 - by0 + 1));
      lo_x = bx0 - ex > lo_x ? bx0 - ex : lo_x;
      hi_x = bx1 + ex < hi_x ? bx1 + ex : hi_x;
      lo_y = by0 - ey > lo_y ? by0 - ey : lo_y;
      hi_y = by1 + ey < hi_y ? by1 + ey : hi_y;
    }
  }
  *x0o = lo_x;
  *x1o = hi_x;
  *y0o = lo_y;
  *y1o = hi_y;
}

// Runs the device initialisation from the staging buffers (or device inputs)
// and checks the outcome.
int finish_init(inpaint_ctx* c) {
  CK(cudaMemcpyAsync(c->h_ctrl, c->st.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (c->h_ctrl->remaining == c->W * c->H) {
    g_last_error = "mask covers every pixel: no known pixel to copy from";
    return INPAINT_ERR_ARG;
  }
  if (c->h_ctrl->status != 0) return c->h_ctrl->status;
  return INPAINT_OK;
}

int check_geometry(int W, int H, int r) {
  if (r < 1 || r > kMaxRadius) {
    g_last_error = "patch radius must be in 1..32";
    return INPAINT_ERR_ARG;
  }
  if (W < 2 * r + 1 || H < 2 * r + 1 || (long long)W * H > (1ll << 30)) {
    g_last_error = "image must be at least (2r+1) x (2r+1) and below 2^30 pixels";
    return INPAINT_ERR_ARG;
  }
  return INPAINT_OK;
}

int launch_iteration(inpaint_ctx* c, int use_cond) {
  if (c->opt.form == INPAINT_FORM_TC)
    CK(launch_search_tc(c->st, c->tc, c->stream));
  else
    CK(launch_search_plain(c->st, c->stream));
  if (c->r <= 8)
    CK(launch_update_fast(c->st, c->cond, use_cond, c->stream));
  else
    CK(launch_update(c->st, 1, c->cond, use_cond, c->stream));
  if (c->opt.debug_checks) CK(launch_verify_count(c->st, c->stream));
  return INPAINT_OK;
}

bool use_engine(const inpaint_ctx* c) {
  if (c->opt.loop_mode == INPAINT_LOOP_GRAPH || c->opt.search_variant != INPAINT_SEARCH_FULL) return false;
  return c->r <= 8;
}

// Rows per warp from an autotuner table: lines "radius max_pixels rows";
// the first line with this radius and max_pixels >= `pixels` (the image's
// pixels per CTA of its team) wins; 0 if none.
int tuned_rows_per_warp(const char* path, int r, long long pixels) {
  if (!path) return 0;
  FILE* f = fopen(path, "r");
  if (!f) return 0;
  int rr = 0, rows = 0, out = 0;
  long long mp = 0;
  while (fscanf(f, "%d %lld %d", &rr, &mp, &rows) == 3) {
    if (rr == r && pixels <= mp && (rows == 1 || rows == 2)) {
      out = rows;
      break;
    }
  }
  fclose(f);
  return out;
}

// Search batch width (a batch is 32 candidate rows x 16 warps x 4 * srw
// candidate columns): srw = 2 (8 candidates per lane, the fewer loads per
// evaluation) when that still gives every CTA of the team a batch, else 1.
int pick_rows_per_warp(const ImgState& s, int grid) {
  const int xb = s.r + ((s.cx0 - s.r) & ~3);
  const long long w2 = eng_batch_cols(2);
  const long long ncg = (s.cx1 - xb + w2) / w2, ch = s.cy1 - s.cy0 + 1;
  return ncg * ((ch + kEngBatchRows - 1) / kEngBatchRows) >= (long long)grid ? 2 : 1;
}

int setup_engine(inpaint_ctx* c) {
  if (c->eng_ready) return INPAINT_OK;
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int sr = c->opt.tile_rows;
  if (sr != 0 && sr != 1 && sr != 2) {
    g_last_error = "tile_rows must be 0, 1 or 2";
    return INPAINT_ERR_ARG;
  }
  const EngineFns* f = engine_fns(c->r);
  if (!f) return INPAINT_ERR_UNSUPPORTED;
  int bps = 0;
  const size_t smem = engine_launch_smem();
  if (smem < f->smem_bytes(2)) {
    g_last_error = "engine kernel does not fit on an SM";
    return INPAINT_ERR_UNSUPPORTED;
  }
  CK(engine_occupancy(smem, &bps));
  if (bps < 1) {
    g_last_error = "engine kernel does not fit on an SM";
    return INPAINT_ERR_UNSUPPORTED;
  }
  const int grid = sms * bps;
  if (!sr) sr = tuned_rows_per_warp(c->opt.tuning_file, c->r, (long long)c->W * c->H / grid);
  if (!sr) sr = pick_rows_per_warp(c->st, grid);
  c->eng_smem = smem;
  c->eng_grid = grid;
  c->eng_sr = sr;
  c->st.srw = sr;
  if (!alloc_n(c, c->d_img, 1) || !alloc_n(c, c->d_tmap, 2) ||
      !alloc_n(c, c->d_ints, (size_t)c->eng_grid + 5) || !alloc_n(c, c->d_team, 1) ||
      !alloc_n(c, c->d_epart, (size_t)c->eng_grid) || !alloc_n(c, c->d_err, 1))
    return INPAINT_ERR_NOMEM;
  if (!c->h_err && cudaMallocHost(&c->h_err, sizeof(int)) != cudaSuccess) return INPAINT_ERR_NOMEM;
  CUtensorMap tm[2];
  if (make_image_tmap(c->st, sr, tm) != 0) {
    g_last_error = "cuTensorMapEncodeTiled failed";
    return INPAINT_ERR_CUDA;
  }
  std::vector<int> ints((size_t)c->eng_grid + 5, 0);  // every CTA in team 0
  ints[c->eng_grid + 0] = 0;
  ints[c->eng_grid + 1] = c->eng_grid;  // team_first = {0, grid}
  ints[c->eng_grid + 2] = 0;
  ints[c->eng_grid + 3] = 1;            // team_img_off = {0, 1}
  ints[c->eng_grid + 4] = 0;            // team_img = {0}
  CK(cudaMemcpyAsync(c->d_img, &c->st, sizeof(ImgState), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->d_tmap, tm, 2 * sizeof(CUtensorMap), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->d_ints, ints.data(), ints.size() * sizeof(int), cudaMemcpyHostToDevice,
                     c->stream));
  CK(cudaStreamSynchronize(c->stream));
  EngineArgs& ea = c->ea;
  ea.imgs = c->d_img;
  ea.tmaps = c->d_tmap;
  ea.cta_team = c->d_ints;
  ea.team_first = c->d_ints + c->eng_grid;
  ea.team_img_off = c->d_ints + c->eng_grid + 2;
  ea.team_img = c->d_ints + c->eng_grid + 4;
  ea.teams = c->d_team;
  ea.partials = c->d_epart;
  ea.err = c->d_err;
  ea.wait_limit_ns = 4000000000ull;  // 4 s: far beyond any iteration
  ea.tc_cols = c->st.planes ? 256 : 0;  // X and S accumulators of N <= 128 columns each
  c->eng_ready = true;
  return INPAINT_OK;
}

int run_engine(inpaint_ctx* c) {
  int rc = setup_engine(c);
  if (rc) return rc;
  CK(cudaMemsetAsync(c->d_team, 0, sizeof(TeamCtl), c->stream));
  CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
  CK(launch_planes(c->st, c->stream));  // the image may have changed since the last launch
  CK(engine_launch(c->eng_smem, c->ea, c->eng_grid, c->stream));
  CK(cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  return INPAINT_OK;
}

int build_run_graph(inpaint_ctx* c) {
  if (c->run_exec) return INPAINT_OK;
  CK(cudaGraphCreate(&c->run_graph, 0));
  cudaGraphConditionalHandle h;
  CK(cudaGraphConditionalHandleCreate(&h, c->run_graph, 1, cudaGraphCondAssignDefault));
  c->cond = (unsigned long long)h;
  cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, c->run_graph, nullptr, nullptr, 0, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(c->stream, body, nullptr, nullptr, 0,
                                   cudaStreamCaptureModeThreadLocal));
  int rc = launch_iteration(c, 1);
  cudaGraph_t captured = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->stream, &captured);
  if (rc != INPAINT_OK) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  CK(cudaGraphInstantiate(&c->run_exec, c->run_graph, 0));
  return INPAINT_OK;
}

int set_limit(inpaint_ctx* c, int limit) {
  *c->h_limit = limit;
  CK(cudaMemcpyAsync(&c->st.ctrl->iter_limit, c->h_limit, sizeof(int), cudaMemcpyHostToDevice,
                     c->stream));
  return INPAINT_OK;
}

int read_ctrl(const inpaint_ctx* c) {
  CK(cudaMemcpyAsync(c->h_ctrl, c->st.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return INPAINT_OK;
}

int create_impl(const uint8_t* rgb, int W, int H, int rgb_stride, const uint8_t* mask,
                int mask_stride, int r, const inpaint_options* opt, inpaint_ctx** out) {
  if (!out) return INPAINT_ERR_ARG;
  *out = nullptr;
  if (!rgb || !mask || rgb_stride < 3 * W || mask_stride < W) {
    g_last_error = "null input or stride smaller than a row";
    return INPAINT_ERR_ARG;
  }
  int rc = check_geometry(W, H, r);
  if (rc) return rc;
  inpaint_options o;
  inpaint_options_default(&o);
  if (opt) o = *opt;
  if (o.form != INPAINT_FORM_PLAIN && o.form != INPAINT_FORM_TC) return INPAINT_ERR_ARG;
  if (o.loop_mode < INPAINT_LOOP_AUTO || o.loop_mode > INPAINT_LOOP_GRAPH) return INPAINT_ERR_ARG;
  if (o.loop_mode == INPAINT_LOOP_ENGINE && r > 8) {
    g_last_error = "the persistent engine supports patch_radius <= 8";
    return INPAINT_ERR_UNSUPPORTED;
  }
  if ((o.dev_alloc == nullptr) != (o.dev_free == nullptr)) {
    g_last_error = "dev_alloc and dev_free must be given together";
    return INPAINT_ERR_ARG;
  }
  if (o.form == INPAINT_FORM_TC && r > 8) {
    g_last_error = "the tensor-core form supports patch_radius <= 8";
    return INPAINT_ERR_UNSUPPORTED;
  }
  if (o.search_variant != INPAINT_SEARCH_FULL && o.search_variant != INPAINT_SEARCH_OVERLAP)
    return INPAINT_ERR_ARG;
  if (o.search_variant == INPAINT_SEARCH_OVERLAP &&
      (o.form != INPAINT_FORM_PLAIN || r > 8 || o.loop_mode == INPAINT_LOOP_ENGINE)) {
    g_last_error = "the partial-overlap search is the plain form, patch_radius <= 8, graph loop";
    return INPAINT_ERR_UNSUPPORTED;
  }

  inpaint_ctx* c = new (std::nothrow) inpaint_ctx();
  if (!c) return INPAINT_ERR_NOMEM;
  c->W = W;
  c->H = H;
  c->r = r;
  c->opt = o;
  auto fail = [&](int code) {
    c->release();
    delete c;
    return code;
  };
  if (o.cuda_stream) {
    c->stream = (cudaStream_t)o.cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess)
      return fail(INPAINT_ERR_CUDA);
    c->own_stream = true;
  }
  if (cudaMallocHost(&c->h_ctrl, sizeof(Ctrl)) != cudaSuccess) return fail(INPAINT_ERR_NOMEM);
  if (cudaMallocHost(&c->h_limit, sizeof(int)) != cudaSuccess) return fail(INPAINT_ERR_NOMEM);

  ImgState& s = c->st;
  s.W = W;
  s.H = H;
  s.r = r;
  search_rect(mask, mask_stride, W, H, r, o.search_alpha, o.search_variant == INPAINT_SEARCH_OVERLAP,
              &s.cx0, &s.cx1, &s.cy0, &s.cy1);
  s.overlap = o.search_variant == INPAINT_SEARCH_OVERLAP ? 1 : 0;
  s.pitch = (W + 3) & ~3;
  s.t0x = (W + kT0 - 1) / kT0;
  s.t0y = (H + kT0 - 1) / kT0;
  s.t1x = (s.t0x + kT1 - 1) / kT1;
  s.t1y = (s.t0y + kT1 - 1) / kT1;
  size_t n_omega = 0;
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) n_omega += mask[(size_t)y * mask_stride + x] != 0;
  s.trace_cap = (int)n_omega + 1;
  const dim3 g = search_plain_grid(s);
  s.n_partial = (int)(g.x * g.y);
  if (o.form == INPAINT_FORM_TC) {
    if (prepare_search_tc(s, &c->tc) != cudaSuccess) {
      g_last_error = "tensor-core search set-up failed";
      return fail(INPAINT_ERR_CUDA);
    }
    s.n_partial = c->tc.grid;
  }
  const size_t n = (size_t)W * H;
  if (!alloc_n(c, s.img, (size_t)s.pitch * H) || !alloc_n(c, s.omega, n) || !alloc_n(c, s.gray, n) ||
      !alloc_n(c, s.conf, n) || !alloc_n(c, s.count, (size_t)s.pitch * H) || !alloc_n(c, s.prio, n) ||
      !alloc_n(c, s.pconf, n) || !alloc_n(c, s.tiles0, (size_t)s.t0x * s.t0y) ||
      !alloc_n(c, s.tiles1, (size_t)s.t1x * s.t1y) ||
      !alloc_n(c, s.ctrl, 1) || !alloc_n(c, s.trace, (size_t)s.trace_cap) ||
      !alloc_n(c, s.partial, (size_t)(s.n_partial > 0 ? s.n_partial : 1)) ||
      !alloc_n(c, c->sat, (size_t)(W + 1) * (H + 1) + (size_t)sat_chunks(H) * W) || !alloc_n(c, c->rgb_stage, 3 * n) ||
      !alloc_n(c, c->mask_stage, n)) {
    g_last_error = "device allocation failed";
    return fail(INPAINT_ERR_NOMEM);
  }
  if (o.form == INPAINT_FORM_TC) {
    // the tensor-core search reads five BF16 planes of the image
    const size_t np = tc_plane_layout(s);
    if (np > 0 && !alloc_n(c, s.planes, np)) {
      g_last_error = "device allocation failed";
      return fail(INPAINT_ERR_NOMEM);
    }
  }
  if (prepare_search_plain(r) != cudaSuccess) return fail(INPAINT_ERR_CUDA);
  *out = c;
  rc = inpaint_reset(c, rgb, rgb_stride, mask, mask_stride, 0);
  if (rc < 0) {
    *out = nullptr;
    return fail(rc);
  }
  return INPAINT_OK;
}

}  // namespace

void inp::set_last_error(const char* msg) { g_last_error = msg; }

extern "C" {

void inpaint_options_default(inpaint_options* opt) {
  if (!opt) return;
  memset(opt, 0, sizeof *opt);
  opt->form = INPAINT_FORM_PLAIN;
  opt->search_alpha = -1.0;
}

int inpaint_create(const uint8_t* rgb, int width, int height, int rgb_stride_bytes,
                   const uint8_t* mask, int mask_stride_bytes, int patch_radius,
                   const inpaint_options* opt, inpaint_ctx** out) {
  try {
    return create_impl(rgb, width, height, rgb_stride_bytes, mask, mask_stride_bytes,
                       patch_radius, opt, out);
  } catch (...) {
    return INPAINT_ERR_NOMEM;
  }
}

int inpaint_reset(inpaint_ctx* c, const uint8_t* rgb, int rgb_stride, const uint8_t* mask,
                  int mask_stride, int input_on_device) {
  if (!c || !rgb || !mask || rgb_stride < 3 * c->W || mask_stride < c->W) return INPAINT_ERR_ARG;
  const int W = c->W, H = c->H;
  const uint8_t* drgb = rgb;
  const uint8_t* dmask = mask;
  int rs = rgb_stride, ms = mask_stride;
  if (!input_on_device) {
    CK(cudaMemcpy2DAsync(c->rgb_stage, 3 * (size_t)W, rgb, rgb_stride, 3 * (size_t)W, H,
                         cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpy2DAsync(c->mask_stage, W, mask, mask_stride, W, H, cudaMemcpyHostToDevice,
                         c->stream));
    drgb = c->rgb_stage;
    dmask = c->mask_stage;
    rs = 3 * W;
    ms = W;
  }
  CK(launch_init(c->st, drgb, rs, dmask, ms, c->sat, nullptr, c->stream));
  return finish_init(c);
}

int inpaint_step(inpaint_ctx* c, inpaint_step_info* info) {
  if (!c) return INPAINT_ERR_ARG;
  int rc = read_ctrl(c);
  if (rc) return rc;
  if (c->h_ctrl->status != 0) return c->h_ctrl->status;
  if (c->h_ctrl->remaining == 0) return INPAINT_DONE;
  if ((rc = set_limit(c, INT_MAX))) return rc;
  CK(launch_planes(c->st, c->stream));  // the image may have changed since the last call
  if ((rc = launch_iteration(c, 0))) return rc;
  if ((rc = read_ctrl(c))) return rc;
  if (c->h_ctrl->status != 0) return c->h_ctrl->status;
  if (info) *info = c->h_ctrl->last;
  return INPAINT_OK;
}

int inpaint_run(inpaint_ctx* c, int max_iters, int* iters_done, inpaint_step_info* trace,
                int trace_cap) {
  if (iters_done) *iters_done = 0;
  if (!c || (trace && trace_cap < 0)) return INPAINT_ERR_ARG;
  if (c->h_err) *c->h_err = 0;
  int rc = read_ctrl(c);
  if (rc) return rc;
  if (c->h_ctrl->status != 0) return c->h_ctrl->status;
  if (c->h_ctrl->remaining == 0) return INPAINT_DONE;
  const int start = c->h_ctrl->iter;
  // Every iteration fills at least one pixel, so |Omega| iterations always
  // suffice: the device loop is bounded even if a kernel misbehaved.
  long long lim = (long long)start + c->h_ctrl->remaining;
  if (max_iters > 0 && (long long)start + max_iters < lim) lim = (long long)start + max_iters;
  if ((rc = set_limit(c, lim > INT_MAX ? INT_MAX : (int)lim))) return rc;
  if (use_engine(c)) {
    if (c->opt.debug_checks) {  // engine has no per-iteration hook: drive it one iteration at a time
      for (long long i = start; i < lim; ++i) {
        if ((rc = set_limit(c, (int)(i + 1)))) return rc;
        if ((rc = run_engine(c))) return rc;
        CK(launch_verify_count(c->st, c->stream));
        if ((rc = read_ctrl(c))) return rc;
        if (*c->h_err || c->h_ctrl->status != 0 || c->h_ctrl->remaining == 0) break;
      }
    } else if ((rc = run_engine(c))) {
      return rc;
    }
  } else {
    if ((rc = build_run_graph(c))) return rc;
    CK(launch_planes(c->st, c->stream));  // the image may have changed since the last call
    CK(cudaGraphLaunch(c->run_exec, c->stream));
  }
  if ((rc = set_limit(c, INT_MAX))) return rc;
  if ((rc = read_ctrl(c))) return rc;
  const int done = c->h_ctrl->iter - start;
  if (iters_done) *iters_done = done;
  if (trace && trace_cap > 0 && done > 0) {
    int n = done < trace_cap ? done : trace_cap;
    if (start + n > c->st.trace_cap) n = c->st.trace_cap - start;
    if (n > 0) {
      CK(cudaMemcpyAsync(trace, c->st.trace + start, (size_t)n * sizeof(inpaint_step_info),
                         cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));
    }
  }
  if (c->h_err && *c->h_err) {
    g_last_error = "a bounded device wait in the persistent engine gave up";
    return INPAINT_ERR_TIMEOUT;
  }
  if (c->h_ctrl->status != 0) return c->h_ctrl->status;
  return INPAINT_OK;
}

int inpaint_result(const inpaint_ctx* c, uint8_t* rgb_out, int stride, uint8_t* mask_out) {
  if (!c || !rgb_out || stride < 3 * c->W) return INPAINT_ERR_ARG;
  CK(launch_export(c->st, c->rgb_stage, c->stream));
  CK(cudaMemcpy2DAsync(rgb_out, stride, c->rgb_stage, 3 * (size_t)c->W, 3 * (size_t)c->W, c->H,
                       cudaMemcpyDeviceToHost, c->stream));
  if (mask_out)
    CK(cudaMemcpyAsync(mask_out, c->st.omega, (size_t)c->W * c->H, cudaMemcpyDeviceToHost,
                       c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return INPAINT_OK;
}

int inpaint_export_state(const inpaint_ctx* c, uint8_t* rgb, uint8_t* omega, double* conf) {
  if (!c) return INPAINT_ERR_ARG;
  const size_t n = (size_t)c->W * c->H;
  if (rgb) {
    CK(launch_export(c->st, c->rgb_stage, c->stream));
    CK(cudaMemcpyAsync(rgb, c->rgb_stage, 3 * n, cudaMemcpyDeviceToHost, c->stream));
  }
  if (omega) CK(cudaMemcpyAsync(omega, c->st.omega, n, cudaMemcpyDeviceToHost, c->stream));
  if (conf)
    CK(cudaMemcpyAsync(conf, c->st.conf, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return INPAINT_OK;
}

int inpaint_import_state(inpaint_ctx* c, const uint8_t* rgb, const uint8_t* omega,
                         const double* conf) {
  if (!c || !rgb || !omega || !conf) return INPAINT_ERR_ARG;
  const size_t n = (size_t)c->W * c->H;
  if (!c->conf_stage && !alloc_n(c, c->conf_stage, n)) return INPAINT_ERR_NOMEM;
  CK(cudaMemcpyAsync(c->rgb_stage, rgb, 3 * n, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->mask_stage, omega, n, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->conf_stage, conf, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CK(launch_import(c->st, c->rgb_stage, c->mask_stage, c->conf_stage, c->sat, nullptr,
                   c->stream));
  return finish_init(c);
}

int inpaint_info(const inpaint_ctx* c, int* width, int* height, int* patch_radius, int* remaining,
                 uint64_t* evals) {
  if (!c) return INPAINT_ERR_ARG;
  int rc = read_ctrl(c);
  if (rc) return rc;
  if (width) *width = c->W;
  if (height) *height = c->H;
  if (patch_radius) *patch_radius = c->r;
  if (remaining) *remaining = c->h_ctrl->remaining;
  if (evals) *evals = c->h_ctrl->evals;
  return INPAINT_OK;
}

int inpaint_time_search(inpaint_ctx* c, int form, int reps, double* ms_per_search,
                        unsigned long long* best_key, unsigned long long* evals) {
  if (!c || reps < 1 || !ms_per_search || (form != INPAINT_FORM_PLAIN && form != INPAINT_FORM_TC))
    return INPAINT_ERR_ARG;
  if (form == INPAINT_FORM_TC && c->r > 8) return INPAINT_ERR_UNSUPPORTED;
  int rc = read_ctrl(c);
  if (rc) return rc;
  const Ctrl h = *c->h_ctrl;
  if (h.status != 0) return h.status;
  if (h.remaining <= 0 || h.px < 0) return INPAINT_DONE;
  ImgState s = c->st;
  TcPlan plan{};
  uint16_t* tmp_planes = nullptr;  // a plain-form context has no planes: build them for the timing
  if (form == INPAINT_FORM_TC) {
    CK(prepare_search_tc(s, &plan));
    s.n_partial = plan.grid;
    if (!s.planes && s.n_partial > 0) {
      const size_t np = tc_plane_layout(s);
      CK(cudaMalloc(&tmp_planes, np * sizeof(uint16_t)));
      s.planes = tmp_planes;
    }
    CK(launch_planes(s, c->stream));
  } else {
    CK(prepare_search_plain(s.r));
    const dim3 g = search_plain_grid(s);
    s.n_partial = (int)(g.x * g.y);
  }
  if (s.n_partial <= 0) return INPAINT_DONE;
  unsigned long long* part = nullptr;
  if (cudaError_t ea = cudaMalloc(&part, sizeof(unsigned long long) * s.n_partial)) {
    if (tmp_planes) cudaFree(tmp_planes);
    return cuda_fail(ea, "cudaMalloc");
  }
  s.partial = part;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto launch = [&]() {
    return form == INPAINT_FORM_TC ? launch_search_tc(s, plan, c->stream) : launch_search_plain(s, c->stream);
  };
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = launch();
  if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
  for (int i = 0; i < reps && e == cudaSuccess; ++i) e = launch();
  if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  std::vector<unsigned long long> keys(s.n_partial);
  if (e == cudaSuccess)
    e = cudaMemcpy(keys.data(), part, sizeof(unsigned long long) * keys.size(), cudaMemcpyDeviceToHost);
  // known pixels of the target patch
  const int r = c->r, P = 2 * r + 1;
  std::vector<uint8_t> om((size_t)P * P, 1);
  const int x0 = std::max(0, h.px - r), x1 = std::min(c->W - 1, h.px + r);
  const int y0 = std::max(0, h.py - r), y1 = std::min(c->H - 1, h.py + r);
  if (e == cudaSuccess)
    e = cudaMemcpy2D(om.data(), P, s.omega + (size_t)y0 * c->W + x0, c->W, x1 - x0 + 1, y1 - y0 + 1,
                     cudaMemcpyDeviceToHost);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(part);
  if (tmp_planes) cudaFree(tmp_planes);
  CK(e);
  long long n_known = 0;
  for (int y = 0; y <= y1 - y0; ++y)
    for (int x = 0; x <= x1 - x0; ++x) n_known += om[(size_t)y * P + x] == 0;
  *ms_per_search = (double)ms / reps;
  if (best_key) *best_key = *std::min_element(keys.begin(), keys.end());
  if (evals) *evals = (unsigned long long)n_known * (unsigned long long)std::max(h.n_valid, 0);
  return INPAINT_OK;
}

namespace {

// Sharded iterations run the plain form's search and update kernels on the
// full search (the variant counts its admissible candidates in the search).
int sharded_ok(const inpaint_ctx* c) {
  if (c->opt.form != INPAINT_FORM_PLAIN || c->opt.search_variant != INPAINT_SEARCH_FULL) {
    g_last_error = "row-sharded iterations need the plain form and the full search";
    return INPAINT_ERR_UNSUPPORTED;
  }
  return INPAINT_OK;
}

}  // namespace

int inpaint_search_rows(inpaint_ctx* c, int y0, int y1, unsigned long long* key_out) {
  if (!c || !key_out || y0 > y1) return INPAINT_ERR_ARG;
  *key_out = INPAINT_KEY_NONE;
  int rc = sharded_ok(c);
  if (rc) return rc;
  if ((rc = read_ctrl(c))) return rc;
  if (c->h_ctrl->status != 0) return c->h_ctrl->status;
  if (c->h_ctrl->remaining == 0) return INPAINT_DONE;
  ImgState s = c->st;
  s.cy0 = std::max(s.cy0, y0);
  s.cy1 = std::min(s.cy1, y1 - 1);
  if (s.cy0 > s.cy1 || s.cx0 > s.cx1) return INPAINT_OK;
  const dim3 g = search_plain_grid(s);
  s.n_partial = (int)(g.x * g.y);  // fewer rows: at most the full rectangle's grid
  if (s.n_partial <= 0 || s.n_partial > c->st.n_partial) return INPAINT_ERR_INTERNAL;
  CK(prepare_search_plain(s.r));
  CK(launch_search_plain(s, c->stream));
  std::vector<unsigned long long> keys(s.n_partial);
  CK(cudaMemcpyAsync(keys.data(), s.partial, sizeof(unsigned long long) * keys.size(),
                     cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  *key_out = *std::min_element(keys.begin(), keys.end());
  return INPAINT_OK;
}

int inpaint_apply_key(inpaint_ctx* c, unsigned long long key, inpaint_step_info* info) {
  if (!c) return INPAINT_ERR_ARG;
  int rc = sharded_ok(c);
  if (rc) return rc;
  if (key != INPAINT_KEY_NONE) {
    const unsigned long long q = key & 0xffffffffull;
    const long long qx = (long long)(q % (unsigned long long)c->W), qy = (long long)(q / (unsigned long long)c->W);
    if (qy >= c->H || qx < c->r || qx > c->W - 1 - c->r || qy < c->r || qy > c->H - 1 - c->r) {
      g_last_error = "the key's centre is not an interior pixel";
      return INPAINT_ERR_ARG;
    }
  }
  if ((rc = read_ctrl(c))) return rc;
  if (c->h_ctrl->status != 0) return c->h_ctrl->status;
  if (c->h_ctrl->remaining == 0) return INPAINT_DONE;
  if (!c->d_key && !alloc_n(c, c->d_key, 1)) return INPAINT_ERR_NOMEM;
  if ((rc = set_limit(c, INT_MAX))) return rc;
  CK(cudaMemcpyAsync(c->d_key, &key, sizeof(key), cudaMemcpyHostToDevice, c->stream));
  ImgState s = c->st;
  s.partial = c->d_key;
  s.n_partial = 1;
  if (c->r <= 8)
    CK(launch_update_fast(s, c->cond, 0, c->stream));
  else
    CK(launch_update(s, 1, c->cond, 0, c->stream));
  if (c->opt.debug_checks) CK(launch_verify_count(c->st, c->stream));
  if ((rc = read_ctrl(c))) return rc;
  if (c->h_ctrl->status != 0) return c->h_ctrl->status;
  if (info) *info = c->h_ctrl->last;
  return INPAINT_OK;
}

int inpaint_run_withheld(inpaint_ctx* c, int rank, double wait_limit_s, int max_iters,
                         int* iters_done) {
  if (iters_done) *iters_done = 0;
  if (!c || rank < 0 || !(wait_limit_s > 0.0) || wait_limit_s > 10.0) return INPAINT_ERR_ARG;
  if (!use_engine(c)) return INPAINT_ERR_UNSUPPORTED;
  int rc = setup_engine(c);
  if (rc) return rc;
  const unsigned long long limit0 = c->ea.wait_limit_ns;
  c->ea.wait_limit_ns = (unsigned long long)(wait_limit_s * 1e9);
  c->ea.withhold = rank + 1;
  rc = inpaint_run(c, max_iters, iters_done, nullptr, 0);
  c->ea.wait_limit_ns = limit0;
  c->ea.withhold = 0;
  return rc;
}

int inpaint_loop_timing(const inpaint_ctx* c, uint64_t* search_ns, uint64_t* update_ns,
                        int* iters) {
  if (!c) return INPAINT_ERR_ARG;
  int rc = read_ctrl(c);
  if (rc) return rc;
  if (search_ns) *search_ns = c->h_ctrl->t_search;
  if (update_ns) *update_ns = c->h_ctrl->t_update;
  if (iters) *iters = c->h_ctrl->timed_iters;
  return INPAINT_OK;
}

int inpaint_search_form_rounds(const inpaint_ctx* c, int* tc_rounds) {
  if (!c || !tc_rounds) return INPAINT_ERR_ARG;
  int rc = read_ctrl(c);
  if (rc) return rc;
  *tc_rounds = c->h_ctrl->tc_rounds;
  return INPAINT_OK;
}

int inpaint_search_rect(const inpaint_ctx* c, int* x0, int* x1, int* y0, int* y1) {
  if (!c) return INPAINT_ERR_ARG;
  if (x0) *x0 = c->st.cx0;
  if (x1) *x1 = c->st.cx1;
  if (y0) *y0 = c->st.cy0;
  if (y1) *y1 = c->st.cy1;
  return INPAINT_OK;
}

void inpaint_destroy(inpaint_ctx* c) {
  if (!c) return;
  c->release();
  delete c;
}

const char* inpaint_status_str(int s) {
  switch (s) {
    case INPAINT_OK: return "ok";
    case INPAINT_DONE: return "done: target region already empty";
    case INPAINT_ERR_ARG: return "invalid argument";
    case INPAINT_ERR_NOMEM: return "out of memory";
    case INPAINT_ERR_CUDA: return "CUDA error";
    case INPAINT_ERR_NO_SOURCE: return "no fully-known source patch";
    case INPAINT_ERR_TIMEOUT: return "device wait timed out";
    case INPAINT_ERR_UNSUPPORTED: return "unsupported";
    case INPAINT_ERR_INTERNAL: return "internal consistency check failed";
    default: return "unknown status";
  }
}

const char* inpaint_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"


// ---------------------------------------------------------------- engine sets

// Device memory owned by a batch or a server (inpaint_options allocator hooks
// when given, else cudaMallocAsync on its stream).
struct DevAlloc {
  inpaint_options opt{};
  cudaStream_t stream = nullptr;
  std::vector<std::pair<void*, size_t>> allocs;
  void* alloc(size_t bytes) {
    void* p = nullptr;
    if (opt.dev_alloc)
      p = opt.dev_alloc(bytes, (void*)stream, opt.alloc_user);
    else if (cudaMallocAsync(&p, bytes, stream) != cudaSuccess)
      p = nullptr;
    if (p) allocs.emplace_back(p, bytes);
    return p;
  }
  void free(void* p) {
    for (size_t i = 0; i < allocs.size(); ++i)
      if (allocs[i].first == p) {
        if (opt.dev_free)
          opt.dev_free(p, allocs[i].second, (void*)stream, opt.alloc_user);
        else
          cudaFreeAsync(p, stream);
        allocs.erase(allocs.begin() + (long)i);
        return;
      }
  }
  void release() {
    while (!allocs.empty()) free(allocs.back().first);
  }
};

// One persistent launch over a set of contexts: team plan, per-image search
// rows and TMA descriptors, and the device arrays the engine reads.
struct EngineSet {
  int grid = 0, n_teams = 0;
  size_t smem = 0;
  std::vector<int> img_team, team_size;
  EngineArgs ea{};
  void* d_block = nullptr;
  size_t d_cap = 0;
  int* d_err = nullptr;
  int* h_pinned = nullptr;  // [0] err, [1..] iteration limits
  Ctrl* h_ctrls = nullptr;
  int h_cap = 0;
};

namespace {

// Teams: with fewer images than CTAs every image gets its own team, sized in
// proportion to its estimated work (|Omega| x valid candidates, i.e. the
// exhaustive evaluation count up to the patch area), at least one CTA; with
// more images than CTAs every CTA is a team and images are dealt longest
// first to the least loaded team.
void plan_teams(const std::vector<double>& work, int grid, std::vector<int>& team_size,
                std::vector<int>& img_team, std::vector<std::vector<int>>& team_imgs) {
  const int n = (int)work.size();
  img_team.assign(n, 0);
  if (n >= grid) {
    team_size.assign(grid, 1);
    team_imgs.assign(grid, {});
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });
    std::vector<double> load(grid, 0.0);
    for (int i : order) {
      const int t = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      load[t] += work[i];
      img_team[i] = t;
      team_imgs[t].push_back(i);
    }
    return;
  }
  // one CTA per image, then each further CTA to the team whose work per CTA
  // is largest (minimises the largest work per CTA, i.e. the batch's end)
  team_size.assign(n, 1);
  team_imgs.assign(n, {});
  std::priority_queue<std::pair<double, int>> pq;
  for (int i = 0; i < n; ++i) pq.emplace(work[i], i);
  for (int k = 0; k < grid - n; ++k) {
    const int i = pq.top().second;
    pq.pop();
    team_size[i] += 1;
    pq.emplace(work[i] / team_size[i], i);
  }
  for (int i = 0; i < n; ++i) {
    img_team[i] = i;
    team_imgs[i].push_back(i);
  }
}

int grid_for(const std::vector<inpaint_ctx*>& cs, int* grid) {
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  size_t smem_min = 0;
  for (inpaint_ctx* c : cs) smem_min = std::max(smem_min, engine_fns(c->r)->smem_bytes(2));
  const size_t smem = engine_launch_smem();
  if (smem < smem_min) return INPAINT_ERR_UNSUPPORTED;
  int bps = 0;
  CK(engine_occupancy(smem, &bps));
  if (bps < 1) return INPAINT_ERR_UNSUPPORTED;
  *grid = sms * bps;
  return INPAINT_OK;
}

// Plans the teams for the contexts (work estimates from their last control
// block mirrors) and uploads everything the engine reads.
int engine_set_prepare(EngineSet& es, const std::vector<inpaint_ctx*>& cs, const std::vector<double>& work,
                       const inpaint_options& opt, DevAlloc& da, cudaStream_t st) {
  const int n = (int)cs.size();
  int rc = grid_for(cs, &es.grid);
  if (rc) return rc;
  std::vector<std::vector<int>> team_imgs;
  plan_teams(work, es.grid, es.team_size, es.img_team, team_imgs);
  es.n_teams = (int)es.team_size.size();
  const int G = es.grid, T = es.n_teams;
  std::vector<ImgState> imgs(n);
  std::vector<CUtensorMap> maps(2 * (size_t)n);
  es.smem = 0;
  for (int i = 0; i < n; ++i) {
    inpaint_ctx* c = cs[i];
    int sr = opt.tile_rows;
    const int tsz = es.team_size[es.img_team[i]];
    if (!sr) sr = tuned_rows_per_warp(opt.tuning_file, c->r, (long long)c->W * c->H / tsz);
    if (!sr) sr = pick_rows_per_warp(c->st, tsz);
    c->st.srw = sr;
    imgs[i] = c->st;
    if (make_image_tmap(c->st, sr, &maps[2 * (size_t)i]) != 0) {
      g_last_error = "cuTensorMapEncodeTiled failed";
      return INPAINT_ERR_CUDA;
    }
  }
  es.smem = engine_launch_smem();
  std::vector<int> first(T + 1, 0), off(T + 1, 0), ints((size_t)G);
  std::vector<int> lst;
  for (int t = 0; t < T; ++t) {
    first[t + 1] = first[t] + es.team_size[t];
    off[t + 1] = off[t] + (int)team_imgs[t].size();
    for (int i : team_imgs[t]) lst.push_back(i);
    for (int k = first[t]; k < first[t + 1]; ++k) ints[k] = t;
  }
  const size_t o_first = ints.size();
  ints.insert(ints.end(), first.begin(), first.end());
  const size_t o_off = ints.size();
  ints.insert(ints.end(), off.begin(), off.end());
  const size_t o_lst = ints.size();
  ints.insert(ints.end(), lst.begin(), lst.end());
  // one device block: states | maps | teams | partials | ints | err
  auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t b_imgs = up(sizeof(ImgState) * n), b_maps = up(sizeof(CUtensorMap) * 2 * n);
  const size_t b_teams = up(sizeof(TeamCtl) * T), b_part = up(sizeof(unsigned long long) * G);
  const size_t b_ints = up(sizeof(int) * ints.size()), b_err = 256;
  const size_t need = b_imgs + b_maps + b_teams + b_part + b_ints + b_err;
  if (need > es.d_cap) {
    if (es.d_block) da.free(es.d_block);
    es.d_block = da.alloc(need * 2);
    if (!es.d_block) return INPAINT_ERR_NOMEM;
    es.d_cap = need * 2;
  }
  if (n + 1 > es.h_cap) {
    if (es.h_pinned) cudaFreeHost(es.h_pinned);
    if (es.h_ctrls) cudaFreeHost(es.h_ctrls);
    es.h_pinned = nullptr;
    es.h_ctrls = nullptr;
    const int cap = 2 * (n + 1);
    if (cudaMallocHost(&es.h_pinned, sizeof(int) * cap) != cudaSuccess ||
        cudaMallocHost(&es.h_ctrls, sizeof(Ctrl) * cap) != cudaSuccess)
      return INPAINT_ERR_NOMEM;
    es.h_cap = cap;
  }
  uint8_t* base = (uint8_t*)es.d_block;
  ImgState* d_imgs = (ImgState*)base;
  CUtensorMap* d_maps = (CUtensorMap*)(base + b_imgs);
  TeamCtl* d_teams = (TeamCtl*)(base + b_imgs + b_maps);
  unsigned long long* d_part = (unsigned long long*)(base + b_imgs + b_maps + b_teams);
  int* d_ints = (int*)(base + b_imgs + b_maps + b_teams + b_part);
  es.d_err = (int*)(base + b_imgs + b_maps + b_teams + b_part + b_ints);
  CK(cudaMemcpyAsync(d_imgs, imgs.data(), sizeof(ImgState) * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_maps, maps.data(), sizeof(CUtensorMap) * 2 * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_ints, ints.data(), sizeof(int) * ints.size(), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));  // the host vectors go out of scope
  EngineArgs& ea = es.ea;
  ea.imgs = d_imgs;
  ea.tmaps = d_maps;
  ea.cta_team = d_ints;
  ea.team_first = d_ints + o_first;
  ea.team_img_off = d_ints + o_off;
  ea.team_img = d_ints + o_lst;
  ea.teams = d_teams;
  ea.partials = d_part;
  ea.err = es.d_err;
  ea.wait_limit_ns = 4000000000ull;
  return INPAINT_OK;
}

// One launch: every context runs until its Omega is empty, it fails, or it
// has done max_iters more iterations (<= 0: no limit).  Control blocks are
// read back into es.h_ctrls.  Returns INPAINT_ERR_TIMEOUT if a bounded
// device wait gave up.
// Runs every member until it is done, or for at most max_iters (> 0) more
// iterations, or until the launch has run tick_ns (> 0; teams stop between
// iterations and resume in the next call).
int engine_set_run(EngineSet& es, const std::vector<inpaint_ctx*>& cs, int max_iters, cudaStream_t st,
                   unsigned long long tick_ns = 0ull) {
  const int n = (int)cs.size();
  for (int i = 0; i < n; ++i)
    CK(cudaMemcpyAsync(es.h_ctrls + i, cs[i]->st.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int i = 0; i < n; ++i) {
    const Ctrl& h = es.h_ctrls[i];
    long long lim = (long long)h.iter + std::max(h.remaining, 0);
    if (max_iters > 0 && (long long)h.iter + max_iters < lim) lim = (long long)h.iter + max_iters;
    es.h_pinned[1 + i] = (int)std::min<long long>(lim, INT_MAX);
    CK(cudaMemcpyAsync(&cs[i]->st.ctrl->iter_limit, &es.h_pinned[1 + i], sizeof(int),
                       cudaMemcpyHostToDevice, st));
  }
  CK(cudaMemsetAsync((void*)es.ea.teams, 0, sizeof(TeamCtl) * es.n_teams, st));
  CK(cudaMemsetAsync(es.d_err, 0, sizeof(int), st));
  es.ea.tick_ns = tick_ns;
  CK(engine_launch(es.smem, es.ea, es.grid, st));
  es.ea.tick_ns = 0ull;
  CK(cudaMemcpyAsync(es.h_pinned, es.d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  for (int i = 0; i < n; ++i)
    CK(cudaMemcpyAsync(es.h_ctrls + i, cs[i]->st.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int i = 0; i < n; ++i) {  // back to the unlimited bound for later calls
    es.h_pinned[1 + i] = INT_MAX;
    CK(cudaMemcpyAsync(&cs[i]->st.ctrl->iter_limit, &es.h_pinned[1 + i], sizeof(int),
                       cudaMemcpyHostToDevice, st));
  }
  CK(cudaStreamSynchronize(st));
  if (es.h_pinned[0]) {
    g_last_error = "a bounded device wait in the persistent engine gave up";
    return INPAINT_ERR_TIMEOUT;
  }
  return INPAINT_OK;
}

void engine_set_free(EngineSet& es) {
  if (es.h_pinned) cudaFreeHost(es.h_pinned);
  if (es.h_ctrls) cudaFreeHost(es.h_ctrls);
  es.h_pinned = nullptr;
  es.h_ctrls = nullptr;
}

// Creates a context for one image on the given stream, with a device copy of
// its input kept for resets.
int make_member(const inpaint_image& im, const inpaint_options& base, cudaStream_t st, int index,
                inpaint_ctx** out) {
  *out = nullptr;
  if (im.patch_radius < 1 || im.patch_radius > 8) {
    char buf[128];
    snprintf(buf, sizeof buf, "image %d: patch radius must be 1..8", index);
    g_last_error = buf;
    return INPAINT_ERR_ARG;
  }
  inpaint_options o = base;
  o.cuda_stream = (void*)st;
  o.loop_mode = INPAINT_LOOP_ENGINE;
  inpaint_ctx* c = nullptr;
  int rc = create_impl(im.rgb, im.width, im.height, im.rgb_stride_bytes, im.mask, im.mask_stride_bytes,
                       im.patch_radius, &o, &c);
  if (rc < 0) {
    char buf[200];
    snprintf(buf, sizeof buf, "image %d: %s", index, g_last_error.c_str());
    g_last_error = buf;
    return rc;
  }
  const size_t px = (size_t)im.width * im.height;
  if (!alloc_n(c, c->orig_rgb, 3 * px) || !alloc_n(c, c->orig_mask, px)) {
    inpaint_destroy(c);
    return INPAINT_ERR_NOMEM;
  }
  if (cudaMemcpyAsync(c->orig_rgb, c->rgb_stage, 3 * px, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(c->orig_mask, c->mask_stage, px, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
    inpaint_destroy(c);
    return INPAINT_ERR_CUDA;
  }
  *out = c;
  return INPAINT_OK;
}

double work_of(const Ctrl& h) {
  return (double)std::max(1, h.remaining) * std::max(1, h.n_valid);
}

}  // namespace

// ---------------------------------------------------------------- batch

struct inpaint_batch {
  int n = 0;
  inpaint_options opt{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<inpaint_ctx*> ctx;
  DevAlloc da;
  EngineSet es;
  // CUDA graphs: every member's initialisation (on kBatchAux parallel
  // branches) and the run to completion (one persistent launch + read-back)
  static constexpr int kBatchAux = 4;
  cudaGraphExec_t reset_exec = nullptr, run_exec = nullptr;
  cudaStream_t aux[kBatchAux] = {};
  cudaEvent_t fork = nullptr, join[kBatchAux] = {};
  void release() {
    if (stream) cudaStreamSynchronize(stream);
    if (reset_exec) cudaGraphExecDestroy(reset_exec);
    if (run_exec) cudaGraphExecDestroy(run_exec);
    reset_exec = run_exec = nullptr;
    for (int k = 0; k < kBatchAux; ++k) {
      if (aux[k]) cudaStreamDestroy(aux[k]);
      if (join[k]) cudaEventDestroy(join[k]);
      aux[k] = nullptr;
      join[k] = nullptr;
    }
    if (fork) cudaEventDestroy(fork);
    fork = nullptr;
    da.release();
    engine_set_free(es);
    for (inpaint_ctx* c : ctx) inpaint_destroy(c);
    ctx.clear();
    if (stream) cudaStreamSynchronize(stream);
    if (own_stream && stream) cudaStreamDestroy(stream);
    stream = nullptr;
  }
};

namespace {

// Captures one stream's work into an executable graph; false (and no graph)
// if anything in the capture fails, so callers keep the direct path.
template <typename F>
bool capture_graph(cudaStream_t st, cudaGraphExec_t* exec, F&& body) {
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const bool ok = body();
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(st, &g);
  bool done = ok && e == cudaSuccess && g && cudaGraphInstantiate(exec, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  if (!done) {
    *exec = nullptr;
    cudaGetLastError();
  }
  return done;
}

void build_batch_graphs(inpaint_batch* b) {
  for (int k = 0; k < inpaint_batch::kBatchAux; ++k)
    if (cudaStreamCreateWithFlags(&b->aux[k], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming) != cudaSuccess)
      return;
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) return;
  capture_graph(b->stream, &b->reset_exec, [&] {
    if (cudaEventRecord(b->fork, b->stream) != cudaSuccess) return false;
    for (int k = 0; k < inpaint_batch::kBatchAux; ++k)
      if (cudaStreamWaitEvent(b->aux[k], b->fork, 0) != cudaSuccess) return false;
    for (int i = 0; i < b->n; ++i) {
      inpaint_ctx* c = b->ctx[i];
      if (launch_init(c->st, c->orig_rgb, 3 * c->W, c->orig_mask, c->W, c->sat, nullptr,
                      b->aux[i % inpaint_batch::kBatchAux]) != cudaSuccess)
        return false;
    }
    for (int k = 0; k < inpaint_batch::kBatchAux; ++k)
      if (cudaEventRecord(b->join[k], b->aux[k]) != cudaSuccess ||
          cudaStreamWaitEvent(b->stream, b->join[k], 0) != cudaSuccess)
        return false;
    return true;
  });
  EngineSet& es = b->es;
  capture_graph(b->stream, &b->run_exec, [&] {
    if (cudaMemsetAsync((void*)es.ea.teams, 0, sizeof(TeamCtl) * es.n_teams, b->stream) != cudaSuccess ||
        cudaMemsetAsync(es.d_err, 0, sizeof(int), b->stream) != cudaSuccess ||
        engine_launch(es.smem, es.ea, es.grid, b->stream) != cudaSuccess ||
        cudaMemcpyAsync(es.h_pinned, es.d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
      return false;
    for (int i = 0; i < b->n; ++i)
      if (cudaMemcpyAsync(es.h_ctrls + i, b->ctx[i]->st.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost,
                          b->stream) != cudaSuccess)
        return false;
    return true;
  });
}

int batch_create_impl(const inpaint_image* images, int n, const inpaint_options* opt, inpaint_batch** out) {
  if (!out || !images || n < 1) return INPAINT_ERR_ARG;
  *out = nullptr;
  inpaint_batch* b = new (std::nothrow) inpaint_batch();
  if (!b) return INPAINT_ERR_NOMEM;
  auto fail = [&](int code) {
    b->release();
    delete b;
    return code;
  };
  inpaint_options_default(&b->opt);
  if (opt) b->opt = *opt;
  if (b->opt.search_variant != INPAINT_SEARCH_FULL) {
    g_last_error = "batches run the persistent engine: full search only";
    return fail(INPAINT_ERR_UNSUPPORTED);
  }
  if (b->opt.form != INPAINT_FORM_PLAIN) {
    g_last_error = "the batched form runs the plain search";
    return fail(INPAINT_ERR_UNSUPPORTED);
  }
  if (b->opt.cuda_stream) {
    b->stream = (cudaStream_t)b->opt.cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(INPAINT_ERR_CUDA);
    b->own_stream = true;
  }
  b->da.opt = b->opt;
  b->da.stream = b->stream;
  b->n = n;
  std::vector<double> work(n);
  for (int i = 0; i < n; ++i) {
    inpaint_ctx* c = nullptr;
    const int rc = make_member(images[i], b->opt, b->stream, i, &c);
    if (rc < 0) return fail(rc);
    b->ctx.push_back(c);
    work[i] = work_of(*c->h_ctrl);
  }
  const int rc = engine_set_prepare(b->es, b->ctx, work, b->opt, b->da, b->stream);
  if (rc < 0) return fail(rc);
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return fail(INPAINT_ERR_CUDA);
  build_batch_graphs(b);
  *out = b;
  return INPAINT_OK;
}

}  // namespace

extern "C" {

int inpaint_batch_create(const inpaint_image* images, int n, const inpaint_options* opt,
                         inpaint_batch** out) {
  try {
    return batch_create_impl(images, n, opt, out);
  } catch (...) {
    return INPAINT_ERR_NOMEM;
  }
}

int inpaint_batch_reset(inpaint_batch* b) {
  if (!b) return INPAINT_ERR_ARG;
  if (b->reset_exec) {
    CK(cudaGraphLaunch(b->reset_exec, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    return INPAINT_OK;
  }
  for (inpaint_ctx* c : b->ctx)
    CK(launch_init(c->st, c->orig_rgb, 3 * c->W, c->orig_mask, c->W, c->sat, nullptr, b->stream));
  CK(cudaStreamSynchronize(b->stream));
  return INPAINT_OK;
}

int inpaint_batch_run_ctx(inpaint_batch* b, int max_iters, int* status_out) {
  if (!b) return INPAINT_ERR_ARG;
  int rc = INPAINT_OK;
  if (max_iters <= 0 && b->run_exec) {
    // run to completion: the iteration bound of every member is unlimited
    // between calls, so the captured launch needs no per-call set-up
    CK(cudaGraphLaunch(b->run_exec, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    if (b->es.h_pinned[0]) {
      g_last_error = "a bounded device wait in the persistent engine gave up";
      rc = INPAINT_ERR_TIMEOUT;
    }
  } else {
    rc = engine_set_run(b->es, b->ctx, max_iters, b->stream);
  }
  if (status_out)
    for (int i = 0; i < b->n; ++i) {
      const Ctrl& h = b->es.h_ctrls[i];
      status_out[i] = h.status != 0 ? h.status : (h.iter == 0 && h.remaining == 0 ? INPAINT_DONE : INPAINT_OK);
    }
  return rc;
}

int inpaint_batch_result(const inpaint_batch* b, int i, uint8_t* rgb_out, int stride_bytes,
                         int* iterations, uint64_t* evals) {
  if (!b || i < 0 || i >= b->n) return INPAINT_ERR_ARG;
  const inpaint_ctx* c = b->ctx[i];
  if (rgb_out) {
    const int rc = inpaint_result(c, rgb_out, stride_bytes, nullptr);
    if (rc) return rc;
  }
  if (iterations || evals) {
    const int rc = read_ctrl(c);
    if (rc) return rc;
    if (iterations) *iterations = c->h_ctrl->iter;
    if (evals) *evals = c->h_ctrl->evals;
  }
  return INPAINT_OK;
}

int inpaint_batch_plan(const inpaint_batch* b, int* grid, int* n_teams, int* team_of_image,
                       int* team_size_of_image, int* rows_per_warp) {
  if (!b) return INPAINT_ERR_ARG;
  if (grid) *grid = b->es.grid;
  if (n_teams) *n_teams = b->es.n_teams;
  for (int i = 0; i < b->n; ++i) {
    if (team_of_image) team_of_image[i] = b->es.img_team[i];
    if (team_size_of_image) team_size_of_image[i] = b->es.team_size[b->es.img_team[i]];
    if (rows_per_warp) rows_per_warp[i] = b->ctx[i]->st.srw;
  }
  return INPAINT_OK;
}

void inpaint_batch_destroy(inpaint_batch* b) {
  if (!b) return;
  b->release();
  delete b;
}

int inpaint_batch_run(int n, const uint8_t* const* rgb, const uint8_t* const* mask, const int* w,
                      const int* h, const int* r, const inpaint_options* opt, uint8_t* const* rgb_out,
                      int* status_out) {
  if (n <= 0 || !rgb || !mask || !w || !h || !r || !rgb_out) {
    g_last_error = "inpaint_batch_run: n must be positive and every array non-null";
    return INPAINT_ERR_ARG;
  }
  std::vector<inpaint_image> ims((size_t)n);
  for (int i = 0; i < n; ++i) {
    if (!rgb[i] || !mask[i] || !rgb_out[i]) {
      g_last_error = "inpaint_batch_run: null image pointer at index " + std::to_string(i);
      return INPAINT_ERR_ARG;
    }
    ims[i] = inpaint_image{rgb[i], w[i], h[i], 3 * w[i], mask[i], w[i], r[i]};
  }
  inpaint_batch* b = nullptr;
  int rc = inpaint_batch_create(ims.data(), n, opt, &b);
  if (rc < 0) return rc;
  rc = inpaint_batch_run_ctx(b, 0, status_out);
  for (int i = 0; rc >= 0 && i < n; ++i) rc = inpaint_batch_result(b, i, rgb_out[i], 3 * w[i], nullptr, nullptr);
  inpaint_batch_destroy(b);
  return rc < 0 ? rc : INPAINT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- server

namespace {

struct SrvReq {
  uint64_t id = 0;
  int W = 0, H = 0, r = 0;
  std::vector<uint8_t> rgb, mask, out;
  double t_submit = 0, t_admit = 0, t_done = 0;
  int status = 0, iters = 0, state = 0;  // state: 0 queued, 1 active, 2 done
  uint64_t evals = 0;
  size_t bytes = 0;
  inpaint_ctx* ctx = nullptr;
};

// Upper estimate of a request's device memory (the buffers create_impl and
// the batch member copy allocate, about 48 bytes per pixel plus the trace).
size_t est_bytes(int W, int H, int n_omega) {
  return (size_t)W * H * 48 + (size_t)(n_omega + 1) * sizeof(inpaint_step_info) + (1u << 20);
}

}  // namespace

// Device time budget of one serving tick: long enough to amortise the
// launch and the host's admission work, short enough to admit new requests
// often.
constexpr unsigned long long kServerTickNs = 20000000ull;

struct inpaint_server {
  size_t budget = 0, used = 0;
  int max_slots = 0, iters_per_tick = 64, device = 0;
  inpaint_options opt{};
  cudaStream_t stream = nullptr;
  DevAlloc da;
  EngineSet es;
  std::mutex mu;
  std::condition_variable cv, cv_idle;
  std::deque<SrvReq*> queue;
  std::vector<SrvReq*> active;
  std::unordered_map<uint64_t, SrvReq*> reqs;
  uint64_t next_id = 1;
  int admitting = 0;  // popped from the queue, not yet active or retired
  bool stop = false;
  std::thread worker;
  std::chrono::steady_clock::time_point t0;
  inpaint_server_stats st{};

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }

  void retire(SrvReq* q, int status) {
    if (q->ctx) {
      if (status >= 0) {
        q->out.resize((size_t)q->W * q->H * 3);
        if (inpaint_result(q->ctx, q->out.data(), 3 * q->W, nullptr) != INPAINT_OK) status = INPAINT_ERR_CUDA;
      }
      inpaint_destroy(q->ctx);
      q->ctx = nullptr;
    }
    q->status = status;
    q->t_done = now();
  }

  void loop() {
    cudaSetDevice(device);
    while (true) {
      std::vector<SrvReq*> admit;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] { return stop || !queue.empty() || !active.empty(); });
        if (stop) return;
        while (!queue.empty() && (int)(active.size() + admit.size()) < max_slots) {
          SrvReq* q = queue.front();
          int n_omega = 0;
          for (uint8_t m : q->mask) n_omega += m != 0;
          const size_t b = est_bytes(q->W, q->H, n_omega);
          if (used + b > budget && !(active.empty() && admit.empty())) break;
          queue.pop_front();
          q->bytes = b;
          used += b;
          admit.push_back(q);
        }
        admitting = (int)admit.size();
      }
      const auto tb = std::chrono::steady_clock::now();
      std::vector<SrvReq*> failed;
      for (SrvReq* q : admit) {
        inpaint_image im{q->rgb.data(), q->W, q->H, 3 * q->W, q->mask.data(), q->W, q->r};
        inpaint_ctx* c = nullptr;
        const int rc = make_member(im, opt, stream, (int)q->id, &c);
        q->t_admit = now();
        if (rc < 0) {
          retire(q, rc);
          failed.push_back(q);
        } else {
          q->ctx = c;
          q->rgb.clear();
          q->rgb.shrink_to_fit();
          q->mask.clear();
          q->mask.shrink_to_fit();
        }
      }
      std::vector<SrvReq*> act;
      {
        std::lock_guard<std::mutex> lk(mu);
        admitting = 0;
        for (SrvReq* q : admit)
          if (q->ctx) {
            q->state = 1;
            active.push_back(q);
            st.admitted++;
          }
        for (SrvReq* q : failed) {
          q->state = 2;
          used -= q->bytes;
          st.failed++;
        }
        act = active;
      }
      std::vector<SrvReq*> done;
      if (!act.empty()) {
        std::vector<inpaint_ctx*> cs;
        std::vector<double> work;
        for (SrvReq* q : act) {
          cs.push_back(q->ctx);
          work.push_back(work_of(*q->ctx->h_ctrl));
        }
        int rc = engine_set_prepare(es, cs, work, opt, da, stream);
        if (rc >= 0) rc = engine_set_run(es, cs, iters_per_tick, stream, kServerTickNs);
        for (size_t i = 0; i < act.size(); ++i) {
          const Ctrl& h = rc >= 0 ? es.h_ctrls[i] : *act[i]->ctx->h_ctrl;
          *act[i]->ctx->h_ctrl = h;  // mirror for the next work estimate
          if (rc < 0 || h.status != 0 || h.remaining == 0) {
            act[i]->iters = h.iter;
            act[i]->evals = h.evals;
            retire(act[i], rc < 0 ? rc : (h.status != 0 ? h.status : INPAINT_OK));
            done.push_back(act[i]);
          }
        }
      }
      std::lock_guard<std::mutex> lk(mu);
      st.ticks++;
      st.busy_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - tb).count();
      for (SrvReq* q : done) {
        q->state = 2;
        used -= q->bytes;
        if (q->status < 0) st.failed++; else st.completed++;
        active.erase(std::find(active.begin(), active.end(), q));
      }
      if (idle()) cv_idle.notify_all();
    }
  }

  bool idle() const { return queue.empty() && active.empty() && admitting == 0; }
};

extern "C" {

int inpaint_server_create(size_t hbm_budget_bytes, int max_slots, int iters_per_tick,
                          const inpaint_options* opt, inpaint_server** out) {
  if (!out || hbm_budget_bytes == 0 || max_slots < 1) return INPAINT_ERR_ARG;
  *out = nullptr;
  inpaint_server* s = new (std::nothrow) inpaint_server();
  if (!s) return INPAINT_ERR_NOMEM;
  inpaint_options_default(&s->opt);
  if (opt) s->opt = *opt;
  if (s->opt.search_variant != INPAINT_SEARCH_FULL) {
    delete s;
    g_last_error = "the server runs the persistent engine: full search only";
    return INPAINT_ERR_UNSUPPORTED;
  }
  s->opt.form = INPAINT_FORM_PLAIN;
  s->budget = hbm_budget_bytes;
  s->max_slots = max_slots;
  s->iters_per_tick = iters_per_tick > 0 ? iters_per_tick : 0;
  if (cudaGetDevice(&s->device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete s;
    return INPAINT_ERR_CUDA;
  }
  s->opt.cuda_stream = (void*)s->stream;
  s->da.opt = s->opt;
  s->da.stream = s->stream;
  s->t0 = std::chrono::steady_clock::now();
  s->st.hbm_budget = hbm_budget_bytes;
  try {
    s->worker = std::thread([s] { s->loop(); });
  } catch (...) {
    cudaStreamDestroy(s->stream);
    delete s;
    return INPAINT_ERR_NOMEM;
  }
  *out = s;
  return INPAINT_OK;
}

int inpaint_server_submit(inpaint_server* s, const inpaint_image* img, uint64_t* id) {
  if (!s || !img || !img->rgb || !img->mask || img->patch_radius < 1 || img->patch_radius > 8 ||
      img->rgb_stride_bytes < 3 * img->width || img->mask_stride_bytes < img->width)
    return INPAINT_ERR_ARG;
  if (check_geometry(img->width, img->height, img->patch_radius)) return INPAINT_ERR_ARG;
  SrvReq* q = new (std::nothrow) SrvReq();
  if (!q) return INPAINT_ERR_NOMEM;
  q->W = img->width;
  q->H = img->height;
  q->r = img->patch_radius;
  q->rgb.resize((size_t)q->W * q->H * 3);
  q->mask.resize((size_t)q->W * q->H);
  for (int y = 0; y < q->H; ++y) {
    memcpy(&q->rgb[(size_t)y * 3 * q->W], img->rgb + (size_t)y * img->rgb_stride_bytes, 3 * (size_t)q->W);
    memcpy(&q->mask[(size_t)y * q->W], img->mask + (size_t)y * img->mask_stride_bytes, (size_t)q->W);
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    q->id = s->next_id++;
    q->t_submit = s->now();
    s->reqs[q->id] = q;
    s->queue.push_back(q);
    s->st.submitted++;
  }
  s->cv.notify_one();
  if (id) *id = q->id;
  return INPAINT_OK;
}

int inpaint_server_poll(inpaint_server* s, uint64_t id, uint8_t* rgb_out, int stride_bytes,
                        inpaint_request_info* info) {
  if (!s) return INPAINT_ERR_ARG;
  SrvReq* q = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return INPAINT_ERR_ARG;
    if (it->second->state != 2) return INPAINT_PENDING;
    q = it->second;
    s->reqs.erase(it);
  }
  if (rgb_out && !q->out.empty())
    for (int y = 0; y < q->H; ++y)
      memcpy(rgb_out + (size_t)y * stride_bytes, &q->out[(size_t)y * 3 * q->W], 3 * (size_t)q->W);
  if (info) {
    info->t_submit = q->t_submit;
    info->t_admit = q->t_admit;
    info->t_done = q->t_done;
    info->status = q->status;
    info->iterations = q->iters;
    info->evals = q->evals;
    info->width = q->W;
    info->height = q->H;
  }
  delete q;
  return INPAINT_OK;
}

int inpaint_server_wait_idle(inpaint_server* s, double timeout_s) {
  if (!s) return INPAINT_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  const bool ok = s->cv_idle.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                      [&] { return s->idle(); });
  return ok ? INPAINT_OK : INPAINT_ERR_TIMEOUT;
}

int inpaint_server_stats_get(inpaint_server* s, inpaint_server_stats* out) {
  if (!s || !out) return INPAINT_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  out->queued = (int)s->queue.size();
  out->active = (int)s->active.size();
  out->hbm_used = s->used;
  out->hbm_budget = s->budget;
  return INPAINT_OK;
}

double inpaint_server_clock(const inpaint_server* s) { return s ? s->now() : 0.0; }

void inpaint_server_destroy(inpaint_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->device);
  for (SrvReq* q : s->active) {
    if (q->ctx) inpaint_destroy(q->ctx);
    q->ctx = nullptr;
  }
  for (auto& kv : s->reqs) {
    if (kv.second->ctx) inpaint_destroy(kv.second->ctx);
    delete kv.second;
  }
  cudaStreamSynchronize(s->stream);
  s->da.release();
  engine_set_free(s->es);
  cudaStreamSynchronize(s->stream);
  cudaStreamDestroy(s->stream);
  delete s;
}

}  // extern "C"
