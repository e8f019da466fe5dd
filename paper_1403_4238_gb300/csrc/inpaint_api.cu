// C-ABI of libinpaint: context lifetime, the iteration loop and host I/O.
//
// The three stages of Sec. 4.2 (initialisation, iterative computation,
// finalisation) map to inpaint_create/inpaint_reset, inpaint_step/inpaint_run
// and inpaint_result.  inpaint_run drives the whole iterative stage from the
// device: one CUDA graph whose conditional while-node repeats
// [findBestPatch search -> copy/update + next selection] until the update
// kernel reports an empty Omega, so no host round trip happens per iteration.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
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

  void* dalloc(size_t bytes) {
    void* p = nullptr;
    if (opt.dev_alloc) {
      p = opt.dev_alloc(bytes, (void*)stream, opt.alloc_user);
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

void search_rect(const uint8_t* mask, int mstride, int W, int H, int r, double alpha,
                 int* x0o, int* x1o, int* y0o, int* y1o) {
  int lo_x = r, hi_x = W - 1 - r, lo_y = r, hi_y = H - 1 - r;
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
  CK(launch_search_plain(c->st, c->stream));
  if (c->r <= 8)
    CK(launch_update_fast(c->st, c->cond, use_cond, c->stream));
  else
    CK(launch_update(c->st, 1, c->cond, use_cond, c->stream));
  if (c->opt.debug_checks) CK(launch_verify_count(c->st, c->stream));
  return INPAINT_OK;
}

bool use_engine(const inpaint_ctx* c) {
  if (c->opt.loop_mode == INPAINT_LOOP_GRAPH) return false;
  return c->r <= 8;
}

// Rows per warp from an autotuner table: lines "radius max_pixels rows";
// the first line with this radius and max_pixels >= W*H wins; 0 if none.
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

// Candidate rows per warp in a search batch (a batch is 16 warps x rows x
// 128 columns): 2 when every CTA still gets about two batches, else 1.
int pick_rows_per_warp(const ImgState& s, int grid) {
  const int xb = s.r + ((s.cx0 - s.r) & ~3);
  const long long ncg = (s.cx1 - xb + 128) / 128, ch = s.cy1 - s.cy0 + 1;
  return ncg * ((ch + 2 * kEngWarps - 1) / (2 * kEngWarps)) >= 2ll * grid ? 2 : 1;
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
  CK(engine_occupancy(f->smem_bytes(2), &bps));
  if (bps < 1) {
    g_last_error = "engine kernel does not fit on an SM";
    return INPAINT_ERR_UNSUPPORTED;
  }
  const int grid = sms * bps;
  if (!sr) sr = tuned_rows_per_warp(c->opt.tuning_file, c->r, (long long)c->W * c->H);
  if (!sr) sr = pick_rows_per_warp(c->st, grid);
  c->eng_smem = f->smem_bytes(sr);
  CK(engine_occupancy(c->eng_smem, &bps));
  const int g2 = sms * (bps < 1 ? 1 : bps);
  c->eng_grid = g2 < grid ? g2 : grid;
  c->eng_sr = sr;
  c->st.srw = sr;
  if (!alloc_n(c, c->d_img, 1) || !alloc_n(c, c->d_tmap, 1) ||
      !alloc_n(c, c->d_ints, (size_t)c->eng_grid + 5) || !alloc_n(c, c->d_team, 1) ||
      !alloc_n(c, c->d_epart, (size_t)c->eng_grid) || !alloc_n(c, c->d_err, 1))
    return INPAINT_ERR_NOMEM;
  if (!c->h_err && cudaMallocHost(&c->h_err, sizeof(int)) != cudaSuccess) return INPAINT_ERR_NOMEM;
  CUtensorMap tm;
  if (make_image_tmap(c->st, sr, &tm) != 0) {
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
  CK(cudaMemcpyAsync(c->d_tmap, &tm, sizeof(CUtensorMap), cudaMemcpyHostToDevice, c->stream));
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
  c->eng_ready = true;
  return INPAINT_OK;
}

int run_engine(inpaint_ctx* c) {
  int rc = setup_engine(c);
  if (rc) return rc;
  CK(cudaMemsetAsync(c->d_team, 0, sizeof(TeamCtl), c->stream));
  CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
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
  if (o.form == INPAINT_FORM_TC) {
    g_last_error = "tensor-core form not built yet";
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
  search_rect(mask, mask_stride, W, H, r, o.search_alpha, &s.cx0, &s.cx1, &s.cy0, &s.cy1);
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
  const size_t n = (size_t)W * H;
  if (!alloc_n(c, s.img, (size_t)s.pitch * H) || !alloc_n(c, s.omega, n) || !alloc_n(c, s.gray, n) ||
      !alloc_n(c, s.conf, n) || !alloc_n(c, s.count, n) || !alloc_n(c, s.prio, n) ||
      !alloc_n(c, s.pconf, n) || !alloc_n(c, s.tiles0, (size_t)s.t0x * s.t0y) ||
      !alloc_n(c, s.tiles1, (size_t)s.t1x * s.t1y) ||
      !alloc_n(c, s.ctrl, 1) || !alloc_n(c, s.trace, (size_t)s.trace_cap) ||
      !alloc_n(c, s.partial, (size_t)(s.n_partial > 0 ? s.n_partial : 1)) ||
      !alloc_n(c, c->sat, (size_t)(W + 1) * (H + 1) + (size_t)sat_chunks(H) * W) || !alloc_n(c, c->rgb_stage, 3 * n) ||
      !alloc_n(c, c->mask_stage, n) || !alloc_n(c, s.spec, 1)) {
    g_last_error = "device allocation failed";
    return fail(INPAINT_ERR_NOMEM);
  }
  if (prepare_search_plain(r) != cudaSuccess) return fail(INPAINT_ERR_CUDA);
  {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || !(s.dtab = data_term_table(dev)))
      return fail(INPAINT_ERR_CUDA);
  }
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

// Per-device table of the data term D = (dot / sqrt(nn)) / 510 (Eq. 2 with
// alpha = 255 and the factor 2 of the central difference), evaluated with
// the same IEEE double operations the kernels would use (sqrt and division
// are correctly rounded on host and device alike).  Built once per device
// and kept for the life of the process.
const double* inp::data_term_table(int device) {
  static std::mutex mu;
  static std::map<int, double*> tabs;
  std::lock_guard<std::mutex> lk(mu);
  auto it = tabs.find(device);
  if (it != tabs.end()) return it->second;
  std::vector<double> h((size_t)kDTabRows * kDTabCols);
  for (int r = 0; r < kDTabRows; ++r) {
    const double root = std::sqrt((double)kDTabNN[r]);
    for (int dot = 0; dot < kDTabCols; ++dot) h[(size_t)r * kDTabCols + dot] = ((double)dot / root) / 510.0;
  }
  double* d = nullptr;
  if (cudaMalloc(&d, h.size() * sizeof(double)) != cudaSuccess) return nullptr;
  if (cudaMemcpy(d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(d);
    return nullptr;
  }
  tabs[device] = d;
  return d;
}

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


// ---------------------------------------------------------------- batch

struct inpaint_batch {
  int n = 0;
  inpaint_options opt{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<inpaint_ctx*> ctx;
  int grid = 0, n_teams = 0;
  size_t smem = 0;
  std::vector<int> img_team, team_size;
  std::vector<std::pair<void*, size_t>> allocs;
  EngineArgs ea{};
  int* d_err = nullptr;
  TeamCtl* d_teams = nullptr;
  int* h_pinned = nullptr;  // [0] err, [1..n] iteration limits
  Ctrl* h_ctrls = nullptr;  // n mirrors

  void* dalloc(size_t bytes) {
    void* p = nullptr;
    if (opt.dev_alloc)
      p = opt.dev_alloc(bytes, (void*)stream, opt.alloc_user);
    else if (cudaMallocAsync(&p, bytes, stream) != cudaSuccess)
      p = nullptr;
    if (p) allocs.emplace_back(p, bytes);
    return p;
  }
  void release() {
    if (stream) cudaStreamSynchronize(stream);
    for (auto& a : allocs) {
      if (opt.dev_free)
        opt.dev_free(a.first, a.second, (void*)stream, opt.alloc_user);
      else
        cudaFreeAsync(a.first, stream);
    }
    allocs.clear();
    for (inpaint_ctx* c : ctx) inpaint_destroy(c);
    ctx.clear();
    if (stream) cudaStreamSynchronize(stream);
    if (h_pinned) cudaFreeHost(h_pinned);
    if (h_ctrls) cudaFreeHost(h_ctrls);
    h_pinned = nullptr;
    h_ctrls = nullptr;
    if (own_stream && stream) cudaStreamDestroy(stream);
    stream = nullptr;
  }
};

namespace {

template <class T>
bool balloc(inpaint_batch* b, T*& p, size_t n) {
  p = static_cast<T*>(b->dalloc(n * sizeof(T)));
  return p != nullptr;
}

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
  double total = 0.0;
  for (double w : work) total += w;
  const int extra = grid - n;
  team_size.assign(n, 1);
  team_imgs.assign(n, {});
  std::vector<std::pair<double, int>> rem;
  int used = 0;
  for (int i = 0; i < n; ++i) {
    const double share = total > 0 ? extra * work[i] / total : (double)extra / n;
    const int k = (int)share;
    team_size[i] += k;
    used += k;
    rem.emplace_back(share - k, i);
  }
  std::sort(rem.begin(), rem.end(), [](const std::pair<double, int>& a, const std::pair<double, int>& b) {
    return a.first > b.first;
  });
  for (int k = 0; k < extra - used; ++k) team_size[rem[k % n].second] += 1;
  for (int i = 0; i < n; ++i) {
    img_team[i] = i;
    team_imgs[i].push_back(i);
  }
}

int batch_create_impl(const inpaint_image* images, int n, const inpaint_options* opt,
                      inpaint_batch** out) {
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
  if (b->opt.form != INPAINT_FORM_PLAIN) {
    g_last_error = "the batched form runs the plain search";
    return fail(INPAINT_ERR_UNSUPPORTED);
  }
  if (b->opt.cuda_stream) {
    b->stream = (cudaStream_t)b->opt.cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess)
      return fail(INPAINT_ERR_CUDA);
    b->own_stream = true;
  }
  b->n = n;
  inpaint_options o = b->opt;
  o.cuda_stream = (void*)b->stream;
  o.loop_mode = INPAINT_LOOP_ENGINE;
  for (int i = 0; i < n; ++i) {
    const inpaint_image& im = images[i];
    if (im.patch_radius < 1 || im.patch_radius > 8) {
      char buf[128];
      snprintf(buf, sizeof buf, "batch image %d: patch radius must be 1..8", i);
      g_last_error = buf;
      return fail(INPAINT_ERR_ARG);
    }
    inpaint_ctx* c = nullptr;
    const int rc = create_impl(im.rgb, im.width, im.height, im.rgb_stride_bytes, im.mask,
                               im.mask_stride_bytes, im.patch_radius, &o, &c);
    if (rc < 0) {
      char buf[160];
      snprintf(buf, sizeof buf, "batch image %d: %s", i, g_last_error.c_str());
      g_last_error = buf;
      return fail(rc);
    }
    b->ctx.push_back(c);
    const size_t px = (size_t)im.width * im.height;
    if (!alloc_n(c, c->orig_rgb, 3 * px) || !alloc_n(c, c->orig_mask, px)) return fail(INPAINT_ERR_NOMEM);
    if (cudaMemcpyAsync(c->orig_rgb, c->rgb_stage, 3 * px, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess ||
        cudaMemcpyAsync(c->orig_mask, c->mask_stage, px, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess)
      return fail(INPAINT_ERR_CUDA);
  }
  // grid and teams
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail(INPAINT_ERR_CUDA);
  size_t smem_max = 0;
  for (inpaint_ctx* c : b->ctx) smem_max = std::max(smem_max, engine_fns(c->r)->smem_bytes(2));
  int bps = 0;
  if (engine_occupancy(smem_max, &bps) != cudaSuccess || bps < 1) return fail(INPAINT_ERR_UNSUPPORTED);
  b->grid = sms * bps;
  std::vector<double> work(n);
  for (int i = 0; i < n; ++i)
    work[i] = (double)std::max(1, b->ctx[i]->h_ctrl->remaining) * std::max(1, b->ctx[i]->h_ctrl->n_valid);
  std::vector<std::vector<int>> team_imgs;
  std::vector<int> tsz;
  plan_teams(work, b->grid, tsz, b->img_team, team_imgs);
  b->n_teams = (int)tsz.size();
  b->team_size = tsz;
  // per-image search rows, tensor maps, device copies of the states
  std::vector<ImgState> imgs(n);
  std::vector<CUtensorMap> maps(n);
  b->smem = 0;
  for (int i = 0; i < n; ++i) {
    inpaint_ctx* c = b->ctx[i];
    int sr = b->opt.tile_rows;
    if (!sr) sr = tuned_rows_per_warp(b->opt.tuning_file, c->r, (long long)c->W * c->H);
    if (!sr) sr = pick_rows_per_warp(c->st, tsz[b->img_team[i]]);
    c->st.srw = sr;
    imgs[i] = c->st;
    if (make_image_tmap(c->st, sr, &maps[i]) != 0) {
      g_last_error = "cuTensorMapEncodeTiled failed";
      return fail(INPAINT_ERR_CUDA);
    }
    b->smem = std::max(b->smem, engine_fns(c->r)->smem_bytes(sr));
  }
  std::vector<int> ints;
  const int G = b->grid, T = b->n_teams;
  std::vector<int> first(T + 1, 0), off(T + 1, 0), lst;
  for (int t = 0; t < T; ++t) {
    first[t + 1] = first[t] + tsz[t];
    off[t + 1] = off[t] + (int)team_imgs[t].size();
    for (int i : team_imgs[t]) lst.push_back(i);
  }
  ints.resize((size_t)G);
  for (int t = 0; t < T; ++t)
    for (int k = first[t]; k < first[t + 1]; ++k) ints[k] = t;
  const size_t o_first = ints.size();
  ints.insert(ints.end(), first.begin(), first.end());
  const size_t o_off = ints.size();
  ints.insert(ints.end(), off.begin(), off.end());
  const size_t o_lst = ints.size();
  ints.insert(ints.end(), lst.begin(), lst.end());
  ImgState* d_imgs = nullptr;
  CUtensorMap* d_maps = nullptr;
  int* d_ints = nullptr;
  unsigned long long* d_part = nullptr;
  if (!balloc(b, d_imgs, n) || !balloc(b, d_maps, n) || !balloc(b, d_ints, ints.size()) ||
      !balloc(b, b->d_teams, T) || !balloc(b, d_part, G) || !balloc(b, b->d_err, 1))
    return fail(INPAINT_ERR_NOMEM);
  if (cudaMallocHost(&b->h_pinned, sizeof(int) * (n + 1)) != cudaSuccess ||
      cudaMallocHost(&b->h_ctrls, sizeof(Ctrl) * n) != cudaSuccess)
    return fail(INPAINT_ERR_NOMEM);
  if (cudaMemcpyAsync(d_imgs, imgs.data(), sizeof(ImgState) * n, cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
      cudaMemcpyAsync(d_maps, maps.data(), sizeof(CUtensorMap) * n, cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
      cudaMemcpyAsync(d_ints, ints.data(), sizeof(int) * ints.size(), cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return fail(INPAINT_ERR_CUDA);
  EngineArgs& ea = b->ea;
  ea.imgs = d_imgs;
  ea.tmaps = d_maps;
  ea.cta_team = d_ints;
  ea.team_first = d_ints + o_first;
  ea.team_img_off = d_ints + o_off;
  ea.team_img = d_ints + o_lst;
  ea.teams = b->d_teams;
  ea.partials = d_part;
  ea.err = b->d_err;
  ea.wait_limit_ns = 4000000000ull;
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
  for (inpaint_ctx* c : b->ctx)
    CK(launch_init(c->st, c->orig_rgb, 3 * c->W, c->orig_mask, c->W, c->sat, nullptr, b->stream));
  CK(cudaStreamSynchronize(b->stream));
  return INPAINT_OK;
}

int inpaint_batch_run(inpaint_batch* b, int max_iters, int* status_out) {
  if (!b) return INPAINT_ERR_ARG;
  const int n = b->n;
  for (int i = 0; i < n; ++i)
    CK(cudaMemcpyAsync(b->h_ctrls + i, b->ctx[i]->st.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, b->stream));
  CK(cudaStreamSynchronize(b->stream));
  for (int i = 0; i < n; ++i) {
    const Ctrl& h = b->h_ctrls[i];
    long long lim = (long long)h.iter + std::max(h.remaining, 0);
    if (max_iters > 0 && (long long)h.iter + max_iters < lim) lim = (long long)h.iter + max_iters;
    b->h_pinned[1 + i] = (int)std::min<long long>(lim, INT_MAX);
    CK(cudaMemcpyAsync(&b->ctx[i]->st.ctrl->iter_limit, &b->h_pinned[1 + i], sizeof(int),
                       cudaMemcpyHostToDevice, b->stream));
  }
  CK(cudaMemsetAsync(b->d_teams, 0, sizeof(TeamCtl) * b->n_teams, b->stream));
  CK(cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream));
  CK(engine_launch(b->smem, b->ea, b->grid, b->stream));
  CK(cudaMemcpyAsync(b->h_pinned, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  for (int i = 0; i < n; ++i)
    CK(cudaMemcpyAsync(b->h_ctrls + i, b->ctx[i]->st.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, b->stream));
  CK(cudaStreamSynchronize(b->stream));
  for (int i = 0; i < n; ++i) {
    // restore the unlimited iteration bound for later calls
    b->h_pinned[1 + i] = INT_MAX;
    CK(cudaMemcpyAsync(&b->ctx[i]->st.ctrl->iter_limit, &b->h_pinned[1 + i], sizeof(int),
                       cudaMemcpyHostToDevice, b->stream));
  }
  CK(cudaStreamSynchronize(b->stream));
  if (status_out)
    for (int i = 0; i < n; ++i) {
      const Ctrl& h = b->h_ctrls[i];
      status_out[i] = h.status != 0 ? h.status : (h.iter == 0 && h.remaining == 0 ? INPAINT_DONE : INPAINT_OK);
    }
  if (b->h_pinned[0]) {
    g_last_error = "a bounded device wait in the persistent engine gave up";
    return INPAINT_ERR_TIMEOUT;
  }
  return INPAINT_OK;
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
  if (grid) *grid = b->grid;
  if (n_teams) *n_teams = b->n_teams;
  for (int i = 0; i < b->n; ++i) {
    if (team_of_image) team_of_image[i] = b->img_team[i];
    if (team_size_of_image) team_size_of_image[i] = b->team_size[b->img_team[i]];
    if (rows_per_warp) rows_per_warp[i] = b->ctx[i]->st.srw;
  }
  return INPAINT_OK;
}

void inpaint_batch_destroy(inpaint_batch* b) {
  if (!b) return;
  b->release();
  delete b;
}

}  // extern "C"
