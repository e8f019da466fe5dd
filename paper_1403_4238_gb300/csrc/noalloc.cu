// findBestPatch for one target patch, with no device allocation.
//
// The paper has no counterpart to this entry point.  It exists for callers
// that cannot call cudaMalloc: a serving process whose device memory is
// reserved up front by another framework's allocator, code that runs while
// a CUDA stream is being captured into a graph whose memory plan is fixed, or
// a real-time loop that forbids allocation after start-up.  Those callers
// hand in device pointers to their own inputs and output; the only scratch
// memory the search needs -- one partial key per CTA and a ticket counter --
// lives in file-scope __device__ arrays of a fixed maximum size, which every
// GPU that loads this library holds until the process exits.
//
// The search is the library's (Sec. 3, Eq. 3-4): over every candidate centre
// whose patch lies inside the image and is fully known, the SSD over the
// known in-image pixels of the target patch; the result is the packed key
// (SSD << 32 | linear index), lowest SSD then lowest index.
#include <mutex>

#include "inpaint_internal.cuh"

namespace {

using inp::block_min_u64;
using inp::pack_rgb;

constexpr int kNaTW = 128;  // candidate columns per CTA
constexpr int kNaTH = 8;    // candidate rows per CTA
constexpr int kNaThreads = 256;
constexpr int kNaMaxR = 8;
constexpr int kNaMaxP = 2 * kNaMaxR + 1;
// Scratch capacity: one partial key per CTA.  4096 tiles of 8 x 128
// candidates cover an interior of up to 4.19 million candidate centres
// (a 4096 x 1024 image, or 2048 x 2048).
constexpr int kNaMaxCtas = 4096;

static __device__ __align__(256) unsigned long long g_na_partial[kNaMaxCtas];
static __device__ __align__(256) unsigned int g_na_ticket[64];

struct NaScratch {
  unsigned long long* partial = nullptr;
  unsigned int* ticket = nullptr;
};

// Set-up once per device (with that device current): the host-side names of
// the arrays are stand-ins, so the kernel gets their device addresses.
int scratch_for_current_device(NaScratch* out) {
  static std::mutex mu;
  static NaScratch table[64];
  static bool ready[64] = {false};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return INPAINT_ERR_CUDA;
  std::lock_guard<std::mutex> lk(mu);
  if (!ready[dev]) {
    NaScratch s;
    if (cudaGetSymbolAddress((void**)&s.partial, g_na_partial) != cudaSuccess) return INPAINT_ERR_CUDA;
    if (cudaGetSymbolAddress((void**)&s.ticket, g_na_ticket) != cudaSuccess) return INPAINT_ERR_CUDA;
    table[dev] = s;
    ready[dev] = true;
  }
  *out = table[dev];
  return INPAINT_OK;
}

__global__ void __launch_bounds__(kNaThreads) k_search_noalloc(const uint8_t* __restrict__ rgb,
                                                              const uint8_t* __restrict__ mask, int W,
                                                              int H, int r, int px, int py,
                                                              unsigned long long* partial,
                                                              unsigned int* ticket,
                                                              unsigned long long* out) {
  const int P = 2 * r + 1;
  const int SW = kNaTW + 2 * r, SH = kNaTH + 2 * r;
  __shared__ uint32_t src[(kNaTH + 2 * kNaMaxR) * (kNaTW + 2 * kNaMaxR)];
  __shared__ uint8_t unk[(kNaTH + 2 * kNaMaxR) * (kNaTW + 2 * kNaMaxR)];
  __shared__ uint16_t colsum[kNaTH * (kNaTW + 2 * kNaMaxR)];
  __shared__ uint32_t koff[kNaMaxP * kNaMaxP], kval[kNaMaxP * kNaMaxP];
  __shared__ unsigned long long red[32];
  __shared__ int nk_s;
  __shared__ bool last_s;
  const int tid = threadIdx.x;
  const int ox = r + blockIdx.x * kNaTW, oy = r + blockIdx.y * kNaTH;  // first candidate of the tile

  // known in-image target pixels (compacted), source tile with unknown flags
  if (tid == 0) {
    int n = 0;
    for (int dy = 0; dy < P; ++dy)
      for (int dx = 0; dx < P; ++dx) {
        const int tx = px + dx - r, ty = py + dy - r;
        if (tx >= 0 && tx < W && ty >= 0 && ty < H && mask[(size_t)ty * W + tx] == 0) {
          const uint8_t* p = rgb + 3 * ((size_t)ty * W + tx);
          koff[n] = dy * SW + dx;
          kval[n] = pack_rgb(p[0], p[1], p[2]);
          ++n;
        }
      }
    nk_s = n;
  }
  for (int i = tid; i < SH * SW; i += blockDim.x) {
    const int xx = ox - r + i % SW, yy = oy - r + i / SW;
    uint32_t w = 0;
    uint8_t u = 1;
    if (xx < W && yy < H) {
      const uint8_t* p = rgb + 3 * ((size_t)yy * W + xx);
      w = pack_rgb(p[0], p[1], p[2]);
      u = mask[(size_t)yy * W + xx] != 0;
    }
    src[i] = w;
    unk[i] = u;
  }
  __syncthreads();
  // unknown pixels per candidate patch: column sums over P rows, then row sums
  for (int i = tid; i < kNaTH * SW; i += blockDim.x) {
    const int row = i / SW, col = i % SW;
    int sacc = 0;
    for (int dy = 0; dy < P; ++dy) sacc += unk[(row + dy) * SW + col];
    colsum[i] = (uint16_t)sacc;
  }
  __syncthreads();

  unsigned long long best = ~0ull;
  const int nk = nk_s;
  for (int c = tid; c < kNaTH * kNaTW; c += blockDim.x) {
    const int row = c / kNaTW, col = c % kNaTW;
    const int qx = ox + col, qy = oy + row;
    if (qx > W - 1 - r || qy > H - 1 - r) continue;
    int cnt = 0;
    for (int dx = 0; dx < P; ++dx) cnt += colsum[row * SW + col + dx];
    if (cnt) continue;
    uint32_t acc = 0;
    const uint32_t* base = src + row * SW + col;
    for (int k = 0; k < nk; ++k) {
      const uint32_t d = __vabsdiffu4(kval[k], base[koff[k]]);
      acc = __dp4a(d, d, acc);
    }
    const unsigned long long key = ((unsigned long long)acc << 32) | (unsigned)(qy * W + qx);
    best = key < best ? key : best;
  }
  best = block_min_u64(best, red);

  // per-CTA partial into the static scratch; the last CTA reduces them
  const unsigned nblocks = gridDim.x * gridDim.y;
  if (tid == 0) {
    partial[blockIdx.y * gridDim.x + blockIdx.x] = best;
    __threadfence();
    last_s = atomicAdd(ticket, 1u) == nblocks - 1u;
  }
  __syncthreads();
  if (last_s) {
    __threadfence();
    unsigned long long b = ~0ull;
    for (unsigned i = tid; i < nblocks; i += blockDim.x) {
      const unsigned long long v = __ldcg(&partial[i]);
      b = v < b ? v : b;
    }
    b = block_min_u64(b, red);
    if (tid == 0) {
      *out = b;
      *ticket = 0u;  // leave the counter at zero for the next call
    }
  }
}

}  // namespace

extern "C" int inpaint_best_patch_noalloc(const uint8_t* d_rgb, const uint8_t* d_mask, int width,
                                          int height, int patch_radius, int px, int py,
                                          uint64_t* d_best_key, void* cuda_stream) {
  const int r = patch_radius, W = width, H = height;
  if (!d_rgb || !d_mask || !d_best_key || r < 1 || r > kNaMaxR || W < 2 * r + 1 ||
      H < 2 * r + 1 || px < 0 || px >= W || py < 0 || py >= H) {
    inp::set_last_error("inpaint_best_patch_noalloc: null pointer, radius outside 1..8, image "
                        "smaller than a patch, or target outside the image");
    return INPAINT_ERR_ARG;
  }
  const int gx = (W - 2 * r + kNaTW - 1) / kNaTW, gy = (H - 2 * r + kNaTH - 1) / kNaTH;
  if ((long long)gx * gy > kNaMaxCtas) {
    inp::set_last_error(
        "inpaint_best_patch_noalloc: image too large for the fixed scratch (at most 4096 tiles of "
        "8 x 128 candidate centres, e.g. 4096 x 1024 or 2048 x 2048 pixels)");
    return INPAINT_ERR_ARG;
  }
  NaScratch sc;
  const int rc = scratch_for_current_device(&sc);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // the ticket must start at zero even if an earlier call was interrupted
  if (cudaMemsetAsync(sc.ticket, 0, sizeof(unsigned int), st) != cudaSuccess) return INPAINT_ERR_CUDA;
  k_search_noalloc<<<dim3(gx, gy), kNaThreads, 0, st>>>(d_rgb, d_mask, W, H, r, px, py, sc.partial,
                                                       sc.ticket,
                                                       reinterpret_cast<unsigned long long*>(d_best_key));
  return cudaGetLastError() == cudaSuccess ? INPAINT_OK : INPAINT_ERR_CUDA;
}
