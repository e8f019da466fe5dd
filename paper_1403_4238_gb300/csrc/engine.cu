// Dispatch of the persistent engine by patch radius, the TMA descriptor of
// an image and the planes of its tensor-core form (the kernels themselves
// are in engine_impl.cuh, instantiated per radius in engine_r<R>.cu).
#include <cuda.h>
#include <cudaTypedefs.h>

#include "inpaint_engine.h"

namespace inp {

const EngineFns* engine_fns(int r) {
  switch (r) {
    case 1: return engine_fns_r1();
    case 2: return engine_fns_r2();
    case 3: return engine_fns_r3();
    case 4: return engine_fns_r4();
    case 5: return engine_fns_r5();
    case 6: return engine_fns_r6();
    case 7: return engine_fns_r7();
    case 8: return engine_fns_r8();
    default: return nullptr;
  }
}

cudaError_t launch_update_fast(const ImgState& s, unsigned long long cond, int use_cond,
                               cudaStream_t st) {
  const EngineFns* f = engine_fns(s.r);
  return f ? f->update_fast(s, cond, use_cond, st) : cudaErrorInvalidValue;
}

cudaError_t launch_prio_init_fast(const ImgState& s, cudaStream_t st) {
  const EngineFns* f = engine_fns(s.r);
  return f ? f->prio_init(s, st) : cudaErrorInvalidValue;
}

// The five BF16 planes of the image's current pixels (zero outside the
// image) in the tiled layout; one thread per (tile column, row, column).
__global__ void k_planes(ImgState s) {
  const size_t n = (size_t)s.tc_ntx * s.prows * s.tc_len;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int xl = (int)(e % s.tc_len);
    const size_t ry = e / s.tc_len;
    const int y = (int)(ry % s.prows), tx = (int)(ry / s.prows);
    const int x = s.tc_xs0 + tx * s.tc_w + xl;
    const uint32_t w = (x < s.W && y < s.H) ? __ldg(&s.img[(size_t)y * s.pitch + x]) : 0x00808080u;
    plane_store_at(s, tx, y, xl, w);  // outside the image: 128 - 128 = 0 everywhere
  }
}

cudaError_t launch_planes(const ImgState& s, cudaStream_t st) {
  if (!s.planes) return cudaSuccess;
  const size_t n = (size_t)s.tc_ntx * s.prows * s.tc_len;
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  k_planes<<<blocks, 256, 0, st>>>(s);
  return cudaGetLastError();
}

// TMA descriptor of a 2-D array of 32-bit words (W x H, row pitch `pitch`
// words), box box_w x box_h words; reads outside the array give 0.
static int encode_2d(void* base, int W, int H, int pitch, int box_w, int box_h, CUtensorMap* out) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return -1;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)H};
  const cuuint64_t strides[1] = {(cuuint64_t)pitch * 4};
  const cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(out, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, base, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -1;
}

int make_image_tmap_box(const ImgState& s, int box_w, int box_h, CUtensorMap* out) {
  return encode_2d(s.img, s.W, s.H, s.pitch, box_w, box_h, out);
}

// The engine's two maps per image: out[0] the search window of RGBA words of
// a batch, eng_tile_width(r, srw) x (32 + 2r); out[1] the validity counts of
// the batch's candidates, eng_count_width(srw) x 32 from a 4-word boundary.
int make_image_tmap(const ImgState& s, int srw, CUtensorMap* out) {
  if (make_image_tmap_box(s, eng_tile_width(s.r, srw), kEngBatchRows + 2 * s.r, out) != 0) return -1;
  return encode_2d(s.count, s.W, s.H, s.pitch, eng_count_width(srw), kEngBatchRows, out + 1);
}

}  // namespace inp
