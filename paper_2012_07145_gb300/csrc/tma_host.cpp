// Host side of TMA: encodes tiled tensor maps through the driver's
// cuTensorMapEncodeTiled, fetched once from the runtime's driver entry point
// (no link against libcuda is needed).
#include <cuda.h>
#include <cuda_runtime.h>

namespace hp {

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    else
      cudaGetLastError();
  }
  return fn;
}

}  // namespace

int encode_tmap_3d(CUtensorMap* map, CUtensorMapDataType dt, int esize, const void* base, int w, int h, int c,
                   long long row_stride, long long plane_stride, int bw, int bh, int bz) {
  EncodeTiledFn fn = encoder();
  if (!fn) return 1;
  if (((unsigned long long)base & 15) || row_stride % 16 || plane_stride % 16 || (bw * esize) % 16 || bw > 256 ||
      bh > 256)
    return 2;
  cuuint64_t dims[3] = {(cuuint64_t)w, (cuuint64_t)h, (cuuint64_t)c};
  cuuint64_t strides[2] = {(cuuint64_t)row_stride, (cuuint64_t)(c > 1 ? plane_stride : row_stride * h)};
  if (bz < 1 || bz > c) return 2;
  cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, (cuuint32_t)bz};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, dt, 3, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : 3;
}

}  // namespace hp
