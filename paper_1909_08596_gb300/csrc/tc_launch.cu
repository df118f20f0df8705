// Tensor-map encoding for the tcgen05 kernels, through the runtime's driver entry point so
// that the library needs no link-time libcuda.

#include <cuda.h>
#include <cuda_runtime.h>

#include "internal.h"

namespace dmet {

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    else
      cudaGetLastError();
  }
  return fn;
}

}  // namespace

namespace {
// element type and size of a precision's slices
void prec_type(int prec, CUtensorMapDataType* t, int* esz) {
  if (prec == 2 || prec == 3) {  // TF32 slices are stored as FP32 words
    *t = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    *esz = 4;
  } else if (prec == 4) {
    *t = CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    *esz = 2;
  } else {
    *t = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    *esz = 2;
  }
}
}  // namespace

cudaError_t make_tmap_3d(CUtensorMap* map, int prec, const void* base, unsigned long long k_elems,
                         unsigned long long rows, unsigned long long slices, unsigned long long row_stride_elems,
                         unsigned long long slice_stride_elems, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  CUtensorMapDataType dt;
  int esz = 2;
  prec_type(prec, &dt, &esz);
  if (((uintptr_t)base & 15) || (row_stride_elems * esz) % 16 || (slice_stride_elems * esz) % 16)
    return cudaErrorInvalidValue;
  const cuuint64_t dims[3] = {k_elems, rows, slices};
  const cuuint64_t strides[2] = {row_stride_elems * esz, slice_stride_elems * esz};
  const cuuint32_t box[3] = {(cuuint32_t)(64 / esz), (cuuint32_t)box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, dt, 3, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t make_tmap_interleaved(CUtensorMap* map, int prec, const void* base, unsigned long long k_elems,
                                  unsigned long long rows, int slices, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  CUtensorMapDataType dt;
  int esz = 2;
  prec_type(prec, &dt, &esz);
  const unsigned long long bk = 64 / esz;
  if (((uintptr_t)base & 15) || k_elems % bk) return cudaErrorInvalidValue;
  // dims (innermost first): element in block, slice, K block, row
  const cuuint64_t dims[4] = {bk, (cuuint64_t)slices, k_elems / bk, rows};
  const cuuint64_t strides[3] = {64, 64ull * slices, (cuuint64_t)slices * k_elems * esz};
  const cuuint32_t box[4] = {(cuuint32_t)bk, 1, 1, (cuuint32_t)box_rows};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = fn(map, dt, 4, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace dmet
