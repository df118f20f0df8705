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

cudaError_t make_tmap_bf16_3d(CUtensorMap* map, const void* base, unsigned long long k_elems,
                              unsigned long long rows, unsigned long long slices, unsigned long long row_stride_elems,
                              unsigned long long slice_stride_elems, int box_k, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  if (((uintptr_t)base & 15) || (row_stride_elems * 2) % 16 || (slice_stride_elems * 2) % 16)
    return cudaErrorInvalidValue;
  const cuuint64_t dims[3] = {k_elems, rows, slices};
  const cuuint64_t strides[2] = {row_stride_elems * 2, slice_stride_elems * 2};
  const cuuint32_t box[3] = {(cuuint32_t)box_k, (cuuint32_t)box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUtensorMapSwizzle sw = box_k * 2 == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t make_tmap_bf16_interleaved(CUtensorMap* map, const void* base, unsigned long long k_elems,
                                       unsigned long long rows, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  if (((uintptr_t)base & 15) || k_elems % 32) return cudaErrorInvalidValue;
  // dims (innermost first): element in block, slice, K block, row
  const cuuint64_t dims[4] = {32, 3, k_elems / 32, rows};
  const cuuint64_t strides[3] = {32 * 2, 96 * 2, 3 * k_elems * 2};
  const cuuint32_t box[4] = {32, 1, 1, (cuuint32_t)box_rows};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace dmet
