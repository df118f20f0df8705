// Entry points of the mixed-precision paths: each dispatches on the operand precision to the
// translation unit compiled for it (mixed_bf16x3.cu, mixed_fp16x2.cu, mixed_tf32.cu, mixed_tf32x3.cu,
// all built from mixed_impl.cuh).
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/dmet_emb.h"
#include "internal.h"
#include "tc_gemm.cuh"

namespace dmet {

cudaError_t launch_mix_scales_bf16x3(int prec, const double2* L, const int4* t1, int E, long long per_block,
                              const double2* const* C, const long long* c_elems, int nspin, int nao, int nrep_max,
                              MixScales* sc, cudaStream_t s);
cudaError_t launch_mix_scales_fp16x2(int prec, const double2* L, const int4* t1, int E, long long per_block,
                              const double2* const* C, const long long* c_elems, int nspin, int nao, int nrep_max,
                              MixScales* sc, cudaStream_t s);
cudaError_t launch_mix_scales_tf32(int prec, const double2* L, const int4* t1, int E, long long per_block,
                              const double2* const* C, const long long* c_elems, int nspin, int nao, int nrep_max,
                              MixScales* sc, cudaStream_t s);
cudaError_t launch_mix_scales_tf32x3(int prec, const double2* L, const int4* t1, int E, long long per_block,
                              const double2* const* C, const long long* c_elems, int nspin, int nao, int nrep_max,
                              MixScales* sc, cudaStream_t s);
cudaError_t launch_split_L_bf16x3(int prec, const double2* L, const int4* t1, int e0, int E, int naux, int nao, int K1,
                           void* Ls, long long sstride, const MixScales* sc, cudaStream_t s);
cudaError_t launch_split_L_fp16x2(int prec, const double2* L, const int4* t1, int e0, int E, int naux, int nao, int K1,
                           void* Ls, long long sstride, const MixScales* sc, cudaStream_t s);
cudaError_t launch_split_L_tf32(int prec, const double2* L, const int4* t1, int e0, int E, int naux, int nao, int K1,
                           void* Ls, long long sstride, const MixScales* sc, cudaStream_t s);
cudaError_t launch_split_L_tf32x3(int prec, const double2* L, const int4* t1, int e0, int E, int naux, int nao, int K1,
                           void* Ls, long long sstride, const MixScales* sc, cudaStream_t s);
cudaError_t launch_build_Cb_bf16x3(int prec, const double2* C, int nk, int nao, int n, int K1, void* Cb, long long sstride,
                            const float* sc, cudaStream_t s);
cudaError_t launch_build_Cb_fp16x2(int prec, const double2* C, int nk, int nao, int n, int K1, void* Cb, long long sstride,
                            const float* sc, cudaStream_t s);
cudaError_t launch_build_Cb_tf32(int prec, const double2* C, int nk, int nao, int n, int K1, void* Cb, long long sstride,
                            const float* sc, cudaStream_t s);
cudaError_t launch_build_Cb_tf32x3(int prec, const double2* C, int nk, int nao, int n, int K1, void* Cb, long long sstride,
                            const float* sc, cudaStream_t s);
cudaError_t launch_build_Cc_bf16x3(int prec, const double2* C, const int4* gather, const int4* t2, int b0, int nq, int nao,
                            int n, int K2, void* Cc, long long sstride, const float* sc, cudaStream_t s);
cudaError_t launch_build_Cc_fp16x2(int prec, const double2* C, const int4* gather, const int4* t2, int b0, int nq, int nao,
                            int n, int K2, void* Cc, long long sstride, const float* sc, cudaStream_t s);
cudaError_t launch_build_Cc_tf32(int prec, const double2* C, const int4* gather, const int4* t2, int b0, int nq, int nao,
                            int n, int K2, void* Cc, long long sstride, const float* sc, cudaStream_t s);
cudaError_t launch_build_Cc_tf32x3(int prec, const double2* C, const int4* gather, const int4* t2, int b0, int nq, int nao,
                            int n, int K2, void* Cc, long long sstride, const float* sc, cudaStream_t s);
cudaError_t launch_pack_split_bf16x3(int prec, const void* ZT, int nq, int naux, int n, int nc, void* Xt, long long sstride,
                              long long Rtot, long long row_base, const float* sx, cudaStream_t s);
cudaError_t launch_pack_split_fp16x2(int prec, const void* ZT, int nq, int naux, int n, int nc, void* Xt, long long sstride,
                              long long Rtot, long long row_base, const float* sx, cudaStream_t s);
cudaError_t launch_pack_split_tf32(int prec, const void* ZT, int nq, int naux, int n, int nc, void* Xt, long long sstride,
                              long long Rtot, long long row_base, const float* sx, cudaStream_t s);
cudaError_t launch_pack_split_tf32x3(int prec, const void* ZT, int nq, int naux, int n, int nc, void* Xt, long long sstride,
                              long long Rtot, long long row_base, const float* sx, cudaStream_t s);
cudaError_t launch_pack_cplx_bf16x3(int prec, const void* ZT, int nq, int naux, int n, int q0, const int* neg, void* Xt,
                             long long sstride, long long Rtot, const float* sx, cudaStream_t s);
cudaError_t launch_pack_cplx_fp16x2(int prec, const void* ZT, int nq, int naux, int n, int q0, const int* neg, void* Xt,
                             long long sstride, long long Rtot, const float* sx, cudaStream_t s);
cudaError_t launch_pack_cplx_tf32(int prec, const void* ZT, int nq, int naux, int n, int q0, const int* neg, void* Xt,
                             long long sstride, long long Rtot, const float* sx, cudaStream_t s);
cudaError_t launch_pack_cplx_tf32x3(int prec, const void* ZT, int nq, int naux, int n, int q0, const int* neg, void* Xt,
                             long long sstride, long long Rtot, const float* sx, cudaStream_t s);
cudaError_t launch_tc_split_t_bf16x3(int prec, int bn, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs,
                              int njobs, const tc::Segment* segs, void* out, long long K2, int nao, int nemb,
                              const tc::TcCtl& ctl, const float* fac, cudaStream_t s);
cudaError_t launch_tc_split_t_fp16x2(int prec, int bn, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs,
                              int njobs, const tc::Segment* segs, void* out, long long K2, int nao, int nemb,
                              const tc::TcCtl& ctl, const float* fac, cudaStream_t s);
cudaError_t launch_tc_split_t_tf32(int prec, int bn, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs,
                              int njobs, const tc::Segment* segs, void* out, long long K2, int nao, int nemb,
                              const tc::TcCtl& ctl, const float* fac, cudaStream_t s);
cudaError_t launch_tc_split_t_tf32x3(int prec, int bn, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs,
                              int njobs, const tc::Segment* segs, void* out, long long K2, int nao, int nemb,
                              const tc::TcCtl& ctl, const float* fac, cudaStream_t s);
cudaError_t launch_tc_pairs_bf16x3(int prec, int bn, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs,
                            int njobs, const tc::Segment* segs, void* out, long long ldo, const tc::TcCtl& ctl,
                            const float* fac, cudaStream_t s);
cudaError_t launch_tc_pairs_fp16x2(int prec, int bn, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs,
                            int njobs, const tc::Segment* segs, void* out, long long ldo, const tc::TcCtl& ctl,
                            const float* fac, cudaStream_t s);
cudaError_t launch_tc_pairs_tf32(int prec, int bn, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs,
                            int njobs, const tc::Segment* segs, void* out, long long ldo, const tc::TcCtl& ctl,
                            const float* fac, cudaStream_t s);
cudaError_t launch_tc_pairs_tf32x3(int prec, int bn, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs,
                            int njobs, const tc::Segment* segs, void* out, long long ldo, const tc::TcCtl& ctl,
                            const float* fac, cudaStream_t s);
cudaError_t launch_tc_rect_bf16x3(int prec, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs, int njobs,
                           const tc::Segment* segs, double* out, long long ldo, double scale, const tc::TcCtl& ctl,
                           const float* fac, cudaStream_t s);
cudaError_t launch_tc_rect_fp16x2(int prec, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs, int njobs,
                           const tc::Segment* segs, double* out, long long ldo, double scale, const tc::TcCtl& ctl,
                           const float* fac, cudaStream_t s);
cudaError_t launch_tc_rect_tf32(int prec, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs, int njobs,
                           const tc::Segment* segs, double* out, long long ldo, double scale, const tc::TcCtl& ctl,
                           const float* fac, cudaStream_t s);
cudaError_t launch_tc_rect_tf32x3(int prec, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs, int njobs,
                           const tc::Segment* segs, double* out, long long ldo, double scale, const tc::TcCtl& ctl,
                           const float* fac, cudaStream_t s);
size_t tc_group_bytes_bf16x3(int kind, int prec);
size_t tc_group_bytes_fp16x2(int kind, int prec);
size_t tc_group_bytes_tf32(int kind, int prec);
size_t tc_group_bytes_tf32x3(int kind, int prec);
cudaError_t tc_group_fill_bf16x3(int kind, int prec, const GroupSpec* specs, int count, void* dst);
cudaError_t tc_group_fill_fp16x2(int kind, int prec, const GroupSpec* specs, int count, void* dst);
cudaError_t tc_group_fill_tf32(int kind, int prec, const GroupSpec* specs, int count, void* dst);
cudaError_t tc_group_fill_tf32x3(int kind, int prec, const GroupSpec* specs, int count, void* dst);
cudaError_t launch_tc_grouped_bf16x3(int kind, int prec, int bn, const void* groups, const tc::TcJob* jobs, int njobs,
                              const tc::TcCtl& ctl, cudaStream_t s);
cudaError_t launch_tc_grouped_fp16x2(int kind, int prec, int bn, const void* groups, const tc::TcJob* jobs, int njobs,
                              const tc::TcCtl& ctl, cudaStream_t s);
cudaError_t launch_tc_grouped_tf32(int kind, int prec, int bn, const void* groups, const tc::TcJob* jobs, int njobs,
                              const tc::TcCtl& ctl, cudaStream_t s);
cudaError_t launch_tc_grouped_tf32x3(int kind, int prec, int bn, const void* groups, const tc::TcJob* jobs, int njobs,
                              const tc::TcCtl& ctl, cudaStream_t s);
cudaError_t launch_tc_herm_bf16x3(int prec, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs, int njobs,
                           const tc::Segment* segs, double* out, long long n2, double scale, const tc::TcCtl& ctl,
                           const float* fac, cudaStream_t s);
cudaError_t launch_tc_herm_fp16x2(int prec, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs, int njobs,
                           const tc::Segment* segs, double* out, long long n2, double scale, const tc::TcCtl& ctl,
                           const float* fac, cudaStream_t s);
cudaError_t launch_tc_herm_tf32(int prec, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs, int njobs,
                           const tc::Segment* segs, double* out, long long n2, double scale, const tc::TcCtl& ctl,
                           const float* fac, cudaStream_t s);
cudaError_t launch_tc_herm_tf32x3(int prec, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs, int njobs,
                           const tc::Segment* segs, double* out, long long n2, double scale, const tc::TcCtl& ctl,
                           const float* fac, cudaStream_t s);
cudaError_t launch_tc_packed_bf16x3(int prec, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs, int njobs,
                             const tc::Segment* segs, double* out, double scale, void* part, const tc::TcCtl& ctl,
                             const float* fac, cudaStream_t s);
cudaError_t launch_tc_packed_fp16x2(int prec, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs, int njobs,
                             const tc::Segment* segs, double* out, double scale, void* part, const tc::TcCtl& ctl,
                             const float* fac, cudaStream_t s);
cudaError_t launch_tc_packed_tf32(int prec, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs, int njobs,
                             const tc::Segment* segs, double* out, double scale, void* part, const tc::TcCtl& ctl,
                             const float* fac, cudaStream_t s);
cudaError_t launch_tc_packed_tf32x3(int prec, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs, int njobs,
                             const tc::Segment* segs, double* out, double scale, void* part, const tc::TcCtl& ctl,
                             const float* fac, cudaStream_t s);

cudaError_t launch_mix_scales(int prec, const double2* L, const int4* t1, int E, long long per_block,
                              const double2* const* C, const long long* c_elems, int nspin, int nao, int nrep_max,
                              MixScales* sc, cudaStream_t s) {
  switch (prec) {
    case DMET_PREC_BF16X3: return launch_mix_scales_bf16x3(prec, L, t1, E, per_block, C, c_elems, nspin, nao, nrep_max, sc, s);
    case DMET_PREC_FP16X2: return launch_mix_scales_fp16x2(prec, L, t1, E, per_block, C, c_elems, nspin, nao, nrep_max, sc, s);
    case DMET_PREC_TF32: return launch_mix_scales_tf32(prec, L, t1, E, per_block, C, c_elems, nspin, nao, nrep_max, sc, s);
    case DMET_PREC_TF32X3: return launch_mix_scales_tf32x3(prec, L, t1, E, per_block, C, c_elems, nspin, nao, nrep_max, sc, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_split_L(int prec, const double2* L, const int4* t1, int e0, int E, int naux, int nao, int K1,
                           void* Ls, long long sstride, const MixScales* sc, cudaStream_t s) {
  switch (prec) {
    case DMET_PREC_BF16X3: return launch_split_L_bf16x3(prec, L, t1, e0, E, naux, nao, K1, Ls, sstride, sc, s);
    case DMET_PREC_FP16X2: return launch_split_L_fp16x2(prec, L, t1, e0, E, naux, nao, K1, Ls, sstride, sc, s);
    case DMET_PREC_TF32: return launch_split_L_tf32(prec, L, t1, e0, E, naux, nao, K1, Ls, sstride, sc, s);
    case DMET_PREC_TF32X3: return launch_split_L_tf32x3(prec, L, t1, e0, E, naux, nao, K1, Ls, sstride, sc, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_build_Cb(int prec, const double2* C, int nk, int nao, int n, int K1, void* Cb, long long sstride,
                            const float* sc, cudaStream_t s) {
  switch (prec) {
    case DMET_PREC_BF16X3: return launch_build_Cb_bf16x3(prec, C, nk, nao, n, K1, Cb, sstride, sc, s);
    case DMET_PREC_FP16X2: return launch_build_Cb_fp16x2(prec, C, nk, nao, n, K1, Cb, sstride, sc, s);
    case DMET_PREC_TF32: return launch_build_Cb_tf32(prec, C, nk, nao, n, K1, Cb, sstride, sc, s);
    case DMET_PREC_TF32X3: return launch_build_Cb_tf32x3(prec, C, nk, nao, n, K1, Cb, sstride, sc, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_build_Cc(int prec, const double2* C, const int4* gather, const int4* t2, int b0, int nq, int nao,
                            int n, int K2, void* Cc, long long sstride, const float* sc, cudaStream_t s) {
  switch (prec) {
    case DMET_PREC_BF16X3: return launch_build_Cc_bf16x3(prec, C, gather, t2, b0, nq, nao, n, K2, Cc, sstride, sc, s);
    case DMET_PREC_FP16X2: return launch_build_Cc_fp16x2(prec, C, gather, t2, b0, nq, nao, n, K2, Cc, sstride, sc, s);
    case DMET_PREC_TF32: return launch_build_Cc_tf32(prec, C, gather, t2, b0, nq, nao, n, K2, Cc, sstride, sc, s);
    case DMET_PREC_TF32X3: return launch_build_Cc_tf32x3(prec, C, gather, t2, b0, nq, nao, n, K2, Cc, sstride, sc, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_pack_split(int prec, const void* ZT, int nq, int naux, int n, int nc, void* Xt, long long sstride,
                              long long Rtot, long long row_base, const float* sx, cudaStream_t s) {
  switch (prec) {
    case DMET_PREC_BF16X3: return launch_pack_split_bf16x3(prec, ZT, nq, naux, n, nc, Xt, sstride, Rtot, row_base, sx, s);
    case DMET_PREC_FP16X2: return launch_pack_split_fp16x2(prec, ZT, nq, naux, n, nc, Xt, sstride, Rtot, row_base, sx, s);
    case DMET_PREC_TF32: return launch_pack_split_tf32(prec, ZT, nq, naux, n, nc, Xt, sstride, Rtot, row_base, sx, s);
    case DMET_PREC_TF32X3: return launch_pack_split_tf32x3(prec, ZT, nq, naux, n, nc, Xt, sstride, Rtot, row_base, sx, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_pack_cplx(int prec, const void* ZT, int nq, int naux, int n, int q0, const int* neg, void* Xt,
                             long long sstride, long long Rtot, const float* sx, cudaStream_t s) {
  switch (prec) {
    case DMET_PREC_BF16X3: return launch_pack_cplx_bf16x3(prec, ZT, nq, naux, n, q0, neg, Xt, sstride, Rtot, sx, s);
    case DMET_PREC_FP16X2: return launch_pack_cplx_fp16x2(prec, ZT, nq, naux, n, q0, neg, Xt, sstride, Rtot, sx, s);
    case DMET_PREC_TF32: return launch_pack_cplx_tf32(prec, ZT, nq, naux, n, q0, neg, Xt, sstride, Rtot, sx, s);
    case DMET_PREC_TF32X3: return launch_pack_cplx_tf32x3(prec, ZT, nq, naux, n, q0, neg, Xt, sstride, Rtot, sx, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_tc_split_t(int prec, int bn, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs,
                              int njobs, const tc::Segment* segs, void* out, long long K2, int nao, int nemb,
                              const tc::TcCtl& ctl, const float* fac, cudaStream_t s) {
  switch (prec) {
    case DMET_PREC_BF16X3: return launch_tc_split_t_bf16x3(prec, bn, A, B, jobs, njobs, segs, out, K2, nao, nemb, ctl, fac, s);
    case DMET_PREC_FP16X2: return launch_tc_split_t_fp16x2(prec, bn, A, B, jobs, njobs, segs, out, K2, nao, nemb, ctl, fac, s);
    case DMET_PREC_TF32: return launch_tc_split_t_tf32(prec, bn, A, B, jobs, njobs, segs, out, K2, nao, nemb, ctl, fac, s);
    case DMET_PREC_TF32X3: return launch_tc_split_t_tf32x3(prec, bn, A, B, jobs, njobs, segs, out, K2, nao, nemb, ctl, fac, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_tc_pairs(int prec, int bn, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs,
                            int njobs, const tc::Segment* segs, void* out, long long ldo, const tc::TcCtl& ctl,
                            const float* fac, cudaStream_t s) {
  switch (prec) {
    case DMET_PREC_BF16X3: return launch_tc_pairs_bf16x3(prec, bn, A, B, jobs, njobs, segs, out, ldo, ctl, fac, s);
    case DMET_PREC_FP16X2: return launch_tc_pairs_fp16x2(prec, bn, A, B, jobs, njobs, segs, out, ldo, ctl, fac, s);
    case DMET_PREC_TF32: return launch_tc_pairs_tf32(prec, bn, A, B, jobs, njobs, segs, out, ldo, ctl, fac, s);
    case DMET_PREC_TF32X3: return launch_tc_pairs_tf32x3(prec, bn, A, B, jobs, njobs, segs, out, ldo, ctl, fac, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_tc_rect(int prec, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs, int njobs,
                           const tc::Segment* segs, double* out, long long ldo, double scale, const tc::TcCtl& ctl,
                           const float* fac, cudaStream_t s) {
  switch (prec) {
    case DMET_PREC_BF16X3: return launch_tc_rect_bf16x3(prec, A, B, jobs, njobs, segs, out, ldo, scale, ctl, fac, s);
    case DMET_PREC_FP16X2: return launch_tc_rect_fp16x2(prec, A, B, jobs, njobs, segs, out, ldo, scale, ctl, fac, s);
    case DMET_PREC_TF32: return launch_tc_rect_tf32(prec, A, B, jobs, njobs, segs, out, ldo, scale, ctl, fac, s);
    case DMET_PREC_TF32X3: return launch_tc_rect_tf32x3(prec, A, B, jobs, njobs, segs, out, ldo, scale, ctl, fac, s);
    default: return cudaErrorInvalidValue;
  }
}

size_t tc_group_bytes(int kind, int prec) {
  switch (prec) {
    case DMET_PREC_BF16X3: return tc_group_bytes_bf16x3(kind, prec);
    case DMET_PREC_FP16X2: return tc_group_bytes_fp16x2(kind, prec);
    case DMET_PREC_TF32: return tc_group_bytes_tf32(kind, prec);
    case DMET_PREC_TF32X3: return tc_group_bytes_tf32x3(kind, prec);
    default: return 0;
  }
}

cudaError_t tc_group_fill(int kind, int prec, const GroupSpec* specs, int count, void* dst) {
  switch (prec) {
    case DMET_PREC_BF16X3: return tc_group_fill_bf16x3(kind, prec, specs, count, dst);
    case DMET_PREC_FP16X2: return tc_group_fill_fp16x2(kind, prec, specs, count, dst);
    case DMET_PREC_TF32: return tc_group_fill_tf32(kind, prec, specs, count, dst);
    case DMET_PREC_TF32X3: return tc_group_fill_tf32x3(kind, prec, specs, count, dst);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_tc_grouped(int kind, int prec, int bn, const void* groups, const tc::TcJob* jobs, int njobs,
                              const tc::TcCtl& ctl, cudaStream_t s) {
  switch (prec) {
    case DMET_PREC_BF16X3: return launch_tc_grouped_bf16x3(kind, prec, bn, groups, jobs, njobs, ctl, s);
    case DMET_PREC_FP16X2: return launch_tc_grouped_fp16x2(kind, prec, bn, groups, jobs, njobs, ctl, s);
    case DMET_PREC_TF32: return launch_tc_grouped_tf32(kind, prec, bn, groups, jobs, njobs, ctl, s);
    case DMET_PREC_TF32X3: return launch_tc_grouped_tf32x3(kind, prec, bn, groups, jobs, njobs, ctl, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_tc_herm(int prec, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs, int njobs,
                           const tc::Segment* segs, double* out, long long n2, double scale, const tc::TcCtl& ctl,
                           const float* fac, cudaStream_t s) {
  switch (prec) {
    case DMET_PREC_BF16X3: return launch_tc_herm_bf16x3(prec, A, B, jobs, njobs, segs, out, n2, scale, ctl, fac, s);
    case DMET_PREC_FP16X2: return launch_tc_herm_fp16x2(prec, A, B, jobs, njobs, segs, out, n2, scale, ctl, fac, s);
    case DMET_PREC_TF32: return launch_tc_herm_tf32(prec, A, B, jobs, njobs, segs, out, n2, scale, ctl, fac, s);
    case DMET_PREC_TF32X3: return launch_tc_herm_tf32x3(prec, A, B, jobs, njobs, segs, out, n2, scale, ctl, fac, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_tc_packed(int prec, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs, int njobs,
                             const tc::Segment* segs, double* out, double scale, void* part, const tc::TcCtl& ctl,
                             const float* fac, cudaStream_t s) {
  switch (prec) {
    case DMET_PREC_BF16X3: return launch_tc_packed_bf16x3(prec, A, B, jobs, njobs, segs, out, scale, part, ctl, fac, s);
    case DMET_PREC_FP16X2: return launch_tc_packed_fp16x2(prec, A, B, jobs, njobs, segs, out, scale, part, ctl, fac, s);
    case DMET_PREC_TF32: return launch_tc_packed_tf32(prec, A, B, jobs, njobs, segs, out, scale, part, ctl, fac, s);
    case DMET_PREC_TF32X3: return launch_tc_packed_tf32x3(prec, A, B, jobs, njobs, segs, out, scale, part, ctl, fac, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dmet
