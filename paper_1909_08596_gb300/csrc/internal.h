// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dmet {

// Message of the last error returned on the calling thread (fixed buffer, no heap).
constexpr int kLastErrorBytes = 512;
char* last_error_buffer();

// Batched complex FP64 GEMM:  D[m][n] = alpha * sum_k opA(m,k) * opB(k,n)  (+ D if beta).
// opA(m,k) = A[k*lda + m] (A_KM) or A[m*lda + k] (A_MK), conjugated if conj_a.
// opB(k,n) = B[k*ldb + n] (B_KN) or B[n*ldb + k] (B_NK).
// Output address: (m/dm_div)*dm_hi + (m%dm_div)*dm_lo + (n/dn_div)*dn_hi + (n%dn_div)*dn_lo.
// Batch z: tab == nullptr -> A += z*sA, B += z*sB, D += z*sD, K = K;
//          else e = tab[tab0 + z] -> A += e.x*sA, B += e.y*sB, D += e.z*sD, K = e.w.
enum { A_KM = 0, A_MK = 1 };
enum { B_KN = 0, B_NK = 1 };

struct ZgemmArgs {
  const double2* A;
  const double2* B;
  double2* D;
  const int4* tab;
  int tab0;
  int M, N, K;
  long long lda, ldb;
  long long sA, sB, sD;
  int dm_div;
  long long dm_hi, dm_lo;
  int dn_div;
  long long dn_hi, dn_lo;
  double alpha;
  int beta;
  int batch;
  int lower;  // nonzero: skip tiles strictly above the diagonal (Hermitian results)
};

cudaError_t launch_zgemm(const ZgemmArgs& a, int a_layout, bool conj_a, int b_layout, cudaStream_t s);

// Real FP64 rank-K product of two [K][*] row-major operands X (ldx) and Y (ldy):
//   mode 0 (8-fold packed, X == Y, M == N): out[m(m+1)/2 + n] += alpha * sum_k X[k][m] X[k][n], m >= n
//   mode 1 (rectangular):                   out[m*ldo + n]    += alpha * sum_k X[k][m] Y[k][n]
struct DsyrkArgs {
  const double* X;
  const double* Y;
  double* out;
  int M, N, K;
  long long ldx, ldy, ldo;
  double alpha;
  int mode;
};

cudaError_t launch_dsyrk(const DsyrkArgs& a, cudaStream_t s);

// C_rep[e][mu][i] = w_e * C[k1_e][mu][i] for the entries e of a table (x = k1, y = half flag).
cudaError_t launch_gather_orbitals(const double2* C, double2* Crep, const int4* tab, int tab0,
                                   int n_entries, int nao, int n, cudaStream_t s);

// Real path: Z[q][P][i][j] -> X[q][P][c][IJ] = Re/Im of s * (Z_ij + Z_ji), c < nc, i >= j.
cudaError_t launch_pack_pairs(const double2* Z, double* X, int nq, int naux, int n, int nc, double s,
                              cudaStream_t st);

// 4-fold packing of a complex ERI block full[i][j][k][l] (the layout of dmet_emb_eri_bytes): a
// same-spin block (rect = 0, na == nb) or the alpha-beta block (rect = 1, rows i >= j, all (k, l)).
cudaError_t launch_pack_s4(const double2* full, int na, int nb, int rect, double2* out, cudaStream_t st);
// Real path 3-index output: Lq[q][P][i][j] = s * (Z_ij + Z_ji), or its complex conjugate if conj.
cudaError_t launch_symmetrize(const double2* Z, double2* Lq, int nq, int naux, int n, double s, int conj,
                              cudaStream_t st);

// Checks. stats layout (doubles, raw maxima): [0] orthonormality, [1] |C^{-k} - conj C^k|,
// [2] |C|, [3] Hermiticity of L, [4] time reversal of L, [5] |L| (the last three component-wise).
// The orthonormality reduction sums ng split-K partial products S_g = C_g^+ C_g first.
// Embedding Fock matrix (fock.cu): F0 = s sum_k Re G[k]; J and K of gamma from the 8-fold packed
// ERI (K must start at zero; n(n+1)/2 + n doubles of shared memory, so n <= 232); out = F0 - J + K/2.
cudaError_t launch_fock_reduce(const double2* G, int nk, int n, double s, double* F0, cudaStream_t st);
cudaError_t launch_coulomb_exchange(const double* eri, const double* gamma, int n, double* J, double* K,
                                    cudaStream_t st);
cudaError_t launch_fock_combine(const double* F0, const double* J, const double* K, int n, double* out,
                                cudaStream_t st);
// FFTDF (fftdf.cu): dst = s exp(sign i q.r) src over the cell grid ([r][x], x < nx), q the mesh point of
// triple nq; buf[G][x] *= v[G].
cudaError_t launch_fftdf_phase(const double2* src, double2* dst, const int grid[3], const int nq[3], const int mesh[3],
                               double sign, double s, long long nx, cudaStream_t st);
cudaError_t launch_fftdf_kernel_mul(double2* buf, const double* v, long long ng, long long nx, cudaStream_t st);
// A dense DFT along the middle axis of [outer][g][inner] for g <= 32 (fftdf_small_axis):
// out[o][k][i] = sum_j F[k g + j] in[o][j][i].
bool fftdf_small_axis(int g);
cudaError_t launch_dft_axis_small(const double2* F, int g, long long outer, long long inner, const double2* in,
                                  double2* out, cudaStream_t st);
// out[i] += sum over the np parts of parts[p n + i] (the K parts of a split GEMM).
cudaError_t launch_sum_parts(const double2* parts, int np, long long n, double2* out, cudaStream_t st);
// The phase for nq_run q values at once (q = qtab[i] for block i; source block by q if by_table, else by i).
cudaError_t launch_fftdf_phase_q(const double2* src, double2* dst, const int* qtab, int nq_run, int by_table,
                                 const int grid[3], const int mesh[3], double sign, double s, long long nx,
                                 cudaStream_t st);
// Density-fitted J and K from the factors L^q (fock.cu), per chunk of z = (q, P) batch entries with
// tab[z] = {z-th factor's index in Lq, the -q factor's index, z, n}:
// v[z] = tr(L^{-q}_P gamma); J += s sum_z v[z] L^q_P; K += s sum_z Kb[z] (Kb[z] = L^q_P gamma L^{-q}_P).
cudaError_t launch_jk_trace(const double2* Lq, const int4* tab, int nz, int n, const double2* gamma, double2* v,
                            cudaStream_t st);
cudaError_t launch_jk_accumulate(const double2* Lq, const int4* tab, const double2* v, const double2* Kb, int nz, int n,
                                 double s, double2* J, double2* K, cudaStream_t st);
// Bath construction (bath.cu). The impurity columns that enter the SVD, by value.
constexpr int kMaxBathCols = 128;
struct BathCols {
  int n;
  int v[kMaxBathCols];
};
constexpr size_t kBathJacobiSmem = 200 * 1024;  // each CTA's rows stay in shared memory up to this size
constexpr int kBathCluster = 8;                  // CTAs (SMs) of the Jacobi SVD's cluster
cudaError_t launch_bath_twiddle(int nk, double2* tw, cudaStream_t st);
cudaError_t launch_bath_offdiag(const double2* gk, const double2* tw, const int mesh[3], int n_lo, const BathCols& val,
                                double* A, double* stats, cudaStream_t st);
size_t bath_jacobi_smem(int m, int n_val);
cudaError_t launch_bath_jacobi(double* A, int m, int n_val, double* B, double* sigma, double* stats,
                               cudaStream_t st);
cudaError_t launch_bath_product(const double2* Clo, const double2* Cb, int nk, int n_lo, int n_val, double2* Cout,
                                cudaStream_t st);
cudaError_t launch_bath_bloch(const double* B, const double2* Clo, const double2* tw, const int mesh[3], int n_lo,
                              int n_val, double2* Cb, double2* Cout, cudaStream_t st);
cudaError_t launch_orth_reduce(const double2* Sg, int ng, int n, double s, double* stat, cudaStream_t st);
cudaError_t launch_c_real_check(const double2* C, const int* neg, int nk, int nao, int n, double* stats,
                                cudaStream_t st);
cudaError_t launch_l_check(const double2* L, const int* neg, int nk, int naux, int nao, double* stats,
                           cudaStream_t st);

}  // namespace dmet

// ---- tensor maps for the tcgen05 kernels (tc_launch.cu) ----
#include <cuda.h>
namespace dmet {
// Tensor maps over the operand slices of precision `prec` (dmet_prec_t; element type bf16, fp16 or
// fp32 for TF32), swizzled to match the UMMA descriptors (64-byte rows):
// 3-D over [slices][rows][K] (K contiguous) with a (64 bytes of K, box_rows, 1) box;
cudaError_t make_tmap_3d(CUtensorMap* map, int prec, const void* base, unsigned long long k_elems,
                         unsigned long long rows, unsigned long long slices, unsigned long long row_stride_elems,
                         unsigned long long slice_stride_elems, int box_rows);
// 4-D over a slice-interleaved operand [rows][K / BK][slices][BK] (BK = 64 bytes of elements) with a
// (BK, 1, 1, box_rows) box: one slice of one K block.
cudaError_t make_tmap_interleaved(CUtensorMap* map, int prec, const void* base, unsigned long long k_elems,
                                  unsigned long long rows, int slices, int box_rows);
}  // namespace dmet

// ---- mixed-precision paths (mixed.cu) ----
namespace dmet {
namespace tc {
struct TcJob;
struct Segment;
struct TcCtl;
}
// Operand scales of the FP16 precision (powers of two; all 1 for the other precisions), computed on
// the device from the maxima mx (float bits) of |L| and |C_s|: Ls = L sL, Cb = Cc = C sC[s],
// A2 = T sT[s] = (step-1 result) f1[s], Z = (step-2 result) f2[s], Xt = (Z + Z^T) sX[s], and block b of
// the contraction = (its result) fc[b].
struct MixScales {
  float sL, sC[2], sT[2], f1[2], f2[2], sX[2], fc[3];
  unsigned int mx[3];
};
int mixed_kblock();             // K padding unit of every operand (elements)
bool prec_scaled(int prec);
int prec_slices(int prec);
int prec_products(int prec);
int prec_elem_bytes(int prec);
cudaError_t launch_mix_scales(int prec, const double2* L, const int4* t1, int E, long long per_block,
                              const double2* const* C, const long long* c_elems, int nspin, int nao, int nrep_max,
                              MixScales* sc, cudaStream_t s);
cudaError_t launch_split_L(int prec, const double2* L, const int4* t1, int e0, int E, int naux, int nao, int K1,
                           void* Ls, long long sstride, const MixScales* sc, cudaStream_t s);
cudaError_t launch_build_Cb(int prec, const double2* C, int nk, int nao, int n, int K1, void* Cb, long long sstride,
                            const float* sc, cudaStream_t s);
cudaError_t launch_build_Cc(int prec, const double2* C, const int4* gather, const int4* t2, int b0, int nq, int nao,
                            int n, int K2, void* Cc, long long sstride, const float* sc, cudaStream_t s);
cudaError_t launch_pack_split(int prec, const void* ZT, int nq, int naux, int n, int nc, void* Xt, long long sstride,
                              long long Rtot, long long row_base, const float* sx, cudaStream_t s);
cudaError_t launch_tc_pairs(int prec, int bn, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs,
                            int njobs, const tc::Segment* segs, void* out, long long ldo, const tc::TcCtl& ctl,
                            const float* fac, cudaStream_t s);
cudaError_t launch_tc_split_t(int prec, int bn, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs,
                              int njobs, const tc::Segment* segs, void* out, long long K2, int nao, int nemb,
                              const tc::TcCtl& ctl, const float* fac, cudaStream_t s);
cudaError_t launch_tc_rect(int prec, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs, int njobs,
                           const tc::Segment* segs, double* out, long long ldo, double scale, const tc::TcCtl& ctl,
                           const float* fac, cudaStream_t s);
cudaError_t launch_tc_packed(int prec, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs, int njobs,
                             const tc::Segment* segs, double* out, double scale, void* part, const tc::TcCtl& ctl,
                             const float* fac, cudaStream_t s);
// L^q of one slot from the step-2 output (two-float pairs): s (Z + Z^T) (pair = 1, real orbitals) or
// s Z (pair = 0), conjugated if conj.
cudaError_t launch_lq_from_pairs(const void* ZT, int naux, int n, double s, int conj, int pair, double2* Lq,
                                 cudaStream_t st);
// The contraction operand of general (complex) orbitals from the step-2 output of slots q0 .. q0+nq-1
// (bra rows ij in the K block of q, ket rows n^2 + 2 kl + c in the K block of -q; mixed.cu).
cudaError_t launch_pack_cplx(int prec, const void* ZT, int nq, int naux, int n, int q0, const int* neg, void* Xt,
                             long long sstride, long long Rtot, const float* sx, cudaStream_t s);
// One same-spin block of complex ERIs, (ij|kl) as (re, im) doubles at out[ij * 2 n2 + 2 kl + c], from
// the tiles with kl <= ij (the others by (kl|ij) = (ij|kl)).
cudaError_t launch_tc_herm(int prec, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs, int njobs,
                           const tc::Segment* segs, double* out, long long n2, double scale, const tc::TcCtl& ctl,
                           const float* fac, cudaStream_t s);
// Grouped tensor-core launches (one persistent launch over the tiles of many problems): the kinds
// of table entry, what an entry holds, its size per precision, the host-side fill and the launch.
enum { kGroupSplitT = 0, kGroupPairs = 1, kGroupContract = 2 };
struct GroupSpec {
  const CUtensorMap* a;
  const CUtensorMap* b;
  const tc::Segment* segs;
  const float* fac;     // device factor, or null
  void* out;            // step 1: the A2 operand; step 2: the Z pairs
  double* const* outp;  // contraction: device slot holding the ERI block's pointer
  long long ld;         // step 1: K2; step 2: 2 n; contraction: the row pitch (mode 1, 2)
  int nao, n;           // step 1
  double scale;         // contraction
  int mode;             // contraction: 0 packed, 1 rectangular, 2 complex same-spin
};
size_t tc_group_bytes(int kind, int prec);
cudaError_t tc_group_fill(int kind, int prec, const GroupSpec* specs, int count, void* host_dst);
cudaError_t launch_tc_grouped(int kind, int prec, int bn, const void* groups, const tc::TcJob* jobs, int njobs,
                              const tc::TcCtl& ctl, cudaStream_t s);
// Sums the K parts of the split tiles of a packed contraction (the parts' jobs: jobs[0 .. ntiles * f)).
cudaError_t launch_combine_parts(const tc::TcJob* jobs, int ntiles, int f, const void* part, double* out, double scale,
                                 cudaStream_t s);
}  // namespace dmet
