// Mixed-precision paths, compiled once per operand precision (a translation unit per precision keeps
// every unit's compile time short): DMET_ONE_PREC is the dmet_prec_t code of the unit, DMET_PREC_TYPE
// its slice type (prec.cuh), DMET_PREC_SUFFIX the suffix of its entry points, which mixed.cu
// dispatches to; DMET_PRIMARY_TU marks the one unit that also defines the precision-free helpers.
//
// Mixed-precision paths of the embedded-ERI transformation: the operand splitting kernels, the
// operand scales of the FP16 precision and the tcgen05 GEMM instantiations with their output
// functors, for every operand precision of prec.cuh (BF16x3, FP16x2, TF32, TF32x3).
//
// Every FP64 operand x is split into slices x = x_0 + x_1 (+ x_2) of the precision's element type,
// each slice the round-to-nearest of what the previous ones left over (the error-free splitting of
// Ozaki et al., applied per element, computed from a two-float form of x so that no FP64
// arithmetic is needed; see split.cuh and prec.cuh). Complex products are written as real GEMMs
// over interleaved (re, im) K indices; the orbital operands carry the signs.
//
// Step 1 (ket side):  T_e[(P,mu)][(j,p)] = sum_(nu,c) L_e[(P,mu)][(nu,c)] Cb^{k2}[(j,p)][(nu,c)]
//   with Cb rows (j, re) = (Cr, -Ci), (j, im) = (Ci, Cr) over (nu, c), so T = L C^{k2}.
// Step 2 (bra side + Fourier sum): Z_q[(P,j)][(i,p)] = sum_(r,mu,c) T[(P,j)][(r,mu,c)] Cc[(i,p)][(r,mu,c)]
//   with Cc rows (i, re) = w_r (Cr, Ci), (i, im) = w_r (-Ci, Cr), so Z = sum_r w_r C^{k1_r +} T_r.
// Contraction: X[(q,P,c)][IJ] = Re/Im of s (Z_ij + Z_ji); (ij|kl) = (1/Nk) sum w_q X^T X.
//
// Scales (FP16x2 only; 1 otherwise): L and C are scaled by powers of two sL, sC that put their
// largest components at or below 2^14; T and X by sT, sX derived from rigorous bounds on their
// magnitudes (a sum of K products is at most K times the largest product); each GEMM's results are
// multiplied back by the exact power of two its operands' scales leave.

#pragma once

#include <cstring>
#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "../../include/dmet_emb.h"
#include "internal.h"
#include "prec.cuh"
#include "split.cuh"
#include "tc_gemm.cuh"

#define DMET_CAT2(a, b) a##b
#define DMET_CAT(a, b) DMET_CAT2(a, b)
#define DMET_P(name) DMET_CAT(name, DMET_PREC_SUFFIX)

namespace dmet {

namespace {

using tc::PrecBF16x3;
using tc::PrecFP16x2;
using tc::PrecTF32;
using tc::PrecTF32x3;

inline int grid_for(long long total, int threads, int cap) {
  long long g = (total + threads - 1) / threads;
  if (g < 1) g = 1;
  return (int)(g < cap ? g : cap);
}

template <class T>
struct __align__(2 * sizeof(T)) Pair2 {
  T a, b;
};

// The slices of the two real components (re = hr + lr, im = hi + li) of one complex element, as
// (re, im) pairs per slice: the precision's own split (prec.cuh), with the two components of each
// 16-bit slice rounded by one paired conversion (the same round-to-nearest of each value).
template <class PREC>
__device__ __forceinline__ void split_pair(float hr, float lr, float hi, float li, Pair2<typename PREC::T>* out) {
  using T = typename PREC::T;
  if constexpr (std::is_same<T, __nv_bfloat16>::value || std::is_same<T, __half>::value) {
    using T2 = typename std::conditional<std::is_same<T, __half>::value, __half2, __nv_bfloat162>::type;
    auto cvt = [](float a, float b) -> T2 {
      if constexpr (std::is_same<T, __half>::value) return __floats2half2_rn(a, b);
      else return __floats2bfloat162_rn(a, b);
    };
    auto back = [](T2 v) -> float2 {
      if constexpr (std::is_same<T, __half>::value) return __half22float2(v);
      else return __bfloat1622float2(v);
    };
    T2 s = cvt(hr, hi);
    out[0] = *reinterpret_cast<Pair2<T>*>(&s);
    float2 f = back(s);
    const float rr = (hr - f.x) + lr, ri = (hi - f.y) + li;
    s = cvt(rr, ri);
    out[1] = *reinterpret_cast<Pair2<T>*>(&s);
    if constexpr (PREC::kSlices == 3) {
      f = back(s);
      s = cvt(rr - f.x, ri - f.y);
      out[2] = *reinterpret_cast<Pair2<T>*>(&s);
    }
  } else {
    T a[3], b[3];
    PREC::split(hr, lr, a);
    PREC::split(hi, li, b);
#pragma unroll
    for (int t = 0; t < PREC::kSlices; ++t) out[t] = Pair2<T>{a[t], b[t]};
  }
}

// x * s as a two-float (hi, lo): the two-float form of the double x, scaled exactly.
__device__ __forceinline__ float2 scaled_ff(double x, float s) {
  const float2 p = d2ff(x);
  return make_float2(p.x * s, p.y * s);
}

// Ls[t][(e - e0) * naux * nao + P * nao + mu][col] for col < K1: L^{k1,k2}_{P, mu, nu}.(re|im) * sL
// at col = 2 nu + c, zero for col >= 2 nao. One thread per (row, nu): it reads the complex
// element (16 bytes; a warp reads a row's run of nu) and writes one (re, im) pair per slice.
// blockIdx.y is the entry; all index arithmetic within an entry is 32-bit.
template <class PREC>
__global__ void __launch_bounds__(256) split_L_kernel(const double2* __restrict__ L, const int4* __restrict__ t1,
                                                      int e0, int naux, int nao, int K1,
                                                      typename PREC::T* __restrict__ Ls, long long sstride,
                                                      const MixScales* __restrict__ sc) {
  using T = typename PREC::T;
  const float s = PREC::kScaled ? sc->sL : 1.f;
  const int el = blockIdx.y;
  const int rows_e = naux * nao, half = K1 >> 1;
  const int total = rows_e * half;
  const long long pair = t1[e0 + el].y;  // block of L
  const double2* src = L + pair * rows_e * nao;
  Pair2<T>* dst = reinterpret_cast<Pair2<T>*>(Ls) + (long long)el * total;
  const long long ss = sstride / 2;
  // Four elements per trip, all loads issued before the first conversion (memory-level parallelism).
  const int stride = gridDim.x * blockDim.x;
  for (int x0 = blockIdx.x * blockDim.x + threadIdx.x; x0 < total; x0 += 4 * stride) {
    double2 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int x = x0 + u * stride;
      const int row = x / half, nu = x - row * half;
      v[u] = make_double2(0.0, 0.0);
      if (x < total && nu < nao) v[u] = src[(long long)row * nao + nu];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int x = x0 + u * stride;
      if (x >= total) break;
      const float2 re = scaled_ff(v[u].x, s), im = scaled_ff(v[u].y, s);
      Pair2<T> pr[3];
      split_pair<PREC>(re.x, re.y, im.x, im.y, pr);
#pragma unroll
      for (int t = 0; t < PREC::kSlices; ++t) dst[x + t * ss] = pr[t];
    }
  }
}

// Cb[t][k * 2n + 2j + p][col], col = 2 nu + c < 2 nao:
//   p = 0: (Cr, -Ci)[c];  p = 1: (Ci, Cr)[c]   of C^k_{nu j} (times sC).
template <class PREC>
__global__ void build_Cb_kernel(const double2* __restrict__ C, int nk, int nao, int n, int K1,
                                typename PREC::T* __restrict__ Cb, long long sstride, const float* __restrict__ psc) {
  const float sc = PREC::kScaled ? *psc : 1.f;
  const long long total = (long long)nk * 2 * n * K1;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total;
       x += (long long)gridDim.x * blockDim.x) {
    const long long row = x / K1;
    const int col = (int)(x % K1);
    const int k = (int)(row / (2 * n));
    const int jp = (int)(row % (2 * n));
    const int j = jp >> 1, p = jp & 1;
    double v = 0.0;
    if (col < 2 * nao) {
      const int nu = col >> 1, c = col & 1;
      const double2 z = C[((long long)k * nao + nu) * n + j];
      v = p == 0 ? (c == 0 ? z.x : -z.y) : (c == 0 ? z.y : z.x);
    }
    const float2 f = scaled_ff(v, sc);
    typename PREC::T a[3];
    PREC::split(f.x, f.y, a);
#pragma unroll
    for (int t = 0; t < PREC::kSlices; ++t) Cb[x + t * sstride] = a[t];
  }
}

// Cc[t][slot * 2n + 2i + p][col], col = r * 2nao + 2 mu + c for r < nrep(slot):
//   p = 0: w_r (Cr, Ci)[c];  p = 1: w_r (-Ci, Cr)[c]  of C^{k1_r}_{mu i} (times sC); zero elsewhere.
template <class PREC>
__global__ void build_Cc_kernel(const double2* __restrict__ C, const int4* __restrict__ gather,
                                const int4* __restrict__ t2, int b0, int nq, int nao, int n, int K2,
                                typename PREC::T* __restrict__ Cc, long long sstride, const float* __restrict__ psc) {
  const float sc = PREC::kScaled ? *psc : 1.f;
  const long long total = (long long)nq * 2 * n * K2;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total;
       x += (long long)gridDim.x * blockDim.x) {
    const long long row = x / K2;
    const int col = (int)(x % K2);
    const int slot = (int)(row / (2 * n));
    const int ip = (int)(row % (2 * n));
    const int i = ip >> 1, p = ip & 1;
    const int4 q = t2[b0 + slot];  // {start, start, slot, nrep * nao}
    double v = 0.0;
    if (col < 2 * q.w) {
      const int r = col / (2 * nao);
      const int mu = (col % (2 * nao)) >> 1, c = col & 1;
      const int4 g = gather[q.x + r];  // {k1, half}
      const double w = g.y ? 0.5 : 1.0;
      const double2 z = C[((long long)g.x * nao + mu) * n + i];
      v = w * (p == 0 ? (c == 0 ? z.x : z.y) : (c == 0 ? -z.y : z.x));
    }
    const float2 f = scaled_ff(v, sc);
    typename PREC::T a[3];
    PREC::split(f.x, f.y, a);
#pragma unroll
    for (int t = 0; t < PREC::kSlices; ++t) Cc[x + t * sstride] = a[t];
  }
}

// Xt[t][IJ][row_base + (slot * naux + P) * nc + c] = split of sX (Z_ij + Z_ji).c for i >= j, where
// each real component of Z_ij (complex) is a two-float pair ZT[slot][(P n + j) 2n + 2i + (re|im)].
// (The factor s of L^q = s (Z + Z^T) is applied, squared, to the contraction's output.)
constexpr int PK_P = 64, PK_B = 4;
template <class PREC>
__global__ void __launch_bounds__(256) pack_split_kernel(const float2* __restrict__ ZT, int naux, int n, int nc,
                                                         typename PREC::T* __restrict__ Xt, long long sstride,
                                                         long long Rtot, long long row_base,
                                                         const float* __restrict__ psx) {
  const float sx = PREC::kScaled ? *psx : 1.f;
  // (re.hi, re.lo, im.hi, im.lo) of (pl, ii, jj) at [pl][ii * PK_B + jj]; the odd row pitch puts
  // consecutive pl (the lanes of the write phase) in different banks.
  constexpr int kPitch = PK_B * PK_B + 1;
  __shared__ float4 za[PK_P][kPitch];
  __shared__ float4 zb[PK_P][kPitch];
  // pair-block decode: lower triangle of ceil(n / PK_B) blocks
  const long long t = blockIdx.x;
  long long bi = (long long)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while (bi * (bi + 1) / 2 > t) --bi;
  while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
  const int bj = (int)(t - bi * (bi + 1) / 2);
  const int i0 = (int)bi * PK_B, j0 = bj * PK_B;
  const int P0 = blockIdx.y * PK_P;
  const int slot = blockIdx.z;
  const float4* z = reinterpret_cast<const float4*>(ZT + (long long)slot * naux * n * 2 * n);
  // All loads of a thread are issued before any is stored (256 threads).
  constexpr int kPer = PK_P * PK_B * PK_B / 256;
  float4 va[kPer], vb[kPer];
#pragma unroll
  for (int r = 0; r < kPer; ++r) {
    const int e = threadIdx.x + r * 256;
    const int pl = e / (PK_B * PK_B), a = (e / PK_B) % PK_B, b = e % PK_B;
    const int P = P0 + pl;
    // za[pl][ii][jj] = Z_{i j} with (ii, jj) = (b, a): consecutive e run over i for fixed j.
    va[r] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (P < naux && i0 + b < n && j0 + a < n) va[r] = z[((long long)P * n + j0 + a) * n + i0 + b];
    // zb[pl][ii][jj] = Z_{j i} with (ii, jj) = (a, b): consecutive e run over j for fixed i.
    vb[r] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (P < naux && i0 + a < n && j0 + b < n) vb[r] = z[((long long)P * n + i0 + a) * n + j0 + b];
  }
#pragma unroll
  for (int r = 0; r < kPer; ++r) {
    const int e = threadIdx.x + r * 256;
    const int pl = e / (PK_B * PK_B), a = (e / PK_B) % PK_B, b = e % PK_B;
    za[pl][b * PK_B + a] = va[r];
    zb[pl][a * PK_B + b] = vb[r];
  }
  __syncthreads();
  const int nr = PK_P * nc;  // rows per pair in this block
  for (int e = threadIdx.x; e < PK_B * PK_B * nr; e += blockDim.x) {
    const int pr = e / nr, rl = e % nr;
    const int ii = pr / PK_B, jj = pr % PK_B;
    const int i = i0 + ii, j = j0 + jj;
    const int pl = rl / nc, c = rl % nc;
    const int P = P0 + pl;
    if (i >= n || j > i || P >= naux) continue;
    const float4 a = za[pl][ii * PK_B + jj], b = zb[pl][ii * PK_B + jj];
    const float ah = c == 0 ? a.x : a.z, al = c == 0 ? a.y : a.w;
    const float bh = c == 0 ? b.x : b.z, bl = c == 0 ? b.y : b.w;
    // (ah + al) + (bh + bl) as a two-float pair: TwoSum of the leading parts.
    const float sh = ah + bh, bv = sh - ah;
    const float sl = ((ah - (sh - bv)) + (bh - bv)) + (al + bl);
    const long long IJ = (long long)i * (i + 1) / 2 + j;
    const long long idx = IJ * Rtot + row_base + ((long long)slot * naux + P) * nc + c;
    typename PREC::T x[3];
    PREC::split(sh * sx, sl * sx, x);
#pragma unroll
    for (int q = 0; q < PREC::kSlices; ++q) Xt[idx + q * sstride] = x[q];
  }
}

// General (complex) orbitals: the contraction operand of spin s holds 3 n^2 rows of Rtot columns.
// Rows ij = i n + j (the bra side) carry, in the K block of q (q * 2 naux), Re L^q_{P,ij} at P and
// Im L^q_{P,ij} at naux + P. Rows n^2 + 2 kl + c (the ket side) carry, in the K block of -q, the
// row of L^q_{P,kl} = y that turns the real dot product into component c of x y for the bra value
// x = L^{-q}: (Re y, -Im y) for c = 0 and (Im y, Re y) for c = 1, since Re(x y) = xr yr - xi yi and
// Im(x y) = xr yi + xi yr. Then (ij|kl) = (1/Nk) sum_q sum_P L^q_ij L^{-q}_kl is one real GEMM of
// the bra rows against the ket rows, whose output row ij is (ij|kl) as (re, im) doubles over kl.
// Z_ij of slot sl is the two-float pair ZT[sl][(P n + j) n + i] (re.hi, re.lo, im.hi, im.lo); the
// factor s of L^q = s Z is applied, squared, to the contraction's output. One block stages a tile
// of 32 P x 32 i at one j (reads coalesced over i), then writes runs of 32 consecutive P per row.
__device__ __forceinline__ float neg_of(float x) { return -x; }
__device__ __forceinline__ __half neg_of(__half x) { return __hneg(x); }
__device__ __forceinline__ __nv_bfloat16 neg_of(__nv_bfloat16 x) { return __hneg(x); }

constexpr int PC_T = 32;
template <class PREC>
__global__ void __launch_bounds__(256) pack_cplx_kernel(const float4* __restrict__ ZT, int naux, int n, int nq,
                                                        int q0, const int* __restrict__ neg,
                                                        typename PREC::T* __restrict__ Xt, long long sstride,
                                                        long long Rtot, const float* __restrict__ psx) {
  using T = typename PREC::T;
  const float sx = PREC::kScaled ? *psx : 1.f;
  __shared__ float4 z[PC_T][PC_T + 1];  // [i][P]
  const int itiles = (n + PC_T - 1) / PC_T;
  const int i0 = (blockIdx.x % itiles) * PC_T, j = blockIdx.x / itiles;
  const int P0 = blockIdx.y * PC_T;
  const int sl = blockIdx.z;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const float4* zs = ZT + (long long)sl * naux * n * n;
#pragma unroll
  for (int r = 0; r < PC_T / 8; ++r) {
    const int pl = ty + r * 8, P = P0 + pl, i = i0 + tx;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (P < naux && i < n) v = zs[((long long)P * n + j) * n + i];
    z[tx][pl] = v;
  }
  __syncthreads();
  const int q = q0 + sl, P = P0 + tx;
  if (P >= naux) return;
  const long long kb = (long long)q * 2 * naux + P, kn = (long long)neg[q] * 2 * naux + P;
  const long long n2 = (long long)n * n;
#pragma unroll
  for (int r = 0; r < PC_T / 8; ++r) {
    const int il = ty + r * 8, i = i0 + il;
    if (i >= n) break;
    const float4 v = z[il][tx];
    T re[3], im[3];
    PREC::split(v.x * sx, v.y * sx, re);
    PREC::split(v.z * sx, v.w * sx, im);
    const long long ij = (long long)i * n + j;
    T* a = Xt + ij * Rtot;
    T* b0 = Xt + (n2 + 2 * ij) * Rtot;
    T* b1 = b0 + Rtot;
#pragma unroll
    for (int t = 0; t < PREC::kSlices; ++t) {
      const long long o = t * sstride;
      a[o + kb] = re[t];
      a[o + kb + naux] = im[t];
      b0[o + kn] = re[t];
      b0[o + kn + naux] = neg_of(im[t]);
      b1[o + kn] = im[t];
      b1[o + kn + naux] = re[t];
    }
  }
}

// Step-1 output functor: element (m = (P, mu) of entry e, n = (j, p)) -> slices of A2 at
// row o2 + P * nemb + j, column k = o3 + 2 mu + p (o2 = slot * naux * nemb, o3 = r * 2 nao).
// A2 keeps the slices of a row side by side in each K block of BK elements,
// A2[row][k / BK][slice][k % BK] (a row is kSlices * K2 elements), so that the slice values a lane
// writes land in one span: with the slices in separate arrays the same bytes went to separate
// streams of short pieces and the step took a third longer. Step 2 reads the layout through a 4D
// tensor map (one slice of one K block per box).
template <class PREC>
struct EpiSplitT {
  using T = typename PREC::T;
  static constexpr int NS = PREC::kSlices;
  static constexpr int BK = tc::kblock_elems<PREC>();
  struct Params {
    T* out;
    long long K2;
    int nao, nemb;
  };
  static constexpr bool kStaged = false;  // lanes already write adjacent columns of one row
  static constexpr bool kAInterleaved = false;
  template <int H>
  static __device__ __forceinline__ void store(const Params& p, const tc::TcJob& j, int row, int col0,
                                               const float* hi, const float* lo) {
    const int m = j.o0 + row;
    const int P = m / p.nao, mu = m % p.nao;
    const long long rbase = (long long)j.o2 + (long long)P * p.nemb;
    const long long cidx = (long long)j.o3 + 2 * mu;
#pragma unroll
    for (int c = 0; c < H; c += 2) {
      if (col0 + c >= j.n_valid) break;
      const int jj = (j.o1 + col0 + c) >> 1;
      Pair2<T> pr[3];  // (re, im) of each slice
      split_pair<PREC>(hi[c], lo[c], hi[c + 1], lo[c + 1], pr);
      T* o = p.out + (rbase + jj) * NS * p.K2 + (cidx / BK) * (NS * BK) + (cidx % BK);
#pragma unroll
      for (int t = 0; t < NS; ++t) *reinterpret_cast<Pair2<T>*>(o + t * BK) = pr[t];
    }
  }
};

// Step-2 output functor: the two-float sum itself, out[(o0 + row) * ldo + o1 + col] = (hi, lo).
struct EpiPairs {
  static constexpr bool kAInterleaved = true;  // A = A2, written slice-interleaved by EpiSplitT
  struct Params {
    float2* out;
    long long ldo;
  };
  static constexpr bool kStaged = true;
  static __device__ __forceinline__ unsigned long long value(const Params&, const tc::TcJob&, float hi, float lo) {
    return (unsigned long long)__float_as_uint(hi) | ((unsigned long long)__float_as_uint(lo) << 32);
  }
  static __device__ __forceinline__ void put(const Params& p, const tc::TcJob& j, int row, int col,
                                             unsigned long long v) {
    if (row < j.m_valid && col < j.n_valid)
      p.out[((long long)j.o0 + row) * p.ldo + j.o1 + col] =
          make_float2(__uint_as_float((unsigned int)v), __uint_as_float((unsigned int)(v >> 32)));
  }
};

template <class PREC, int BN, class EPI>
cudaError_t launch_tc_bn(const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs, int njobs,
                         const tc::Segment* segs, const typename EPI::Params& ep, const tc::TcCtl& ctl, const float* fac,
                         cudaStream_t s, const tc::TcGroup<EPI>* groups = nullptr) {
  using Cfg = tc::TcCfg<PREC, BN, EPI::kStaged>;
  static bool attr = false;
  if (!attr) {
    // The register split inside the kernel assumes exactly kLaunchRegs registers per thread at
    // launch; with fewer, setmaxnreg.inc could never be satisfied, so refuse to launch.
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, tc::tc_gemm_kernel<PREC, BN, EPI>);
    if (e != cudaSuccess) return e;
    if (fa.numRegs != tc::kLaunchRegs) return cudaErrorInvalidKernelImage;
    e = cudaFuncSetAttribute(tc::tc_gemm_kernel<PREC, BN, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             Cfg::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (njobs <= 0) return cudaSuccess;
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
  }
  const int grid = njobs < nsm ? njobs : nsm;
  tc::tc_gemm_kernel<PREC, BN, EPI><<<grid, tc::kThreads, Cfg::SMEM, s>>>(A, B, jobs, njobs, segs, ep, ctl, fac,
                                                                          groups);
  return cudaGetLastError();
}

template <class PREC, class EPI>
cudaError_t launch_tc(int bn, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs, int njobs,
                      const tc::Segment* segs, const typename EPI::Params& ep, const tc::TcCtl& ctl, const float* fac,
                      cudaStream_t s) {
  switch (bn) {
    case 128: return launch_tc_bn<PREC, 128, EPI>(A, B, jobs, njobs, segs, ep, ctl, fac, s);
    case 112: return launch_tc_bn<PREC, 112, EPI>(A, B, jobs, njobs, segs, ep, ctl, fac, s);
    case 96: return launch_tc_bn<PREC, 96, EPI>(A, B, jobs, njobs, segs, ep, ctl, fac, s);
    default: return cudaErrorInvalidValue;
  }
}

// A grouped launch of the functor EPI: the maps, segments, factors and parameters come from the
// device table `groups`; the kernel's own map and parameter arguments are unused placeholders.
template <class PREC, class EPI>
cudaError_t launch_tc_group(int bn, const void* groups, const tc::TcJob* jobs, int njobs, const tc::TcCtl& ctl,
                            cudaStream_t s) {
  static const CUtensorMap none{};
  const typename EPI::Params ep{};
  const auto* g = static_cast<const tc::TcGroup<EPI>*>(groups);
  switch (bn) {
    case 128: return launch_tc_bn<PREC, 128, EPI>(none, none, jobs, njobs, nullptr, ep, ctl, nullptr, s, g);
    case 112: return launch_tc_bn<PREC, 112, EPI>(none, none, jobs, njobs, nullptr, ep, ctl, nullptr, s, g);
    case 96: return launch_tc_bn<PREC, 96, EPI>(none, none, jobs, njobs, nullptr, ep, ctl, nullptr, s, g);
    default: return cudaErrorInvalidValue;
  }
}

// Runs f(PREC{}) for this translation unit's precision code (dmet_prec_t); other codes are not
// compiled here.
template <class F>
cudaError_t with_prec(int prec, F&& f) {
  if (prec != DMET_ONE_PREC) return cudaErrorInvalidValue;
  return f(DMET_PREC_TYPE{});
}

// The split tiles of a packed contraction: tile t (its first part is jobs[t * f]) is the sum of
// its f K parts, part[t * f + p][row][col] = (hi, lo); the sum is formed with TwoSum, scaled as
// the contraction's own epilogue does, and stored where that epilogue would have stored it.
__global__ void __launch_bounds__(256) combine_parts_kernel(const tc::TcJob* __restrict__ jobs, int f,
                                                            const uint2* __restrict__ part, double* __restrict__ out,
                                                            float sh, float sl) {
  const tc::TcJob j = jobs[(long long)blockIdx.x * f];
  const int T = tc::kTile;
  for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < T * T; e += gridDim.y * blockDim.x) {
    const int row = e / T, col = e % T;
    if (row >= j.m_valid || col >= j.n_valid) continue;
    const long long m = (long long)j.o0 + row, n = (long long)j.o1 + col;
    if (n > m) continue;
    float hi = 0.f, lo = 0.f;
    for (int q = 0; q < f; ++q) {
      const uint2 v = part[((long long)blockIdx.x * f + q) * T * T + e];
      tc::two_sum_acc(hi, lo, __uint_as_float(v.x));
      lo += __uint_as_float(v.y);
    }
    out[m * (m + 1) / 2 + n] = tc::scaled_pair(hi, lo, sh, sl);
  }
}

// Largest |component| of the L blocks t1[e0 .. e0 + E).y, as float bits (atomicMax on the bits of a
// non-negative float orders like the value).
__global__ void __launch_bounds__(256) absmax_L_kernel(const double2* __restrict__ L, const int4* __restrict__ t1,
                                                       int e0, long long per_block, unsigned int* __restrict__ out) {
  const double2* src = L + (long long)t1[e0 + blockIdx.y].y * per_block;
  double m = 0.0;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < per_block;
       x += (long long)gridDim.x * blockDim.x) {
    const double2 v = src[x];
    m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
  }
  float mf = (float)m;
#pragma unroll
  for (int o = 16; o; o >>= 1) mf = fmaxf(mf, __shfl_xor_sync(0xffffffffu, mf, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(mf));
}

__global__ void __launch_bounds__(256) absmax_kernel(const double* __restrict__ x, long long n,
                                                     unsigned int* __restrict__ out) {
  double m = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    m = fmax(m, fabs(x[i]));
  float mf = (float)m;
#pragma unroll
  for (int o = 16; o; o >>= 1) mf = fmaxf(mf, __shfl_xor_sync(0xffffffffu, mf, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(mf));
}

// Power of two s = 2^e with b * s < 2^14 (b >= 0; s = 1 for b = 0), e clamped to FP32's range.
__device__ int scale_exp(double b) {
  if (!(b > 0.0)) return 0;
  int k = 0;
  frexp(b, &k);  // b = m 2^k, 0.5 <= m < 1, so b < 2^k
  const int e = 14 - k;
  return e < -120 ? -120 : (e > 120 ? 120 : e);
}

__device__ float pow2f(int e) {
  e = e < -126 ? -126 : (e > 127 ? 127 : e);
  return __uint_as_float((unsigned int)(e + 127) << 23);
}

// The FP16 precision's scales from the maxima in sc->mx: |L| <= mL, |C_s| <= mC_s component-wise;
// |T_s| <= 2 nao mL mC_s (a sum of 2 nao products); |Z_s| <= 2 nrep nao |T_s| mC_s (2 nrep nao
// products, orbital weights <= 1); |X_s| <= 2 |Z_s|.
__global__ void make_scales_kernel(MixScales* sc, int nao, int nrep_max, int nspin) {
  if (threadIdx.x || blockIdx.x) return;
  const double mL = (double)__uint_as_float(sc->mx[0]);
  const int eL = scale_exp(mL);
  int eC[2] = {0, 0}, eT[2] = {0, 0}, eX[2] = {0, 0};
  for (int s = 0; s < nspin; ++s) {
    const double mC = (double)__uint_as_float(sc->mx[1 + s]);
    const double bT = 2.0 * nao * mL * mC;
    const double bX = 2.0 * (2.0 * nrep_max * nao * bT * mC);
    eC[s] = scale_exp(mC);
    eT[s] = scale_exp(bT);
    eX[s] = scale_exp(bX);
  }
  sc->sL = pow2f(eL);
  for (int s = 0; s < 2; ++s) {
    sc->sC[s] = pow2f(eC[s]);
    sc->sT[s] = pow2f(eT[s]);
    sc->f1[s] = pow2f(eT[s] - eL - eC[s]);
    sc->f2[s] = pow2f(-eT[s] - eC[s]);
    sc->sX[s] = pow2f(eX[s]);
  }
  const int sa[3] = {0, 0, 1}, sb[3] = {0, 1, 1};
  for (int b = 0; b < 3; ++b) sc->fc[b] = pow2f(-eX[sa[b]] - eX[nspin == 2 ? sb[b] : 0]);
}

// Lq[P][i][j] = s (Z_ij + Z_ji) (conj: its complex conjugate) from the step-2 output of one slot,
// Z_ij = (re, im), each a two-float (hi, lo) at ZT[(P n + j) n + i] (a float4), summed exactly in FP64.
__global__ void lq_from_pairs_kernel(const float4* __restrict__ ZT, int naux, int n, double s, double sim, int pair,
                                     double2* __restrict__ Lq) {
  const long long nn = (long long)n * n, total = (long long)naux * nn;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total;
       x += (long long)gridDim.x * blockDim.x) {
    const long long P = x / nn;
    const int i = (int)((x % nn) / n), j = (int)(x % n);
    const float4 a = ZT[(P * n + j) * n + i];
    const float4 b = pair ? ZT[(P * n + i) * n + j] : make_float4(0.f, 0.f, 0.f, 0.f);
    const double re = ((double)a.x + (double)a.y) + ((double)b.x + (double)b.y);
    const double im = ((double)a.z + (double)a.w) + ((double)b.z + (double)b.w);
    Lq[x] = make_double2(s * re, sim * im);
  }
}

}  // namespace

#if DMET_PRIMARY_TU
cudaError_t launch_lq_from_pairs(const void* ZT, int naux, int n, double s, int conj, int pair, double2* Lq,
                                 cudaStream_t st) {
  const long long total = (long long)naux * n * n;
  lq_from_pairs_kernel<<<grid_for(total, 256, 152 * 16), 256, 0, st>>>((const float4*)ZT, naux, n, s, conj ? -s : s,
                                                                        pair, Lq);
  return cudaGetLastError();
}

cudaError_t launch_combine_parts(const tc::TcJob* jobs, int ntiles, int f, const void* part, double* out, double scale,
                                 cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  const float sh = (float)scale;
  combine_parts_kernel<<<dim3((unsigned)ntiles, 8), 256, 0, s>>>(jobs, f, (const uint2*)part, out, sh,
                                                                 (float)(scale - (double)sh));
  return cudaGetLastError();
}

int mixed_kblock() { return 32; }

bool prec_scaled(int prec) { return prec == DMET_PREC_FP16X2; }
int prec_slices(int prec) {
  return prec == DMET_PREC_BF16X3 ? 3 : (prec == DMET_PREC_TF32 ? 1 : 2);
}
int prec_products(int prec) {
  return prec == DMET_PREC_BF16X3 ? 6 : (prec == DMET_PREC_TF32 ? 1 : 3);
}
int prec_elem_bytes(int prec) { return (prec == DMET_PREC_TF32 || prec == DMET_PREC_TF32X3) ? 4 : 2; }

#endif  // DMET_PRIMARY_TU

cudaError_t DMET_P(launch_mix_scales)(int prec, const double2* L, const int4* t1, int E, long long per_block,
                              const double2* const* C, const long long* c_elems, int nspin, int nao, int nrep_max,
                              MixScales* sc, cudaStream_t s) {
  if (!prec_scaled(prec)) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(sc->mx, 0, sizeof(sc->mx), s);
  if (e != cudaSuccess) return e;
  for (int e0 = 0; e0 < E; e0 += 65535) {
    const int n = E - e0 < 65535 ? E - e0 : 65535;
    const long long gx = (152LL * 8 + n - 1) / n;
    absmax_L_kernel<<<dim3((unsigned)(gx > 1 ? gx : 1), (unsigned)n), 256, 0, s>>>(L, t1, e0, per_block, &sc->mx[0]);
  }
  for (int sp = 0; sp < nspin; ++sp)
    absmax_kernel<<<grid_for(2 * c_elems[sp], 256, 152 * 4), 256, 0, s>>>((const double*)C[sp], 2 * c_elems[sp],
                                                                           &sc->mx[1 + sp]);
  make_scales_kernel<<<1, 32, 0, s>>>(sc, nao, nrep_max, nspin);
  return cudaGetLastError();
}

cudaError_t DMET_P(launch_split_L)(int prec, const double2* L, const int4* t1, int e0, int E, int naux, int nao, int K1,
                           void* Ls, long long sstride, const MixScales* sc, cudaStream_t s) {
  if (E <= 0) return cudaSuccess;
  if ((long long)naux * nao * (K1 / 2) >= (1LL << 30) || E > 65535) return cudaErrorInvalidValue;
  // about 16 blocks of 256 threads per SM over all entries, at least one per entry
  const long long per_entry = (long long)naux * nao * (K1 / 2);
  long long gx = (152LL * 16 + E - 1) / E;
  const long long need = (per_entry + 1023) / 1024;  // four elements per thread at least
  if (gx > need) gx = need;
  if (gx < 1) gx = 1;
  return with_prec(prec, [&](auto tag) -> cudaError_t {
    using P = decltype(tag);
    split_L_kernel<P><<<dim3((unsigned)gx, (unsigned)E), 256, 0, s>>>(L, t1, e0, naux, nao, K1,
                                                                       (typename P::T*)Ls, sstride, sc);
    return cudaGetLastError();
  });
}

cudaError_t DMET_P(launch_build_Cb)(int prec, const double2* C, int nk, int nao, int n, int K1, void* Cb, long long sstride,
                            const float* sc, cudaStream_t s) {
  const long long total = (long long)nk * 2 * n * K1;
  return with_prec(prec, [&](auto tag) -> cudaError_t {
    using P = decltype(tag);
    build_Cb_kernel<P><<<grid_for(total, 256, 152 * 16), 256, 0, s>>>(C, nk, nao, n, K1, (typename P::T*)Cb, sstride,
                                                                      sc);
    return cudaGetLastError();
  });
}

cudaError_t DMET_P(launch_build_Cc)(int prec, const double2* C, const int4* gather, const int4* t2, int b0, int nq, int nao,
                            int n, int K2, void* Cc, long long sstride, const float* sc, cudaStream_t s) {
  const long long total = (long long)nq * 2 * n * K2;
  return with_prec(prec, [&](auto tag) -> cudaError_t {
    using P = decltype(tag);
    build_Cc_kernel<P><<<grid_for(total, 256, 152 * 16), 256, 0, s>>>(C, gather, t2, b0, nq, nao, n, K2,
                                                                      (typename P::T*)Cc, sstride, sc);
    return cudaGetLastError();
  });
}

cudaError_t DMET_P(launch_pack_split)(int prec, const void* ZT, int nq, int naux, int n, int nc, void* Xt, long long sstride,
                              long long Rtot, long long row_base, const float* sx, cudaStream_t s) {
  const long long nb = (n + PK_B - 1) / PK_B;
  const dim3 grid((unsigned)(nb * (nb + 1) / 2), (naux + PK_P - 1) / PK_P, nq);
  return with_prec(prec, [&](auto tag) -> cudaError_t {
    using P = decltype(tag);
    pack_split_kernel<P><<<grid, 256, 0, s>>>((const float2*)ZT, naux, n, nc, (typename P::T*)Xt, sstride, Rtot,
                                              row_base, sx);
    return cudaGetLastError();
  });
}

cudaError_t DMET_P(launch_pack_cplx)(int prec, const void* ZT, int nq, int naux, int n, int q0, const int* neg, void* Xt,
                             long long sstride, long long Rtot, const float* sx, cudaStream_t s) {
  const long long gx = (long long)((n + PC_T - 1) / PC_T) * n;
  if (gx > 0x7fffffffLL || nq > 65535 || (naux + PC_T - 1) / PC_T > 65535) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)gx, (naux + PC_T - 1) / PC_T, nq);
  return with_prec(prec, [&](auto tag) -> cudaError_t {
    using P = decltype(tag);
    pack_cplx_kernel<P><<<grid, 256, 0, s>>>((const float4*)ZT, naux, n, nq, q0, neg, (typename P::T*)Xt, sstride,
                                             Rtot, sx);
    return cudaGetLastError();
  });
}

cudaError_t DMET_P(launch_tc_split_t)(int prec, int bn, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs,
                              int njobs, const tc::Segment* segs, void* out, long long K2, int nao, int nemb,
                              const tc::TcCtl& ctl, const float* fac, cudaStream_t s) {
  return with_prec(prec, [&](auto tag) -> cudaError_t {
    using P = decltype(tag);
    typename EpiSplitT<P>::Params p{(typename P::T*)out, K2, nao, nemb};
    return launch_tc<P, EpiSplitT<P>>(bn, A, B, jobs, njobs, segs, p, ctl, fac, s);
  });
}

cudaError_t DMET_P(launch_tc_pairs)(int prec, int bn, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs,
                            int njobs, const tc::Segment* segs, void* out, long long ldo, const tc::TcCtl& ctl,
                            const float* fac, cudaStream_t s) {
  EpiPairs::Params p{(float2*)out, ldo};
  return with_prec(prec, [&](auto tag) -> cudaError_t {
    using P = decltype(tag);
    return launch_tc<P, EpiPairs>(bn, A, B, jobs, njobs, segs, p, ctl, fac, s);
  });
}

cudaError_t DMET_P(launch_tc_rect)(int prec, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs, int njobs,
                           const tc::Segment* segs, double* out, long long ldo, double scale, const tc::TcCtl& ctl,
                           const float* fac, cudaStream_t s) {
  const float sh = (float)scale;
  tc::EpiRect::Params p{out, ldo, sh, (float)(scale - (double)sh)};
  return with_prec(prec, [&](auto tag) -> cudaError_t {
    using P = decltype(tag);
    return launch_tc_bn<P, 128, tc::EpiRect>(A, B, jobs, njobs, segs, p, ctl, fac, s);
  });
}

// Host side of the grouped launches: the table entry of each kind, filled from a GroupSpec.
template <class EPI>
void fill_group(tc::TcGroup<EPI>* g, const GroupSpec& sp, const typename EPI::Params& ep) {
  std::memset((void*)g, 0, sizeof(*g));
  std::memcpy(&g->a, sp.a, sizeof(CUtensorMap));
  std::memcpy(&g->b, sp.b, sizeof(CUtensorMap));
  g->segs = sp.segs;
  g->fac = sp.fac;
  g->ep = ep;
}

size_t DMET_P(tc_group_bytes)(int kind, int prec) {
  size_t b = 0;
  with_prec(prec, [&](auto tag) -> cudaError_t {
    using P = decltype(tag);
    b = kind == kGroupSplitT ? sizeof(tc::TcGroup<EpiSplitT<P>>)
                             : (kind == kGroupPairs ? sizeof(tc::TcGroup<EpiPairs>) : sizeof(tc::TcGroup<tc::EpiAny>));
    return cudaSuccess;
  });
  return b;
}

cudaError_t DMET_P(tc_group_fill)(int kind, int prec, const GroupSpec* specs, int count, void* dst) {
  return with_prec(prec, [&](auto tag) -> cudaError_t {
    using P = decltype(tag);
    for (int i = 0; i < count; ++i) {
      const GroupSpec& sp = specs[i];
      if (kind == kGroupSplitT) {
        typename EpiSplitT<P>::Params ep{(typename P::T*)sp.out, sp.ld, sp.nao, sp.n};
        fill_group(static_cast<tc::TcGroup<EpiSplitT<P>>*>(dst) + i, sp, ep);
      } else if (kind == kGroupPairs) {
        EpiPairs::Params ep{(float2*)sp.out, sp.ld};
        fill_group(static_cast<tc::TcGroup<EpiPairs>*>(dst) + i, sp, ep);
      } else if (kind == kGroupContract) {
        const float sh = (float)sp.scale;
        tc::EpiAny::Params ep{sp.outp, nullptr, sp.ld, sh, (float)(sp.scale - (double)sh), sp.mode};
        fill_group(static_cast<tc::TcGroup<tc::EpiAny>*>(dst) + i, sp, ep);
      } else {
        return cudaErrorInvalidValue;
      }
    }
    return cudaSuccess;
  });
}

cudaError_t DMET_P(launch_tc_grouped)(int kind, int prec, int bn, const void* groups, const tc::TcJob* jobs, int njobs,
                              const tc::TcCtl& ctl, cudaStream_t s) {
  return with_prec(prec, [&](auto tag) -> cudaError_t {
    using P = decltype(tag);
    if (kind == kGroupSplitT) return launch_tc_group<P, EpiSplitT<P>>(bn, groups, jobs, njobs, ctl, s);
    if (kind == kGroupPairs) return launch_tc_group<P, EpiPairs>(bn, groups, jobs, njobs, ctl, s);
    if (kind == kGroupContract && bn == 128) return launch_tc_group<P, tc::EpiAny>(128, groups, jobs, njobs, ctl, s);
    return cudaErrorInvalidValue;
  });
}

cudaError_t DMET_P(launch_tc_herm)(int prec, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs, int njobs,
                           const tc::Segment* segs, double* out, long long n2, double scale, const tc::TcCtl& ctl,
                           const float* fac, cudaStream_t s) {
  const float sh = (float)scale;
  tc::EpiHerm::Params p{out, 2 * n2, sh, (float)(scale - (double)sh)};
  return with_prec(prec, [&](auto tag) -> cudaError_t {
    using P = decltype(tag);
    return launch_tc_bn<P, 128, tc::EpiHerm>(A, B, jobs, njobs, segs, p, ctl, fac, s);
  });
}

cudaError_t DMET_P(launch_tc_packed)(int prec, const CUtensorMap& A, const CUtensorMap& B, const tc::TcJob* jobs, int njobs,
                             const tc::Segment* segs, double* out, double scale, void* part, const tc::TcCtl& ctl,
                             const float* fac, cudaStream_t s) {
  const float sh = (float)scale;
  tc::EpiPacked::Params p{out, sh, (float)(scale - (double)sh), (unsigned long long*)part};
  return with_prec(prec, [&](auto tag) -> cudaError_t {
    using P = decltype(tag);
    return launch_tc_bn<P, 128, tc::EpiPacked>(A, B, jobs, njobs, segs, p, ctl, fac, s);
  });
}

}  // namespace dmet
