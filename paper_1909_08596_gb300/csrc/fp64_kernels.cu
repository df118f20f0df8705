// FP64 kernels of the embedded-ERI transformation (Algorithm 1, section 2.1).
//
// GB300 executes FP64 fused multiply-adds on the CUDA cores at a small fraction of its
// FP32 rate, so the plain-FP64 path is bound by the DFMA pipe, not by memory: every
// kernel here keeps its operands in shared memory and registers and spends its issue
// slots on DFMAs. Tiles are 64x64 outputs per 256-thread CTA (4x4 outputs per thread);
// a warp owns 8 consecutive rows of the tile and skips its FMAs when all of them lie
// past the matrix edge, so small dimensions (n_emb) waste no DFMAs beyond a multiple of 8.

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "internal.h"

namespace dmet {

namespace {

constexpr int TM = 64;   // tile rows
constexpr int TN = 64;   // tile columns
constexpr int ZBK = 8;   // complex k-step
constexpr int DBK = 16;  // real k-step

__device__ __forceinline__ long long map2(int x, int div, long long hi, long long lo) {
  return (long long)(x / div) * hi + (long long)(x % div) * lo;
}

template <int AL, bool CJ, int BL>
__global__ void __launch_bounds__(256, 2) zgemm_fp64_kernel(const ZgemmArgs d) {
  __shared__ __align__(16) double2 As[ZBK][TM];
  __shared__ __align__(16) double2 Bs[ZBK][TN];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  if (d.lower && n0 >= m0 + TM) return;  // the whole CTA leaves together
  const double2* A = d.A;
  const double2* B = d.B;
  double2* D = d.D;
  int K = d.K;
  if (d.tab) {
    const int4 e = d.tab[d.tab0 + blockIdx.z];
    A += e.x * d.sA;
    B += e.y * d.sB;
    D += e.z * d.sD;
    K = e.w;
  } else {
    A += (long long)blockIdx.z * d.sA;
    B += (long long)blockIdx.z * d.sB;
    D += (long long)blockIdx.z * d.sD;
  }
  const bool active = (m0 + (tid >> 5) * 8) < d.M;

  double2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);

  for (int k0 = 0; k0 < K; k0 += ZBK) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int e = tid + r * 256;
      int kk, mm, nn;
      if (AL == A_KM) { kk = e >> 6; mm = e & 63; } else { mm = e >> 3; kk = e & 7; }
      int gk = k0 + kk, gm = m0 + mm;
      double2 v = make_double2(0.0, 0.0);
      if (gk < K && gm < d.M) v = (AL == A_KM) ? A[gk * d.lda + gm] : A[gm * d.lda + gk];
      if (CJ) v.y = -v.y;
      As[kk][mm] = v;
      if (BL == B_KN) { kk = e >> 6; nn = e & 63; } else { nn = e >> 3; kk = e & 7; }
      gk = k0 + kk;
      const int gn = n0 + nn;
      double2 w = make_double2(0.0, 0.0);
      if (gk < K && gn < d.N) w = (BL == B_KN) ? B[gk * d.ldb + gn] : B[gn * d.ldb + gk];
      Bs[kk][nn] = w;
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int kk = 0; kk < ZBK; ++kk) {
        double2 a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            acc[i][j].x = fma(a[i].x, b[j].x, acc[i][j].x);
            acc[i][j].x = fma(-a[i].y, b[j].y, acc[i][j].x);
            acc[i][j].y = fma(a[i].x, b[j].y, acc[i][j].y);
            acc[i][j].y = fma(a[i].y, b[j].x, acc[i][j].y);
          }
      }
    }
    __syncthreads();
  }
  if (!active) return;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= d.M) continue;
    const long long rm = map2(m, d.dm_div, d.dm_hi, d.dm_lo);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= d.N) continue;
      const long long addr = rm + map2(n, d.dn_div, d.dn_hi, d.dn_lo);
      double2 v = make_double2(d.alpha * acc[i][j].x, d.alpha * acc[i][j].y);
      if (d.beta) {
        const double2 o = D[addr];
        v.x += o.x;
        v.y += o.y;
      }
      D[addr] = v;
    }
  }
}

__global__ void __launch_bounds__(256, 2) dsyrk_fp64_kernel(const DsyrkArgs d) {
  __shared__ __align__(16) double Xs[DBK][TM];
  __shared__ __align__(16) double Ys[DBK][TN];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  int m0, n0;
  if (d.mode == 0) {
    const long long t = blockIdx.x;
    long long ti = (long long)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (ti * (ti + 1) / 2 > t) --ti;
    while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
    m0 = (int)ti * TM;
    n0 = (int)(t - ti * (ti + 1) / 2) * TN;
  } else {
    m0 = blockIdx.y * TM;
    n0 = blockIdx.x * TN;
  }
  const double* Y = d.mode == 0 ? d.X : d.Y;
  const long long ldy = d.mode == 0 ? d.ldx : d.ldy;
  const int wrow = m0 + (tid >> 5) * 8;
  // In the packed mode a warp whose 8 rows all lie above the tile's columns has no m >= n.
  const bool active = wrow < d.M && (d.mode != 0 || wrow + 7 >= n0);

  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int k0 = 0; k0 < d.K; k0 += DBK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + r * 256;
      const int kk = e >> 6, mm = e & 63;
      const int gk = k0 + kk;
      double v = 0.0, w = 0.0;
      if (gk < d.K && m0 + mm < d.M) v = d.X[gk * d.ldx + m0 + mm];
      if (gk < d.K && n0 + mm < d.N) w = Y[gk * ldy + n0 + mm];
      Xs[kk][mm] = v;
      Ys[kk][mm] = w;
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int kk = 0; kk < DBK; ++kk) {
        double a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = Xs[kk][ty * 4 + i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Ys[kk][tx * 4 + j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
    }
    __syncthreads();
  }
  if (!active) return;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= d.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= d.N) continue;
      long long addr;
      if (d.mode == 0) {
        if (n > m) continue;
        addr = (long long)m * (m + 1) / 2 + n;
      } else {
        addr = (long long)m * d.ldo + n;
      }
      d.out[addr] += d.alpha * acc[i][j];
    }
  }
}

__global__ void gather_orbitals_kernel(const double2* __restrict__ C, double2* __restrict__ Crep,
                                       const int4* __restrict__ tab, int tab0, int nao, int n) {
  const int e = blockIdx.y;
  const int4 t = tab[tab0 + e];
  const double w = t.y ? 0.5 : 1.0;
  const long long sz = (long long)nao * n;
  const double2* src = C + t.x * sz;
  double2* dst = Crep + e * sz;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < sz;
       x += (long long)gridDim.x * blockDim.x) {
    const double2 v = src[x];
    dst[x] = make_double2(w * v.x, w * v.y);
  }
}

__device__ __forceinline__ void pair_of(long long ij, int& i, int& j) {
  long long r = (long long)((sqrt(8.0 * (double)ij + 1.0) - 1.0) * 0.5);
  while (r * (r + 1) / 2 > ij) --r;
  while ((r + 1) * (r + 2) / 2 <= ij) ++r;
  i = (int)r;
  j = (int)(ij - r * (r + 1) / 2);
}

__global__ void pack_pairs_kernel(const double2* __restrict__ Z, double* __restrict__ X, int nq, int naux,
                                  int n, int nc, double s) {
  const long long npair = (long long)n * (n + 1) / 2;
  const long long total = (long long)nq * naux * nc * npair;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total;
       x += (long long)gridDim.x * blockDim.x) {
    const long long ij = x % npair;
    const long long row = x / npair;  // (q, P, c)
    const int c = (int)(row % nc);
    const long long qp = row / nc;    // q * naux + P
    int i, j;
    pair_of(ij, i, j);
    const double2* z = Z + qp * n * (long long)n;
    const double2 a = z[(long long)i * n + j], b = z[(long long)j * n + i];
    X[x] = s * (c == 0 ? a.x + b.x : a.y + b.y);
  }
}

__global__ void symmetrize_kernel(const double2* __restrict__ Z, double2* __restrict__ Lq, int nq, int naux,
                                  int n, double s, double sim) {
  const long long nn = (long long)n * n;
  const long long total = (long long)nq * naux * nn;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total;
       x += (long long)gridDim.x * blockDim.x) {
    const long long base = x - x % nn;
    const int i = (int)((x % nn) / n), j = (int)(x % n);
    const double2 a = Z[x], b = Z[base + (long long)j * n + i];
    Lq[x] = make_double2(s * (a.x + b.x), sim * (a.y + b.y));
  }
}

// Max of non-negative doubles through their bit patterns (NaN compares above +inf).
__device__ __forceinline__ double wmax(double a, double b) { return (isnan(a) || a > b) ? a : b; }

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = wmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ void atomic_max_nonneg(double* p, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(p), (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ void block_max_commit(double v, double* out) {
  __shared__ double red[32];
  v = warp_max(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    v = warp_max(v);
    if (lane == 0) atomic_max_nonneg(out, v);
  }
  __syncthreads();
}

// S = s * sum_g S_g (ng split-K partial products of C^+ C); stat = max |S_ij - delta_ij| over
// the lower triangle j <= i (S is Hermitian, and only those tiles of S_g are computed).
__global__ void orth_reduce_kernel(const double2* __restrict__ Sg, int ng, int n, double s, double* stat) {
  double v = 0.0;
  const long long nn = (long long)n * n;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < nn;
       x += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(x / n), j = (int)(x % n);
    if (j > i) continue;
    double re = 0.0, im = 0.0;
    for (int g = 0; g < ng; ++g) {
      const double2 e = Sg[g * nn + x];
      re += e.x;
      im += e.y;
    }
    re = s * re - (i == j ? 1.0 : 0.0);
    im = s * im;
    v = wmax(v, sqrt(re * re + im * im));
  }
  block_max_commit(v, stat);
}

__global__ void c_real_check_kernel(const double2* __restrict__ C, const int* __restrict__ neg, int nk,
                                    int nao, int n, double* stats) {
  double dv = 0.0, mv = 0.0;
  const long long per = (long long)nao * n, total = per * nk;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total;
       x += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(x / per);
    const double2 a = C[x], b = C[neg[k] * per + x % per];
    const double dr = b.x - a.x, di = b.y + a.y;
    dv = wmax(dv, sqrt(dr * dr + di * di));
    mv = wmax(mv, sqrt(a.x * a.x + a.y * a.y));
  }
  block_max_commit(dv, stats + 1);
  block_max_commit(mv, stats + 2);
}

// |x| of a double as its bit pattern with the sign cleared: for non-negative doubles the
// integer order is the numeric order (NaN patterns sort above +inf).
__device__ __forceinline__ unsigned long long abits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

__device__ __forceinline__ unsigned long long warp_umax(unsigned long long v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// Symmetries of L over a chunk of aux indices of one k pair (k1, k2): Hermiticity against
// L[k2][k1][P][nu][mu] (checked once per unordered pair, k1 <= k2) and time reversal against
// L[-k1][-k2][P][mu][nu] (checked once per pair of pairs). The transposed partner is read
// through the read-only cache, where the block's other warps have brought its lines.
// Records max-norm differences (component-wise) and max |L| (component-wise) as bit patterns.
constexpr int LCHK_P = 8;
__global__ void __launch_bounds__(256) l_check_kernel(const double2* __restrict__ L, const int* __restrict__ neg,
                                                      int nk, int naux, int nao, double* stats) {
  const int pchunks = (naux + LCHK_P - 1) / LCHK_P;
  const long long nwork = (long long)nk * nk * pchunks;
  unsigned long long hv = 0, tv = 0, mv = 0;
  for (long long w = blockIdx.x; w < nwork; w += gridDim.x) {
    const long long kk = w / pchunks;
    const int P0 = (int)(w % pchunks) * LCHK_P;
    const int k1 = (int)(kk / nk), k2 = (int)(kk % nk);
    const long long kt = (long long)neg[k1] * nk + neg[k2];
    const bool do_h = k1 <= k2, do_t = kk <= kt;
    const long long blk = (long long)nao * nao, pair = blk * naux;
    const double2* a_pair = L + kk * pair;
    const double2* h_pair = L + ((long long)k2 * nk + k1) * pair;
    const double2* t_pair = L + kt * pair;
    const int pend = min(naux, P0 + LCHK_P);
    for (int P = P0; P < pend; ++P) {
      const long long base = (long long)P * blk;
      for (long long e = threadIdx.x; e < blk; e += blockDim.x) {
        const double2 a = a_pair[base + e];
        mv = max(mv, max(abits(a.x), abits(a.y)));
        if (do_h) {
          const int mu = (int)(e / nao), nu = (int)(e % nao);
          const double2 h = __ldg(h_pair + base + (long long)nu * nao + mu);
          hv = max(hv, max(abits(h.x - a.x), abits(h.y + a.y)));
        }
        if (do_t) {
          const double2 t = t_pair[base + e];
          tv = max(tv, max(abits(t.x - a.x), abits(t.y + a.y)));
        }
      }
    }
  }
  hv = warp_umax(hv);
  tv = warp_umax(tv);
  mv = warp_umax(mv);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(reinterpret_cast<unsigned long long*>(stats + 3), hv);
    atomicMax(reinterpret_cast<unsigned long long*>(stats + 4), tv);
    atomicMax(reinterpret_cast<unsigned long long*>(stats + 5), mv);
  }
}

inline int grid_for(long long total, int threads, int cap) {
  long long g = (total + threads - 1) / threads;
  if (g < 1) g = 1;
  return (int)(g < cap ? g : cap);
}

// Largest t with t(t+1)/2 <= x (the row of a lower-triangle index), exact for x < 2^50.
__device__ __forceinline__ long long tri_row(long long x) {
  long long t = (long long)((sqrt(8.0 * (double)x + 1.0) - 1.0) * 0.5);
  while (t * (t + 1) / 2 > x) --t;
  while ((t + 1) * (t + 2) / 2 <= x) ++t;
  return t;
}

// out[pos] = full[i][j][k][l] for the (i, j, k, l) that packed position pos stands for.
__global__ void pack_s4_kernel(const double2* __restrict__ full, int na, int nb, int rect, double2* __restrict__ out) {
  const long long np = (long long)na * (na + 1) / 2, ns = (long long)na * (na - 1) / 2;
  const long long nA = np * (np + 1) / 2;
  const long long total = rect ? np * nb * nb : nA + ns * (ns + 1) / 2;
  const long long nb2 = (long long)nb * nb;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total;
       x += (long long)gridDim.x * blockDim.x) {
    long long i, j, k, l;
    if (rect) {
      const long long I = x / nb2, kl = x % nb2;
      i = tri_row(I);
      j = I - i * (i + 1) / 2;
      k = kl / nb;
      l = kl % nb;
    } else if (x < nA) {
      const long long I = tri_row(x), K = x - I * (I + 1) / 2;
      i = tri_row(I);
      j = I - i * (i + 1) / 2;
      k = tri_row(K);
      l = K - k * (k + 1) / 2;
    } else {
      // a = i(i-1)/2 + j with i > j, b = l(l-1)/2 + k with l > k
      const long long y = x - nA, a = tri_row(y), b = y - a * (a + 1) / 2;
      i = tri_row(a) + 1;
      j = a - i * (i - 1) / 2;
      l = tri_row(b) + 1;
      k = b - l * (l - 1) / 2;
    }
    out[x] = full[((i * na + j) * nb + k) * nb + l];
  }
}

}  // namespace

cudaError_t launch_zgemm(const ZgemmArgs& a, int a_layout, bool conj_a, int b_layout, cudaStream_t s) {
  if (a.M <= 0 || a.N <= 0 || a.batch <= 0) return cudaSuccess;
  const dim3 grid((a.N + TN - 1) / TN, (a.M + TM - 1) / TM, a.batch);
  if (a_layout == A_KM && conj_a && b_layout == B_KN)
    zgemm_fp64_kernel<A_KM, true, B_KN><<<grid, 256, 0, s>>>(a);
  else if (a_layout == A_KM && !conj_a && b_layout == B_KN)
    zgemm_fp64_kernel<A_KM, false, B_KN><<<grid, 256, 0, s>>>(a);
  else if (a_layout == A_KM && !conj_a && b_layout == B_NK)
    zgemm_fp64_kernel<A_KM, false, B_NK><<<grid, 256, 0, s>>>(a);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_dsyrk(const DsyrkArgs& a, cudaStream_t s) {
  if (a.M <= 0 || a.N <= 0) return cudaSuccess;
  dim3 grid;
  if (a.mode == 0) {
    const long long nt = (a.M + TM - 1) / TM;
    grid = dim3((unsigned)(nt * (nt + 1) / 2), 1, 1);
  } else {
    grid = dim3((a.N + TN - 1) / TN, (a.M + TM - 1) / TM, 1);
  }
  dsyrk_fp64_kernel<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_gather_orbitals(const double2* C, double2* Crep, const int4* tab, int tab0, int n_entries,
                                   int nao, int n, cudaStream_t s) {
  if (n_entries <= 0) return cudaSuccess;
  const dim3 grid(grid_for((long long)nao * n, 256, 64), n_entries, 1);
  gather_orbitals_kernel<<<grid, 256, 0, s>>>(C, Crep, tab, tab0, nao, n);
  return cudaGetLastError();
}

cudaError_t launch_pack_pairs(const double2* Z, double* X, int nq, int naux, int n, int nc, double sc,
                              cudaStream_t s) {
  const long long total = (long long)nq * naux * nc * ((long long)n * (n + 1) / 2);
  pack_pairs_kernel<<<grid_for(total, 256, 152 * 16), 256, 0, s>>>(Z, X, nq, naux, n, nc, sc);
  return cudaGetLastError();
}

cudaError_t launch_symmetrize(const double2* Z, double2* Lq, int nq, int naux, int n, double sc, int conj,
                              cudaStream_t s) {
  const long long total = (long long)nq * naux * n * n;
  symmetrize_kernel<<<grid_for(total, 256, 152 * 16), 256, 0, s>>>(Z, Lq, nq, naux, n, sc, conj ? -sc : sc);
  return cudaGetLastError();
}

cudaError_t launch_orth_reduce(const double2* Sg, int ng, int n, double sc, double* stat, cudaStream_t s) {
  orth_reduce_kernel<<<grid_for((long long)n * n, 256, 152), 256, 0, s>>>(Sg, ng, n, sc, stat);
  return cudaGetLastError();
}

cudaError_t launch_c_real_check(const double2* C, const int* neg, int nk, int nao, int n, double* stats,
                                cudaStream_t s) {
  c_real_check_kernel<<<grid_for((long long)nk * nao * n, 256, 152 * 4), 256, 0, s>>>(C, neg, nk, nao, n,
                                                                                        stats);
  return cudaGetLastError();
}

cudaError_t launch_l_check(const double2* L, const int* neg, int nk, int naux, int nao, double* stats,
                           cudaStream_t s) {
  const long long pchunks = (naux + LCHK_P - 1) / LCHK_P;
  const long long nwork = (long long)nk * nk * pchunks;
  l_check_kernel<<<(unsigned)(nwork < (1LL << 30) ? nwork : (1LL << 30)), 256, 0, s>>>(L, neg, nk, naux, nao, stats);
  return cudaGetLastError();
}

cudaError_t launch_pack_s4(const double2* full, int na, int nb, int rect, double2* out, cudaStream_t st) {
  const long long np = (long long)na * (na + 1) / 2, ns = (long long)na * (na - 1) / 2;
  const long long total = rect ? np * nb * nb : np * (np + 1) / 2 + ns * (ns + 1) / 2;
  pack_s4_kernel<<<grid_for(total, 256, 152 * 16), 256, 0, st>>>(full, na, nb, rect, out);
  return cudaGetLastError();
}

}  // namespace dmet
