// DMET bath and embedding orbitals (section 2.1): the environment-impurity block of the
// mean-field density matrix brought to real space (Eq. "bath R SVD" needs gamma^{R != 0, 0}),
// its singular value decomposition by one-sided Jacobi rotations, the block form of Eq.
// "C loemb R" and the two transformations of Eq. "C loemb k". FP64 throughout.

#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <stdint.h>

#include "internal.h"

namespace dmet {

namespace {

// k.R in units of 2 pi / Nk: sum_d (n_d m_d mod N_d) Nk / N_d, exact in integers (C-order index).
__device__ __forceinline__ int k_dot_r(int k, int r, int n1, int n2, int n3) {
  const int k1 = k / (n2 * n3), k2 = (k / n3) % n2, k3 = k % n3;
  const int r1 = r / (n2 * n3), r2 = (r / n3) % n2, r3 = r % n3;
  const int nk = n1 * n2 * n3;
  return (((k1 * r1) % n1) * (nk / n1) + ((k2 * r2) % n2) * (nk / n2) + ((k3 * r3) % n3) * (nk / n3)) % nk;
}

// Non-negative doubles order like their bit patterns.
__device__ __forceinline__ void atomic_max_nonneg(double* p, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(p), (unsigned long long)__double_as_longlong(v));
}

// A[c][r] = Re gamma^{R,0}_{i, val[c]}, r = (R - 1) n_lo + i for the cells R = 1 .. Nk - 1, with
// gamma^{R,0} = (1/Nk) sum_k exp(+i k.R) gamma^k. stats[0] / stats[1] collect the largest |Re| and
// |Im| of the block.
__global__ void __launch_bounds__(256) bath_offdiag_kernel(const double2* __restrict__ gk, int n1, int n2, int n3,
                                                           int n_lo, BathCols val, double* __restrict__ A,
                                                           double* __restrict__ stats) {
  const int nk = n1 * n2 * n3;
  const long long m = (long long)(nk - 1) * n_lo, total = m * val.n;
  const double inv = 1.0 / nk;
  double mre = 0.0, mim = 0.0;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total; x += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(x / m);
    const int r = (int)(x % m);
    const int R = 1 + r / n_lo, i = r % n_lo, j = val.v[c];
    double re = 0.0, im = 0.0;
    for (int k = 0; k < nk; ++k) {
      double s, co;
      sincospi(2.0 * k_dot_r(k, R, n1, n2, n3) * inv, &s, &co);
      const double2 g = gk[((long long)k * n_lo + i) * n_lo + j];
      re = fma(g.x, co, fma(-g.y, s, re));
      im = fma(g.x, s, fma(g.y, co, im));
    }
    re *= inv;
    im *= inv;
    A[x] = re;
    mre = fmax(mre, fabs(re));
    mim = fmax(mim, fabs(im));
  }
  for (int o = 16; o; o >>= 1) {
    mre = fmax(mre, __shfl_xor_sync(0xffffffffu, mre, o));
    mim = fmax(mim, __shfl_xor_sync(0xffffffffu, mim, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(&stats[0], mre);
    atomic_max_nonneg(&stats[1], mim);
  }
}

constexpr int kJacobiThreads = 512;
constexpr int kJacobiWarps = kJacobiThreads / 32;
constexpr int kMaxSweeps = 40;
constexpr double kRotTol = 1e-14;  // rotate a pair while |a_p.a_q| > kRotTol ||a_p|| ||a_q||

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One-sided Jacobi SVD (Hestenes 1958; the rotation angle as in Rutishauser's symmetric Jacobi
// method) of the m x n_val block A (column-major), in one CTA. Sweeps visit every column pair in
// n_pad - 1 rounds of the round-robin ordering (n_pad = n_val rounded up to even; the pad column
// is an all-zero column and never rotates), one warp per pair of a round. After convergence
// column c is sigma_c u_c. The columns are written in decreasing sigma, each scaled by
// sign / sigma with the sign that makes its largest-magnitude entry (the first of equal ones)
// positive: B[r][rank] = u. A zero singular value leaves a zero column. stats[2] = sweeps,
// stats[3] = largest pair cosine |a_p.a_q| / (||a_p|| ||a_q||) of the last sweep,
// stats[4] = sigma_min / sigma_max.
__global__ void __launch_bounds__(kJacobiThreads) bath_jacobi_kernel(double* __restrict__ Ag, int m, int n_val,
                                                                     int in_smem, double* __restrict__ B,
                                                                     double* __restrict__ sigma_out,
                                                                     double* __restrict__ stats) {
  extern __shared__ double sm[];
  __shared__ double s_sigma[kMaxBathCols];
  __shared__ int s_rank[kMaxBathCols];
  __shared__ int s_rot;
  __shared__ double s_off[kJacobiWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* A = Ag;
  if (in_smem) {
    A = sm;
    for (long long x = threadIdx.x; x < (long long)m * n_val; x += blockDim.x) A[x] = Ag[x];
  }
  __syncthreads();
  const int n_pad = n_val + (n_val & 1);
  const int half = n_pad / 2;
  int sweeps = 0;
  double off = 0.0;
  for (int sweep = 0; sweep < kMaxSweeps && n_val > 1; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    double woff = 0.0;
    __syncthreads();
    for (int round = 0; round < n_pad - 1; ++round) {
      for (int j = warp; j < half; j += kJacobiWarps) {
        // round-robin: position n_pad - 1 stays, the others turn one step per round
        int p = j == 0 ? n_pad - 1 : (round + j) % (n_pad - 1);
        int q = j == 0 ? round : (round - j + n_pad - 1) % (n_pad - 1);
        if (p >= n_val || q >= n_val) continue;
        double* ap = A + (long long)p * m;
        double* aq = A + (long long)q * m;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int r = lane; r < m; r += 32) {
          const double x = ap[r], y = aq[r];
          al = fma(x, x, al);
          be = fma(y, y, be);
          ga = fma(x, y, ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        const double nrm = sqrt(al) * sqrt(be);
        if (!(nrm > 0.0)) continue;
        const double cosine = fabs(ga) / nrm;
        woff = fmax(woff, cosine);
        if (cosine <= kRotTol) continue;
        // t = tan of the angle that makes the rotated columns orthogonal: the root of smaller
        // magnitude of t^2 + 2 zeta t - 1 = 0, zeta = (be - al) / (2 ga)
        const double zeta = (be - al) / (2.0 * ga);
        const double t = fabs(zeta) > 1e150 ? 0.5 / zeta
                                            : copysign(1.0, zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
        const double c = 1.0 / sqrt(fma(t, t, 1.0)), s = c * t;
        for (int r = lane; r < m; r += 32) {
          const double x = ap[r], y = aq[r];
          ap[r] = fma(c, x, -s * y);
          aq[r] = fma(s, x, c * y);
        }
        if (lane == 0) s_rot = 1;
      }
      __syncthreads();
    }
    if (lane == 0) s_off[warp] = woff;
    __syncthreads();
    ++sweeps;
    off = 0.0;
    for (int w = 0; w < kJacobiWarps; ++w) off = fmax(off, s_off[w]);
    const int rotated = s_rot;
    __syncthreads();
    if (!rotated) break;
  }
  // singular values and their ranks (decreasing; equal values keep column order)
  for (int c = warp; c < n_val; c += kJacobiWarps) {
    const double* ac = A + (long long)c * m;
    double ss = 0.0;
    for (int r = lane; r < m; r += 32) ss = fma(ac[r], ac[r], ss);
    ss = warp_sum(ss);
    if (lane == 0) s_sigma[c] = sqrt(ss);
  }
  __syncthreads();
  if (threadIdx.x < n_val) {
    const int c = threadIdx.x;
    const double sc = s_sigma[c];
    int rk = 0;
    for (int d = 0; d < n_val; ++d) rk += (s_sigma[d] > sc) || (s_sigma[d] == sc && d < c);
    s_rank[c] = rk;
    if (sigma_out) sigma_out[rk] = sc;
  }
  __syncthreads();
  for (int c = warp; c < n_val; c += kJacobiWarps) {
    const double* ac = A + (long long)c * m;
    double best = -1.0;
    int at = 0;
    for (int r = lane; r < m; r += 32) {
      const double v = fabs(ac[r]);
      if (v > best) {
        best = v;
        at = r;
      }
    }
    for (int o = 16; o; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oa = __shfl_xor_sync(0xffffffffu, at, o);
      if (ob > best || (ob == best && oa < at)) {
        best = ob;
        at = oa;
      }
    }
    const double sg = s_sigma[c];
    const double scale = sg > 0.0 ? (ac[at] < 0.0 ? -1.0 : 1.0) / sg : 0.0;
    const int rk = s_rank[c];
    for (int r = lane; r < m; r += 32) B[(long long)r * n_val + rk] = ac[r] * scale;
  }
  if (threadIdx.x == 0) {
    double smax = 0.0, smin = INFINITY;
    for (int c = 0; c < n_val; ++c) {
      smax = fmax(smax, s_sigma[c]);
      smin = fmin(smin, s_sigma[c]);
    }
    stats[2] = sweeps;
    stats[3] = off;
    stats[4] = smax > 0.0 ? smin / smax : 0.0;
  }
}

// Cb[k][i][b] = sum_{R != 0} exp(-i k.R) B[(R - 1) n_lo + i][b] (the Bloch sum of the bath columns
// of Eq. "C loemb R"), and the impurity columns of C^{k,AO,EO}: C_out[k][mu][j] = C^{k,AO,LO}[k][mu][j]
// for j < n_lo (the identity block of Eq. "C loemb R" times C^{k,AO,LO}).
__global__ void __launch_bounds__(256) bath_bloch_kernel(const double* __restrict__ B, const double2* __restrict__ Clo,
                                                         int n1, int n2, int n3, int n_lo, int n_val,
                                                         double2* __restrict__ Cb, double2* __restrict__ Cout) {
  const int nk = n1 * n2 * n3;
  const int n_emb = n_lo + n_val;
  const long long nb = (long long)nk * n_lo * n_val, ni = (long long)nk * n_lo * n_lo;
  const double inv = 1.0 / nk;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < nb + ni; x += (long long)gridDim.x * blockDim.x) {
    if (x < nb) {
      const int b = (int)(x % n_val);
      const int i = (int)((x / n_val) % n_lo);
      const int k = (int)(x / ((long long)n_val * n_lo));
      double re = 0.0, im = 0.0;
      for (int R = 1; R < nk; ++R) {
        double s, c;
        sincospi(2.0 * k_dot_r(k, R, n1, n2, n3) * inv, &s, &c);
        const double v = B[((long long)(R - 1) * n_lo + i) * n_val + b];
        re = fma(v, c, re);
        im = fma(-v, s, im);
      }
      Cb[x] = make_double2(re, im);
    } else {
      const long long y = x - nb;
      const int j = (int)(y % n_lo);
      const long long kmu = y / n_lo;
      Cout[kmu * n_emb + j] = Clo[y];
    }
  }
}

}  // namespace

cudaError_t launch_bath_offdiag(const double2* gk, const int mesh[3], int n_lo, const BathCols& val, double* A,
                                double* stats, cudaStream_t st) {
  const long long total = (long long)(mesh[0] * mesh[1] * mesh[2] - 1) * n_lo * val.n;
  if (total <= 0) return cudaSuccess;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 8);
  bath_offdiag_kernel<<<blocks, 256, 0, st>>>(gk, mesh[0], mesh[1], mesh[2], n_lo, val, A, stats);
  return cudaGetLastError();
}

size_t bath_jacobi_smem(int m, int n_val) { return (size_t)m * n_val * sizeof(double); }

cudaError_t launch_bath_jacobi(double* A, int m, int n_val, double* B, double* sigma, double* stats,
                               cudaStream_t st) {
  const size_t need = bath_jacobi_smem(m, n_val);
  const bool in_smem = need <= kBathJacobiSmem;
  if (in_smem) {
    cudaError_t e = cudaFuncSetAttribute(bath_jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kBathJacobiSmem);
    if (e != cudaSuccess) return e;
  }
  bath_jacobi_kernel<<<1, kJacobiThreads, in_smem ? need : 0, st>>>(A, m, n_val, in_smem ? 1 : 0, B, sigma, stats);
  return cudaGetLastError();
}

cudaError_t launch_bath_bloch(const double* B, const double2* Clo, const int mesh[3], int n_lo, int n_val,
                              double2* Cb, double2* Cout, cudaStream_t st) {
  const int nk = mesh[0] * mesh[1] * mesh[2];
  const long long total = (long long)nk * n_lo * (n_val + n_lo);
  const int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 8);
  bath_bloch_kernel<<<blocks, 256, 0, st>>>(B, Clo, mesh[0], mesh[1], mesh[2], n_lo, n_val, Cb, Cout);
  return cudaGetLastError();
}

}  // namespace dmet
