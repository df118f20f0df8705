// DMET bath and embedding orbitals (section 2.1): the environment-impurity block of the
// mean-field density matrix brought to real space (Eq. "bath R SVD" needs gamma^{R != 0, 0}),
// its singular value decomposition by one-sided Jacobi rotations on one thread-block cluster,
// the block form of Eq. "C loemb R" and the two transformations of Eq. "C loemb k". FP64
// throughout; every phase factor comes from one table of the Nk roots of unity.

#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <stdint.h>

#include <cooperative_groups.h>

#include "internal.h"

namespace cg = cooperative_groups;

namespace dmet {

namespace {

// k.R = 2 pi t / Nk with t = sum_d k_d R_d Nk / N_d (mod Nk). For a fixed point x of the mesh
// (a k-point or a cell, C-order index) step_of gives the three steps a_d = x_d Nk / N_d mod Nk, so
// that walking the other index y over the mesh in C order only adds a_3 per step of y_3 (a_2, a_1
// on the carries): the phase index of (x, y) without a division in the loop.
struct MeshSteps {
  int a1, a2, a3;
};
__device__ __forceinline__ MeshSteps step_of(int x, int n1, int n2, int n3) {
  const int nk = n1 * n2 * n3;
  const int x1 = x / (n2 * n3), x2 = (x / n3) % n2, x3 = x % n3;
  return {x1 * (nk / n1), x2 * (nk / n2), x3 * (nk / n3)};
}
__device__ __forceinline__ int add_mod(int a, int b, int n) {
  const int s = a + b;
  return s >= n ? s - n : s;
}

// Non-negative doubles order like their bit patterns.
__device__ __forceinline__ void atomic_max_nonneg(double* p, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(p), (unsigned long long)__double_as_longlong(v));
}

// tw[t] = exp(+2 pi i t / Nk) = (cos, sin), t < Nk: every phase factor of the mesh (k.R is an
// integer multiple of 2 pi / Nk).
__global__ void bath_twiddle_kernel(int nk, double2* __restrict__ tw) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nk; t += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * t / nk, &s, &c);
    tw[t] = make_double2(c, s);
  }
}

// A[c][r] = Re gamma^{R,0}_{i, val[c]}, r = (R - 1) n_lo + i for the cells R = 1 .. Nk - 1, with
// gamma^{R,0} = (1/Nk) sum_k exp(+i k.R) gamma^k. stats[0] / stats[1] collect the largest |Re| and
// |Im| of the block.
__global__ void __launch_bounds__(128) bath_offdiag_kernel(const double2* __restrict__ gk, const double2* __restrict__ tw,
                                                           int n1, int n2, int n3, int n_lo, BathCols val,
                                                           double* __restrict__ A, double* __restrict__ stats) {
  const int nk = n1 * n2 * n3;
  const long long m = (long long)(nk - 1) * n_lo, total = m * val.n;
  const double inv = 1.0 / nk;
  double mre = 0.0, mim = 0.0;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total; x += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(x / m);
    const int r = (int)(x % m);
    const int R = 1 + r / n_lo, i = r % n_lo, j = val.v[c];
    double re = 0.0, im = 0.0;
    const MeshSteps st = step_of(R, n1, n2, n3);
    const double2* g = gk + (long long)i * n_lo + j;
    const long long gs = (long long)n_lo * n_lo;
    for (int k1 = 0, t1 = 0; k1 < n1; ++k1, t1 = add_mod(t1, st.a1, nk))
      for (int k2 = 0, t2 = t1; k2 < n2; ++k2, t2 = add_mod(t2, st.a2, nk))
        for (int k3 = 0, t = t2; k3 < n3; ++k3, t = add_mod(t, st.a3, nk), g += gs) {
          const double2 e = tw[t];
          const double2 v = *g;
          re = fma(v.x, e.x, fma(-v.y, e.y, re));
          im = fma(v.x, e.y, fma(v.y, e.x, im));
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
constexpr float kRotTol = 1e-14f;  // rotate a pair while |a_p.a_q| > kRotTol ||a_p|| ||a_q||

// Pair slot j of round `round` of the round-robin ordering of n_pad columns: position n_pad - 1
// stays, the others turn one step per round, so n_pad - 1 rounds meet every pair once.
__device__ __forceinline__ void pair_of(int round, int j, int n_pad, int& p, int& q) {
  p = j == 0 ? n_pad - 1 : (round + j) % (n_pad - 1);
  q = j == 0 ? round : (round - j + n_pad - 1) % (n_pad - 1);
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One-sided Jacobi SVD (Hestenes 1958; the rotation angle as in Rutishauser's symmetric Jacobi
// method) of the m x n_val block A (column-major), on one cluster of kBathCluster CTAs: CTA rank
// r owns the rows [r mc, (r + 1) mc) of every column (mc = ceil(m / kBathCluster)), in shared
// memory when they fit, else in place in global memory. A sweep visits every column pair in
// n_pad - 1 rounds of the round-robin ordering (n_pad = n_val rounded up to even; the pad column
// never rotates), one warp per pair of a round (the FP64 pipe of a sub-partition is charged per
// warp instruction, idle lanes included, so the pairs go to different warps and the warps of a
// round to different sub-partitions). Per round each CTA forms
// the pair's three dot products over its rows, the cluster barrier publishes them, and every CTA
// adds the partials in the same fixed order (the same numbers in the same order, so every CTA
// takes the same rotation and the same convergence decision, and all pass the same barriers),
// then rotates its own rows. The partials alternate between two buffers, so one barrier per
// round suffices. The rotation angle is taken in FP32 and the rotation then made orthogonal in
// FP64 (an angle off by 1e-7 relative leaves a cosine 1e-7 times the old one, which the next
// sweep removes; the rotation itself never loses orthogonality). After convergence
// column c is sigma_c u_c. The columns are written in decreasing sigma, each scaled by
// sign / sigma with the sign that makes its largest-magnitude entry (the first of equal ones)
// positive: B[r][rank] = u. A zero singular value leaves a zero column. stats[2] = sweeps,
// stats[3] = largest pair cosine |a_p.a_q| / (||a_p|| ||a_q||) of the last sweep,
// stats[4] = sigma_min / sigma_max.
__global__ void __cluster_dims__(kBathCluster, 1, 1) __launch_bounds__(kJacobiThreads)
    bath_jacobi_kernel(double* __restrict__ Ag, int m, int n_val, int in_smem, double* __restrict__ B,
                       double* __restrict__ sigma_out, double* __restrict__ stats) {
  extern __shared__ double sm[];
  __shared__ double part[2][kMaxBathCols / 2][3];
  __shared__ double s_norm2[kMaxBathCols];   // this CTA's share of ||a_c||^2
  __shared__ double s_big[kMaxBathCols];     // this CTA's largest |a_c| entry, signed
  __shared__ int s_big_row[kMaxBathCols];    // and its global row (m if the CTA has no rows)
  __shared__ double s_sigma[kMaxBathCols];
  __shared__ double s_sign[kMaxBathCols];
  __shared__ int s_rank[kMaxBathCols];
  __shared__ int s_rot;
  __shared__ double s_off[kJacobiWarps];
  cg::cluster_group cl = cg::this_cluster();
  const int crank = (int)cl.block_rank();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int mc = (m + kBathCluster - 1) / kBathCluster;
  const int r0 = min(m, crank * mc), ml = min(m, r0 + mc) - r0;
  double* A = Ag + r0;
  long long ld = m;
  if (in_smem) {
    A = sm;
    ld = mc;
    for (long long x = threadIdx.x; x < (long long)n_val * mc; x += blockDim.x) {
      const int c = (int)(x / mc), r = (int)(x % mc);
      if (r < ml) sm[x] = Ag[(long long)c * m + r0 + r];
    }
  }
  __syncthreads();
  const int n_pad = n_val + (n_val & 1);
  const int half = n_pad / 2;
  int sweeps = 0, buf = 0;
  double off = 0.0;
  for (int sweep = 0; sweep < kMaxSweeps && n_val > 1; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    double woff = 0.0;
    __syncthreads();
    for (int round = 0; round < n_pad - 1; ++round) {
      // dot products of this CTA's rows, one warp per pair slot j (j = warp, warp + 16, ...)
      for (int j = warp; j < half; j += kJacobiWarps) {
        int p, q;
        pair_of(round, j, n_pad, p, q);
        if (p >= n_val || q >= n_val) continue;
        const double* ap = A + p * ld;
        const double* aq = A + q * ld;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int r = lane; r < ml; r += 32) {
          const double x = ap[r], y = aq[r];
          al = fma(x, x, al);
          be = fma(y, y, be);
          ga = fma(x, y, ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (lane == 0) {
          part[buf][j][0] = al;
          part[buf][j][1] = be;
          part[buf][j][2] = ga;
        }
      }
      cl.sync();
      for (int j = warp; j < half; j += kJacobiWarps) {
        int p, q;
        pair_of(round, j, n_pad, p, q);
        if (p >= n_val || q >= n_val) continue;
        // lane g < 8 reads CTA g's three partials; a fixed shuffle tree adds them
        double al = 0.0, be = 0.0, ga = 0.0;
        if (lane < kBathCluster) {
          const double* rp = cl.map_shared_rank(&part[buf][j][0], lane);
          al = rp[0];
          be = rp[1];
          ga = rp[2];
        }
        for (int o = kBathCluster / 2; o; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        al = __shfl_sync(0xffffffffu, al, 0);
        be = __shfl_sync(0xffffffffu, be, 0);
        ga = __shfl_sync(0xffffffffu, ga, 0);
        // The angle in FP32 (its error only slows convergence a little), the rotation made
        // orthogonal to FP64 rounding: (c, s) scaled by 1/sqrt(c^2 + s^2) = 1 - d/2 + 3d^2/8,
        // d = c^2 + s^2 - 1 = O(1e-7). A zero column gives a NaN cosine and never rotates.
        const float ga32 = (float)ga;
        const float cs = fabsf(ga32) * rsqrtf((float)al) * rsqrtf((float)be);
        if (cs == cs) woff = fmax(woff, (double)cs);
        if (!(cs > kRotTol)) continue;
        // t = tan of the angle that makes the rotated columns orthogonal: the root of smaller
        // magnitude of t^2 + 2 zeta t - 1 = 0, zeta = (be - al) / (2 ga)
        const float zeta = (float)(be - al) / (2.0f * ga32);
        const float t = fabsf(zeta) > 1e18f ? 0.5f / zeta
                                            : copysignf(1.0f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.0f)));
        const float c32 = rsqrtf(fmaf(t, t, 1.0f));
        const double cd = c32, sd = (double)(c32 * t);
        const double d = fma(cd, cd, fma(sd, sd, -1.0));
        const double nr = fma(0.375 * d, d, fma(-0.5, d, 1.0));
        const double c = cd * nr, sn = sd * nr;
        double* ap = A + p * ld;
        double* aq = A + q * ld;
        for (int r = lane; r < ml; r += 32) {
          const double x = ap[r], y = aq[r];
          ap[r] = fma(c, x, -sn * y);
          aq[r] = fma(sn, x, c * y);
        }
        if (lane == 0) s_rot = 1;
      }
      buf ^= 1;
      __syncthreads();
    }
    for (int o = 16; o; o >>= 1) woff = fmax(woff, __shfl_xor_sync(0xffffffffu, woff, o));
    if (lane == 0) s_off[warp] = woff;
    __syncthreads();
    ++sweeps;
    off = 0.0;
    for (int w = 0; w < kJacobiWarps; ++w) off = fmax(off, s_off[w]);
    const int rotated = s_rot;
    __syncthreads();
    if (!rotated) break;
  }
  // this CTA's shares of the column norms and of the largest-magnitude entries
  for (int c = warp; c < n_val; c += kJacobiWarps) {
    const double* ac = A + c * ld;
    double ss = 0.0, best = -1.0, val = 0.0;
    int at = m;
    for (int r = lane; r < ml; r += 32) {
      const double v = ac[r];
      ss = fma(v, v, ss);
      if (fabs(v) > best) {
        best = fabs(v);
        val = v;
        at = r0 + r;
      }
    }
    ss = warp_sum(ss);
    for (int o = 16; o; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const double ov = __shfl_xor_sync(0xffffffffu, val, o);
      const int oa = __shfl_xor_sync(0xffffffffu, at, o);
      if (ob > best || (ob == best && oa < at)) {
        best = ob;
        val = ov;
        at = oa;
      }
    }
    if (lane == 0) {
      s_norm2[c] = ss;
      s_big[c] = val;
      s_big_row[c] = at;
    }
  }
  cl.sync();
  if (threadIdx.x < n_val) {
    const int c = threadIdx.x;
    double n2 = 0.0;
    for (int r = 0; r < kBathCluster; ++r) n2 += *cl.map_shared_rank(&s_norm2[c], r);
    s_sigma[c] = sqrt(n2);
    double best = -1.0, val = 0.0;
    int at = m;
    for (int r = 0; r < kBathCluster; ++r) {
      const double v = *cl.map_shared_rank(&s_big[c], r);
      const int a = *cl.map_shared_rank(&s_big_row[c], r);
      if (fabs(v) > best || (fabs(v) == best && a < at)) {
        best = fabs(v);
        val = v;
        at = a;
      }
    }
    s_sign[c] = val < 0.0 ? -1.0 : 1.0;
  }
  __syncthreads();
  if (threadIdx.x < n_val) {
    const int c = threadIdx.x;
    const double sc = s_sigma[c];
    int rk = 0;
    for (int d = 0; d < n_val; ++d) rk += (s_sigma[d] > sc) || (s_sigma[d] == sc && d < c);
    s_rank[c] = rk;
    if (sigma_out && crank == 0) sigma_out[rk] = sc;
  }
  __syncthreads();
  for (int c = warp; c < n_val; c += kJacobiWarps) {
    const double* ac = A + c * ld;
    const double sg = s_sigma[c];
    const double scale = sg > 0.0 ? s_sign[c] / sg : 0.0;
    const int rk = s_rank[c];
    for (int r = lane; r < ml; r += 32) B[(long long)(r0 + r) * n_val + rk] = ac[r] * scale;
  }
  if (threadIdx.x == 0 && crank == 0) {
    double smax = 0.0, smin = INFINITY;
    for (int c = 0; c < n_val; ++c) {
      smax = fmax(smax, s_sigma[c]);
      smin = fmin(smin, s_sigma[c]);
    }
    stats[2] = sweeps;
    stats[3] = off;
    stats[4] = smax > 0.0 ? smin / smax : 0.0;
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

// Cb[k][i][b] = sum_{R != 0} exp(-i k.R) B[(R - 1) n_lo + i][b] (the Bloch sum of the bath columns
// of Eq. "C loemb R"), and the impurity columns of C^{k,AO,EO}: C_out[k][mu][j] = C^{k,AO,LO}[k][mu][j]
// for j < n_lo (the identity block of Eq. "C loemb R" times C^{k,AO,LO}).
__global__ void __launch_bounds__(128) bath_bloch_kernel(const double* __restrict__ B, const double2* __restrict__ Clo,
                                                         const double2* __restrict__ tw, int n1, int n2, int n3,
                                                         int n_lo, int n_val, double2* __restrict__ Cb,
                                                         double2* __restrict__ Cout) {
  const int nk = n1 * n2 * n3;
  const int n_emb = n_lo + n_val;
  const long long nb = (long long)nk * n_lo * n_val, ni = (long long)nk * n_lo * n_lo;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < nb + ni; x += (long long)gridDim.x * blockDim.x) {
    if (x < nb) {
      const int b = (int)(x % n_val);
      const int i = (int)((x / n_val) % n_lo);
      const int k = (int)(x / ((long long)n_val * n_lo));
      double re = 0.0, im = 0.0;
      const MeshSteps st = step_of(k, n1, n2, n3);
      int R = 0;
      for (int r1 = 0, t1 = 0; r1 < n1; ++r1, t1 = add_mod(t1, st.a1, nk))
        for (int r2 = 0, t2 = t1; r2 < n2; ++r2, t2 = add_mod(t2, st.a2, nk))
          for (int r3 = 0, t = t2; r3 < n3; ++r3, t = add_mod(t, st.a3, nk), ++R) {
            if (R == 0) continue;  // the bath has no weight in the reference cell
            const double2 e = tw[t];
            const double bv = B[((long long)(R - 1) * n_lo + i) * n_val + b];
            re = fma(bv, e.x, re);
            im = fma(-bv, e.y, im);
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

// The bath columns of C^{k,AO,EO}: C_out[k][mu][n_lo + b] = sum_i C_lo[k][mu][i] Cb[k][i][b], one
// thread per output element (the products are n_lo x n_lo by n_lo x n_val per k: far too small
// for a tiled GEMM, whose tiles would be mostly padding).
__global__ void __launch_bounds__(128) bath_product_kernel(const double2* __restrict__ Clo, const double2* __restrict__ Cb,
                                                           int nk, int n_lo, int n_val, double2* __restrict__ Cout) {
  const int n_emb = n_lo + n_val;
  const long long total = (long long)nk * n_lo * n_val;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total; x += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(x % n_val);
    const long long kmu = x / n_val;  // k n_lo + mu
    const int k = (int)(kmu / n_lo);
    const double2* a = Clo + kmu * n_lo;
    const double2* c = Cb + (long long)k * n_lo * n_val + b;
    double re = 0.0, im = 0.0;
    for (int i = 0; i < n_lo; ++i) {
      const double2 u = a[i], v = c[(long long)i * n_val];
      re = fma(u.x, v.x, fma(-u.y, v.y, re));
      im = fma(u.x, v.y, fma(u.y, v.x, im));
    }
    Cout[kmu * n_emb + n_lo + b] = make_double2(re, im);
  }
}

}  // namespace

cudaError_t launch_bath_product(const double2* Clo, const double2* Cb, int nk, int n_lo, int n_val, double2* Cout,
                                cudaStream_t st) {
  const long long total = (long long)nk * n_lo * n_val;
  const int blocks = (int)std::min<long long>((total + 127) / 128, 152LL * 16);
  bath_product_kernel<<<blocks, 128, 0, st>>>(Clo, Cb, nk, n_lo, n_val, Cout);
  return cudaGetLastError();
}

cudaError_t launch_bath_twiddle(int nk, double2* tw, cudaStream_t st) {
  bath_twiddle_kernel<<<(nk + 255) / 256, 256, 0, st>>>(nk, tw);
  return cudaGetLastError();
}

cudaError_t launch_bath_offdiag(const double2* gk, const double2* tw, const int mesh[3], int n_lo, const BathCols& val,
                                double* A, double* stats, cudaStream_t st) {
  const long long total = (long long)(mesh[0] * mesh[1] * mesh[2] - 1) * n_lo * val.n;
  if (total <= 0) return cudaSuccess;
  const int blocks = (int)std::min<long long>((total + 127) / 128, 152LL * 16);
  bath_offdiag_kernel<<<blocks, 128, 0, st>>>(gk, tw, mesh[0], mesh[1], mesh[2], n_lo, val, A, stats);
  return cudaGetLastError();
}

size_t bath_jacobi_smem(int m, int n_val) {
  return (size_t)((m + kBathCluster - 1) / kBathCluster) * n_val * sizeof(double);
}

cudaError_t launch_bath_jacobi(double* A, int m, int n_val, double* B, double* sigma, double* stats,
                               cudaStream_t st) {
  const size_t need = bath_jacobi_smem(m, n_val);
  const bool in_smem = need <= kBathJacobiSmem;
  if (in_smem) {
    cudaError_t e = cudaFuncSetAttribute(bath_jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kBathJacobiSmem);
    if (e != cudaSuccess) return e;
  }
  bath_jacobi_kernel<<<kBathCluster, kJacobiThreads, in_smem ? need : 0, st>>>(A, m, n_val, in_smem ? 1 : 0, B, sigma,
                                                                                stats);
  return cudaGetLastError();
}

cudaError_t launch_bath_bloch(const double* B, const double2* Clo, const double2* tw, const int mesh[3], int n_lo,
                              int n_val, double2* Cb, double2* Cout, cudaStream_t st) {
  const int nk = mesh[0] * mesh[1] * mesh[2];
  const long long total = (long long)nk * n_lo * (n_val + n_lo);
  const int blocks = (int)std::min<long long>((total + 127) / 128, 152LL * 16);
  bath_bloch_kernel<<<blocks, 128, 0, st>>>(B, Clo, tw, mesh[0], mesh[1], mesh[2], n_lo, n_val, Cb, Cout);
  return cudaGetLastError();
}

}  // namespace dmet
