// The embedding one-particle Hamiltonian (section 2.1): the reduction of the transformed Fock
// matrices over k (Eq. "fock transform") and the Coulomb / exchange double counting evaluated
// with the 8-fold packed embedding ERIs (Eq. "fock double counting"). FP64 throughout.

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace dmet {

namespace {

// F0[i][j] = s * sum_k Re G[k][i][j], G[k] = C^{k+} F^k C^k.
__global__ void fock_reduce_kernel(const double2* __restrict__ G, int nk, int n, double s, double* __restrict__ F0) {
  const int nn = n * n;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nn; x += gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int k = 0; k < nk; ++k) v += G[(long long)k * nn + x].x;
    F0[x] = s * v;
  }
}

// One block per pair row A = {i, k}, i >= k: the block stages the row of the packed ERI in shared
// memory, V[B] = (ik|B) for every pair B (the element at max(A,B)(max+1)/2 + min), and then
//   thread j:  K_ij += sum_l (ik|lj) gamma_kl   and, for i != k,   K_kj += sum_l (ki|lj) gamma_il,
//   all:       J_ik  = J_ki = sum_{l,j} (ik|lj) gamma_jl = sum_B V[B] gamma_B (2 - delta_B),
// with V[{l, j}] = (ik|lj) = (ki|lj) (real orbitals). Each row is read once; the exchange rows are
// added to K (which starts at zero) with one atomic add per element and block.
__global__ void __launch_bounds__(256) coulomb_exchange_kernel(const double* __restrict__ eri,
                                                               const double* __restrict__ gamma, int n,
                                                               double* __restrict__ J, double* __restrict__ K) {
  extern __shared__ double sm[];
  const long long npair = (long long)n * (n + 1) / 2;
  double* row = sm;             // [npair]
  double* gi = sm + npair;      // gamma row i [n]
  double* gk = gi + n;          // gamma row k [n]
  __shared__ double red[8];
  for (long long A = blockIdx.x; A < npair; A += gridDim.x) {
    // (i, k) of A: i = floor((sqrt(8A + 1) - 1) / 2), made exact
    long long il = (long long)((sqrt(8.0 * (double)A + 1.0) - 1.0) * 0.5);
    while (il * (il + 1) / 2 > A) --il;
    while ((il + 1) * (il + 2) / 2 <= A) ++il;
    const int i = (int)il, k = (int)(A - il * (il + 1) / 2);
    const long long rowA = A * (A + 1) / 2;
    __syncthreads();  // the previous row's readers are done
    for (long long B = threadIdx.x; B < npair; B += blockDim.x)
      row[B] = B <= A ? eri[rowA + B] : eri[B * (B + 1) / 2 + A];
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      gi[t] = gamma[(long long)i * n + t];
      gk[t] = gamma[(long long)k * n + t];
    }
    __syncthreads();
    // The exchange rows: nsplit groups of n threads each take a share of l for every j (so that a
    // block of 256 threads keeps busy when n is below 256); their partial sums meet in the atomic adds.
    // (Pair indices fit 32 bits: n <= 2047.)
    const int nsplit = n < (int)blockDim.x ? (int)blockDim.x / n : 1;
    for (int t = threadIdx.x; t < nsplit * n; t += blockDim.x) {
      const int j = t % n, h = t / n;
      const int l0 = h * n / nsplit, l1 = (h + 1) * n / nsplit;
      double si = 0.0, sk = 0.0;
      const int jj = j * (j + 1) / 2;
      for (int l = l0; l < l1; ++l) {
        const double v = row[l >= j ? l * (l + 1) / 2 + j : jj + l];
        si = fma(v, gk[l], si);
        sk = fma(v, gi[l], sk);
      }
      atomicAdd(&K[(long long)i * n + j], si);
      if (i != k) atomicAdd(&K[(long long)k * n + j], sk);
    }
    double js = 0.0;
    for (int l = threadIdx.x >> 5; l < n; l += blockDim.x >> 5) {
      const long long base = (long long)l * (l + 1) / 2;
      for (int j = threadIdx.x & 31; j <= l; j += 32)
        js = fma(row[base + j], (l == j ? 1.0 : 2.0) * gamma[(long long)l * n + j], js);
    }
    for (int o = 16; o; o >>= 1) js += __shfl_xor_sync(0xffffffffu, js, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = js;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      J[(long long)i * n + k] = t;
      J[(long long)k * n + i] = t;
    }
  }
}

// out = F0 - (J - K / 2)
__global__ void fock_combine_kernel(const double* __restrict__ F0, const double* __restrict__ J,
                                    const double* __restrict__ K, int nn, double* __restrict__ out) {
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nn; x += gridDim.x * blockDim.x)
    out[x] = F0[x] - (J[x] - 0.5 * K[x]);
}

inline int blocks_for(long long total, int threads, int cap) {
  long long b = (total + threads - 1) / threads;
  return (int)(b < 1 ? 1 : (b < cap ? b : cap));
}

// v[z] = tr(L^{-q}_P gamma) = sum_{k,l} Lm[z][k][l] gamma[l][k] for the batch entries z = (q, P) of a
// chunk: Lm[z] = Lq[tab[z].y] (the -q factor). One block per z.
__global__ void __launch_bounds__(256) jk_trace_kernel(const double2* __restrict__ Lq, const int4* __restrict__ tab,
                                                       int n, const double2* __restrict__ gamma, double2* __restrict__ v) {
  const long long nn = (long long)n * n;
  const double2* m = Lq + (long long)tab[blockIdx.x].y * nn;
  double re = 0.0, im = 0.0;
  for (long long x = threadIdx.x; x < nn; x += blockDim.x) {
    const int k = (int)(x / n), l = (int)(x % n);
    const double2 a = m[x], g = gamma[(long long)l * n + k];
    re = fma(a.x, g.x, fma(-a.y, g.y, re));
    im = fma(a.x, g.y, fma(a.y, g.x, im));
  }
  __shared__ double sr[8], si[8];
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sr[threadIdx.x >> 5] = re;
    si[threadIdx.x >> 5] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += sr[w];
      b += si[w];
    }
    v[blockIdx.x] = make_double2(a, b);
  }
}

// J[x] += s sum_z v[z] Lq[tab[z].x][x] and K[x] += s sum_z Kb[z][x] over the nz entries of a chunk.
__global__ void __launch_bounds__(256) jk_accumulate_kernel(const double2* __restrict__ Lq, const int4* __restrict__ tab,
                                                            const double2* __restrict__ v, const double2* __restrict__ Kb,
                                                            int nz, long long nn, double s, double2* __restrict__ J,
                                                            double2* __restrict__ K) {
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < nn; x += (long long)gridDim.x * blockDim.x) {
    double jr = 0.0, ji = 0.0, kr = 0.0, ki = 0.0;
    for (int z = 0; z < nz; ++z) {
      const double2 a = Lq[(long long)tab[z].x * nn + x], w = v[z], b = Kb[(long long)z * nn + x];
      jr = fma(a.x, w.x, fma(-a.y, w.y, jr));
      ji = fma(a.x, w.y, fma(a.y, w.x, ji));
      kr += b.x;
      ki += b.y;
    }
    J[x] = make_double2(J[x].x + s * jr, J[x].y + s * ji);
    K[x] = make_double2(K[x].x + s * kr, K[x].y + s * ki);
  }
}

}  // namespace

cudaError_t launch_fock_reduce(const double2* G, int nk, int n, double s, double* F0, cudaStream_t st) {
  fock_reduce_kernel<<<blocks_for((long long)n * n, 256, 152 * 8), 256, 0, st>>>(G, nk, n, s, F0);
  return cudaGetLastError();
}

cudaError_t launch_coulomb_exchange(const double* eri, const double* gamma, int n, double* J, double* K,
                                    cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (n > 1024) return cudaErrorInvalidValue;
  const long long npair = (long long)n * (n + 1) / 2;
  const size_t smem = (size_t)(npair + 2 * n) * sizeof(double);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;  // the caller checks the size first
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(coulomb_exchange_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int grid = (int)(npair < 152 * 16 ? npair : 152 * 16);
  coulomb_exchange_kernel<<<grid, 256, smem, st>>>(eri, gamma, n, J, K);
  return cudaGetLastError();
}

cudaError_t launch_fock_combine(const double* F0, const double* J, const double* K, int n, double* out,
                                cudaStream_t st) {
  fock_combine_kernel<<<blocks_for((long long)n * n, 256, 152 * 8), 256, 0, st>>>(F0, J, K, n * n, out);
  return cudaGetLastError();
}

cudaError_t launch_jk_trace(const double2* Lq, const int4* tab, int nz, int n, const double2* gamma, double2* v,
                            cudaStream_t st) {
  if (nz <= 0) return cudaSuccess;
  jk_trace_kernel<<<nz, 256, 0, st>>>(Lq, tab, n, gamma, v);
  return cudaGetLastError();
}

cudaError_t launch_jk_accumulate(const double2* Lq, const int4* tab, const double2* v, const double2* Kb, int nz, int n,
                                 double s, double2* J, double2* K, cudaStream_t st) {
  const long long nn = (long long)n * n;
  long long blocks = (nn + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  jk_accumulate_kernel<<<(unsigned)(blocks > 0 ? blocks : 1), 256, 0, st>>>(Lq, tab, v, Kb, nz, nn, s, J, K);
  return cudaGetLastError();
}

}  // namespace dmet
