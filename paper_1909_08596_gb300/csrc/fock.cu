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

// pairs[P] = (l, j) with l >= j, P = l(l+1)/2 + j; g[P] = gamma_lj (2 - delta_lj).
__global__ void pair_table_kernel(const double* __restrict__ gamma, int n, int2* __restrict__ pairs,
                                  double* __restrict__ g) {
  for (int l = blockIdx.x; l < n; l += gridDim.x)
    for (int j = threadIdx.x; j <= l; j += blockDim.x) {
      const long long P = (long long)l * (l + 1) / 2 + j;
      pairs[P] = make_int2(l, j);
      g[P] = (l == j ? 1.0 : 2.0) * gamma[(long long)l * n + j];
    }
}

// One pair row A = (i, k), i >= k, per block, over every pair column B = (l, j), l >= j, with
// v = (ik|lj) read from the packed lower triangle (the element at max(A,B)(max+1)/2 + min):
//   J[i][k] = J[k][i] = sum_B v g[B];
//   K[a][d] += v gamma_bc for each image (a b | c d) of (ik|lj) with its bra from {(i,k), (k,i)}
//   and its ket from {(l,j), (j,l)} (distinct images only); the images with bra and ket
//   exchanged are added when the row B is processed, so every ordered image counts once.
// The exchange rows i and k accumulate in shared memory and are added to K once per block.
__global__ void __launch_bounds__(256) coulomb_exchange_kernel(const double* __restrict__ eri,
                                                               const int2* __restrict__ pairs,
                                                               const double* __restrict__ g,
                                                               const double* __restrict__ gamma, int n,
                                                               double* __restrict__ J, double* __restrict__ K) {
  extern __shared__ double sm[];
  double* gi = sm;          // gamma row i
  double* gk = sm + n;      // gamma row k
  double* ki = sm + 2 * n;  // exchange row i
  double* kk = sm + 3 * n;  // exchange row k
  __shared__ double red[32];
  const long long npair = (long long)n * (n + 1) / 2;
  for (long long A = blockIdx.x; A < npair; A += gridDim.x) {
    const int2 ik = pairs[A];
    const int i = ik.x, k = ik.y;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      gi[t] = gamma[(long long)i * n + t];
      gk[t] = gamma[(long long)k * n + t];
      ki[t] = 0.0;
      kk[t] = 0.0;
    }
    __syncthreads();
    double jsum = 0.0;
    const long long rowA = A * (A + 1) / 2;
    for (long long B = threadIdx.x; B < npair; B += blockDim.x) {
      const double v = B <= A ? eri[rowA + B] : eri[B * (B + 1) / 2 + A];
      const int2 lj = pairs[B];
      const int l = lj.x, j = lj.y;
      jsum += v * g[B];
      atomicAdd(&ki[j], v * gk[l]);
      if (l != j) atomicAdd(&ki[l], v * gk[j]);
      if (i != k) {
        atomicAdd(&kk[j], v * gi[l]);
        if (l != j) atomicAdd(&kk[l], v * gi[j]);
      }
    }
    // block sum of jsum
    for (int o = 16; o; o >>= 1) jsum += __shfl_xor_sync(0xffffffffu, jsum, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = jsum;
    __syncthreads();
    if (threadIdx.x < 32) {
      double s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
      for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (threadIdx.x == 0) {
        J[(long long)i * n + k] = s;
        J[(long long)k * n + i] = s;
      }
    }
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      atomicAdd(&K[(long long)i * n + t], ki[t]);
      if (i != k) atomicAdd(&K[(long long)k * n + t], kk[t]);
    }
    __syncthreads();
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

}  // namespace

cudaError_t launch_fock_reduce(const double2* G, int nk, int n, double s, double* F0, cudaStream_t st) {
  fock_reduce_kernel<<<blocks_for((long long)n * n, 256, 152 * 8), 256, 0, st>>>(G, nk, n, s, F0);
  return cudaGetLastError();
}

cudaError_t launch_coulomb_exchange(const double* eri, const double* gamma, int n, void* pairs, double* g, double* J,
                                    double* K, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  pair_table_kernel<<<n < 1024 ? n : 1024, 128, 0, st>>>(gamma, n, (int2*)pairs, g);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long npair = (long long)n * (n + 1) / 2;
  const size_t smem = (size_t)4 * n * sizeof(double);
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(coulomb_exchange_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int grid = (int)(npair < 152 * 8 ? npair : 152 * 8);
  coulomb_exchange_kernel<<<grid, 256, smem, st>>>(eri, (const int2*)pairs, g, gamma, n, J, K);
  return cudaGetLastError();
}

cudaError_t launch_fock_combine(const double* F0, const double* J, const double* K, int n, double* out,
                                cudaStream_t st) {
  fock_combine_kernel<<<blocks_for((long long)n * n, 256, 152 * 8), 256, 0, st>>>(F0, J, K, n * n, out);
  return cudaGetLastError();
}

}  // namespace dmet
