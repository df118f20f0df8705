// The FFTDF variant of the embedded-ERI transformation (Appendix B, Algorithm 2): the pointwise
// steps around the Fourier transforms of the transformed pair densities. The transforms themselves
// are dense DFTs along each grid axis, run as batched complex GEMMs (zgemm_fp64_kernel); FP64.

#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace dmet {

namespace {

inline int grid_for(long long total, int threads, int cap) {
  long long g = (total + threads - 1) / threads;
  if (g < 1) g = 1;
  return (int)(g < cap ? g : cap);
}

// dst[r][x] = s exp(sign * i q.r) src[r][x], q.r = 2 pi sum_d (j_d / g_d)(n_d / N_d) for grid point
// r = (j_1, j_2, j_3) (C order) and the mesh triple n of q.
__global__ void fftdf_phase_kernel(const double2* __restrict__ src, double2* __restrict__ dst, int g0, int g1, int g2,
                                   double f0, double f1, double f2, double sign, double s, long long nx) {
  const long long total = (long long)g0 * g1 * g2 * nx;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long r = t / nx;
    const int j2 = (int)(r % g2), j1 = (int)((r / g2) % g1), j0 = (int)(r / ((long long)g1 * g2));
    // exp(sign * 2 pi i (j0 f0 + j1 f1 + j2 f2)), f_d = n_d / (N_d g_d)
    double sn, cs;
    sincospi(2.0 * sign * (j0 * f0 + j1 * f1 + j2 * f2), &sn, &cs);
    const double2 a = src[t];
    dst[t] = make_double2(s * (a.x * cs - a.y * sn), s * (a.x * sn + a.y * cs));
  }
}

// The same phase for a run of q values at once: blockIdx.y is the local index i of a q in the run,
// qtab[i] its q (mesh triple from the mesh, C order). Source block: src + qtab[i] * ng * nx if by_table,
// else src + i * ng * nx; destination block dst + i * ng * nx.
__global__ void fftdf_phase_q_kernel(const double2* __restrict__ src, double2* __restrict__ dst,
                                     const int* __restrict__ qtab, int by_table, int g0, int g1, int g2, int m0,
                                     int m1, int m2, double sign, double s, long long nx) {
  const long long ngx = (long long)g0 * g1 * g2 * nx;
  const int i = blockIdx.y, q = qtab[i];
  const int n0 = q / (m1 * m2), n1 = (q / m2) % m1, n2 = q % m2;
  const double f0 = (double)n0 / ((double)m0 * g0), f1 = (double)n1 / ((double)m1 * g1),
               f2 = (double)n2 / ((double)m2 * g2);
  const double2* in = src + (long long)(by_table ? q : i) * ngx;
  double2* out = dst + (long long)i * ngx;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ngx;
       t += (long long)gridDim.x * blockDim.x) {
    const long long r = t / nx;
    const int j2 = (int)(r % g2), j1 = (int)((r / g2) % g1), j0 = (int)(r / ((long long)g1 * g2));
    double sn, cs;
    sincospi(2.0 * sign * (j0 * f0 + j1 * f1 + j2 * f2), &sn, &cs);
    const double2 a = in[t];
    out[t] = make_double2(s * (a.x * cs - a.y * sn), s * (a.x * sn + a.y * cs));
  }
}

// buf[G][x] *= v[G]
__global__ void fftdf_kernel_mul(double2* __restrict__ buf, const double* __restrict__ v, long long ng, long long nx) {
  const long long total = ng * nx;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const double w = v[t / nx];
    buf[t] = make_double2(buf[t].x * w, buf[t].y * w);
  }
}

// A dense DFT along the middle axis of [outer][g][inner]: out[o][k][i] = sum_j F[k g + j] in[o][j][i],
// for axes of at most kMaxDftAxis points. One thread per (o, i) column keeps the column's g inputs
// in registers and F in shared memory; the reads and writes of a warp are runs of consecutive i.
constexpr int kMaxDftAxis = 32;
__global__ void __launch_bounds__(256) dft_axis_kernel(const double2* __restrict__ F, int g, long long outer,
                                                      long long inner, const double2* __restrict__ in,
                                                      double2* __restrict__ out) {
  __shared__ double2 f[kMaxDftAxis * kMaxDftAxis];
  for (int t = threadIdx.x; t < g * g; t += blockDim.x) f[t] = F[t];
  __syncthreads();
  const long long total = outer * inner;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < total;
       c += (long long)gridDim.x * blockDim.x) {
    const long long o = c / inner, i = c - o * inner;
    const long long base = o * g * inner + i;
    double2 x[kMaxDftAxis];
#pragma unroll
    for (int j = 0; j < kMaxDftAxis; ++j)
      if (j < g) x[j] = in[base + j * inner];
    for (int k = 0; k < g; ++k) {
      double re = 0.0, im = 0.0;
#pragma unroll
      for (int j = 0; j < kMaxDftAxis; ++j)
        if (j < g) {
          const double2 a = f[k * g + j];
          re = fma(a.x, x[j].x, fma(-a.y, x[j].y, re));
          im = fma(a.x, x[j].y, fma(a.y, x[j].x, im));
        }
      out[base + k * inner] = make_double2(re, im);
    }
  }
}

// out[i] += sum_p parts[p n + i]
__global__ void sum_parts_kernel(const double2* __restrict__ parts, int np, long long n, double2* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double2 a = out[i];
    for (int p = 0; p < np; ++p) {
      const double2 b = parts[(long long)p * n + i];
      a.x += b.x;
      a.y += b.y;
    }
    out[i] = a;
  }
}

}  // namespace

bool fftdf_small_axis(int g) { return g >= 1 && g <= kMaxDftAxis; }

cudaError_t launch_dft_axis_small(const double2* F, int g, long long outer, long long inner, const double2* in,
                                  double2* out, cudaStream_t st) {
  if (!fftdf_small_axis(g)) return cudaErrorInvalidValue;
  dft_axis_kernel<<<grid_for(outer * inner, 256, 152 * 8), 256, 0, st>>>(F, g, outer, inner, in, out);
  return cudaGetLastError();
}

cudaError_t launch_sum_parts(const double2* parts, int np, long long n, double2* out, cudaStream_t st) {
  sum_parts_kernel<<<grid_for(n, 256, 152 * 16), 256, 0, st>>>(parts, np, n, out);
  return cudaGetLastError();
}

cudaError_t launch_fftdf_phase(const double2* src, double2* dst, const int grid[3], const int nq[3], const int mesh[3],
                               double sign, double s, long long nx, cudaStream_t st) {
  const long long total = (long long)grid[0] * grid[1] * grid[2] * nx;
  fftdf_phase_kernel<<<grid_for(total, 256, 152 * 16), 256, 0, st>>>(
      src, dst, grid[0], grid[1], grid[2], (double)nq[0] / ((double)mesh[0] * grid[0]),
      (double)nq[1] / ((double)mesh[1] * grid[1]), (double)nq[2] / ((double)mesh[2] * grid[2]), sign, s, nx);
  return cudaGetLastError();
}

cudaError_t launch_fftdf_phase_q(const double2* src, double2* dst, const int* qtab, int nq_run, int by_table,
                                 const int grid[3], const int mesh[3], double sign, double s, long long nx,
                                 cudaStream_t st) {
  if (nq_run <= 0) return cudaSuccess;
  if (nq_run > 65535) return cudaErrorInvalidValue;
  const long long per = (long long)grid[0] * grid[1] * grid[2] * nx;
  const int gx = grid_for(per, 256, std::max(1, 152 * 16 / nq_run));
  fftdf_phase_q_kernel<<<dim3(gx, nq_run), 256, 0, st>>>(src, dst, qtab, by_table, grid[0], grid[1], grid[2], mesh[0],
                                                         mesh[1], mesh[2], sign, s, nx);
  return cudaGetLastError();
}

cudaError_t launch_fftdf_kernel_mul(double2* buf, const double* v, long long ng, long long nx, cudaStream_t st) {
  fftdf_kernel_mul<<<grid_for(ng * nx, 256, 152 * 16), 256, 0, st>>>(buf, v, ng, nx);
  return cudaGetLastError();
}

}  // namespace dmet
