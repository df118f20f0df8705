// Device implementation of synth.counter_normals (synth/lattice.py): the same counter-based
// definition (SplitMix64 of Steele, Lea & Flood 2014 used as a hash of (seed, stream, counter),
// then the Box-Muller transform), for seeded inputs too large to draw on the host. It produces
// input numbers only; none of the embedded-ERI method's arithmetic is here.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kM1 = 0xBF58476D1CE4E5B9ull;
constexpr uint64_t kM2 = 0x94D049BB133111EBull;

__host__ __device__ inline uint64_t mix(uint64_t z) {
  z = (z ^ (z >> 30)) * kM1;
  z = (z ^ (z >> 27)) * kM2;
  return z ^ (z >> 31);
}

__host__ __device__ inline uint64_t stream_key(uint64_t seed, uint64_t stream) {
  const uint64_t k0 = mix(seed + kGamma);
  return mix(k0 + (stream + 1) * kGamma);
}

// out[s * per + t] = normal t of stream stream0 + s, for s < n_streams, t < per.
__global__ void normals_kernel(double* __restrict__ out, uint64_t seed, uint64_t stream0, long long n_streams,
                               long long per) {
  const long long total = n_streams * per;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total;
       x += (long long)gridDim.x * blockDim.x) {
    const long long s = x / per, t = x - s * per;
    const uint64_t key = stream_key(seed, stream0 + (uint64_t)s);
    const uint64_t h1 = mix(key + (2ull * (uint64_t)t + 1ull) * kGamma) >> 11;
    const uint64_t h2 = mix(key + (2ull * (uint64_t)t + 2ull) * kGamma) >> 11;
    const double u1 = ((double)h1 + 1.0) * 0x1p-53;
    const double u2 = (double)h2 * (0x1p-53 * 2.0 * 3.141592653589793);
    out[x] = sqrt(-2.0 * log(u1)) * cos(u2);
  }
}

}  // namespace

extern "C" __attribute__((visibility("default"))) int synth_counter_normals(double* out, uint64_t seed,
                                                                             uint64_t stream0, long long n_streams,
                                                                             long long per, void* stream) {
  if (!out || n_streams < 0 || per < 0) return (int)cudaErrorInvalidValue;
  if (n_streams * per == 0) return 0;
  long long blocks = (n_streams * per + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  normals_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(out, seed, stream0, n_streams, per);
  return (int)cudaGetLastError();
}
