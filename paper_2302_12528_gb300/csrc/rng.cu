// Seeded N(0,1) start blocks on the device, for a solve called without a
// start block.  Algorithm 3 takes any full-rank start block X0; this file
// only defines which one a seed stands for.
//
// Generator: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC 2011), counter-based, so every element is
// computed independently.  Block element e = i + n j (column-major) belongs to
// pair p = e / 2 (real) or p = e (complex).  The pair's counter is
// (p mod 2^32, p / 2^32, 0, 0) and the key is the 64-bit seed.  The four output
// words give two uniforms with 53 random bits each,
//   u1 = ((x0 >> 5) 2^26 + (x1 >> 6) + 1/2) 2^-53 in (0, 1),  u2 from x2, x3,
// and the Box-Muller transform turns them into z0 = r cos(2 pi u2) and
// z1 = r sin(2 pi u2), r = sqrt(-2 ln u1).  A real element is z0 (even e) or z1
// (odd e).  A complex element is (z0 s, z1 s), s the double nearest 1 / sqrt 2.
#include <algorithm>

#include "common.cuh"
#include "rng.cuh"

namespace mpl {

namespace {

constexpr uint32_t PH_M0 = 0xD2511F53u, PH_M1 = 0xCD9E8D57u;  // round multipliers
constexpr uint32_t PH_W0 = 0x9E3779B9u, PH_W1 = 0xBB67AE85u;  // key increments

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += PH_W0;
      k1 += PH_W1;
    }
    const uint32_t hi0 = __umulhi(PH_M0, c.x), lo0 = PH_M0 * c.x;
    const uint32_t hi1 = __umulhi(PH_M1, c.z), lo1 = PH_M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

__device__ __forceinline__ double uniform53(uint32_t a, uint32_t b) {
  return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6) + 0.5) * 0x1p-53;
}

__device__ __forceinline__ void normal_pair(unsigned long long p, unsigned long long seed, double& z0,
                                            double& z1) {
  const uint4 x = philox4x32_10(make_uint4((uint32_t)p, (uint32_t)(p >> 32), 0u, 0u), (uint32_t)seed,
                                (uint32_t)(seed >> 32));
  const double u1 = uniform53(x.x, x.y), u2 = uniform53(x.z, x.w);
  const double r = sqrt(-2.0 * log(u1));
  const double t = 2.0 * 3.141592653589793 * u2;
  z0 = r * cos(t);
  z1 = r * sin(t);
}

// Real block: one thread per pair of consecutive elements.
__global__ void start_block_real_kernel(long long ne, unsigned long long seed, double* __restrict__ X) {
  const long long np = (ne + 1) / 2;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np;
       p += (long long)gridDim.x * blockDim.x) {
    double z0, z1;
    normal_pair((unsigned long long)p, seed, z0, z1);
    X[2 * p] = z0;
    if (2 * p + 1 < ne) X[2 * p + 1] = z1;
  }
}

// Complex block: one thread per element (interleaved re, im).
__global__ void start_block_complex_kernel(long long ne, unsigned long long seed, double* __restrict__ X) {
  const double s = 0.70710678118654752440;  // 1 / sqrt(2), the nearest double
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne;
       e += (long long)gridDim.x * blockDim.x) {
    double z0, z1;
    normal_pair((unsigned long long)e, seed, z0, z1);
    X[2 * e] = z0 * s;
    X[2 * e + 1] = z1 * s;
  }
}

}  // namespace

void start_block(cudaStream_t st, bool cx, long long n, int m, unsigned long long seed, double* X) {
  const long long ne = n * (long long)m;
  const long long work = cx ? ne : (ne + 1) / 2;
  if (work <= 0) return;
  const int grid = (int)std::min<long long>((work + 255) / 256, 8LL * NUM_SMS);
  count_launch();
  if (cx) start_block_complex_kernel<<<grid, 256, 0, st>>>(ne, seed, X);
  else start_block_real_kernel<<<grid, 256, 0, st>>>(ne, seed, X);
}

}  // namespace mpl

#include "mplobpcg_steps.h"

extern "C" mpl_status mpl_start_block(int dtype, int64_t n, int m, uint64_t seed, void* X, void* stream) {
  if ((dtype != MPL_R64 && dtype != MPL_C128) || n < 1 || m < 1 || !X) return MPL_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  mpl::start_block(st, dtype == MPL_C128, n, m, seed, static_cast<double*>(X));
  if (cudaGetLastError() != cudaSuccess) return MPL_ECUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? MPL_OK : MPL_ECUDA;
}
