// Tensor-core trailing update of the 16-bit factor stage: C -= A A^T (A A^H
// for complex) on the lower triangle, A (n x k) holding values of the 16-bit
// format (fp16 or bf16), products accumulated in FP32, the result optionally
// rounded to the format -- the contraction of the blocked Cholesky step with
// the factor stored in the lower precision.
//
// One CTA (8 warps) computes one 128 x 128 lower-triangle tile with
// tcgen05.mma (kind::f16, FP32 accumulator in tensor memory): the operand
// tiles (128 rows x K <= 128, K-major, converted to the format on the way
// in) are staged in shared memory in the canonical no-swizzle layout of
// 8-row x 16-byte core matrices, one thread issues the K/16 MMAs, their
// completion is committed to an mbarrier (waited on with an iteration
// limit), and each warp reads 32 accumulator lanes x 64 columns back with
// tcgen05.ld.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "common.cuh"

namespace mpl {

constexpr int TC_M = 128, TC_N = 128, TC_KMAX = 128;
constexpr int TC_THREADS = 256;  // two warpgroups: both stage operands, each reads half the columns
constexpr long long TC_WAIT_LIMIT = 1LL << 22;  // mbarrier polls before giving up (tens of ns each)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor, no swizzle, K-major: lbo = byte distance
// between core matrices adjacent along K, sbo = along M / N.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of this architecture
  return d;               // base offset 0, relative LBO, swizzle none
}

// Instruction descriptor of kind::f16: FP32 accumulator, A and B in the
// 16-bit format fmt (0 fp16, 1 bf16), both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_f16(int fmt, int M, int N) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

template <int FMT>
__device__ __forceinline__ uint16_t to16(float v) {
  if constexpr (FMT == 0) return __half_as_ushort(__float2half_rn(v));
  else return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}
template <int FMT>
__device__ __forceinline__ float round_to(float v) {
  if constexpr (FMT == 0) return __half2float(__float2half_rn(v));
  else return __bfloat162float(__float2bfloat16_rn(v));
}

// Core-matrix layout of a rows x K tile: element (r, kcol) at byte offset
// ((r / 8) * (KMAX / 8) + kcol / 8) * 128 + (r % 8) * 16 + (kcol % 8) * 2.
__device__ __forceinline__ int core_off(int r, int kc) {
  return (((r >> 3) * (TC_KMAX / 8) + (kc >> 3)) << 7) + ((r & 7) << 4) + ((kc & 7) << 1);
}

// Real: C -= A A^T with one accumulator.  Complex (CX, A and C interleaved
// re/im): with A = Ar + i Ai the Hermitian update C -= A A^H is two real
// products of depth 2k sharing the operand B = [Ar Ai]:
//   Re: [Ar Ai] B^T = Ar Ar^T + Ai Ai^T,   Im: [Ai -Ar] B^T = Ai Ar^T - Ar Ai^T,
// accumulated in two 128-column halves of tensor memory.  ROUND: the
// updated entries are rounded to the format (the factor's storage) in the
// epilogue.
template <int FMT, bool CX>
__global__ void __launch_bounds__(TC_THREADS)
tc_syrk_kernel(int n, int k, const float* __restrict__ A, long long lda, float* __restrict__ C, long long ldc,
               int round_out, int* err, long long wait_limit) {
  constexpr int NACC = CX ? 2 : 1;
  constexpr int TILE_BYTES = TC_M * TC_KMAX * 2;
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* Bs = sm;                      // [Ar Ai] rows of the column tile
  unsigned char* As0 = sm + TILE_BYTES;        // [Ar Ai] rows of the row tile
  unsigned char* As1 = sm + 2 * TILE_BYTES;    // [Ai -Ar] rows of the row tile (complex)
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  // tile (tm, tn), tn <= tm: blockIdx.x enumerates the lower triangle of tiles
  int tm = 0, t = blockIdx.x;
  while (t > tm) { t -= tm + 1; ++tm; }
  const int tn = t;
  const int m0 = tm * TC_M, n0 = tn * TC_N;
  const int keff = CX ? 2 * k : k;
  const int kp = (keff + 15) & ~15;  // depth padded to the MMA's K

  if (wid == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(NACC * TC_N));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // operands, converted to the format (exact for values of the format): a
  // thread takes one row and 8 consecutive depth indices -- one 16-byte row
  // of a core matrix, stored at once; consecutive threads take consecutive
  // rows (coalesced global loads, conflict-free 16-byte shared stores)
  for (int e = tid; e < TC_M * (kp / 8); e += TC_THREADS) {
    const int r = e % TC_M, k8 = (e / TC_M) * 8;
    const int ga = m0 + r, gb = n0 + r;
    uint32_t pa[4], pb[4], pi[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t wa = 0, wb = 0, wi = 0;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int kc = k8 + 2 * q + h;
        if constexpr (!CX) {
          const float va = (ga < n && kc < k) ? A[ga + (long long)kc * lda] : 0.0f;
          const float vb = (gb < n && kc < k) ? A[gb + (long long)kc * lda] : 0.0f;
          wa |= (uint32_t)to16<FMT>(va) << (16 * h);
          wb |= (uint32_t)to16<FMT>(vb) << (16 * h);
        } else {
          const bool hi = kc >= k;  // second half of the depth: the imaginary parts
          const int l = hi ? kc - k : kc;
          const bool in = kc < keff;
          float2 x = make_float2(0.f, 0.f), y = make_float2(0.f, 0.f);
          if (in && ga < n) x = *reinterpret_cast<const float2*>(A + 2 * (ga + (long long)l * lda));
          if (in && gb < n) y = *reinterpret_cast<const float2*>(A + 2 * (gb + (long long)l * lda));
          wa |= (uint32_t)to16<FMT>(hi ? x.y : x.x) << (16 * h);
          wi |= (uint32_t)to16<FMT>(hi ? -x.x : x.y) << (16 * h);
          wb |= (uint32_t)to16<FMT>(hi ? y.y : y.x) << (16 * h);
        }
      }
      pa[q] = wa;
      pb[q] = wb;
      pi[q] = wi;
    }
    const int off = core_off(r, k8);
    *reinterpret_cast<uint4*>(As0 + off) = make_uint4(pa[0], pa[1], pa[2], pa[3]);
    *reinterpret_cast<uint4*>(Bs + off) = make_uint4(pb[0], pb[1], pb[2], pb[3]);
    if constexpr (CX) *reinterpret_cast<uint4*>(As1 + off) = make_uint4(pi[0], pi[1], pi[2], pi[3]);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic stores -> tensor-core reads
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  if (tid == 0) {
    constexpr uint32_t LBO = 128, SBO = (TC_KMAX / 8) * 128;
    const uint32_t idesc = idesc_f16(FMT, TC_M, TC_N);
    const uint32_t b0 = smem_u32(Bs);
#pragma unroll
    for (int h = 0; h < NACC; ++h) {
      const uint32_t a0 = smem_u32(h == 0 ? As0 : As1);
      for (int kk = 0; kk < kp / 16; ++kk) {
        const uint64_t da = smem_desc(a0 + kk * 2 * 128, LBO, SBO);
        const uint64_t db = smem_desc(b0 + kk * 2 * 128, LBO, SBO);
        const uint32_t acc = kk > 0 ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t"
            "}" ::"r"(tmem + (uint32_t)(h * TC_N)), "l"(da), "l"(db), "r"(idesc), "r"(acc)
            : "memory");
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(&mbar))
                 : "memory");
  }
  // wait for the MMAs: at most wait_limit non-blocking polls
  uint32_t done = 0;
  for (long long it = 0; it < wait_limit && !done; ++it) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t"
        "}"
        : "=r"(done)
        : "r"(smem_u32(&mbar)), "r"(0u)
        : "memory");
  }
  done = __syncthreads_and(done);  // uniform: the epilogue's tcgen05.ld is warp-synchronous
  if (!done && tid == 0) {
    atomicExch(err, 1);
    // the wait gave up: let the MMAs that were issued finish (bounded, at the
    // normal limit) before their tensor memory is released
    uint32_t drained = 0;
    for (long long it = 0; it < TC_WAIT_LIMIT && !drained; ++it) {
      asm volatile(
          "{\n\t.reg .pred p;\n\t"
          "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t"
          "}"
          : "=r"(drained)
          : "r"(smem_u32(&mbar)), "r"(0u)
          : "memory");
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (done) {
    // warp w may read accumulator lanes (rows) 32 (w % 4) .. + 31 only; the
    // two warpgroups split the columns
    const int lg = wid & 3, ch = wid >> 2;
    const int row = m0 + 32 * lg + lane;
    for (int c0 = ch * (TC_N / 2); c0 < (ch + 1) * (TC_N / 2); c0 += 16) {
      uint32_t v[NACC][16];
#pragma unroll
      for (int h = 0; h < NACC; ++h) {
        const uint32_t taddr = tmem + ((uint32_t)(32 * lg) << 16) + (uint32_t)(h * TC_N + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15}, [%16];"
            : "=r"(v[h][0]), "=r"(v[h][1]), "=r"(v[h][2]), "=r"(v[h][3]), "=r"(v[h][4]), "=r"(v[h][5]),
              "=r"(v[h][6]), "=r"(v[h][7]), "=r"(v[h][8]), "=r"(v[h][9]), "=r"(v[h][10]), "=r"(v[h][11]),
              "=r"(v[h][12]), "=r"(v[h][13]), "=r"(v[h][14]), "=r"(v[h][15])
            : "r"(taddr));
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int col = n0 + c0 + j;
        if (row < n && col < n && row >= col) {
          if constexpr (!CX) {
            float* c = C + row + (long long)col * ldc;
            const float r = *c - __uint_as_float(v[0][j]);
            *c = round_out ? round_to<FMT>(r) : r;
          } else {
            float2* c = reinterpret_cast<float2*>(C + 2 * (row + (long long)col * ldc));
            float2 x = *c;
            x.x -= __uint_as_float(v[0][j]);
            x.y -= __uint_as_float(v[1][j]);
            if (round_out) x = make_float2(round_to<FMT>(x.x), round_to<FMT>(x.y));
            *c = x;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (wid == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NACC * TC_N));
}

template <int FMT, bool CX>
static void launch_tc(cudaStream_t st, int tiles, int n, int k, const float* A, long long lda, float* C,
                      long long ldc, int round_out, int* err, long long wait_limit) {
  const size_t sm = (size_t)(CX ? 3 : 2) * TC_M * TC_KMAX * 2;
  // one attribute call per instantiation (thread-safe static initialisation)
  static const bool opened =
      cudaFuncSetAttribute(tc_syrk_kernel<FMT, CX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) ==
      cudaSuccess;
  (void)opened;
  count_launch();
  tc_syrk_kernel<FMT, CX><<<tiles, TC_THREADS, sm, st>>>(n, k, A, lda, C, ldc, round_out, err, wait_limit);
}

// C (n x n, ld ldc, lower triangle) -= A A^T (A A^H when cx: A, C complex
// interleaved, ld in complex elements), A n x k holding values of the format
// fmt (1 fp16, 2 bf16), k <= 128 (64 complex); round_out: round the updated
// entries to the format.  Returns false when k or fmt is out of range (the
// caller then uses the CUDA-core GEMM).
bool tc_syrk(cudaStream_t st, int fmt, bool cx, int n, int k, const float* A, long long lda, float* C,
             long long ldc, bool round_out, int* err, long long wait_polls) {
  const long long wl = wait_polls > 0 ? std::min(wait_polls, TC_WAIT_LIMIT) : TC_WAIT_LIMIT;
  if (n <= 0 || k <= 0) return true;
  if ((cx ? 2 * k : k) > TC_KMAX || (fmt != 1 && fmt != 2)) return false;
  const int nt = (n + TC_M - 1) / TC_M;
  const int tiles = nt * (nt + 1) / 2;
  const int r = round_out ? 1 : 0;
  if (fmt == 1) {
    if (cx) launch_tc<0, true>(st, tiles, n, k, A, lda, C, ldc, r, err, wl);
    else launch_tc<0, false>(st, tiles, n, k, A, lda, C, ldc, r, err, wl);
  } else {
    if (cx) launch_tc<1, true>(st, tiles, n, k, A, lda, C, ldc, r, err, wl);
    else launch_tc<1, false>(st, tiles, n, k, A, lda, C, ldc, r, err, wl);
  }
  return true;
}

}  // namespace mpl

// ---- C ABI: the update as a step of the factorisation (for checks) --------
#include "mplobpcg_steps.h"

extern "C" mpl_status mpl_step_lowp_syrk(int fmt, int is_complex, int64_t n, int64_t k, const void* A, int64_t lda,
                                         void* C, int64_t ldc, int round_out, int64_t wait_polls, void* stream) {
  const int64_t kmax = is_complex ? mpl::TC_KMAX / 2 : mpl::TC_KMAX;
  if ((fmt != 1 && fmt != 2) || n < 0 || k < 1 || k > kmax || !A || !C || lda < n || ldc < n ||
      n > (1LL << 31) - 1)
    return MPL_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int* err = nullptr;
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return MPL_ENOMEM;
  }
  int h = 0;
  mpl_status s = MPL_OK;
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) s = MPL_ECUDA;
  if (s == MPL_OK)
    mpl::tc_syrk(st, fmt, is_complex != 0, (int)n, (int)k, static_cast<const float*>(A), lda,
                 static_cast<float*>(C), ldc, round_out != 0, err, wait_polls);
  if (s == MPL_OK && cudaGetLastError() != cudaSuccess) s = MPL_ECUDA;
  if (s == MPL_OK && (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                      cudaStreamSynchronize(st) != cudaSuccess))
    s = MPL_ECUDA;
  if (s == MPL_OK && h != 0) s = MPL_ECUDA;  // the MMA completion wait gave up
  cudaFree(err);
  return s;
}
