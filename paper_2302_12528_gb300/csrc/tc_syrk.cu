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

// ------------------------------------------------------------------------
// FP32 trailing update on the tensor cores by 3xTF32 splitting: every FP32
// value x is cut into big = tf32(x) (round to nearest at the 10-bit mantissa)
// and small = tf32(x - big) (x - big is exact in FP32), and
//   A B^T ~ big_A big_B^T + big_A small_B^T + small_A big_B^T
// is accumulated in FP32 tensor memory by tcgen05.mma kind::tf32; each
// product of TF32 values is exact in FP32 and the dropped small_A small_B^T
// term and the rounding of small weigh about 2^-22 of the product.  Same
// tiles, operand construction (real; complex as [Ar Ai] / [Ai -Ar]) and
// epilogue as the 16-bit update above, without rounding to a format; the
// depth goes through shared memory in chunks of TF_KC.
constexpr int TF_KC = 32;                              // depth of a staged chunk
constexpr int TF_TILE = TC_M * TF_KC * 4;              // bytes of one operand tile (16 KB)

// Core-matrix layout of a 128 x TF_KC tile of 32-bit values: element (r, kc)
// at byte ((r / 8) * (TF_KC / 4) + kc / 4) * 128 + (r % 8) * 16 + (kc % 4) * 4.
__device__ __forceinline__ int core_off_tf(int r, int kc) {
  return (((r >> 3) * (TF_KC / 4) + (kc >> 2)) << 7) + ((r & 7) << 4) + ((kc & 3) << 2);
}

// Instruction descriptor of kind::tf32: FP32 accumulator, A and B TF32, both
// K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t tf32_rn(float x) {
  const uint32_t b = __float_as_uint(x);
  if ((b & 0x7F800000u) == 0x7F800000u) return b;      // Inf / NaN unchanged
  return (b + 0xFFFu + ((b >> 13) & 1u)) & 0xFFFFE000u;
}

template <bool CX>
__global__ void __launch_bounds__(TC_THREADS)
tf32x3_syrk_kernel(int n, int k, const float* __restrict__ A, long long lda, float* __restrict__ C, long long ldc,
                   int* err, long long wait_limit) {
  constexpr int NACC = CX ? 2 : 1;
  constexpr int NT = CX ? 6 : 4;                       // B big/small, A0 big/small (, A1 big/small)
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  int tm = 0, t = blockIdx.x;
  while (t > tm) { t -= tm + 1; ++tm; }
  const int tn = t;
  const int m0 = tm * TC_M, n0 = tn * TC_N;
  const int keff = CX ? 2 * k : k;
  const int nch = (keff + TF_KC - 1) / TF_KC;

  if (wid == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(NACC * TC_N));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  bool done = true;
  for (int c = 0; c < nch && done; ++c) {
    // stage chunk c: a thread takes one row and 4 consecutive depth indices
    // (one 16-byte row of a core matrix) of every operand tile
    for (int e = tid; e < TC_M * (TF_KC / 4); e += TC_THREADS) {
      const int r = e % TC_M, k4 = (e / TC_M) * 4;
      const int ga = m0 + r, gb = n0 + r;
      uint32_t ab[4], as_[4], bb[4], bs[4], ib[4], is_[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int kc = c * TF_KC + k4 + q;
        float va = 0.f, vb = 0.f, vi = 0.f;
        if constexpr (!CX) {
          if (kc < k) {
            if (ga < n) va = A[ga + (long long)kc * lda];
            if (gb < n) vb = A[gb + (long long)kc * lda];
          }
        } else {
          if (kc < keff) {
            const bool hi = kc >= k;  // second half of the depth: the imaginary parts
            const int l = hi ? kc - k : kc;
            float2 x = make_float2(0.f, 0.f), y = make_float2(0.f, 0.f);
            if (ga < n) x = *reinterpret_cast<const float2*>(A + 2 * (ga + (long long)l * lda));
            if (gb < n) y = *reinterpret_cast<const float2*>(A + 2 * (gb + (long long)l * lda));
            va = hi ? x.y : x.x;
            vi = hi ? -x.x : x.y;
            vb = hi ? y.y : y.x;
          }
        }
        ab[q] = tf32_rn(va);
        as_[q] = tf32_rn(va - __uint_as_float(ab[q]));
        bb[q] = tf32_rn(vb);
        bs[q] = tf32_rn(vb - __uint_as_float(bb[q]));
        ib[q] = tf32_rn(vi);
        is_[q] = tf32_rn(vi - __uint_as_float(ib[q]));
      }
      const int off = core_off_tf(r, k4);
      *reinterpret_cast<uint4*>(sm + 0 * TF_TILE + off) = make_uint4(bb[0], bb[1], bb[2], bb[3]);
      *reinterpret_cast<uint4*>(sm + 1 * TF_TILE + off) = make_uint4(bs[0], bs[1], bs[2], bs[3]);
      *reinterpret_cast<uint4*>(sm + 2 * TF_TILE + off) = make_uint4(ab[0], ab[1], ab[2], ab[3]);
      *reinterpret_cast<uint4*>(sm + 3 * TF_TILE + off) = make_uint4(as_[0], as_[1], as_[2], as_[3]);
      if constexpr (CX) {
        *reinterpret_cast<uint4*>(sm + 4 * TF_TILE + off) = make_uint4(ib[0], ib[1], ib[2], ib[3]);
        *reinterpret_cast<uint4*>(sm + 5 * TF_TILE + off) = make_uint4(is_[0], is_[1], is_[2], is_[3]);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic stores -> tensor-core reads
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      constexpr uint32_t LBO = 128, SBO = (TF_KC / 4) * 128;
      constexpr uint32_t idesc = idesc_tf32(TC_M, TC_N);
      const uint32_t base = smem_u32(sm);
#pragma unroll
      for (int h = 0; h < NACC; ++h) {
        const uint32_t abig = base + (2 + 2 * h) * TF_TILE, asml = abig + TF_TILE;
        const uint32_t bbig = base, bsml = base + TF_TILE;
#pragma unroll
        for (int kk = 0; kk < TF_KC / 8; ++kk) {
#pragma unroll
          for (int pr = 0; pr < 3; ++pr) {  // big big, big small, small big
            const uint64_t da = smem_desc((pr == 2 ? asml : abig) + kk * 256, LBO, SBO);
            const uint64_t db = smem_desc((pr == 1 ? bsml : bbig) + kk * 256, LBO, SBO);
            const uint32_t acc = (c > 0 || kk > 0 || pr > 0) ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "setp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t"
                "}" ::"r"(tmem + (uint32_t)(h * TC_N)),
                "l"(da), "l"(db), "r"(idesc), "r"(acc)
                : "memory");
          }
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&mbar))
                   : "memory");
    }
    // wait for this chunk's MMAs (their operands are overwritten next): at
    // most wait_limit non-blocking polls
    uint32_t ok = 0;
    for (long long it = 0; it < wait_limit && !ok; ++it) {
      asm volatile(
          "{\n\t.reg .pred p;\n\t"
          "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t"
          "}"
          : "=r"(ok)
          : "r"(smem_u32(&mbar)), "r"((uint32_t)(c & 1))
          : "memory");
    }
    done = __syncthreads_and(ok);
    if (!done && tid == 0) {
      atomicExch(err, 1);
      // let the MMAs that were issued finish (bounded, at the normal limit)
      uint32_t drained = 0;
      for (long long it = 0; it < TC_WAIT_LIMIT && !drained; ++it) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t"
            "}"
            : "=r"(drained)
            : "r"(smem_u32(&mbar)), "r"((uint32_t)(c & 1))
            : "memory");
      }
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  if (done) {
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
            C[row + (long long)col * ldc] -= __uint_as_float(v[0][j]);
          } else {
            float2* cp = reinterpret_cast<float2*>(C + 2 * (row + (long long)col * ldc));
            float2 x = *cp;
            x.x -= __uint_as_float(v[0][j]);
            x.y -= __uint_as_float(v[1][j]);
            *cp = x;
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

template <bool CX>
static void launch_tf32x3(cudaStream_t st, int tiles, int n, int k, const float* A, long long lda, float* C,
                          long long ldc, int* err, long long wait_limit) {
  const size_t sm = (size_t)(CX ? 6 : 4) * TF_TILE;
  static const bool opened =
      cudaFuncSetAttribute(tf32x3_syrk_kernel<CX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) ==
      cudaSuccess;
  (void)opened;
  count_launch();
  tf32x3_syrk_kernel<CX><<<tiles, TC_THREADS, sm, st>>>(n, k, A, lda, C, ldc, err, wait_limit);
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
  if ((cx ? 2 * k : k) > TC_KMAX || fmt < 1 || fmt > 3) return false;
  const int nt = (n + TC_M - 1) / TC_M;
  const int tiles = nt * (nt + 1) / 2;
  if (fmt == 3) {  // FP32 values, 3xTF32 products (round_out has no format to round to)
    if (cx) launch_tf32x3<true>(st, tiles, n, k, A, lda, C, ldc, err, wl);
    else launch_tf32x3<false>(st, tiles, n, k, A, lda, C, ldc, err, wl);
    return true;
  }
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
  if (fmt < 1 || fmt > 3 || n < 0 || k < 1 || k > kmax || !A || !C || lda < n || ldc < n ||
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
