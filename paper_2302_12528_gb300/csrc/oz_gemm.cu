// FP64-accurate products C = A B on the bf16 tensor cores by error-free
// splitting (Ozaki, Ogita, Oishi & Rump, "Error-free transformations of
// matrix multiplication by using fast routines of matrix multiplication and
// its applications", Numer. Algorithms 59, 2012), for the working-precision
// A X of the dense operator.
//
// Splitting.  Row r of A is scaled by its exponent e_r (|A_rk| < 2^e_r) and
// cut into OZ_S signed 8-bit digits by rounding to nearest:
//   u = A_rk 2^(8 - e_r),  q_i = rint(u),  u <- 256 (u - q_i),
// so A_rk = 2^(e_r - 8) sum_i q_i 2^(-8i) + O(2^(e_r - 8 - 8 OZ_S)), with
// |q_0| <= 256 and |q_i| <= 128 after it; every q_i 2^(-8i) is exact in
// bf16.  Columns of B likewise with exponents f_c.  All steps are exact in
// FP64 (u - rint(u) and the scaling by 256 round nothing).
//
// Products.  Slice pairs (i, j) with i + j = g share the scale 2^(-8g).
// Groups g < OZ_G are accumulated in their own FP32 tensor-memory
// accumulator over a window of OZ_WIN = 128 depth indices: every partial sum
// is an integer multiple of 2^(-8g) below 2^24 of it, so FP32 adds nothing
// to it.  The pairs with g >= OZ_G (relative weight <= 2^-32) share one FP32
// accumulator.  After each window the accumulators are folded into an int64
// fixed-point sum 2^S sum_g I_g 2^(-8g) (the tail rounded to the nearest
// unit 2^-S) on the integer pipes -- GB300 executes FP64 at 1/64 of FP32 --
// and depth splits of one tile add their int64 sums with exact, order-free
// atomics.  C = 2^(e_r + f_c - 16 - S) T, one FP64 scaling per entry.
//
// Tiles.  One CTA (16 warps) per 128-row tile and depth split; a depth chunk
// of 64 brings all OZ_S slices of A (7 x 16 KB) and of B (7 x NPAD x 128 B)
// into shared memory with bulk copies (the slices are stored pre-blocked in
// the canonical no-swizzle K-major core-matrix layout), one thread issues
// the 28 pairs x 4 tcgen05.mma (kind::f16, bf16, M = 128, N = NPAD), the
// completion is committed to an mbarrier; every wait has an iteration limit
// after which the CTA records an error, waits once more (bounded) for what
// it issued, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>

#include "common.cuh"
#include "oz_gemm.cuh"

namespace mpl {

namespace {

constexpr int OZ_BM = 128;                       // rows of a tile
constexpr int OZ_BK = 64;                        // depth of a chunk
constexpr int OZ_WIN_CHUNKS = OZ_WIN / OZ_BK;    // chunks per exact window
constexpr int OZ_THREADS = 512;  // four warpgroups: each reads a quarter of the columns back
constexpr int OZ_TILE_A = OZ_BM * OZ_BK;         // elements of one A slice block
constexpr long long OZ_WAIT_LIMIT = 1LL << 22;   // mbarrier polls before giving up
static_assert(OZ_WIN % OZ_BK == 0, "window of whole chunks");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// element offset of (r, kc) in a rows x 64 block, K-major core matrices
// (8 rows x 8 elements = 128 bytes; 8 of them along the chunk's depth)
__host__ __device__ __forceinline__ int core_off64(int r, int kc) {
  return (((r >> 3) * (OZ_BK / 8) + (kc >> 3)) << 6) + ((r & 7) << 3) + (kc & 7);
}

// Shared-memory matrix descriptor, no swizzle, K-major (LBO: next core
// matrix along K, SBO: next 8-row group), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// kind::f16 instruction descriptor: FP32 accumulator, bf16 A and B, K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// value of the real operand selected by mode from real (mode 0) or
// interleaved complex storage: 1 re, 2 im, 3 re + im (the 3M sum, in FP64);
// of the conjugate: 4 -im, 5 re - im
__device__ __forceinline__ double pick(const double* A, long long idx, int mode) {
  if (mode == 0) return A[idx];
  const double re = A[2 * idx], im = A[2 * idx + 1];
  switch (mode) {
    case 1: return re;
    case 2: return im;
    case 3: return re + im;
    case 4: return -im;
    default: return re - im;
  }
}

__device__ __forceinline__ int exp_of(double amax) {
  if (!(amax > 0.0)) return INT_MIN;
  int e;
  frexp(amax, &e);  // amax = f 2^e, f in [0.5, 1): |x| <= amax < 2^e
  return e;
}

__global__ void fill_int_kernel(int n, int* p, int v) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = v;
}

// e[r] = max over k of the exponent of |A(r, k)| (rows: threads, depth: grid y)
__global__ void row_exp_kernel(int n, int k, const double* __restrict__ A, long long lda, int mode,
                               int* __restrict__ e) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int k0 = blockIdx.y * 256, k1 = min(k, k0 + 256);
  double m = 0.0;
  for (int kk = k0; kk < k1; ++kk) m = fmax(m, fabs(pick(A, r + (long long)kk * lda, mode)));
  const int ex = exp_of(m);
  if (ex != INT_MIN) atomicMax(e + r, ex);
}

// f[c] = max over k of the exponent of |B(k, c)| (one block per column)
__global__ void col_exp_kernel(int k, const double* __restrict__ B, long long ldb, int mode, int* __restrict__ f) {
  __shared__ double red[256];
  const int c = blockIdx.x;
  double m = 0.0;
  for (int kk = threadIdx.x; kk < k; kk += blockDim.x) m = fmax(m, fabs(pick(B, kk + (long long)c * ldb, mode)));
  red[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int ex = exp_of(red[0]);
    f[c] = ex == INT_MIN ? 0 : ex;
  }
}

__global__ void clamp_exp_kernel(int n, int* e) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (e[i] == INT_MIN) e[i] = 0;
}

__device__ __forceinline__ uint16_t bf16_bits_exact(double q, int i) {
  // q integer, |q| <= 256: q 2^(-8i) has <= 8 significant bits
  return __bfloat16_as_ushort(__float2bfloat16_rn((float)ldexp(q, -8 * i)));
}

// The OZ_S digits of one element u = x 2^(8 - ex) (|u| <= 256).
__device__ __forceinline__ void digits(double x, int ex, uint16_t out[OZ_S]) {
  double u = ldexp(x, 8 - ex);
#pragma unroll
  for (int i = 0; i < OZ_S; ++i) {
    const double q = rint(u);
    out[i] = bf16_bits_exact(q, i);
    u = (u - q) * 256.0;
  }
}

// Row slices of A (rows padded to ntile * 128, depth to nchunk * 64, zeros
// outside): slice i of tile t, chunk c is the 128 x 64 block at
// ((i * ntile + t) * nchunk + c) * 8192.
__global__ void split_rows_kernel(int n, int k, const double* __restrict__ A, long long lda, int mode,
                                  const int* __restrict__ e, int ntile, int nchunk, uint16_t* __restrict__ Q) {
  const long long rows = (long long)ntile * OZ_BM, tot = rows * ((long long)nchunk * OZ_BK);
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < tot;
       id += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(id % rows), kk = (int)(id / rows);
    const double x = (r < n && kk < k) ? pick(A, r + (long long)kk * lda, mode) : 0.0;
    uint16_t d[OZ_S];
    digits(x, r < n ? e[r] : 0, d);
    const int t = r / OZ_BM, c = kk / OZ_BK;
    const int off = core_off64(r % OZ_BM, kk % OZ_BK);
#pragma unroll
    for (int i = 0; i < OZ_S; ++i) Q[(((long long)i * ntile + t) * nchunk + c) * OZ_TILE_A + off] = d[i];
  }
}

// The same row slices of op(A) = A^T (A^H through the conjugate modes) from
// storage k x n (ld lda): depth runs along the stored columns (coalesced).
__global__ void split_rows_t_kernel(int n, int k, const double* __restrict__ A, long long lda, int mode,
                                    const int* __restrict__ e, int ntile, int nchunk, uint16_t* __restrict__ Q) {
  const long long kpad = (long long)nchunk * OZ_BK, tot = (long long)ntile * OZ_BM * kpad;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < tot;
       id += (long long)gridDim.x * blockDim.x) {
    const int kk = (int)(id % kpad), r = (int)(id / kpad);
    const double x = (r < n && kk < k) ? pick(A, kk + (long long)r * lda, mode) : 0.0;
    uint16_t d[OZ_S];
    digits(x, r < n ? e[r] : 0, d);
    const int t = r / OZ_BM, c = kk / OZ_BK;
    const int off = core_off64(r % OZ_BM, kk % OZ_BK);
#pragma unroll
    for (int i = 0; i < OZ_S; ++i) Q[(((long long)i * ntile + t) * nchunk + c) * OZ_TILE_A + off] = d[i];
  }
}

// Column slices of B (k x m; columns padded to npad, depth to nchunk * 64):
// slice j of chunk c is the npad x 64 block at (j * nchunk + c) * npad * 64.
__global__ void split_cols_kernel(int k, int m, const double* __restrict__ B, long long ldb, int mode,
                                  const int* __restrict__ f, int nchunk, int npad, uint16_t* __restrict__ P) {
  const long long tot = (long long)npad * nchunk * OZ_BK;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < tot;
       id += (long long)gridDim.x * blockDim.x) {
    const int kk = (int)(id % ((long long)nchunk * OZ_BK)), c = (int)(id / ((long long)nchunk * OZ_BK));
    const double x = (c < m && kk < k) ? pick(B, kk + (long long)c * ldb, mode) : 0.0;
    uint16_t d[OZ_S];
    digits(x, c < m ? f[c] : 0, d);
    const int ch = kk / OZ_BK;
    const int off = core_off64(c, kk % OZ_BK);
#pragma unroll
    for (int j = 0; j < OZ_S; ++j) P[((long long)j * nchunk + ch) * npad * OZ_BK + off] = d[j];
  }
}

// The same column slices of op(B) = B^T (B^H through the conjugate modes)
// from storage m x k (ld ldb).
__global__ void split_cols_t_kernel(int k, int m, const double* __restrict__ B, long long ldb, int mode,
                                    const int* __restrict__ f, int nchunk, int npad, uint16_t* __restrict__ P) {
  const long long tot = (long long)npad * nchunk * OZ_BK;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < tot;
       id += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(id % npad), kk = (int)(id / npad);
    const double x = (c < m && kk < k) ? pick(B, c + (long long)kk * ldb, mode) : 0.0;
    uint16_t d[OZ_S];
    digits(x, c < m ? f[c] : 0, d);
    const int ch = kk / OZ_BK;
    const int off = core_off64(c, kk % OZ_BK);
#pragma unroll
    for (int j = 0; j < OZ_S; ++j) P[((long long)j * nchunk + ch) * npad * OZ_BK + off] = d[j];
  }
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  for (long long it = 0; it < OZ_WAIT_LIMIT && !done; ++it) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t"
        "}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
  }
  return done != 0;
}

// T (rows x NPAD int64, column-major, ld = ntile * 128) += the fixed-point
// product of the slices of tile blockIdx.x over the chunks of split
// blockIdx.y.
template <int NPAD>
__global__ void __launch_bounds__(OZ_THREADS, 1)
oz_mma_kernel(int ntile, int nchunk, int chunks_per_split, const uint16_t* __restrict__ QA,
              const uint16_t* __restrict__ PB, long long* __restrict__ T, int S, int* err) {
  static_assert(NPAD % 32 == 0 && NPAD >= 32 && NPAD <= 96, "N of the tile");
  constexpr int NACC = OZ_G + 1;                       // exact groups + the tail
  constexpr int A_BYTES = OZ_TILE_A * 2, B_BYTES = NPAD * OZ_BK * 2;
  constexpr int QCOLS = NPAD / 4;                      // columns a warp reads back
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* sA = sm;                              // OZ_S slices of A
  unsigned char* sB = sm + OZ_S * A_BYTES;             // OZ_S slices of B
  __shared__ __align__(8) uint64_t bar_load, bar_mma;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  const int t = blockIdx.x;
  const int c0 = blockIdx.y * chunks_per_split, c1 = min(nchunk, c0 + chunks_per_split);

  if (wid == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_load)), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_mma)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t bl = smem_u32(&bar_load), bm = smem_u32(&bar_mma);

  long long acc[QCOLS];
#pragma unroll
  for (int q = 0; q < QCOLS; ++q) acc[q] = 0;
  const int lg = wid & 3, ch = wid >> 2;               // accumulator lanes 32 lg.., columns ch * QCOLS..
  uint32_t fresh = (1u << NACC) - 1;                   // bit g: accumulator g starts a new window
  bool ok = true;
  uint32_t phase = 0;

  for (int c = c0; c < c1 && ok; ++c, phase ^= 1u) {
    if (tid == 0) {
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bl),
                   "r"((uint32_t)(OZ_S * (A_BYTES + B_BYTES)))
                   : "memory");
      for (int i = 0; i < OZ_S; ++i) {
        const uint16_t* ga = QA + (((long long)i * ntile + t) * nchunk + c) * OZ_TILE_A;
        const uint16_t* gb = PB + ((long long)i * nchunk + c) * NPAD * OZ_BK;
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(sA + i * A_BYTES)),
            "l"(ga), "r"((uint32_t)A_BYTES), "r"(bl)
            : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(sB + i * B_BYTES)),
            "l"(gb), "r"((uint32_t)B_BYTES), "r"(bl)
            : "memory");
      }
    }
    ok = __syncthreads_and(mbar_wait(bl, phase));
    if (!ok) break;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      constexpr uint32_t LBO = 128, SBO = (OZ_BK / 8) * 128;
      constexpr uint32_t idesc = idesc_bf16(OZ_BM, NPAD);
      for (int i = 0; i < OZ_S; ++i)
        for (int j = 0; i + j < OZ_S; ++j) {
          const int g = min(i + j, OZ_G);
          const uint32_t d_tmem = tmem + (uint32_t)(g * NPAD);
#pragma unroll
          for (int kk = 0; kk < OZ_BK / 16; ++kk) {
            const uint64_t da = smem_desc(smem_u32(sA + i * A_BYTES) + kk * 256, LBO, SBO);
            const uint64_t db = smem_desc(smem_u32(sB + j * B_BYTES) + kk * 256, LBO, SBO);
            const uint32_t accum = ((fresh >> g) & 1u) ? 0u : 1u;
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "setp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t"
                "}" ::"r"(d_tmem),
                "l"(da), "l"(db), "r"(idesc), "r"(accum)
                : "memory");
            fresh &= ~(1u << g);
          }
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bm)
                   : "memory");
    }
    ok = __syncthreads_and(mbar_wait(bm, phase));
    if (!ok) break;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const bool flush = ((c - c0) % OZ_WIN_CHUNKS == OZ_WIN_CHUNKS - 1) || (c == c1 - 1);
    if (flush) {
      // fold the window into the int64 sum: group g holds I_g 2^(-8g) exactly
#pragma unroll
      for (int c8 = 0; c8 < QCOLS; c8 += 8) {
#pragma unroll
        for (int g = 0; g < NACC; ++g) {
          uint32_t v[8];
          const uint32_t taddr = tmem + ((uint32_t)(32 * lg) << 16) + (uint32_t)(g * NPAD + ch * QCOLS + c8);
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                       : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                         "=r"(v[7])
                       : "r"(taddr));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float x = __uint_as_float(v[q]);
            if (g < OZ_G)  // I_g = x 2^(8g), an integer below 2^24: exact conversions
              acc[c8 + q] += (long long)__float2int_rn(ldexpf(x, 8 * g)) * (1LL << (S - 8 * g));
            else           // the tail, rounded to the unit 2^-S
              acc[c8 + q] += __float2ll_rn(ldexpf(x, S));
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      fresh = (1u << NACC) - 1;
    }
  }
  if (!ok) {
    if (tid == 0) atomicExch(err, 1);
    // let whatever was issued finish (bounded) before the memory is released
    mbar_wait(bl, phase);
    mbar_wait(bm, phase);
  } else {
    const long long ldt = (long long)ntile * OZ_BM;
    const long long row = (long long)t * OZ_BM + 32 * lg + lane;
#pragma unroll
    for (int q = 0; q < QCOLS; ++q)
      atomicAdd(reinterpret_cast<unsigned long long*>(T + row + (long long)(ch * QCOLS + q) * ldt),
                (unsigned long long)acc[q]);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (wid == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// C(r, c) = 2^(e_r + f_c - 16 - S) T(r, c)   (real), or the 3M combination
// of three such products (complex): Re = T1 - T2, Im = T3 - T1 - T2.
__global__ void combine_real_kernel(int n, int m, const long long* __restrict__ T, long long ldt,
                                    const int* __restrict__ e, const int* __restrict__ f, int S, double alpha,
                                    double beta, int lower_only, int col0, double* __restrict__ C, long long ldc) {
  const long long tot = (long long)n * m;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < tot;
       id += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(id % n), c = (int)(id / n);
    if (lower_only && r < col0 + c) continue;
    double v = alpha * ldexp((double)T[r + c * ldt], e[r] + f[c] - 16 - S);
    if (beta != 0.0) v += beta * C[r + c * ldc];
    C[r + c * ldc] = v;
  }
}

__global__ void combine_3m_kernel(int n, int m, const long long* __restrict__ T, long long ldt, long long tstride,
                                  const int* __restrict__ e, int estride, const int* __restrict__ f, int fstride,
                                  int S, double alpha, double beta, int lower_only, int col0, double* __restrict__ C,
                                  long long ldc) {
  const long long tot = (long long)n * m;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < tot;
       id += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(id % n), c = (int)(id / n);
    if (lower_only && r < col0 + c) continue;
    double p[3];
#pragma unroll
    for (int q = 0; q < 3; ++q)
      p[q] = ldexp((double)T[q * tstride + r + c * ldt], e[q * estride + r] + f[q * fstride + c] - 16 - S);
    double re = alpha * (p[0] - p[1]), im = alpha * (p[2] - p[0] - p[1]);
    if (beta != 0.0) {
      re += beta * C[2 * (r + c * ldc)];
      im += beta * C[2 * (r + c * ldc) + 1];
    }
    C[2 * (r + c * ldc)] = re;
    C[2 * (r + c * ldc) + 1] = im;
  }
}

inline int grid_for(long long tot) { return (int)std::min<long long>((tot + 255) / 256, 16LL * NUM_SMS); }

}  // namespace

// Fixed-point shift: with W windows of depth 128 the int64 sum stays below
// W * 2^(23.01 + S) < 2^63.
int oz_shift(long long k) {
  const long long w = std::max<long long>(1, (k + OZ_WIN - 1) / OZ_WIN);
  int lw = 0;
  while ((1LL << lw) < w) ++lw;
  return std::min(32, 39 - lw);
}

size_t oz_a_elems(int n, int k) {
  const long long ntile = (n + OZ_BM - 1) / OZ_BM, nchunk = (k + OZ_BK - 1) / OZ_BK;
  return (size_t)OZ_S * ntile * OZ_BM * nchunk * OZ_BK;
}
size_t oz_b_elems(int k, int npad) {
  const long long nchunk = (k + OZ_BK - 1) / OZ_BK;
  return (size_t)OZ_S * npad * nchunk * OZ_BK;
}
int oz_npad(int m) { return m <= 32 ? 32 : m <= 64 ? 64 : 96; }

void oz_split_a(cudaStream_t st, int mode, int n, int k, const double* A, long long lda, int* e, uint16_t* Q,
                bool trans) {
  const int ntile = (n + OZ_BM - 1) / OZ_BM, nchunk = (k + OZ_BK - 1) / OZ_BK;
  if (trans) {
    // row r of op(A) is stored column r: one block per row reduces its exponent
    count_launch(2);
    col_exp_kernel<<<n, 256, 0, st>>>(k, A, lda, mode, e);
    const long long tot = (long long)ntile * OZ_BM * nchunk * OZ_BK;
    split_rows_t_kernel<<<grid_for(tot), 256, 0, st>>>(n, k, A, lda, mode, e, ntile, nchunk, Q);
    return;
  }
  count_launch(3);
  fill_int_kernel<<<grid_for(n), 256, 0, st>>>(n, e, INT_MIN);
  row_exp_kernel<<<dim3((n + 255) / 256, (k + 255) / 256), 256, 0, st>>>(n, k, A, lda, mode, e);
  clamp_exp_kernel<<<grid_for(n), 256, 0, st>>>(n, e);
  const long long tot = (long long)ntile * OZ_BM * nchunk * OZ_BK;
  count_launch();
  split_rows_kernel<<<grid_for(tot), 256, 0, st>>>(n, k, A, lda, mode, e, ntile, nchunk, Q);
}

void oz_split_b(cudaStream_t st, int mode, int k, int m, const double* B, long long ldb, int* f, uint16_t* P,
                bool trans) {
  const int npad = oz_npad(m), nchunk = (k + OZ_BK - 1) / OZ_BK;
  if (trans) {
    // column c of op(B) is stored row c: row maxima by atomics
    count_launch(4);
    fill_int_kernel<<<grid_for(m), 256, 0, st>>>(m, f, INT_MIN);
    row_exp_kernel<<<dim3((m + 255) / 256, (k + 255) / 256), 256, 0, st>>>(m, k, B, ldb, mode, f);
    clamp_exp_kernel<<<grid_for(m), 256, 0, st>>>(m, f);
    const long long tot = (long long)npad * nchunk * OZ_BK;
    split_cols_t_kernel<<<grid_for(tot), 256, 0, st>>>(k, m, B, ldb, mode, f, nchunk, npad, P);
    return;
  }
  count_launch(2);
  col_exp_kernel<<<m, 256, 0, st>>>(k, B, ldb, mode, f);
  const long long tot = (long long)npad * nchunk * OZ_BK;
  split_cols_kernel<<<grid_for(tot), 256, 0, st>>>(k, m, B, ldb, mode, f, nchunk, npad, P);
}

template <int NPAD>
static void launch_mma(cudaStream_t st, int ntile, int nchunk, int nsplit, int cps, const uint16_t* Q,
                       const uint16_t* P, long long* T, int S, int* err) {
  const size_t sm = (size_t)OZ_S * (OZ_TILE_A * 2 + NPAD * OZ_BK * 2);
  // one attribute call per instantiation (thread-safe static initialisation)
  static const bool opened =
      cudaFuncSetAttribute(oz_mma_kernel<NPAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) ==
      cudaSuccess;
  (void)opened;
  count_launch();
  oz_mma_kernel<NPAD><<<dim3(ntile, nsplit), OZ_THREADS, sm, st>>>(ntile, nchunk, cps, Q, P, T, S, err);
}

// T (ntile * 128 x npad int64, zeroed by the caller) += fixed-point A B.
void oz_mma(cudaStream_t st, int n, int k, int m, const uint16_t* Q, const uint16_t* P, long long* T, int* err) {
  const int ntile = (n + OZ_BM - 1) / OZ_BM, nchunk = (k + OZ_BK - 1) / OZ_BK;
  const int npad = oz_npad(m);
  // depth splits of whole windows: about 8 waves of one CTA per SM per launch
  const int want = std::max(1, (8 * NUM_SMS + ntile - 1) / ntile);
  const int nwin = (nchunk + OZ_WIN_CHUNKS - 1) / OZ_WIN_CHUNKS;
  const int nsplit = std::min(want, nwin);
  const int cps = ((nwin + nsplit - 1) / nsplit) * OZ_WIN_CHUNKS;
  const int nsp = (nchunk + cps - 1) / cps;
  const int S = oz_shift(k);
  if (npad == 32) launch_mma<32>(st, ntile, nchunk, nsp, cps, Q, P, T, S, err);
  else if (npad == 64) launch_mma<64>(st, ntile, nchunk, nsp, cps, Q, P, T, S, err);
  else launch_mma<96>(st, ntile, nchunk, nsp, cps, Q, P, T, S, err);
}

void oz_combine_real(cudaStream_t st, int n, int m, const long long* T, long long ldt, const int* e, const int* f,
                     int S, double* C, long long ldc, double alpha, double beta, bool lower_only, int col0) {
  count_launch();
  combine_real_kernel<<<grid_for((long long)n * m), 256, 0, st>>>(n, m, T, ldt, e, f, S, alpha, beta,
                                                                   lower_only ? 1 : 0, col0, C, ldc);
}

void oz_combine_3m(cudaStream_t st, int n, int m, const long long* T, long long ldt, long long tstride, const int* e,
                   int estride, const int* f, int fstride, int S, double* C, long long ldc, double alpha, double beta,
                   bool lower_only, int col0) {
  count_launch();
  combine_3m_kernel<<<grid_for((long long)n * m), 256, 0, st>>>(n, m, T, ldt, tstride, e, estride, f, fstride, S,
                                                                 alpha, beta, lower_only ? 1 : 0, col0, C, ldc);
}

long long oz_t_rows(int n) { return (long long)((n + OZ_BM - 1) / OZ_BM) * OZ_BM; }

}  // namespace mpl

// ---- C = alpha op(A) op(B) + beta C through the split product -------------
namespace mpl {
namespace {
struct OzPool {
  void* p[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // e, f, Q, P, T
  size_t bytes[5] = {0, 0, 0, 0, 0};
  int* err = nullptr;
  bool grow(int i, size_t b) {
    if (b <= bytes[i]) return true;
    if (p[i]) cudaFree(p[i]);
    p[i] = nullptr;
    bytes[i] = 0;
    if (cudaMalloc(&p[i], b) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    bytes[i] = b;
    return true;
  }
};
std::mutex& pool_mutex() {
  static std::mutex m;
  return m;
}
std::map<cudaStream_t, OzPool>& pools() {
  static std::map<cudaStream_t, OzPool> p;
  return p;
}
}  // namespace

bool oz_gemm_requested() {
  static const bool on = [] {
    const char* v = std::getenv("MPL_GEMM_SPLIT");
    return v && v[0] == '1';
  }();
  return on;
}

bool oz_gemm_fp64(cudaStream_t st, bool cx, bool ta, bool tb, int M, int N, int K, double alpha, const double* A,
                  long long lda, const double* B, long long ldb, double beta, double* C, long long ldc,
                  bool lower_only) {
  if (M < 1 || N < 1 || K < 1 || K > (1 << 21) || oz_shift(K) < 24 || !(beta == 0.0 || beta == 1.0)) return false;
  std::lock_guard<std::mutex> lock(pool_mutex());
  OzPool& P = pools()[st];
  const int np = cx ? 3 : 1, elt = cx ? 2 : 1;
  const size_t qa = oz_a_elems(M, K), pb = oz_b_elems(K, 96);
  const long long trows = oz_t_rows(M);
  const size_t tt = (size_t)trows * 96;
  if (!P.err) {
    if (cudaMalloc(&P.err, sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      P.err = nullptr;
      return false;
    }
    cudaMemsetAsync(P.err, 0, sizeof(int), st);
  }
  if (!P.grow(0, sizeof(int) * np * M) || !P.grow(1, sizeof(int) * np * 96) || !P.grow(2, 2 * np * qa) ||
      !P.grow(3, 2 * np * pb) || !P.grow(4, sizeof(long long) * np * tt))
    return false;
  int* e = static_cast<int*>(P.p[0]);
  int* f = static_cast<int*>(P.p[1]);
  uint16_t* Q = static_cast<uint16_t*>(P.p[2]);
  uint16_t* Pb = static_cast<uint16_t*>(P.p[3]);
  long long* T = static_cast<long long*>(P.p[4]);
  // 3M operands: re, im, re + im; of a conjugate transpose: re, -im, re - im
  auto mode_of = [&](int p, bool t) { return !cx ? 0 : !t ? p + 1 : (p == 0 ? 1 : p == 1 ? 4 : 5); };
  for (int p = 0; p < np; ++p) oz_split_a(st, mode_of(p, ta), M, K, A, lda, e + p * M, Q + p * qa, ta);
  const int S = oz_shift(K);
  for (int c0 = 0; c0 < N; c0 += 96) {
    const int nb = std::min(96, N - c0);
    // columns c0.. of op(B): stored columns (no transpose) or stored rows
    const double* Bc = B + (size_t)elt * (tb ? (size_t)c0 : (size_t)c0 * ldb);
    cudaMemsetAsync(T, 0, sizeof(long long) * np * tt, st);
    for (int p = 0; p < np; ++p) oz_split_b(st, mode_of(p, tb), K, nb, Bc, ldb, f + p * 96, Pb + p * pb, tb);
    for (int p = 0; p < np; ++p) oz_mma(st, M, K, nb, Q + p * qa, Pb + p * pb, T + p * tt, P.err);
    double* Cc = C + (size_t)elt * c0 * ldc;
    if (cx) oz_combine_3m(st, M, nb, T, trows, (long long)tt, e, M, f, 96, S, Cc, ldc, alpha, beta, lower_only, c0);
    else oz_combine_real(st, M, nb, T, trows, e, f, S, Cc, ldc, alpha, beta, lower_only, c0);
  }
  return true;
}

int oz_take_error(cudaStream_t st) {
  std::lock_guard<std::mutex> lock(pool_mutex());
  auto it = pools().find(st);
  if (it == pools().end() || !it->second.err) return 0;
  int h = 0;
  cudaMemcpyAsync(&h, it->second.err, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  if (h) cudaMemsetAsync(it->second.err, 0, sizeof(int), st);
  return h;
}

}  // namespace mpl

// ---- C ABI: the product as a step (for checks) -----------------------------
#include <vector>

#include "mplobpcg_steps.h"

extern "C" mpl_status mpl_step_split_gemm(int is_complex, int trans_a, int64_t n, int64_t k, int64_t m,
                                          const void* A, int64_t lda, const void* B, int64_t ldb, void* C,
                                          int64_t ldc, void* stream) {
  if (n < 1 || k < 1 || m < 1 || m > 96 || !A || !B || !C || lda < (trans_a ? k : n) || ldb < k || ldc < n ||
      n > (1LL << 30) || k > (1LL << 21) || mpl::oz_shift(k) < 24)
    return MPL_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int np = is_complex ? 3 : 1;
  const int npad = mpl::oz_npad((int)m);
  const long long trows = mpl::oz_t_rows((int)n);
  const size_t qa = mpl::oz_a_elems((int)n, (int)k), pb = mpl::oz_b_elems((int)k, npad);
  const size_t tt = (size_t)trows * npad;
  int *e = nullptr, *f = nullptr, *err = nullptr;
  uint16_t *Q = nullptr, *P = nullptr;
  long long* T = nullptr;
  mpl_status s = MPL_OK;
  auto alloc = [&](void** p, size_t bytes) {
    if (s == MPL_OK && cudaMalloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      s = MPL_ENOMEM;
    }
  };
  alloc((void**)&e, sizeof(int) * np * n);
  alloc((void**)&f, sizeof(int) * np * m);
  alloc((void**)&err, sizeof(int));
  alloc((void**)&Q, sizeof(uint16_t) * np * qa);
  alloc((void**)&P, sizeof(uint16_t) * np * pb);
  alloc((void**)&T, sizeof(long long) * np * tt);
  int h = 0;
  if (s == MPL_OK) {
    const double* a = static_cast<const double*>(A);
    const double* b = static_cast<const double*>(B);
    cudaMemsetAsync(err, 0, sizeof(int), st);
    cudaMemsetAsync(T, 0, sizeof(long long) * np * tt, st);
    for (int p = 0; p < np; ++p) {
      const int mode = is_complex ? p + 1 : 0;  // 3M: re, im, re + im
      // op(A) = A^H: re, -im, re - im of the stored matrix
      const int amode = (is_complex && trans_a) ? (p == 0 ? 1 : p == 1 ? 4 : 5) : mode;
      mpl::oz_split_a(st, amode, (int)n, (int)k, a, lda, e + p * n, Q + p * qa, trans_a != 0);
      mpl::oz_split_b(st, mode, (int)k, (int)m, b, ldb, f + p * m, P + p * pb);
    }
    for (int p = 0; p < np; ++p)
      mpl::oz_mma(st, (int)n, (int)k, (int)m, Q + p * qa, P + p * pb, T + p * tt, err);
    const int S = mpl::oz_shift(k);
    if (is_complex)
      mpl::oz_combine_3m(st, (int)n, (int)m, T, trows, (long long)tt, e, (int)n, f, (int)m, S,
                         static_cast<double*>(C), ldc, 1.0, 0.0, false, 0);
    else
      mpl::oz_combine_real(st, (int)n, (int)m, T, trows, e, f, S, static_cast<double*>(C), ldc, 1.0, 0.0, false, 0);
    if (cudaGetLastError() != cudaSuccess) s = MPL_ECUDA;
    if (s == MPL_OK && (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                        cudaStreamSynchronize(st) != cudaSuccess))
      s = MPL_ECUDA;
    if (s == MPL_OK && h != 0) s = MPL_ECUDA;  // a completion wait gave up
  }
  for (void* p : {(void*)e, (void*)f, (void*)err, (void*)Q, (void*)P, (void*)T})
    if (p) cudaFree(p);
  return s;
}
