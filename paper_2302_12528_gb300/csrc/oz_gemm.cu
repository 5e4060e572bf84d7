// FP64-accurate products C = A B on the bf16 tensor cores by error-free
// splitting (Ozaki, Ogita, Oishi & Rump, "Error-free transformations of
// matrix multiplication by using fast routines of matrix multiplication and
// its applications", Numer. Algorithms 59, 2012), for the working-precision
// products of Algorithm 3 (A X and, on request, the large Gram and update
// products).
//
// Splitting.  Row r of A is scaled by its exponent e_r (|A_rk| < 2^e_r) and
// cut into OZ_S = 8 balanced signed 8-bit digits by rounding to nearest:
//   u = A_rk 2^(7 - e_r),  q_i = rint(u),  u <- 256 (u - q_i),
// so |q_i| <= 128 (exact in bf16) and A_rk = 2^(e_r - 7) sum_i q_i 2^(-8i)
// up to 2^(e_r - 71).  Columns of B likewise with exponents f_c.  Every step
// is exact in FP64 (u - rint(u) and the scaling by 256 round nothing); the
// kernels compute the same digits from the bit pattern on the integer pipes
// (oz_fixed.cuh).
//
// Products.  The slice pairs (i, j) with i + j = g <= 7 (36 pairs; the
// dropped ones weigh <= 2^-64 of the leading product) are accumulated per
// shift group g in their own FP32 tensor-memory accumulator, over windows of
// OZ_WIN = 128 depth indices.  Every partial sum of group g is an integer of
// magnitude <= (g + 1) 2^14 x 128 <= 2^24, so the tensor core's FP32 sums
// are exact.  After each window the eight integers I_g are folded on the
// integer pipes into two int64 sums, hi = sum_{g<4} I_g 2^(24-8g) and
// lo = sum_{g>=4} I_g 2^(56-8g) (|hi| < 2^59, |lo| < 2^62 for depth <= 2^21),
// and the depth splits of a tile add theirs with exact, order-free int64
// atomics.  The product is then exact for the truncated digits:
//   C = 2^(e_r + f_c - 14) (hi 2^-24 + lo 2^-56),
// rounded once to FP64 in the combination kernel (oz_fixed_value) -- no
// rounding inside the dot product at all, unlike an FP64 GEMM.
//
// Tiles.  A CTA owns 128 rows of A, one block of NPAD <= 64 columns of B
// (8 accumulators x NPAD <= 512 tensor-memory columns) and a range of depth.
// Two column blocks of one row tile run as adjacent CTAs, so the second
// read of A's slices is served by L2.  The slices are stored pre-blocked per
// OZ_BK-deep chunk in the canonical no-swizzle K-major core-matrix layout,
// the eight slices of a chunk contiguous, so one bulk copy brings a chunk of
// A (64 KB) and one a chunk of B.  Warp roles: warp 0 copies (two stages in
// flight), warp 1 issues the 36 x 2 tcgen05.mma of a stage (ordered by A
// slice, so that each block of A is read from shared memory once and kept
// in the tensor core's collector buffer for its 8 - i products) and commits
// their completion, warps 2-17 fold the accumulators after each window
// (one lane polls the accumulator barrier, the other warps sleep on a
// hardware barrier).
//
// What bounds it (ncu, one real product at n = 8192, N = 48): the tensor
// pipe is active a third of the time, about 80 cycles per M = 128, N = 48,
// K = 16 MMA against about 24 of tensor work, and neither halving the
// shared-memory operand reads (collector reuse: tensor-core shared-memory
// wavefronts 61 % -> 28 %), nor four copies in flight instead of one, nor
// fewer launch waves changes the time; DRAM runs at 28 %, L2 at 17 %.  The
// product is bound by the number of MMA instructions, which the eight
// shift-group accumulators (8 x N <= 512 tensor-memory columns) cap at
// 128 x 64 outputs each; a CTA pair (cta_group::2, M = 256) would double
// the work per instruction.
//
// Every wait has an iteration limit; a role that gives up records an error
// and raises the CTA's abort flag, the others leave their waits, and the CTA
// waits (bounded) for the copies and MMAs it issued before it frees its
// tensor memory.
#include <cuda_bf16.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>

#include "common.cuh"
#include "oz_fixed.cuh"
#include "oz_gemm.cuh"

namespace mpl {

namespace {

constexpr int OZ_BM = 128;                         // rows of a tile
constexpr int OZ_STAGES_PER_WIN = OZ_WIN / OZ_BK;  // stages per exact window
constexpr int OZ_FOLD_WARPS = 16;
constexpr int OZ_THREADS = 32 * (2 + OZ_FOLD_WARPS);
constexpr int OZ_TILE_A = OZ_BM * OZ_BK;           // elements of one slice block of A
constexpr long long OZ_WAIT_LIMIT = 1LL << 22;     // mbarrier polls before giving up
static_assert(OZ_WIN % OZ_BK == 0, "window of whole stages");
static_assert(OZ_BK % 16 == 0, "whole MMA depth steps per stage");

// The stage ring of the product kernel for a column block of NPAD: NST
// stages of OZ_BK depth (A's and B's eight slices).  Two 32-deep stages:
// a ring of five 16-deep stages (four copies in flight instead of one)
// measured 11 % slower -- the product is bound by the issue of its small
// MMAs, not by operand delivery (see the header).
template <int NPAD>
struct OzRing {
  static constexpr int A_BYTES = OZ_S * OZ_TILE_A * 2;      // the 8 slices of one chunk of the row tile
  static constexpr int B_BYTES = OZ_S * NPAD * OZ_BK * 2;   // the 8 slices of one chunk of the column block
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr int NST = 2;
  static_assert(NST * STAGE <= 227 * 1024, "the ring fits the shared memory of a CTA");
  static_assert(STAGE % 1024 == 0, "stages keep the 1024-byte alignment of the buffer");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// element offset of (r, kc) in a rows x OZ_BK block, K-major core matrices
// (8 rows x 8 elements = 128 bytes; OZ_BK / 8 of them along the chunk's depth)
__host__ __device__ __forceinline__ int core_off32(int r, int kc) {
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


// Exponent of |x| as frexp gives it (|x| < 2^e, |x| >= 2^(e-1)); INT_MIN for
// zero.  From the bit pattern except for subnormal numbers.
__device__ __forceinline__ int exp_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFULL;
  if (b == 0) return INT_MIN;
  const int E = (int)(b >> 52);
  if (E) return E - 1022;
  int e;
  frexp(x, &e);
  return e;
}

// The NP real operands one stored entry feeds: NP = 1, the value `pick`
// selects by mode; NP = 3, the 3M operands of complex storage, (re, im,
// re + im) for mode 0 and those of the conjugate (re, -im, re - im) for
// mode 1.  One read of the entry serves all three.
template <int NP>
__device__ __forceinline__ void operands(const double* A, long long idx, int mode, double v[NP]) {
  if constexpr (NP == 1) {
    v[0] = pick(A, idx, mode);
  } else {
    const double re = A[2 * idx], im = A[2 * idx + 1];
    v[0] = re;
    v[1] = mode ? -im : im;
    v[2] = mode ? re - im : re + im;
  }
}

// exponent slots of NP operands (slot p of entry r at e[p * estride + r]):
// "no nonzero entry yet" before the maxima, 0 for all-zero rows after them
__global__ void fill_exp_kernel(int n, int* e, long long estride) {
  int* ep = e + blockIdx.y * estride;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) ep[i] = INT_MIN;
}

__global__ void clamp_exp_kernel(int n, int* e, long long estride) {
  int* ep = e + blockIdx.y * estride;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (ep[i] == INT_MIN) ep[i] = 0;
}

// e[p][r] = max over k of the exponent of operand p of A(r, k) (rows:
// threads, depth: grid y in chunks of kc -- 32 unless the grid would exceed
// its y limit -- enough blocks to keep many loads in flight on the thin
// operands of the basis updates)
inline int row_exp_chunk(int k) { return std::max(32, (k + 65534) / 65535); }
template <int NP>
__global__ void row_exp_kernel(int n, int k, int kc, const double* __restrict__ A, long long lda, int mode,
                               int* __restrict__ e, long long estride) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int k0 = blockIdx.y * kc, k1 = min(k, k0 + kc);
  int m[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) m[p] = INT_MIN;
#pragma unroll 4
  for (int kk = k0; kk < k1; ++kk) {
    double v[NP];
    operands<NP>(A, r + (long long)kk * lda, mode, v);
#pragma unroll
    for (int p = 0; p < NP; ++p) m[p] = max(m[p], exp_bits(v[p]));
  }
#pragma unroll
  for (int p = 0; p < NP; ++p)
    if (m[p] != INT_MIN) atomicMax(e + p * estride + r, m[p]);
}

// f[p][c] = max over k of the exponent of operand p of B(k, c): grid x
// columns, grid y chunks of OZ_EXP_CHUNK depth (256 threads x 8 independent
// loads each), a block reduction and one atomic per operand
constexpr int OZ_EXP_CHUNK = 2048;
template <int NP>
__global__ void __launch_bounds__(256) col_exp_kernel(int k, const double* __restrict__ B, long long ldb, int mode,
                                                      int* __restrict__ f, long long fstride) {
  __shared__ int red[NP][8];
  const int c = blockIdx.x, k0 = blockIdx.y * OZ_EXP_CHUNK;
  int m[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) m[p] = INT_MIN;
#pragma unroll
  for (int j = 0; j < OZ_EXP_CHUNK / 256; ++j) {
    const int kk = k0 + j * 256 + threadIdx.x;
    if (kk < k) {
      double v[NP];
      operands<NP>(B, kk + (long long)c * ldb, mode, v);
#pragma unroll
      for (int p = 0; p < NP; ++p) m[p] = max(m[p], exp_bits(v[p]));
    }
  }
#pragma unroll
  for (int p = 0; p < NP; ++p) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m[p] = max(m[p], __shfl_xor_sync(0xffffffffu, m[p], o));
    if ((threadIdx.x & 31) == 0) red[p][threadIdx.x >> 5] = m[p];
  }
  __syncthreads();
  if (threadIdx.x < NP) {
    int mm = INT_MIN;
#pragma unroll
    for (int w = 0; w < 8; ++w) mm = max(mm, red[threadIdx.x][w]);
    if (mm != INT_MIN) atomicMax(f + threadIdx.x * fstride + c, mm);
  }
}

__device__ __forceinline__ void store8(uint16_t* dst, const uint16_t v[8]) {
  uint4 w;
  w.x = (uint32_t)v[0] | ((uint32_t)v[1] << 16);
  w.y = (uint32_t)v[2] | ((uint32_t)v[3] << 16);
  w.z = (uint32_t)v[4] | ((uint32_t)v[5] << 16);
  w.w = (uint32_t)v[6] | ((uint32_t)v[7] << 16);
  *reinterpret_cast<uint4*>(dst) = w;
}

// Row slices of op(A) (n x k; rows padded to ntile * 128, depth to
// nchunk * OZ_BK, zeros outside) for each of the NP operands (slices of operand
// p at Q + p * qstride, exponents at e + p * estride): slice i of tile t,
// chunk c is the 128 x OZ_BK block at ((t * nchunk + c) * OZ_S + i) * 128 OZ_BK.
// One thread per row and 8 consecutive depth indices (one read of the
// stored entries for all operands; 16-byte stores into one core-matrix
// row), rows fastest across threads so that 8 neighbours fill a 128-byte
// core-matrix row group; trans: op(A) = A^T (A^H through the conjugate
// modes) from storage k x n (each thread then reads 128 contiguous bytes).
template <bool TRANS, int NP>
__global__ void split_rows_kernel(int n, int k, const double* __restrict__ A, long long lda, int mode,
                                  const int* __restrict__ e, long long estride, int ntile, int nchunk,
                                  uint16_t* __restrict__ Q, long long qstride) {
  const long long rows = (long long)ntile * OZ_BM, k8 = (long long)nchunk * (OZ_BK / 8);
  const long long tot = rows * k8;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < tot;
       id += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(id % rows), kb = (int)(id / rows);
    double x[8][NP];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int kk = kb * 8 + q;
      if (r < n && kk < k) {
        operands<NP>(A, TRANS ? kk + (long long)r * lda : r + (long long)kk * lda, mode, x[q]);
      } else {
#pragma unroll
        for (int p = 0; p < NP; ++p) x[q][p] = 0.0;
      }
    }
    const int t = r / OZ_BM, c = (kb * 8) / OZ_BK;
    const int off = core_off32(r % OZ_BM, (kb * 8) % OZ_BK);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const int ex = r < n ? e[p * estride + r] : 0;
      uint16_t d[OZ_S][8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        uint16_t dq[OZ_S];
        oz_digits(x[q][p], ex, dq);
#pragma unroll
        for (int i = 0; i < OZ_S; ++i) d[i][q] = dq[i];
      }
#pragma unroll
      for (int i = 0; i < OZ_S; ++i)
        store8(Q + p * qstride + (((long long)t * nchunk + c) * OZ_S + i) * OZ_TILE_A + off, d[i]);
    }
  }
}

// Column slices of op(B) (k x m; columns padded to ncb * npad, depth to
// nchunk * OZ_BK) for each of the NP operands (at P + p * pstride, exponents
// at f + p * fstride): slice j of column block b, chunk c is the npad x OZ_BK
// block at ((b * nchunk + c) * OZ_S + j) * npad * OZ_BK.  One thread per
// column and 8 consecutive depth indices, columns fastest across threads
// (8 neighbours fill a 128-byte core-matrix row group; with trans their
// loads are contiguous too); trans: op(B) = B^T (B^H) from storage m x k.
template <bool TRANS, int NP>
__global__ void split_cols_kernel(int k, int m, const double* __restrict__ B, long long ldb, int mode,
                                  const int* __restrict__ f, long long fstride, int nchunk, int npad, int ncb,
                                  uint16_t* __restrict__ P, long long pstride) {
  const long long k8 = (long long)nchunk * (OZ_BK / 8), cols = (long long)ncb * npad, tot = cols * k8;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < tot;
       id += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(id % cols), kb = (int)(id / cols);
    double x[8][NP];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int kk = kb * 8 + q;
      if (c < m && kk < k) {
        operands<NP>(B, TRANS ? c + (long long)kk * ldb : kk + (long long)c * ldb, mode, x[q]);
      } else {
#pragma unroll
        for (int p = 0; p < NP; ++p) x[q][p] = 0.0;
      }
    }
    const int b = c / npad, cc = c % npad, ch = (kb * 8) / OZ_BK;
    const int off = core_off32(cc, (kb * 8) % OZ_BK);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const int ex = c < m ? f[p * fstride + c] : 0;
      uint16_t d[OZ_S][8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        uint16_t dq[OZ_S];
        oz_digits(x[q][p], ex, dq);
#pragma unroll
        for (int j = 0; j < OZ_S; ++j) d[j][q] = dq[j];
      }
#pragma unroll
      for (int j = 0; j < OZ_S; ++j)
        store8(P + p * pstride + (((long long)b * nchunk + ch) * OZ_S + j) * npad * OZ_BK + off, d[j]);
    }
  }
}

// Bounded wait on an mbarrier phase; leaves early when the CTA aborts and
// raises the abort flag when the limit runs out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  for (long long it = 0; it < OZ_WAIT_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t"
        "}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (*abort_flag) return false;
  }
  *abort_flag = 1;
  return false;
}

// The same wait without the abort exit (teardown: waits for what was issued).
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < OZ_WAIT_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t"
        "}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return;
  }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// T (hi at T, lo at T + tlo; column-major, ld ldt) += the exact fixed-point
// product of row tile blockIdx.x / ncb with column block blockIdx.x % ncb
// over the chunks of split blockIdx.y.
template <int NPAD, bool COLLECT>
__global__ void __launch_bounds__(OZ_THREADS, 1)
oz_mma_kernel(int ncb, int nchunk, int chunks_per_split, const uint16_t* __restrict__ QA,
              const uint16_t* __restrict__ PB, long long* __restrict__ T, long long ldt, long long tlo, int* err,
              int single_split) {
  static_assert(NPAD % 16 == 0 && NPAD >= 16 && NPAD <= 64, "N of the tile");
  constexpr int A_BYTES = OzRing<NPAD>::A_BYTES;
  constexpr int B_BYTES = OzRing<NPAD>::B_BYTES;
  constexpr int STAGE = OzRing<NPAD>::STAGE;
  constexpr int NST = OzRing<NPAD>::NST;                 // stages in the ring
  constexpr int QC = NPAD / 4;                           // columns a fold warp reads back
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t bar_full[NST], bar_empty[NST], bar_accf, bar_acce;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  __shared__ int issued, committed;                      // stages copied / whose MMAs were committed
  __shared__ volatile int fold_go[2];                     // the accumulator poll's answer, by window parity
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  const int tile = blockIdx.x / ncb, cb = blockIdx.x % ncb;
  const int c0 = blockIdx.y * chunks_per_split, c1 = min(nchunk, c0 + chunks_per_split);
  const int nst = c1 - c0;
  const int nwin = (nst + OZ_STAGES_PER_WIN - 1) / OZ_STAGES_PER_WIN;

  if (tid == 0) {
    for (int b = 0; b < NST; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_full[b])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_empty[b])), "r"(1));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_accf)), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_acce)), "r"(OZ_FOLD_WARPS));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_flag = 0;
    issued = 0;
    committed = 0;
  }
  if (wid == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t sbase = smem_u32(sm);

  if (wid == 0) {
    // ---- producer: one bulk copy of A's and one of B's slices per stage
    if (lane == 0) {
      for (int s = 0; s < nst; ++s) {
        const int b = s % NST, r = s / NST;
        if (r > 0 && !mbar_wait(smem_u32(&bar_empty[b]), (r - 1) & 1, &abort_flag)) break;
        const uint32_t fb = smem_u32(&bar_full[b]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"((uint32_t)STAGE)
                     : "memory");
        const uint16_t* ga = QA + ((long long)tile * nchunk + c0 + s) * OZ_S * OZ_TILE_A;
        const uint16_t* gb = PB + ((long long)cb * nchunk + c0 + s) * OZ_S * NPAD * OZ_BK;
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                sbase + b * STAGE),
            "l"(ga), "r"((uint32_t)A_BYTES), "r"(fb)
            : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                sbase + b * STAGE + A_BYTES),
            "l"(gb), "r"((uint32_t)B_BYTES), "r"(fb)
            : "memory");
        issued = s + 1;
      }
    }
  } else if (wid == 1) {
    // ---- MMA issuer: 36 slice pairs x 2 depth steps per stage
    if (lane == 0) {
      constexpr uint32_t LBO = 128, SBO = (OZ_BK / 8) * 128;
      constexpr uint32_t idesc = idesc_bf16(OZ_BM, NPAD);
      for (int s = 0; s < nst; ++s) {
        const int b = s % NST, r = s / NST, w = s / OZ_STAGES_PER_WIN;
        const bool first = (s % OZ_STAGES_PER_WIN) == 0;
        if (first && w > 0 && !mbar_wait(smem_u32(&bar_acce), (w - 1) & 1, &abort_flag)) break;
        if (!mbar_wait(smem_u32(&bar_full[b]), r & 1, &abort_flag)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // the first MMA of each group in a window overwrites its accumulator
        const uint32_t acc0 = first ? 0u : 1u;
        const uint32_t sa = sbase + b * STAGE, sb = sa + A_BYTES;
        // descriptors of slice 0 / depth step 0; the others differ only in the
        // start address field (bytes >> 4), so constant offsets are added
        const uint64_t da0 = smem_desc(sa, LBO, SBO), db0 = smem_desc(sb, LBO, SBO);
        // A slice i at depth step kk feeds the groups g = i..7 with B slices
        // g - i: with COLLECT the consecutive MMAs of one (i, kk) keep A in
        // the tensor core's collector buffer (filled by the first, released
        // by the last), so each 128 x 16 block of A is read from shared
        // memory once per stage instead of 8 - i times (the operand reads of
        // small-N MMAs otherwise saturate shared memory before the tensor
        // pipe).  The first MMA into every accumulator is still
        // (i = 0, kk = 0).
#pragma unroll
        for (int i = 0; i < OZ_S; ++i) {
#pragma unroll
          for (int kk = 0; kk < OZ_BK / 16; ++kk) {
            const uint64_t da = da0 + (uint64_t)((i * (OZ_TILE_A * 2) + kk * 256) >> 4);
#pragma unroll
            for (int g = i; g < OZ_S; ++g) {
              const uint32_t d_tmem = tmem + (uint32_t)(g * NPAD);
              const uint64_t db = db0 + (uint64_t)(((g - i) * (NPAD * OZ_BK * 2) + kk * 256) >> 4);
              const uint32_t accum = (i == 0 && kk == 0) ? acc0 : 1u;
              if (!COLLECT || i == OZ_S - 1) {
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t"
                    "}" ::"r"(d_tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(accum)
                    : "memory");
              } else if (g == i) {
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%0], %1, %2, %3, p;\n\t"
                    "}" ::"r"(d_tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(accum)
                    : "memory");
              } else if (g == OZ_S - 1) {
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [%0], %1, %2, %3, p;\n\t"
                    "}" ::"r"(d_tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(accum)
                    : "memory");
              } else {
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16.collector::a::use [%0], %1, %2, %3, p;\n\t"
                    "}" ::"r"(d_tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(accum)
                    : "memory");
              }
            }
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&bar_empty[b]))
                     : "memory");
        if ((s % OZ_STAGES_PER_WIN) == OZ_STAGES_PER_WIN - 1 || s == nst - 1)
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(&bar_accf))
                       : "memory");
        committed = s + 1;
      }
    }
  } else {
    // ---- fold warps: accumulator lanes 32 (wid % 4) .., columns QC * ((wid - 2) / 4) ..
    const int lg = wid & 3, ch = (wid - 2) >> 2;
    long long hi[QC], lo[QC];
#pragma unroll
    for (int q = 0; q < QC; ++q) hi[q] = lo[q] = 0;
    bool ok = true;
    for (int w = 0; w < nwin && ok; ++w) {
      // one lane of one fold warp polls the accumulator barrier (every poll
      // is a shared-memory access that competes with the MMAs' operand
      // reads); the other fold warps sleep on hardware barrier 1 until it
      // has the answer.  The answer is double-buffered by window so that a
      // late reader of window w never sees window w + 1's: the poller
      // cannot pass the next barrier before every fold warp has.
      if (wid == 2 && lane == 0) fold_go[w & 1] = mbar_wait(smem_u32(&bar_accf), w & 1, &abort_flag) ? 1 : 0;
      asm volatile("bar.sync 1, %0;" ::"n"(32 * OZ_FOLD_WARPS) : "memory");
      ok = fold_go[w & 1] != 0;
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int c4 = 0; c4 < QC; c4 += 4) {
        // the eight groups' values of 4 columns: all loads in flight, one wait
        uint32_t v[OZ_S][4];
#pragma unroll
        for (int g = 0; g < OZ_S; ++g) {
          const uint32_t taddr = tmem + ((uint32_t)(32 * lg) << 16) + (uint32_t)(g * NPAD + ch * QC + c4);
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                       : "=r"(v[g][0]), "=r"(v[g][1]), "=r"(v[g][2]), "=r"(v[g][3])
                       : "r"(taddr));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int g = 0; g < OZ_S; ++g)
#pragma unroll
          for (int q = 0; q < 4; ++q) asm volatile("" : "+r"(v[g][q]));  // uses stay after the wait
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          // integers below 2^24 in magnitude: exact FP32 -> int32 conversions
          long long h = 0, l = 0;
#pragma unroll
          for (int g = 0; g < 4; ++g) h += (long long)__float2int_rn(__uint_as_float(v[g][q])) * (1LL << (24 - 8 * g));
#pragma unroll
          for (int g = 4; g < OZ_S; ++g) l += (long long)__float2int_rn(__uint_as_float(v[g][q])) * (1LL << (56 - 8 * g));
          hi[c4 + q] += h;
          lo[c4 + q] += l;
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bar_acce));
    }
    if (ok) {
      const long long row = (long long)tile * OZ_BM + 32 * lg + lane;
#pragma unroll
      for (int q = 0; q < QC; ++q) {
        const long long col = (long long)cb * NPAD + ch * QC + q;
        if (single_split) {  // the only writer of this tile: no zeroing, no atomics
          T[row + col * ldt] = hi[q];
          T[tlo + row + col * ldt] = lo[q];
        } else {
          atomicAdd(reinterpret_cast<unsigned long long*>(T + row + col * ldt), (unsigned long long)hi[q]);
          atomicAdd(reinterpret_cast<unsigned long long*>(T + tlo + row + col * ldt), (unsigned long long)lo[q]);
        }
      }
    }
  }
  __syncthreads();
  if (abort_flag) {
    if (tid == 0) {
      atomicExch(err, 1);
      // let the copies and MMAs that were issued finish (bounded) before the
      // shared and tensor memory are released
      for (int s = max(0, issued - NST); s < issued; ++s) mbar_drain(smem_u32(&bar_full[s % NST]), (s / NST) & 1);
      for (int s = max(0, committed - NST); s < committed; ++s)
        mbar_drain(smem_u32(&bar_empty[s % NST]), (s / NST) & 1);
    }
    __syncthreads();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (wid == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// C(r, c) = alpha 2^(e_r + f_c - 14) (hi 2^-24 + lo 2^-56) (+ beta C); rows
// by grid x (grid-stride), columns by grid y
__global__ void combine_real_kernel(int n, int m, const long long* __restrict__ T, long long ldt, long long tlo,
                                    const int* __restrict__ e, const int* __restrict__ f, double alpha, double beta,
                                    int lower_only, int col0, double* __restrict__ C, long long ldc) {
  const int c = blockIdx.y;
  const int fc = f[c] - 14;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    if (lower_only && r < col0 + c) continue;
    const long long t = r + c * ldt;
    double v = oz_fixed_value(T[t], T[tlo + t], e[r] + fc);
    if (alpha != 1.0) v *= alpha;
    if (beta != 0.0) v += beta * C[r + c * ldc];
    C[r + c * ldc] = v;
  }
}

// The 3M combination of three such products: Re = T1 - T2, Im = T3 - T1 - T2.
__global__ void combine_3m_kernel(int n, int m, const long long* __restrict__ T, long long ldt, long long tlo,
                                  long long tstride, const int* __restrict__ e, int estride,
                                  const int* __restrict__ f, int fstride, double alpha, double beta, int lower_only,
                                  int col0, double* __restrict__ C, long long ldc) {
  const int c = blockIdx.y;
  int fc[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) fc[q] = f[q * fstride + c] - 14;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    if (lower_only && r < col0 + c) continue;
    double p[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const long long t = q * tstride + r + c * ldt;
      p[q] = oz_fixed_value(T[t], T[tlo + t], e[q * estride + r] + fc[q]);
    }
    double re = p[0] - p[1], im = p[2] - p[0] - p[1];
    if (alpha != 1.0) {
      re *= alpha;
      im *= alpha;
    }
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

int oz_npad(int m) { return m <= 16 ? 16 : m <= 32 ? 32 : m <= 48 ? 48 : m <= 64 ? 64 : m <= 96 ? 48 : 64; }
int oz_ncb(int m) { return (m + oz_npad(m) - 1) / oz_npad(m); }
long long oz_t_rows(int n) { return (long long)((n + OZ_BM - 1) / OZ_BM) * OZ_BM; }
size_t oz_t_elems(int n, int m) { return (size_t)2 * oz_t_rows(n) * oz_ncb(m) * oz_npad(m); }

size_t oz_a_elems(int n, int k) {
  const long long ntile = (n + OZ_BM - 1) / OZ_BM, nchunk = (k + OZ_BK - 1) / OZ_BK;
  return (size_t)OZ_S * ntile * OZ_BM * nchunk * OZ_BK;
}
size_t oz_b_elems(int k, int m) {
  const long long nchunk = (k + OZ_BK - 1) / OZ_BK;
  return (size_t)OZ_S * oz_ncb(m) * oz_npad(m) * nchunk * OZ_BK;
}

namespace {
// exponents of the NP operands: every stored entry is read once per pass
// (maxima, then digits); four launches whatever NP is
template <int NP>
void split_a_np(cudaStream_t st, int mode, int n, int k, const double* A, long long lda, int* e, long long estride,
                uint16_t* Q, long long qstride, bool trans) {
  const int ntile = (n + OZ_BM - 1) / OZ_BM, nchunk = (k + OZ_BK - 1) / OZ_BK;
  const long long tot = (long long)ntile * OZ_BM * nchunk * (OZ_BK / 8);
  const int gx = std::min((n + 255) / 256, 4 * NUM_SMS);
  count_launch(4);
  fill_exp_kernel<<<dim3(gx, NP), 256, 0, st>>>(n, e, estride);
  if (trans)  // row r of op(A) is stored column r (contiguous along the depth)
    col_exp_kernel<NP><<<dim3(n, (k + OZ_EXP_CHUNK - 1) / OZ_EXP_CHUNK), 256, 0, st>>>(k, A, lda, mode, e, estride);
  else
    row_exp_kernel<NP><<<dim3((n + 255) / 256, (k + row_exp_chunk(k) - 1) / row_exp_chunk(k)), 256, 0, st>>>(
        n, k, row_exp_chunk(k), A, lda, mode, e, estride);
  clamp_exp_kernel<<<dim3(gx, NP), 256, 0, st>>>(n, e, estride);
  if (trans)
    split_rows_kernel<true, NP><<<grid_for(tot), 256, 0, st>>>(n, k, A, lda, mode, e, estride, ntile, nchunk, Q,
                                                               qstride);
  else
    split_rows_kernel<false, NP><<<grid_for(tot), 256, 0, st>>>(n, k, A, lda, mode, e, estride, ntile, nchunk, Q,
                                                                qstride);
}

template <int NP>
void split_b_np(cudaStream_t st, int mode, int k, int m, const double* B, long long ldb, int* f, long long fstride,
                uint16_t* P, long long pstride, bool trans) {
  const int npad = oz_npad(m), ncb = oz_ncb(m), nchunk = (k + OZ_BK - 1) / OZ_BK;
  const long long tot = (long long)ncb * npad * nchunk * (OZ_BK / 8);
  const int gx = std::min((m + 255) / 256, 4 * NUM_SMS);
  count_launch(4);
  fill_exp_kernel<<<dim3(gx, NP), 256, 0, st>>>(m, f, fstride);
  if (trans)  // column c of op(B) is stored row c
    row_exp_kernel<NP><<<dim3((m + 255) / 256, (k + row_exp_chunk(k) - 1) / row_exp_chunk(k)), 256, 0, st>>>(
        m, k, row_exp_chunk(k), B, ldb, mode, f, fstride);
  else
    col_exp_kernel<NP><<<dim3(m, (k + OZ_EXP_CHUNK - 1) / OZ_EXP_CHUNK), 256, 0, st>>>(k, B, ldb, mode, f, fstride);
  clamp_exp_kernel<<<dim3(gx, NP), 256, 0, st>>>(m, f, fstride);
  if (trans)
    split_cols_kernel<true, NP><<<grid_for(tot), 256, 0, st>>>(k, m, B, ldb, mode, f, fstride, nchunk, npad, ncb, P,
                                                               pstride);
  else
    split_cols_kernel<false, NP><<<grid_for(tot), 256, 0, st>>>(k, m, B, ldb, mode, f, fstride, nchunk, npad, ncb,
                                                                P, pstride);
}
}  // namespace

void oz_split_a(cudaStream_t st, int mode, int n, int k, const double* A, long long lda, int* e, uint16_t* Q,
                bool trans) {
  split_a_np<1>(st, mode, n, k, A, lda, e, 0, Q, 0, trans);
}

void oz_split_b(cudaStream_t st, int mode, int k, int m, const double* B, long long ldb, int* f, uint16_t* P,
                bool trans) {
  split_b_np<1>(st, mode, k, m, B, ldb, f, 0, P, 0, trans);
}

void oz_split_a_3m(cudaStream_t st, bool conj, int n, int k, const double* A, long long lda, int* e,
                   long long estride, uint16_t* Q, long long qstride, bool trans) {
  split_a_np<3>(st, conj ? 1 : 0, n, k, A, lda, e, estride, Q, qstride, trans);
}

void oz_split_b_3m(cudaStream_t st, bool conj, int k, int m, const double* B, long long ldb, int* f,
                   long long fstride, uint16_t* P, long long pstride, bool trans) {
  split_b_np<3>(st, conj ? 1 : 0, k, m, B, ldb, f, fstride, P, pstride, trans);
}

// Depth splits of whole windows.  One CTA fits an SM (tensor memory and
// shared memory), so a launch of C CTAs of w windows each takes about
// ceil(C / NUM_SMS) rounds of w windows plus a fixed start (first copies,
// tensor-memory allocation; about half a window): the split count with the
// fewest half-window units wins, ties to fewer splits (fewer atomics).
static void oz_plan(int n, int k, int m, int* nsp, int* cps) {
  const int ntile = (n + OZ_BM - 1) / OZ_BM, nchunk = (k + OZ_BK - 1) / OZ_BK;
  const long long tiles = (long long)ntile * oz_ncb(m);
  const int nwin = (nchunk + OZ_STAGES_PER_WIN - 1) / OZ_STAGES_PER_WIN;
  const int maxsp = (int)std::min<long long>(nwin, std::max<long long>(1, (32LL * NUM_SMS + tiles - 1) / tiles));
  int best_cw = nwin;
  long long best = LLONG_MAX;
  for (int s = 1; s <= maxsp; ++s) {
    const int cw = (nwin + s - 1) / s;                 // windows per split
    const long long ctas = tiles * ((nwin + cw - 1) / cw);
    const long long cost = ((ctas + NUM_SMS - 1) / NUM_SMS) * (2LL * cw + 1);
    if (cost < best) {
      best = cost;
      best_cw = cw;
    }
  }
  *cps = best_cw * OZ_STAGES_PER_WIN;
  *nsp = (nchunk + *cps - 1) / *cps;
}

bool oz_mma_accumulates(int n, int k, int m) {
  int nsp, cps;
  oz_plan(n, k, m, &nsp, &cps);
  return nsp > 1;
}

// MPL_OZ_COLLECTOR=0 issues every MMA with its A operand read from shared
// memory (no collector-buffer reuse); same products, for comparison.
static bool oz_collector() {
  static const bool on = [] {
    const char* v = std::getenv("MPL_OZ_COLLECTOR");
    return !(v && v[0] == '0');
  }();
  return on;
}

template <int NPAD, bool COLLECT>
static void launch_mma_as(cudaStream_t st, int ntile, int ncb, int nchunk, int nsplit, int cps, const uint16_t* Q,
                          const uint16_t* P, long long* T, long long ldt, long long tlo, int* err) {
  const size_t sm = (size_t)OzRing<NPAD>::NST * OzRing<NPAD>::STAGE;
  // one attribute call per instantiation (thread-safe static initialisation)
  static const bool opened =
      cudaFuncSetAttribute(oz_mma_kernel<NPAD, COLLECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) ==
      cudaSuccess;
  (void)opened;
  count_launch();
  oz_mma_kernel<NPAD, COLLECT><<<dim3(ntile * ncb, nsplit), OZ_THREADS, sm, st>>>(ncb, nchunk, cps, Q, P, T, ldt,
                                                                                   tlo, err, nsplit == 1 ? 1 : 0);
}

template <int NPAD>
static void launch_mma(cudaStream_t st, int ntile, int ncb, int nchunk, int nsplit, int cps, const uint16_t* Q,
                       const uint16_t* P, long long* T, long long ldt, long long tlo, int* err) {
  if (oz_collector()) launch_mma_as<NPAD, true>(st, ntile, ncb, nchunk, nsplit, cps, Q, P, T, ldt, tlo, err);
  else launch_mma_as<NPAD, false>(st, ntile, ncb, nchunk, nsplit, cps, Q, P, T, ldt, tlo, err);
}

void oz_mma(cudaStream_t st, int n, int k, int m, const uint16_t* Q, const uint16_t* P, long long* T, int* err) {
  const int ntile = (n + OZ_BM - 1) / OZ_BM, nchunk = (k + OZ_BK - 1) / OZ_BK;
  const int npad = oz_npad(m), ncb = oz_ncb(m);
  int nsp, cps;
  oz_plan(n, k, m, &nsp, &cps);
  const long long ldt = oz_t_rows(n), tlo = ldt * ncb * npad;
  switch (npad) {
    case 16: launch_mma<16>(st, ntile, ncb, nchunk, nsp, cps, Q, P, T, ldt, tlo, err); break;
    case 32: launch_mma<32>(st, ntile, ncb, nchunk, nsp, cps, Q, P, T, ldt, tlo, err); break;
    case 48: launch_mma<48>(st, ntile, ncb, nchunk, nsp, cps, Q, P, T, ldt, tlo, err); break;
    default: launch_mma<64>(st, ntile, ncb, nchunk, nsp, cps, Q, P, T, ldt, tlo, err); break;
  }
}

void oz_combine_real(cudaStream_t st, int n, int m, const long long* T, const int* e, const int* f, double* C,
                     long long ldc, double alpha, double beta, bool lower_only, int col0) {
  const long long ldt = oz_t_rows(n), tlo = (long long)oz_t_elems(n, m) / 2;
  count_launch();
  const dim3 grid(std::min((n + 255) / 256, 64), m);  // columns by grid y: no index division
  combine_real_kernel<<<grid, 256, 0, st>>>(n, m, T, ldt, tlo, e, f, alpha, beta, lower_only ? 1 : 0, col0, C, ldc);
}

void oz_combine_3m(cudaStream_t st, int n, int m, const long long* T, const int* e, int estride, const int* f,
                   int fstride, double* C, long long ldc, double alpha, double beta, bool lower_only, int col0) {
  const long long ldt = oz_t_rows(n), tt = (long long)oz_t_elems(n, m), tlo = tt / 2;
  count_launch();
  const dim3 grid(std::min((n + 255) / 256, 64), m);
  combine_3m_kernel<<<grid, 256, 0, st>>>(n, m, T, ldt, tlo, tt, e, estride, f, fstride, alpha, beta,
                                          lower_only ? 1 : 0, col0, C, ldc);
}

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

int oz_gemm_mode() {
  static const int mode = [] {
    const char* v = std::getenv("MPL_GEMM_SPLIT");
    if (v && v[0] == '0') return 0;
    return (v && v[0] == '1') ? 1 : 2;
  }();
  return mode;
}
bool oz_gemm_enabled() { return oz_gemm_mode() != 0; }

bool oz_gemm_fp64(cudaStream_t st, bool cx, bool ta, bool tb, int M, int N, int K, double alpha, const double* A,
                  long long lda, const double* B, long long ldb, double beta, double* C, long long ldc,
                  bool lower_only) {
  if (M < 1 || N < 1 || K < 1 || K > (1 << 21) || !(beta == 0.0 || beta == 1.0)) return false;
  std::lock_guard<std::mutex> lock(pool_mutex());
  OzPool& P = pools()[st];
  const int np = cx ? 3 : 1, elt = cx ? 2 : 1;
  // column chunks: <= 96 as one call, wider products in chunks of 1536 (24 blocks of 64)
  const int CW = N <= OZ_MAXM ? N : std::min(N, 1536);
  const size_t qa = oz_a_elems(M, K), pb = oz_b_elems(K, CW), tmax = oz_t_elems(M, CW);
  if (!P.err) {
    if (cudaMalloc(&P.err, sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      P.err = nullptr;
      return false;
    }
    cudaMemsetAsync(P.err, 0, sizeof(int), st);
  }
  if (!P.grow(0, sizeof(int) * np * M) || !P.grow(1, sizeof(int) * np * CW) || !P.grow(2, 2 * np * qa) ||
      !P.grow(3, 2 * np * pb) || !P.grow(4, sizeof(long long) * np * tmax))
    return false;
  int* e = static_cast<int*>(P.p[0]);
  int* f = static_cast<int*>(P.p[1]);
  uint16_t* Q = static_cast<uint16_t*>(P.p[2]);
  uint16_t* Pb = static_cast<uint16_t*>(P.p[3]);
  long long* T = static_cast<long long*>(P.p[4]);
  // 3M operands: re, im, re + im; of a conjugate transpose: re, -im, re - im
  if (cx) oz_split_a_3m(st, ta, M, K, A, lda, e, M, Q, (long long)qa, ta);
  else oz_split_a(st, 0, M, K, A, lda, e, Q, ta);
  for (int c0 = 0; c0 < N; c0 += CW) {
    const int nb = std::min(CW, N - c0);
    const size_t tt = oz_t_elems(M, nb);
    // columns c0.. of op(B): stored columns (no transpose) or stored rows
    const double* Bc = B + (size_t)elt * (tb ? (size_t)c0 : (size_t)c0 * ldb);
    if (oz_mma_accumulates(M, K, nb)) cudaMemsetAsync(T, 0, sizeof(long long) * np * tt, st);
    if (cx) oz_split_b_3m(st, tb, K, nb, Bc, ldb, f, CW, Pb, (long long)pb, tb);
    else oz_split_b(st, 0, K, nb, Bc, ldb, f, Pb, tb);
    for (int p = 0; p < np; ++p) oz_mma(st, M, K, nb, Q + p * qa, Pb + p * pb, T + p * tt, P.err);
    double* Cc = C + (size_t)elt * c0 * ldc;
    if (cx) oz_combine_3m(st, M, nb, T, e, M, f, CW, Cc, ldc, alpha, beta, lower_only, c0);
    else oz_combine_real(st, M, nb, T, e, f, Cc, ldc, alpha, beta, lower_only, c0);
  }
  return true;
}

// Every stream's flag (the sparse factorisation runs fronts on auxiliary
// streams joined into the caller's): read after synchronising with the
// caller's stream, cleared when set.
int oz_take_error(cudaStream_t st) {
  std::lock_guard<std::mutex> lock(pool_mutex());
  int any = 0;
  cudaStreamSynchronize(st);
  for (auto& kv : pools()) {
    if (!kv.second.err) continue;
    int h = 0;
    cudaMemcpy(&h, kv.second.err, sizeof(int), cudaMemcpyDeviceToHost);
    if (h) {
      cudaMemset(kv.second.err, 0, sizeof(int));
      any = 1;
    }
  }
  return any;
}

}  // namespace mpl

// ---- C ABI: the product as a step (for checks) -----------------------------
#include <vector>

#include "mplobpcg_steps.h"

extern "C" mpl_status mpl_step_split_gemm(int is_complex, int trans_a, int64_t n, int64_t k, int64_t m,
                                          const void* A, int64_t lda, const void* B, int64_t ldb, void* C,
                                          int64_t ldc, void* stream) {
  if (n < 1 || k < 1 || m < 1 || m > mpl::OZ_MAXM || !A || !B || !C || lda < (trans_a ? k : n) || ldb < k ||
      ldc < n || n > (1LL << 30) || k > (1LL << 21))
    return MPL_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int np = is_complex ? 3 : 1;
  const size_t qa = mpl::oz_a_elems((int)n, (int)k), pb = mpl::oz_b_elems((int)k, (int)m);
  const size_t tt = mpl::oz_t_elems((int)n, (int)m);
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
    if (mpl::oz_mma_accumulates((int)n, (int)k, (int)m)) cudaMemsetAsync(T, 0, sizeof(long long) * np * tt, st);
    for (int p = 0; p < np; ++p) {
      const int mode = is_complex ? p + 1 : 0;  // 3M: re, im, re + im
      // op(A) = A^H: re, -im, re - im of the stored matrix
      const int amode = (is_complex && trans_a) ? (p == 0 ? 1 : p == 1 ? 4 : 5) : mode;
      mpl::oz_split_a(st, amode, (int)n, (int)k, a, lda, e + p * n, Q + p * qa, trans_a != 0);
      mpl::oz_split_b(st, mode, (int)k, (int)m, b, ldb, f + p * m, P + p * pb);
    }
    for (int p = 0; p < np; ++p) mpl::oz_mma(st, (int)n, (int)k, (int)m, Q + p * qa, P + p * pb, T + p * tt, err);
    if (is_complex)
      mpl::oz_combine_3m(st, (int)n, (int)m, T, e, (int)n, f, (int)m, static_cast<double*>(C), ldc, 1.0, 0.0, false,
                         0);
    else
      mpl::oz_combine_real(st, (int)n, (int)m, T, e, f, static_cast<double*>(C), ldc, 1.0, 0.0, false, 0);
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
