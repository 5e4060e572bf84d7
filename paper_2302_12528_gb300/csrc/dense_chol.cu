// Dense lower-precision Cholesky factor and the multi-right-hand-side
// triangular sweeps that apply T = L^-* L^-1 (Section 5.1: the preconditioner
// is applied as a forward and a backward triangular solve in the lower
// precision).
//
// Factor: blocked right-looking.  Per NB-column step k one CTA factors the
// diagonal block in shared memory and also writes its inverse Dinv_k; the
// panel L_ik = A_ik Dinv_k^* and the lower-triangular trailing update
// A_ij -= L_ik L_jk^* are GEMMs.  Dinv is kept for the sweeps.
//
// Sweeps: one persistent launch per sweep over work items (block row of NBS
// rows, tile of right-hand sides), claimed in dependency order; the owner of
// a block row accumulates its updates from the finished rows above it
// (left-looking), applies the inverse diagonal block and publishes the row
// through a flag.  The backward sweep does the same with (L_ji)^* and Dinv^*.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>

#include "dense_chol.cuh"

namespace mpl {

template <typename T, int NB>
__global__ void __launch_bounds__(256)
potrf_diag_kernel(int kb, T* A, long long lda, T* Dinv, int col0, int* info) {
  using R = real_t<T>;
  extern __shared__ unsigned char sm[];
  constexpr int LD = NB + 1;
  T* S = reinterpret_cast<T*>(sm);      // factor, [c * LD + r]
  T* Si = S + NB * LD;                  // inverse
  __shared__ R piv;
  __shared__ int bad;
  const int tid = threadIdx.x;
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    const int r = e % NB, c = e / NB;
    S[c * LD + r] = (r < kb && c < kb && r >= c) ? A[r + (long long)c * lda] : zero_<T>();
  }
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    if (tid == 0) {
      R d = re_(S[j * LD + j]);
      if (!(d > R(0)) || !isfinite((double)d)) {
        if (bad == 0) bad = j + 1;
        d = R(1);
      }
      d = (sizeof(R) == 8) ? (R)sqrt((double)d) : (R)sqrtf((float)d);
      S[j * LD + j] = from_real<T>(d);
      piv = R(1) / d;
    }
    __syncthreads();
    const R rs = piv;
    for (int i = j + 1 + tid; i < kb; i += blockDim.x) S[j * LD + i] = S[j * LD + i] * rs;
    __syncthreads();
    const int w = kb - j - 1;
    for (int e = tid; e < w * w; e += blockDim.x) {
      const int i = j + 1 + e % w, l = j + 1 + e / w;
      if (i >= l) S[l * LD + i] = S[l * LD + i] - S[j * LD + i] * conj_(S[j * LD + l]);
    }
    __syncthreads();
  }
  // inverse of the lower-triangular block, one column per thread
  for (int c = tid; c < NB; c += blockDim.x) {
    for (int i = 0; i < NB; ++i) {
      T s = zero_<T>();
      if (c < kb && i >= c && i < kb) {
        s = (i == c) ? from_real<T>(R(1)) : zero_<T>();
        for (int l = c; l < i; ++l) s = s - S[l * LD + i] * Si[c * LD + l];
        const R dii = re_(S[i * LD + i]);
        s = s * (R(1) / dii);
      }
      Si[c * LD + i] = s;
    }
  }
  __syncthreads();
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    const int r = e % NB, c = e / NB;
    if (r < kb && c < kb) A[r + (long long)c * lda] = (r >= c) ? S[c * LD + r] : zero_<T>();
    Dinv[r + c * NB] = Si[c * LD + r];
  }
  if (tid == 0 && bad != 0) atomicCAS(info, 0, col0 + bad);
}

template <typename T>
__global__ void copy_block_kernel(int rows, int cols, const T* __restrict__ S, long long lds,
                                  T* __restrict__ D, long long ldd) {
  const long long total = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e % rows), c = (int)(e / rows);
    D[r + c * ldd] = S[r + c * lds];
  }
}

// ---- 16-bit storage format of the factor ---------------------------------
// Rounding to fp16 / bf16 at the points where a factorisation that stores
// its matrix in the format would store (scaled input, diagonal block, panel,
// trailing update); arithmetic stays FP32.
__device__ __forceinline__ float round16(float v, int fmt) {
  return fmt == 1 ? __half2float(__float2half_rn(v)) : __bfloat162float(__float2bfloat16_rn(v));
}
__device__ __forceinline__ float round16v(float v, int fmt) { return round16(v, fmt); }
__device__ __forceinline__ zf round16v(zf v, int fmt) { return {round16(v.x, fmt), round16(v.y, fmt)}; }
__device__ __forceinline__ double round16v(double v, int) { return v; }
__device__ __forceinline__ zd round16v(zd v, int) { return v; }

template <typename T>
__global__ void round_block_kernel(int rows, int cols, T* A, long long lda, int fmt, int lower_only) {
  const long long tot = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % rows), j = (int)(e / rows);
    if (lower_only && i < j) continue;
    T* a = A + i + (long long)j * lda;
    *a = round16v(*a, fmt);
  }
}

template <typename T>
void round_block(cudaStream_t st, int rows, int cols, T* A, long long lda, int fmt, bool lower_only) {
  if (fmt == 0 || fmt == 3 || rows <= 0 || cols <= 0) return;  // 3: FP32 storage, nothing to round
  const long long tot = (long long)rows * cols;
  count_launch();
  round_block_kernel<T><<<(int)std::min<long long>((tot + 255) / 256, 8 * NUM_SMS), 256, 0, st>>>(
      rows, cols, A, lda, fmt, lower_only ? 1 : 0);
}

template <typename T>
void dense_cholesky(cudaStream_t st, DenseFactor<T>& F, T* tmp, int* info, Scratch scr, int nfact,
                    long long col_offset, bool reset_info, int fmt16, int* tc_err) {
  constexpr int NB = CholBlock<T>::NB;
  const int n = F.n;
  if (nfact < 0 || nfact > n) nfact = n;
  F.nb = NB;
  F.nblk = ceil_div(nfact, NB);
  const long long lda = F.ldl;
  const size_t sm = 2 * (size_t)NB * (NB + 1) * sizeof(T);
  cudaFuncSetAttribute(potrf_diag_kernel<T, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (reset_info) cudaMemsetAsync(info, 0, sizeof(int), st);
  if (nfact == n) zero_upper<T>(st, n, F.L, lda);
  for (int b = 0; b < F.nblk; ++b) {
    const int k = b * NB;
    const int kb = (nfact - k < NB) ? (nfact - k) : NB;
    T* Akk = F.L + k + (long long)k * lda;
    T* Db = F.Dinv + (size_t)b * NB * NB;
    count_launch();
    potrf_diag_kernel<T, NB><<<1, 256, sm, st>>>(kb, Akk, lda, Db, (int)(col_offset + k), info);
    round_block<T>(st, kb, kb, Akk, lda, fmt16, true);
    const int rest = n - k - kb;
    if (rest <= 0) continue;
    T* Aik = F.L + (k + kb) + (long long)k * lda;
    // panel: L_ik = A_ik Dinv^*  (out of place, then copied back)
    gemm<T>(st, false, true, rest, kb, kb, real_t<T>(1), Aik, lda, Db, NB, real_t<T>(0), tmp, rest,
            false, scr);
    long long tot = (long long)rest * kb;
    int blocks = (int)((tot + 255) / 256);
    if (blocks > 8 * NUM_SMS) blocks = 8 * NUM_SMS;
    count_launch();
    copy_block_kernel<T><<<blocks, 256, 0, st>>>(rest, kb, tmp, rest, Aik, lda);
    round_block<T>(st, rest, kb, Aik, lda, fmt16, false);
    // trailing update, lower triangle only
    T* Att = F.L + (k + kb) + (long long)(k + kb) * lda;
    bool on_tc = false;
    if constexpr (sizeof(real_t<T>) == 4)
      if (fmt16 && tc_err)
        on_tc = tc_syrk(st, fmt16, tr<T>::cx, rest, kb, reinterpret_cast<const float*>(Aik), lda,
                        reinterpret_cast<float*>(Att), lda, true, tc_err);
    if (!on_tc) {
      gemm<T>(st, false, true, rest, rest, kb, real_t<T>(-1), Aik, lda, Aik, lda, real_t<T>(1), Att,
              lda, true, scr);
      round_block<T>(st, rest, rest, Att, lda, fmt16, true);
    }
  }
}

// d_i = 1 / sqrt(re A_ii) (FP64 arithmetic, stored FP32).
template <typename TW>
__global__ void diag_rsqrt_kernel(int n, const TW* __restrict__ A, long long lda, float* __restrict__ d) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    d[i] = (float)(1.0 / sqrt((double)re_(A[i + (long long)i * lda])));
}

// L = T(D A D) (lower triangle and diagonal; the upper is cleared by the factorisation).
template <typename T, typename TW>
__global__ void cast_scaled_kernel(int n, const TW* __restrict__ A, long long lda, const float* __restrict__ d,
                                   T* __restrict__ L, long long ldl) {
  const long long tot = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    if (i < j) continue;
    const double s = (double)d[i] * (double)d[j];
    L[i + (long long)j * ldl] = cvt<T, TW>(s * A[i + (long long)j * lda]);
  }
}

template <typename T, typename TW>
void scaled_lower_copy(cudaStream_t st, int n, const TW* A, long long lda, float* d, T* L, long long ldl) {
  count_launch();
  diag_rsqrt_kernel<TW><<<ceil_div(n, 256), 256, 0, st>>>(n, A, lda, d);
  const long long tot = (long long)n * n;
  count_launch();
  cast_scaled_kernel<T, TW><<<(int)std::min<long long>((tot + 255) / 256, 16 * NUM_SMS), 256, 0, st>>>(n, A, lda, d,
                                                                                                      L, ldl);
}

// B(i, :) *= d_i for B n x m (ld ldb).
template <typename T>
__global__ void scale_rows_kernel(int n, int m, T* B, long long ldb, const float* __restrict__ d) {
  const int j = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    B[i + (long long)j * ldb] = (real_t<T>)d[i] * B[i + (long long)j * ldb];
}

template <typename T>
void scale_rows(cudaStream_t st, int n, int m, T* B, long long ldb, const float* d) {
  if (n <= 0 || m <= 0) return;
  count_launch();
  scale_rows_kernel<T><<<dim3(std::min(ceil_div(n, 256), 64), m), 256, 0, st>>>(n, m, B, ldb, d);
}

// ------------------------------------------------------------------------
// triangular sweeps
// ------------------------------------------------------------------------
// Sweep geometry.  One persistent launch per sweep: work items are (sweep
// block row i, tile of CT right-hand sides), claimed in dependency order
// from an atomic counter.  The CTA that owns item (i, c) accumulates
// B_i - sum_j L_ij Y_j over the finished blocks j in a fixed order (so the
// result is bitwise reproducible), waiting on block j's flag before reading
// Y_j, then applies the inverse diagonal sub-block and publishes Y_i with a
// release store of its flag.  Items are claimed in order, so every item an
// owner waits for was claimed earlier by a CTA that is already running: the
// launch makes progress without co-residency guarantees.  The diagonal
// NBS x NBS sub-blocks of the stored Dinv_k are the inverses of the diagonal
// sub-blocks of the triangular L_kk.  FP32 types use NBS = 64, FP64 types 32;
// every CTA works on CT = 32 right-hand sides with a 16 x 16 thread grid,
// each thread owning an (NBS/16) x 2 register tile.  Each flag wait has an
// iteration limit; a CTA that gives up records an error word (read by the
// host after the solve) and still publishes its block, so no wait runs on
// indefinitely.
// NBS: rows of a block row; CT: right-hand sides per item; DB: two tile
// buffers (the next tile is loaded while the current one is multiplied).
// The FP32 sweeps wait on memory and take DB; the FP64 ones are bound by the
// FP64 pipe, where twice the shared memory per CTA only lowers the number of
// resident CTAs.
template <typename T> struct Sweep { static constexpr int NBS = 32, CT = 32; static constexpr bool DB = false; };
template <> struct Sweep<float> { static constexpr int NBS = 64, CT = 32; static constexpr bool DB = true; };
template <> struct Sweep<zf> { static constexpr int NBS = 64, CT = 32; static constexpr bool DB = true; };

constexpr long long SWEEP_WAIT_LIMIT = 1LL << 24;  // flag polls (with a short sleep) before giving up

// Loads that bypass L1 (another CTA wrote the value; L1 is not coherent).
__device__ __forceinline__ float ldcg_(const float* p) { return __ldcg(p); }
__device__ __forceinline__ double ldcg_(const double* p) { return __ldcg(p); }
__device__ __forceinline__ zf ldcg_(const zf* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return {v.x, v.y};
}
__device__ __forceinline__ zd ldcg_(const zd* p) {
  const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return {v.x, v.y};
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Asynchronous element copies global -> shared (cp.async; 4, 8 or 16 bytes,
// the element's own alignment, so any leading dimension works).  The factor
// is read-only during a sweep, so L1-cached copies are fine for it.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  if constexpr (sizeof(T) == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(src), "n"((int)sizeof(T)) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// sync: [0] claim counter (zeroed before the launch), [1] error word,
// [2 + i * nct + c] the flag of item (i, c) (= epoch once published).
// Per tile update one barrier: the next factor tile is copied asynchronously
// and the next Y block read into registers (each thread acquires the row's
// flag itself) while the current tile is multiplied; two buffers alternate.
// The single-buffer form (the FP64 sweeps): the factor tile is staged by
// plain loads (the backward tile conjugate-transposed) before waiting for
// Y_j, thread 0 waits, and three barriers bracket each tile.  Bound by the
// FP64 pipe, it gains nothing from overlapping the loads and keeps more
// CTAs resident.
template <typename T, int NBS, int CT, bool BACK>
__global__ void __launch_bounds__(256)
trsm_sweep_1buf_kernel(int n, int nsb, int nct, const T* __restrict__ L, long long ldl, const T* __restrict__ Dinv,
                  int dnb, T* B, long long ldb, int m, unsigned* sync, unsigned epoch) {
  constexpr int LDS = NBS + 1;
  constexpr int TM = NBS / 16, TN = CT / 16;
  extern __shared__ unsigned char sm[];
  T* Ls = reinterpret_cast<T*>(sm);  // Ls[kk * LDS + r]
  T* Ys = Ls + NBS * LDS;            // Ys[kk * CT + c]
  __shared__ int item, gave_up;
  const int tid = threadIdx.x;
  const int tr = tid & 15, tc = tid >> 4;
  unsigned* flags = sync + 2;
  const int nitems = nsb * nct;
  for (;;) {
    if (tid == 0) {
      item = (int)atomicAdd(sync, 1u);
      gave_up = 0;
    }
    __syncthreads();
    const int t = item;
    if (t >= nitems) break;
    const int step = t / nct, c = t % nct;
    const int i = BACK ? nsb - 1 - step : step;
    const int ct0 = c * CT, cw = min(CT, m - ct0);
    const int r0 = i * NBS, rb = min(NBS, n - r0);

    T acc[TM][TN];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TN; ++b) {
        const int r = tr + 16 * a, cc = tc + 16 * b;
        acc[a][b] = (r < rb && cc < cw) ? ldcg_(B + (r0 + r) + (long long)(ct0 + cc) * ldb) : zero_<T>();
      }
    for (int s2 = 0; s2 < step; ++s2) {
      const int j = BACK ? nsb - 1 - s2 : s2;
      const int rk0 = j * NBS, kb = min(NBS, n - rk0);
      // the factor tile is final: stage it before waiting for Y_j
      for (int e = tid; e < NBS * NBS; e += 256) {
        const int a = e % NBS, b = e / NBS;
        if (!BACK) {  // L_ij(r = a, kk = b)
          Ls[b * LDS + a] = (a < rb && b < kb) ? L[(r0 + a) + (long long)(rk0 + b) * ldl] : zero_<T>();
        } else {      // (L_ji)^*(r = b, kk = a) = conj(L_ji(a, b))
          Ls[a * LDS + b] = (a < kb && b < rb) ? conj_(L[(rk0 + a) + (long long)(r0 + b) * ldl]) : zero_<T>();
        }
      }
      if (tid == 0 && !gave_up) {
        const unsigned* f = flags + (size_t)j * nct + c;
        long long it = 0;
        while (ld_acquire(f) != epoch) {
          if (++it >= SWEEP_WAIT_LIMIT) {
            gave_up = 1;
            atomicExch(sync + 1, 1u);
            break;
          }
          __nanosleep(32);
        }
      }
      __syncthreads();
      for (int e = tid; e < NBS * CT; e += 256) {
        const int kk = e % NBS, cc = e / NBS;
        Ys[kk * CT + cc] = (kk < kb && cc < cw) ? ldcg_(B + (rk0 + kk) + (long long)(ct0 + cc) * ldb) : zero_<T>();
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < NBS; ++kk) {
        T av[TM], bv[TN];
#pragma unroll
        for (int a = 0; a < TM; ++a) av[a] = -Ls[kk * LDS + tr + 16 * a];
#pragma unroll
        for (int b = 0; b < TN; ++b) bv[b] = Ys[kk * CT + tc + 16 * b];
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
          for (int b = 0; b < TN; ++b) fma_(acc[a][b], av[a], bv[b]);
      }
      __syncthreads();
    }
    // Y_i = Dinv_ii (B_i - sum_j L_ij Y_j)   (backward: the conjugate transpose)
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TN; ++b) Ys[(tr + 16 * a) * CT + tc + 16 * b] = acc[a][b];
    const int fb = r0 / dnb, off = r0 % dnb;
    const T* Di = Dinv + (size_t)fb * dnb * dnb + off + (size_t)off * dnb;
    for (int e = tid; e < NBS * NBS; e += 256) {
      const int a = e % NBS, b = e / NBS;
      const T v = (a < rb && b < rb) ? Di[a + (size_t)b * dnb] : zero_<T>();
      if (!BACK) Ls[b * LDS + a] = v;           // Dinv(r = a, kk = b)
      else Ls[a * LDS + b] = conj_(v);          // Dinv^*(r = b, kk = a)
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TN; ++b) acc[a][b] = zero_<T>();
#pragma unroll 4
    for (int kk = 0; kk < NBS; ++kk) {
      T av[TM], bv[TN];
#pragma unroll
      for (int a = 0; a < TM; ++a) av[a] = Ls[kk * LDS + tr + 16 * a];
#pragma unroll
      for (int b = 0; b < TN; ++b) bv[b] = Ys[kk * CT + tc + 16 * b];
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TN; ++b) fma_(acc[a][b], av[a], bv[b]);
    }
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TN; ++b) {
        const int r = tr + 16 * a, cc = tc + 16 * b;
        if (r < rb && cc < cw) B[(r0 + r) + (long long)(ct0 + cc) * ldb] = acc[a][b];
      }
    __threadfence();
    __syncthreads();
    if (tid == 0) st_release(flags + (size_t)i * nct + c, epoch);
  }
}

template <typename T, int NBS, int CT, bool BACK>
__global__ void __launch_bounds__(256, 2)
trsm_sweep_kernel(int n, int nsb, int nct, const T* __restrict__ L, long long ldl, const T* __restrict__ Dinv,
                  int dnb, const T* __restrict__ Mla, T* B, long long ldb, int m, unsigned* sync, unsigned epoch) {
  constexpr int LDS = NBS + 1;
  constexpr int TM = NBS / 16, TN = CT / 16;
  constexpr int YPT = NBS * CT / 256;  // elements of a Y block per thread
  static_assert(NBS * CT % 256 == 0, "whole Y block per thread");
  extern __shared__ unsigned char sm[];
  // buffer q: factor tile at L0 + q NBS LDS, Y block at Y0 + q NBS CT ([kk * CT + c])
  T* const L0 = reinterpret_cast<T*>(sm);
  T* const Y0 = L0 + 2 * NBS * LDS;
  __shared__ int item;
  const int tid = threadIdx.x, lane = tid & 31;
  const int tr = tid & 15, tc = tid >> 4;
  unsigned* flags = sync + 2;
  const int nitems = nsb * nct;
  bool gave_up = false;
  for (;;) {
    if (tid == 0) item = (int)atomicAdd(sync, 1u);
    __syncthreads();
    const int t = item;
    if (t >= nitems) break;
    const int step = t / nct, c = t % nct;
    const int i = BACK ? nsb - 1 - step : step;
    const int ct0 = c * CT, cw = min(CT, m - ct0);
    const int r0 = i * NBS, rb = min(NBS, n - r0);
    auto jof = [&](int s2) { return BACK ? nsb - 1 - s2 : s2; };
    // the factor tile (i, j) into buffer q, asynchronously and as stored
    // (backward: L_ji(kk, r) at [r * LDS + kk], conjugated when read)
    auto stage_L = [&](int q, int j) {
      const int rk0 = j * NBS, kb = min(NBS, n - rk0);
      T* Ls = L0 + q * NBS * LDS;
      for (int e = tid; e < NBS * NBS; e += 256) {
        if (!BACK) {  // L_ij(r, kk) at [kk * LDS + r]
          const int r = e % NBS, kk = e / NBS;
          if (r < rb && kk < kb) cp_async_elem(Ls + kk * LDS + r, L + (r0 + r) + (long long)(rk0 + kk) * ldl);
          else Ls[kk * LDS + r] = zero_<T>();
        } else {
          const int kk = e % NBS, r = e / NBS;
          if (r < rb && kk < kb) cp_async_elem(Ls + r * LDS + kk, L + (rk0 + kk) + (long long)(r0 + r) * ldl);
          else Ls[r * LDS + kk] = zero_<T>();
        }
      }
      cp_async_commit();
    };
    // Y_j's flag, read by lane 0 of each warp (one poller per warp keeps the
    // polling traffic off the L2 slices that hold the flags) and passed on
    // with a warp barrier, which orders lane 0's acquire before the other
    // lanes' loads: poll once, or wait (bounded) for it
    auto flag_ready = [&](int j) {
      int r = 1;
      if (lane == 0 && !gave_up) r = ld_acquire(flags + (size_t)j * nct + c) == epoch;
      r = __shfl_sync(0xffffffffu, r, 0);
      __syncwarp();
      return r != 0;
    };
    auto wait_flag = [&](int j) {
      int g = gave_up ? 1 : 0;
      if (lane == 0 && !g) {
        long long it = 0;
        while (ld_acquire(flags + (size_t)j * nct + c) != epoch) {
          if (++it >= SWEEP_WAIT_LIMIT) {
            g = 1;
            atomicExch(sync + 1, 1u);
            break;
          }
          __nanosleep(32);
        }
      }
      gave_up = __shfl_sync(0xffffffffu, g, 0) != 0;
      __syncwarp();
    };
    // this thread's elements of Y_j into registers (after its flag was seen)
    T yr[YPT];
    auto load_Y = [&](int j) {
      const int rk0 = j * NBS, kb = min(NBS, n - rk0);
#pragma unroll
      for (int q = 0; q < YPT; ++q) {
        const int e = tid + 256 * q, kk = e % NBS, cc = e / NBS;
        yr[q] = (kk < kb && cc < cw) ? ldcg_(B + (rk0 + kk) + (long long)(ct0 + cc) * ldb) : zero_<T>();
      }
    };
    auto put_Y = [&](int q) {
#pragma unroll
      for (int u = 0; u < YPT; ++u) {
        const int e = tid + 256 * u, kk = e % NBS, cc = e / NBS;
        Y0[q * NBS * CT + kk * CT + cc] = yr[u];
      }
    };

    T acc[TM][TN];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TN; ++b) {
        const int r = tr + 16 * a, cc = tc + 16 * b;
        acc[a][b] = (r < rb && cc < cw) ? ldcg_(B + (r0 + r) + (long long)(ct0 + cc) * ldb) : zero_<T>();
      }
    // with the look-ahead products M_i (Mla), the last tile (the row that
    // finishes just before this one) is left out of the accumulation:
    // Y_i = Dinv_ii (B_i - sum_{j < last} L_ij Y_j) - M_i Y_last, so only one
    // product follows the wait for Y_last
    const bool la = Mla != nullptr && step > 0;
    const int nacc = la ? step - 1 : step;
    if (nacc > 0) {
      stage_L(0, jof(0));
      wait_flag(jof(0));
      load_Y(jof(0));
      put_Y(0);
      cp_async_wait_all();
      __syncthreads();
      for (int s2 = 0; s2 < nacc; ++s2) {
        const int q = s2 & 1;
        const bool more = s2 + 1 < nacc;
        // the next tile's factor part is always prefetched; its Y part only
        // when already published (else read after this tile's product, so
        // that a row still in flight does not hold up the product)
        bool early = false;
        if (more) {
          stage_L(q ^ 1, jof(s2 + 1));
          early = flag_ready(jof(s2 + 1));
          if (early) load_Y(jof(s2 + 1));
        }
        const T* Ls = L0 + q * NBS * LDS;
        const T* Ys = Y0 + q * NBS * CT;
#pragma unroll 4
        for (int kk = 0; kk < NBS; ++kk) {
          T av[TM], bv[TN];
#pragma unroll
          for (int a = 0; a < TM; ++a)
            av[a] = BACK ? -conj_(Ls[(tr + 16 * a) * LDS + kk]) : -Ls[kk * LDS + tr + 16 * a];
#pragma unroll
          for (int b = 0; b < TN; ++b) bv[b] = Ys[kk * CT + tc + 16 * b];
#pragma unroll
          for (int a = 0; a < TM; ++a)
#pragma unroll
            for (int b = 0; b < TN; ++b) fma_(acc[a][b], av[a], bv[b]);
        }
        if (more) {
          if (!early) {
            wait_flag(jof(s2 + 1));
            load_Y(jof(s2 + 1));
          }
          put_Y(q ^ 1);
        }
        cp_async_wait_all();
        __syncthreads();
      }
    }
    if (la) {  // M_i into buffer 1 while the diagonal product runs
      const T* Mi = Mla + (size_t)i * NBS * NBS;
      T* Lm = L0 + NBS * LDS;
      for (int e = tid; e < NBS * NBS; e += 256) {
        const int r = e % NBS, kk = e / NBS;
        cp_async_elem(Lm + kk * LDS + r, Mi + e);
      }
      cp_async_commit();
    }
    // Y_i = Dinv_ii (B_i - sum_j L_ij Y_j)   (backward: the conjugate transpose)
    T* Ls = L0;
    T* Ys = Y0;
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TN; ++b) Ys[(tr + 16 * a) * CT + tc + 16 * b] = acc[a][b];
    const int fb = r0 / dnb, off = r0 % dnb;
    const T* Di = Dinv + (size_t)fb * dnb * dnb + off + (size_t)off * dnb;
    for (int e = tid; e < NBS * NBS; e += 256) {
      const int a = e % NBS, b = e / NBS;
      const T v = (a < rb && b < rb) ? Di[a + (size_t)b * dnb] : zero_<T>();
      if (!BACK) Ls[b * LDS + a] = v;           // Dinv(r = a, kk = b)
      else Ls[a * LDS + b] = conj_(v);          // Dinv^*(r = b, kk = a)
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TN; ++b) acc[a][b] = zero_<T>();
#pragma unroll 4
    for (int kk = 0; kk < NBS; ++kk) {
      T av[TM], bv[TN];
#pragma unroll
      for (int a = 0; a < TM; ++a) av[a] = Ls[kk * LDS + tr + 16 * a];
#pragma unroll
      for (int b = 0; b < TN; ++b) bv[b] = Ys[kk * CT + tc + 16 * b];
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TN; ++b) fma_(acc[a][b], av[a], bv[b]);
    }
    if (la) {  // - M_i Y_last, after Y_last is published
      const int jl = jof(step - 1);
      wait_flag(jl);
      load_Y(jl);
      put_Y(1);
      cp_async_wait_all();
      __syncthreads();
      const T* Lm = L0 + NBS * LDS;
      const T* Ym = Y0 + NBS * CT;
#pragma unroll 4
      for (int kk = 0; kk < NBS; ++kk) {
        T av[TM], bv[TN];
#pragma unroll
        for (int a = 0; a < TM; ++a) av[a] = Lm[kk * LDS + tr + 16 * a];
#pragma unroll
        for (int b = 0; b < TN; ++b) bv[b] = Ym[kk * CT + tc + 16 * b];
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
          for (int b = 0; b < TN; ++b) fms_(acc[a][b], av[a], bv[b]);
      }
    }
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TN; ++b) {
        const int r = tr + 16 * a, cc = tc + 16 * b;
        if (r < rb && cc < cw) B[(r0 + r) + (long long)(ct0 + cc) * ldb] = acc[a][b];
      }
    __threadfence();
    __syncthreads();
    if (tid == 0) st_release(flags + (size_t)i * nct + c, epoch);
  }
}

template <typename T>
static size_t sweep_smem() {
  constexpr int NBS = Sweep<T>::NBS, CT = Sweep<T>::CT;
  return (Sweep<T>::DB ? 2 : 1) * ((size_t)NBS * (NBS + 1) + (size_t)NBS * CT) * sizeof(T);
}

// Per-stream synchronisation words of the persistent sweeps (claim counter,
// error word, item flags) and the epoch that marks a flag as published in
// the current launch; sweeps on one stream run in order, so one area per
// stream suffices.
namespace {
struct SweepSync {
  unsigned* d = nullptr;
  size_t words = 0;
  unsigned epoch = 0;
};
std::mutex& sweep_mutex() {
  static std::mutex mtx;
  return mtx;
}
std::map<cudaStream_t, SweepSync>& sweep_syncs() {
  static std::map<cudaStream_t, SweepSync> m;
  return m;
}
}  // namespace

// Look-ahead products of the double-buffered sweeps: for block row i,
// forward M_i = Dinv_ii L_{i,i-1}, backward M_i = Dinv_ii^* L_{i+1,i}^*
// (NBS x NBS, column-major at M + i NBS^2; zero where the neighbour does not
// exist).  Computed once per factorisation, in the factor's precision.
template <typename T, int NBS, bool BACK>
__global__ void __launch_bounds__(256) sweep_lookahead_kernel(int n, int nsb, const T* __restrict__ L, long long ldl,
                                                              const T* __restrict__ Dinv, int dnb, T* M) {
  constexpr int LDS = NBS + 1;
  extern __shared__ unsigned char sm[];
  T* Ds = reinterpret_cast<T*>(sm);  // Ds[t * LDS + r] = (Dinv or Dinv^*)(r, t)
  T* Ls = Ds + NBS * LDS;            // Ls[kk * LDS + t] = (L_{i,i-1} or L_{i+1,i}^*)(t, kk)
  const int i = blockIdx.x, tid = threadIdx.x;
  const int jl = BACK ? i + 1 : i - 1;
  T* Mi = M + (size_t)i * NBS * NBS;
  if (jl < 0 || jl >= nsb) {
    for (int e = tid; e < NBS * NBS; e += 256) Mi[e] = zero_<T>();
    return;
  }
  const int r0 = i * NBS, rb = min(NBS, n - r0);
  const int rk0 = jl * NBS, kb = min(NBS, n - rk0);
  const int fb = r0 / dnb, off = r0 % dnb;
  const T* Di = Dinv + (size_t)fb * dnb * dnb + off + (size_t)off * dnb;
  for (int e = tid; e < NBS * NBS; e += 256) {
    const int a = e % NBS, b = e / NBS;
    if (!BACK) {
      Ds[b * LDS + a] = (a < rb && b < rb) ? Di[a + (size_t)b * dnb] : zero_<T>();                  // Dinv(a, b)
      Ls[b * LDS + a] = (a < rb && b < kb) ? L[(r0 + a) + (long long)(rk0 + b) * ldl] : zero_<T>();  // L(r0+a, rk0+b)
    } else {
      Ds[a * LDS + b] = (a < rb && b < rb) ? conj_(Di[a + (size_t)b * dnb]) : zero_<T>();           // Dinv^*(b, a)
      Ls[a * LDS + b] = (a < kb && b < rb) ? conj_(L[(rk0 + a) + (long long)(r0 + b) * ldl]) : zero_<T>();  // L^*(b, a)
    }
  }
  __syncthreads();
  for (int e = tid; e < NBS * NBS; e += 256) {
    const int r = e % NBS, kk = e / NBS;
    T acc = zero_<T>();
    for (int t = 0; t < NBS; ++t) fma_(acc, Ds[t * LDS + r], Ls[kk * LDS + t]);
    Mi[e] = acc;
  }
}

template <typename T>
size_t dense_lookahead_elems(int n) {
  constexpr int NBS = Sweep<T>::NBS;
  return Sweep<T>::DB ? 2 * (size_t)ceil_div(n, NBS) * NBS * NBS : 0;
}

template <typename T>
void dense_sweep_lookahead(cudaStream_t st, DenseFactor<T>& F, T* ws) {
  F.Mf = F.Mb = nullptr;
  if constexpr (Sweep<T>::DB) {
    constexpr int NBS = Sweep<T>::NBS, NB = CholBlock<T>::NB;
    const int nsb = ceil_div(F.n, NBS);
    if (!ws || nsb < 2) return;
    const size_t sm = 2 * (size_t)NBS * (NBS + 1) * sizeof(T);
    static const bool opened = [&] {
      cudaFuncSetAttribute(sweep_lookahead_kernel<T, NBS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      cudaFuncSetAttribute(sweep_lookahead_kernel<T, NBS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      return true;
    }();
    (void)opened;
    count_launch(2);
    sweep_lookahead_kernel<T, NBS, false><<<nsb, 256, sm, st>>>(F.n, nsb, F.L, F.ldl, F.Dinv, NB, ws);
    sweep_lookahead_kernel<T, NBS, true><<<nsb, 256, sm, st>>>(F.n, nsb, F.L, F.ldl, F.Dinv, NB, ws + (size_t)nsb * NBS * NBS);
    F.Mf = ws;
    F.Mb = ws + (size_t)nsb * NBS * NBS;
  }
}

template <typename T, bool BACK>
static void dense_sweep(cudaStream_t st, const DenseFactor<T>& F, T* B, long long ldb, int m) {
  constexpr int NB = CholBlock<T>::NB, NBS = Sweep<T>::NBS, CT = Sweep<T>::CT;
  static_assert(NB % NBS == 0, "sweep block must divide the factor block");
  const int n = F.n, nsb = ceil_div(n, NBS), nct = ceil_div(m, CT);
  if (n <= 0 || m <= 0) return;
  const size_t sm = sweep_smem<T>();
  auto kern = [] {
    if constexpr (Sweep<T>::DB) return trsm_sweep_kernel<T, NBS, CT, BACK>;
    else return trsm_sweep_1buf_kernel<T, NBS, CT, BACK>;
  }();
  const T* Mla = BACK ? F.Mb : F.Mf;
  // as many CTAs as fit at once (measured: faster than one per SM -- the
  // off-chain updates need the throughput more than the chain needs an SM
  // of its own)
  static const int resident = [&] {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, sm) != cudaSuccess || per_sm < 1) {
      cudaGetLastError();
      per_sm = 1;
    }
    return per_sm * NUM_SMS;
  }();
  unsigned* sync;
  unsigned epoch;
  {
    std::lock_guard<std::mutex> lock(sweep_mutex());
    SweepSync& S = sweep_syncs()[st];
    const size_t need = 2 + (size_t)nsb * nct;
    if (need > S.words) {
      if (S.d) {
        cudaStreamSynchronize(st);
        cudaFree(S.d);
      }
      S.d = nullptr;
      S.words = 0;
      if (cudaMalloc(&S.d, sizeof(unsigned) * need) != cudaSuccess) {
        cudaGetLastError();
        S.d = nullptr;
        throw std::bad_alloc();
      }
      cudaMemsetAsync(S.d, 0, sizeof(unsigned) * need, st);
      S.words = need;
      S.epoch = 0;
    }
    if (++S.epoch == 0) {  // wrapped: clear the flags once
      cudaMemsetAsync(S.d + 2, 0, sizeof(unsigned) * (S.words - 2), st);
      S.epoch = 1;
    }
    sync = S.d;
    epoch = S.epoch;
  }
  cudaMemsetAsync(sync, 0, sizeof(unsigned), st);  // claim counter (launch errors surface at the caller's check)
  const int grid = std::max(1, std::min(nsb * nct, resident));
  count_launch();
  if constexpr (Sweep<T>::DB) kern<<<grid, 256, sm, st>>>(n, nsb, nct, F.L, F.ldl, F.Dinv, NB, Mla, B, ldb, m, sync, epoch);
  else kern<<<grid, 256, sm, st>>>(n, nsb, nct, F.L, F.ldl, F.Dinv, NB, B, ldb, m, sync, epoch);
}

int sweep_take_error(cudaStream_t st) {
  std::lock_guard<std::mutex> lock(sweep_mutex());
  cudaStreamSynchronize(st);
  int any = 0;
  for (auto& kv : sweep_syncs()) {
    if (!kv.second.d) continue;
    unsigned h = 0;
    cudaMemcpy(&h, kv.second.d + 1, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (h) {
      cudaMemset(kv.second.d + 1, 0, sizeof(unsigned));
      any = 1;
    }
  }
  return any;
}

template <typename T>
void dense_trsm_fwd(cudaStream_t st, const DenseFactor<T>& F, T* B, long long ldb, int m) {
  dense_sweep<T, false>(st, F, B, ldb, m);
}

template <typename T>
void dense_trsm_bwd(cudaStream_t st, const DenseFactor<T>& F, T* B, long long ldb, int m) {
  dense_sweep<T, true>(st, F, B, ldb, m);
}

template <typename T>
void dense_precond(cudaStream_t st, const DenseFactor<T>& F, T* B, long long ldb, int m) {
  dense_trsm_fwd<T>(st, F, B, ldb, m);   // L Y = B
  dense_trsm_bwd<T>(st, F, B, ldb, m);   // L^* Z = Y
}

#define MPL_INST_CHOL(T)                                                                      \
  template void dense_cholesky<T>(cudaStream_t, DenseFactor<T>&, T*, int*, Scratch, int,     \
                                  long long, bool, int, int*);                               \
  template void scale_rows<T>(cudaStream_t, int, int, T*, long long, const float*);         \
  template void round_block<T>(cudaStream_t, int, int, T*, long long, int, bool);           \
  template void dense_precond<T>(cudaStream_t, const DenseFactor<T>&, T*, long long, int);   \
  template void dense_trsm_fwd<T>(cudaStream_t, const DenseFactor<T>&, T*, long long, int);  \
  template void dense_trsm_bwd<T>(cudaStream_t, const DenseFactor<T>&, T*, long long, int);  \
  template size_t dense_lookahead_elems<T>(int);                                             \
  template void dense_sweep_lookahead<T>(cudaStream_t, DenseFactor<T>&, T*);
MPL_INST_CHOL(float)
MPL_INST_CHOL(double)
MPL_INST_CHOL(zf)
MPL_INST_CHOL(zd)
#undef MPL_INST_CHOL
template void scaled_lower_copy<float, double>(cudaStream_t, int, const double*, long long, float*, float*, long long);
template void scaled_lower_copy<zf, zd>(cudaStream_t, int, const zd*, long long, float*, zf*, long long);

}  // namespace mpl
