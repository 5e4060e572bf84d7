// Sparse lower-precision Cholesky on the GPU (Section 5.1: Pi^* A Pi = L L^*,
// "computed in single precision"; the paper used a single-precision CHOLMOD).
//
// Multifrontal over the blocks of the symbolic analysis (nested-dissection
// leaf boxes and separator planes).  Each block b owns a dense front F_b of
// nrows_b x nrows_b (column-major); its first ncols_b columns become the
// columns of L, the trailing part is the update matrix U_b passed to the
// parent.  Schedule, level by level from the leaves (level = height in the
// block tree):
//   1. extend-add: U_c of every child c is added into its parent's front at
//      the parent-relative row positions (children in fixed order: one launch
//      per child rank, so no two writers ever meet -- deterministic);
//   2. partial factorisation of every front at the level: one CTA per small
//      front, the blocked dense Cholesky (GEMM trailing updates) for large
//      fronts.
// Solves (all m right-hand sides at once) follow the same tree: forward from
// the leaves, each block gathering its children's contribution blocks, solving
// with its diagonal block and producing its own contribution; backward from
// the root, each block reading the already solved rows of its ancestors.
#include <algorithm>

#include "sparse.cuh"

namespace mpl {

constexpr int BIG_NCOLS = 256;
constexpr int BIG_NROWS = 1536;
constexpr int EA_COLS = 32;  // child columns per extend-add CTA

template <typename T>
struct SparseFactorSolve<T>::Impl {
  long long n = 0, nb = 0, nnzl = 0, ftotal = 0;
  int maxlevel = 0;
  std::vector<long long> start, rowptr, fptr, cptr;
  std::vector<int> ncols, nrows;
  std::vector<std::vector<int>> small_lv, big_lv;
  int ncmax_small = 1;  // largest ncols among the small fronts
  std::vector<int> small_nrmax;  // largest nrows among a level's small fronts
  std::vector<long long> small_off;  // offsets into d_small per level
  struct Round { long long off; int cnt; int maxchunks; };
  std::vector<std::vector<Round>> rounds;
  std::vector<long long> big_dinv;   // Dinv offset per block (-1 if small)
  std::vector<std::vector<int>> children;

  DevMem F, d_rows, d_rowptr, d_relpos, d_fptr, d_amap, d_avals, d_dmap, d_start, d_ncols, d_nrows,
      d_chptr, d_chlist, d_small, d_pairs, d_cptr, dinv, tmp, info, contrib, gbuf, scr_mem;
  Scratch scr;
  int mcap = 0;
  int maxnbl = 1;
  // The dense (big) fronts of one level are independent in both sweeps: they
  // run concurrently on these streams, forked from and joined back into the
  // caller's stream with events; each stream has its own split-K scratch
  // and gather buffer.
  static constexpr int NAUX = 8;
  static constexpr size_t AUX_SCR = (size_t)16 << 20;
  cudaStream_t aux[NAUX] = {};
  cudaEvent_t fork = nullptr, join[NAUX] = {};
  DevMem aux_scr, aux_gbuf, aux_tmp;
  bool aux_ready = false;
  size_t tmp_elems = 0;  // per-stream factor panel buffer (elements)
  void ensure_aux() {
    if (aux_ready) return;
    for (int i = 0; i < NAUX; ++i) {
      MPL_CUDA(cudaStreamCreateWithFlags(&aux[i], cudaStreamNonBlocking));
      MPL_CUDA(cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming));
    }
    MPL_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    aux_scr.alloc(AUX_SCR * NAUX);
    aux_ready = true;
  }
  void fork_aux(cudaStream_t main) {
    MPL_CUDA(cudaEventRecord(fork, main));
    for (int i = 0; i < NAUX; ++i) MPL_CUDA(cudaStreamWaitEvent(aux[i], fork, 0));
  }
  void join_aux(cudaStream_t main, int used) {
    for (int i = 0; i < NAUX && i < used; ++i) {
      MPL_CUDA(cudaEventRecord(join[i], aux[i]));
      MPL_CUDA(cudaStreamWaitEvent(main, join[i], 0));
    }
  }
  Scratch aux_scratch(int i) {
    Scratch sc;
    sc.ptr = static_cast<unsigned char*>(aux_scr.ptr()) + (size_t)i * AUX_SCR;
    sc.bytes = AUX_SCR;
    return sc;
  }
  ~Impl() {
    for (int i = 0; i < NAUX; ++i) {
      if (aux[i]) cudaStreamDestroy(aux[i]);
      if (join[i]) cudaEventDestroy(join[i]);
    }
    if (fork) cudaEventDestroy(fork);
  }
};

// ---- kernels -------------------------------------------------------------
template <typename T>
__global__ void assemble_kernel(long long nnz, const long long* __restrict__ amap,
                                const double* __restrict__ vals, T* __restrict__ F) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nnz;
       q += (long long)gridDim.x * blockDim.x)
    F[amap[q]] = (T)vals[q];
}

template <typename T>
__global__ void add_sigma_kernel(long long n, const long long* __restrict__ dmap, T* F, double sigma) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x)
    F[dmap[j]] += (T)sigma;
}

// U_c (lower part) of the child into the parent's front.
template <typename T>
__global__ void __launch_bounds__(256)
extend_add_kernel(const int2* __restrict__ pairs, T* F, const long long* __restrict__ fptr,
                  const long long* __restrict__ rowptr, const int* __restrict__ relpos,
                  const int* __restrict__ ncols, const int* __restrict__ nrows) {
  const int2 pr = pairs[blockIdx.x];
  const int c = pr.x, s = pr.y;
  const int ncc = ncols[c], nrc = nrows[c], nbc = nrc - ncc;
  const int nrs = nrows[s];
  const int j0 = blockIdx.y * EA_COLS;
  if (j0 >= nbc) return;
  const int j1 = min(nbc, j0 + EA_COLS);
  const T* Fc = F + fptr[c];
  T* Fs = F + fptr[s];
  const int* rp = relpos + rowptr[c] + ncc;
  for (int jc = j0; jc < j1; ++jc) {
    const int tc = rp[jc];
    const T* col = Fc + (long long)(ncc + jc) * nrc + ncc;
    T* tcol = Fs + (long long)tc * nrs;
    for (int ic = jc + threadIdx.x; ic < nbc; ic += blockDim.x) tcol[rp[ic]] += col[ic];
  }
}

// Partial Cholesky of a small front: the first nc columns, Schur update of
// the rest (one CTA per front).
// Small-front factorisation by column panels of PW held in shared memory:
// the panel (rows j0.., PW columns) is factored there column by column, then
// written back, and the trailing lower triangle receives one rank-PW update
// per panel (a warp per column, lanes down the rows) -- one global
// read-modify-write per element and panel instead of per column.
template <typename T, int PW>
__global__ void __launch_bounds__(256)
factor_front_kernel(const int* __restrict__ list, T* F, const long long* __restrict__ fptr,
                    const int* __restrict__ ncols, const int* __restrict__ nrows,
                    const long long* __restrict__ start, int* info, int nrmax) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* P = reinterpret_cast<T*>(smraw);  // P[r + jj * LDP], r relative to j0
  const int LDP = nrmax + 1;
  const int b = list[blockIdx.x];
  const int nc = ncols[b], nr = nrows[b];
  T* A = F + fptr[b];
  __shared__ T piv;
  __shared__ int bad;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  if (tid == 0) bad = 0;
  for (int j0 = 0; j0 < nc; j0 += PW) {
    const int pw = min(PW, nc - j0), rws = nr - j0;
    for (int e = tid; e < rws * pw; e += nt) {
      const int r = e % rws, jj = e / rws;
      P[r + jj * LDP] = A[(j0 + r) + (long long)(j0 + jj) * nr];
    }
    __syncthreads();
    for (int jj = 0; jj < pw; ++jj) {
      if (tid == 0) {
        T d = P[jj + jj * LDP];
        if (!(d > T(0)) || !isfinite((double)d)) {
          if (bad == 0) bad = j0 + jj + 1;
          d = T(1);
        }
        d = (sizeof(T) == 8) ? (T)sqrt((double)d) : (T)sqrtf((float)d);
        P[jj + jj * LDP] = d;
        piv = T(1) / d;
      }
      __syncthreads();
      const T rs = piv;
      for (int r = jj + 1 + tid; r < rws; r += nt) P[r + jj * LDP] *= rs;
      __syncthreads();
      const int h = rws - jj - 1, w = pw - jj - 1;
      for (int e = tid; e < h * w; e += nt) {
        const int r = jj + 1 + e % h, c = jj + 1 + e / h;
        if (r >= c) P[r + c * LDP] -= P[r + jj * LDP] * P[c + jj * LDP];
      }
      __syncthreads();
    }
    for (int e = tid; e < rws * pw; e += nt) {
      const int r = e % rws, jj = e / rws;
      if (r >= jj) A[(j0 + r) + (long long)(j0 + jj) * nr] = P[r + jj * LDP];
    }
    for (int col = j0 + pw + wid; col < nr; col += nw) {
      T fj[PW];
#pragma unroll
      for (int jj = 0; jj < PW; ++jj) fj[jj] = jj < pw ? P[(col - j0) + jj * LDP] : T(0);
      T* ac = A + (long long)col * nr;
      for (int row = col + lane; row < nr; row += 32) {
        T acc = ac[row];
        const T* pr = P + (row - j0);
#pragma unroll
        for (int jj = 0; jj < PW; ++jj)
          if (jj < pw) acc -= pr[jj * LDP] * fj[jj];  // columns past pw are not loaded
        ac[row] = acc;
      }
    }
    __syncthreads();
  }
  if (tid == 0 && bad != 0) atomicCAS(info, 0, (int)(start[b] + bad));
}

template <typename T> struct FrontPanel { static constexpr int PW = 32; };
template <> struct FrontPanel<double> { static constexpr int PW = 16; };

template <typename T>
__global__ void __launch_bounds__(256)
factor_small_kernel(const int* __restrict__ list, T* F, const long long* __restrict__ fptr,
                    const int* __restrict__ ncols, const int* __restrict__ nrows,
                    const long long* __restrict__ start, int* info) {
  const int b = list[blockIdx.x];
  const int nc = ncols[b], nr = nrows[b];
  T* A = F + fptr[b];
  __shared__ T piv;
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  for (int j = 0; j < nc; ++j) {
    if (threadIdx.x == 0) {
      T d = A[j + (long long)j * nr];
      if (!(d > T(0)) || !isfinite((double)d)) {
        if (bad == 0) bad = j + 1;
        d = T(1);
      }
      d = (sizeof(T) == 8) ? (T)sqrt((double)d) : (T)sqrtf((float)d);
      A[j + (long long)j * nr] = d;
      piv = T(1) / d;
    }
    __syncthreads();
    const T rs = piv;
    T* cj = A + (long long)j * nr;
    for (int i = j + 1 + threadIdx.x; i < nr; i += blockDim.x) cj[i] *= rs;
    __syncthreads();
    // lower-triangular trailing update: one warp per column, lanes down the rows
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int col = j + 1 + wid; col < nr; col += nw) {
      const T f = cj[col];
      T* ac = A + (long long)col * nr;
      for (int row = col + lane; row < nr; row += 32) ac[row] -= cj[row] * f;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && bad != 0) atomicCAS(info, 0, (int)(start[b] + bad));
}

// Forward solve of the small blocks of one level: gather the children's
// contributions, y = L11^-1 t, contribution = t_below - L21 y.
template <typename T>
__global__ void __launch_bounds__(256)
fwd_small_kernel(const int* __restrict__ list, int single, const T* __restrict__ F,
                 const long long* __restrict__ fptr,
                 const int* __restrict__ ncols, const int* __restrict__ nrows,
                 const long long* __restrict__ start, const long long* __restrict__ rowptr,
                 const int* __restrict__ relpos, const int* __restrict__ chptr,
                 const int* __restrict__ chlist, const long long* __restrict__ cptr, T* contrib,
                 T* B, long long ldb, int m, int gather_only) {
  const int b = single >= 0 ? single : list[blockIdx.x];
  const int nc = ncols[b], nr = nrows[b], nbl = nr - nc;
  const long long f = start[b];
  const T* A = F + fptr[b];
  T* Cb = contrib + cptr[b] * m;
  for (long long e = threadIdx.x; e < (long long)nbl * m; e += blockDim.x) Cb[e] = T(0);
  __syncthreads();
  for (int q = chptr[b]; q < chptr[b + 1]; ++q) {
    const int ch = chlist[q];
    const int ncc = ncols[ch], nbc = nrows[ch] - ncc;
    const T* Cc = contrib + cptr[ch] * m;
    const int* rp = relpos + rowptr[ch] + ncc;
    for (long long e = threadIdx.x; e < (long long)nbc * m; e += blockDim.x) {
      const int i = (int)(e % nbc), c = (int)(e / nbc);
      const int pos = rp[i];
      const T v = Cc[i + (long long)c * nbc];
      if (pos < nc) B[(f + pos) + (long long)c * ldb] += v;
      else Cb[(pos - nc) + (long long)c * nbl] += v;
    }
    __syncthreads();
  }
  if (gather_only) return;
  for (int j = 0; j < nc; ++j) {
    const T ljj = A[j + (long long)j * nr];
    for (int c = threadIdx.x; c < m; c += blockDim.x) B[(f + j) + (long long)c * ldb] /= ljj;
    __syncthreads();
    const int w = nr - j - 1;
    for (long long e = threadIdx.x; e < (long long)w * m; e += blockDim.x) {
      const int i = j + 1 + (int)(e % w), c = (int)(e / w);
      const T v = A[i + (long long)j * nr] * B[(f + j) + (long long)c * ldb];
      if (i < nc) B[(f + i) + (long long)c * ldb] -= v;
      else Cb[(i - nc) + (long long)c * nbl] -= v;
    }
    __syncthreads();
  }
}

// Backward solve of the small blocks of one level: t = y - L21^T x_below,
// x = L11^-T t.
template <typename T>
__global__ void __launch_bounds__(256)
bwd_small_kernel(const int* __restrict__ list, const T* __restrict__ F, const long long* __restrict__ fptr,
                 const int* __restrict__ ncols, const int* __restrict__ nrows,
                 const long long* __restrict__ start, const long long* __restrict__ rowptr,
                 const int* __restrict__ rows, T* B, long long ldb, int m) {
  const int b = list[blockIdx.x];
  const int nc = ncols[b], nr = nrows[b];
  const long long f = start[b];
  const T* A = F + fptr[b];
  const int* rw = rows + rowptr[b];
  for (long long e = threadIdx.x; e < (long long)nc * m; e += blockDim.x) {
    const int i = (int)(e % nc), c = (int)(e / nc);
    T acc = B[(f + i) + (long long)c * ldb];
    const T* li = A + (long long)i * nr;
    for (int q = nc; q < nr; ++q) acc -= li[q] * B[rw[q] + (long long)c * ldb];
    B[(f + i) + (long long)c * ldb] = acc;
  }
  __syncthreads();
  for (int j = nc - 1; j >= 0; --j) {
    const T ljj = A[j + (long long)j * nr];
    for (int c = threadIdx.x; c < m; c += blockDim.x) B[(f + j) + (long long)c * ldb] /= ljj;
    __syncthreads();
    for (long long e = threadIdx.x; e < (long long)j * m; e += blockDim.x) {
      const int i = (int)(e % j), c = (int)(e / j);
      B[(f + i) + (long long)c * ldb] -= A[j + (long long)i * nr] * B[(f + j) + (long long)c * ldb];
    }
    __syncthreads();
  }
}

// gather G(q, c) = B(rows[q], c) for the below-rows of a (large) block
// Front solves with the front's top nc x m block held in shared memory
// (small fronts: nc < 256).  Forward: extend-add of the children, then
// L11 y = b by 32-column panels -- the diagonal block by one warp per
// right-hand side (lanes = rows, registers and shuffles), the rows below it
// in one parallel pass -- and finally C_b -= L21 y with one thread per row
// and 16 right-hand sides per pass (each L21 element loaded once per pass).
constexpr int FPW = 32;
constexpr int BW_ACC = 48;  // outputs per thread of the backward L21^T pass

template <typename T>
__global__ void __launch_bounds__(256)
fwd_front_kernel(const int* __restrict__ list, const T* __restrict__ F, const long long* __restrict__ fptr,
                 const int* __restrict__ ncols, const int* __restrict__ nrows, const long long* __restrict__ start,
                 const long long* __restrict__ rowptr, const int* __restrict__ relpos, const int* __restrict__ chptr,
                 const int* __restrict__ chlist, const long long* __restrict__ cptr, T* contrib, T* B, long long ldb,
                 int m, int ncmax) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* Y = reinterpret_cast<T*>(smraw);  // nc x m, ld nc
  T* Lp = Y + (size_t)ncmax * m;       // panel rows j0.., ld LDP
  const int LDP = ncmax + 1;
  const int b = list[blockIdx.x];
  const int nc = ncols[b], nr = nrows[b], nbl = nr - nc;
  const long long f = start[b];
  const T* A = F + fptr[b];
  T* Cb = contrib + cptr[b] * m;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  for (long long e = tid; e < (long long)nbl * m; e += nt) Cb[e] = T(0);
  __syncthreads();
  for (int q = chptr[b]; q < chptr[b + 1]; ++q) {
    const int ch = chlist[q];
    const int ncc = ncols[ch], nbc = nrows[ch] - ncc;
    const T* Cc = contrib + cptr[ch] * m;
    const int* rp = relpos + rowptr[ch] + ncc;
    for (long long e = tid; e < (long long)nbc * m; e += nt) {
      const int i = (int)(e % nbc), c = (int)(e / nbc);
      const int pos = rp[i];
      const T v = Cc[i + (long long)c * nbc];
      if (pos < nc) B[(f + pos) + (long long)c * ldb] += v;
      else Cb[(pos - nc) + (long long)c * nbl] += v;
    }
    __syncthreads();
  }
  for (int e = tid; e < nc * m; e += nt) Y[e] = B[(f + e % nc) + (long long)(e / nc) * ldb];
  __syncthreads();
  for (int j0 = 0; j0 < nc; j0 += FPW) {
    const int pw = min(FPW, nc - j0), rws = nc - j0;
    for (int e = tid; e < rws * pw; e += nt) {
      const int r = e % rws, jj = e / rws;
      Lp[r + jj * LDP] = A[(j0 + r) + (long long)(j0 + jj) * nr];
    }
    __syncthreads();
    for (int c = wid; c < m; c += nw) {
      T y = lane < pw ? Y[j0 + lane + c * nc] : T(0);
      for (int jj = 0; jj < pw; ++jj) {
        if (lane == jj) y = y / Lp[jj + jj * LDP];
        const T yj = __shfl_sync(0xffffffffu, y, jj);
        if (lane > jj && lane < pw) y -= Lp[lane + jj * LDP] * yj;
      }
      if (lane < pw) Y[j0 + lane + c * nc] = y;
    }
    __syncthreads();
    const int below = rws - pw;
    for (int e = tid; e < below * m; e += nt) {
      const int r = pw + e % below, c = e / below;
      T acc = Y[j0 + r + c * nc];
#pragma unroll 8
      for (int jj = 0; jj < pw; ++jj) acc -= Lp[r + jj * LDP] * Y[j0 + jj + c * nc];
      Y[j0 + r + c * nc] = acc;
    }
    __syncthreads();
  }
  for (int e = tid; e < nc * m; e += nt) B[(f + e % nc) + (long long)(e / nc) * ldb] = Y[e];
  for (int c0 = 0; c0 < m; c0 += 16) {
    const int qc = min(16, m - c0);
    for (int i = tid; i < nbl; i += nt) {
      T acc[16];
#pragma unroll
      for (int cc = 0; cc < 16; ++cc) acc[cc] = T(0);
      const T* a = A + nc + i;
      for (int j = 0; j < nc; ++j) {
        const T lij = a[(long long)j * nr];
        const T* yj = Y + j + (long long)c0 * nc;
#pragma unroll
        for (int cc = 0; cc < 16; ++cc)
          if (cc < qc) acc[cc] += lij * yj[(long long)cc * nc];
      }
      for (int cc = 0; cc < qc; ++cc) Cb[i + (long long)(c0 + cc) * nbl] -= acc[cc];
    }
  }
}

// Backward: t = y - L21^T x_below into shared memory, then L11^T x = t by
// 32-row panels from the bottom (the panel's rows of L staged in shared
// memory with coalesced row loads), the diagonal block by one warp per
// right-hand side, the rows above the panel in one parallel pass.
template <typename T>
__global__ void __launch_bounds__(256)
bwd_front_kernel(const int* __restrict__ list, const T* __restrict__ F, const long long* __restrict__ fptr,
                 const int* __restrict__ ncols, const int* __restrict__ nrows, const long long* __restrict__ start,
                 const long long* __restrict__ rowptr, const int* __restrict__ rows, T* B, long long ldb, int m,
                 int ncmax) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* Y = reinterpret_cast<T*>(smraw);  // nc x m, ld nc
  T* Lp = Y + (size_t)ncmax * m;       // rows j0..j0+pw of L, Lp[jj + i * (FPW + 1)]
  constexpr int L1 = FPW + 1;
  const int b = list[blockIdx.x];
  const int nc = ncols[b], nr = nrows[b];
  const long long f = start[b];
  const T* A = F + fptr[b];
  const int* rw = rows + rowptr[b];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  // t = y - L21^T x_below, by 32-row chunks of L21 and of the gathered
  // x_below staged in shared memory (each thread owns <= BW_ACC outputs)
  const int tot = nc * m;
  if (tot <= BW_ACC * nt) {
    T* Ls = Lp;                          // 32 rows of L21: Ls[qq + i * L1]
    T* Xs = Lp + (size_t)L1 * ncmax;     // 32 rows of x_below: Xs[qq + c * FPW]
    T acc[BW_ACC];
#pragma unroll
    for (int k = 0; k < BW_ACC; ++k) acc[k] = T(0);
    for (int q0 = nc; q0 < nr; q0 += FPW) {
      const int qw = min(FPW, nr - q0);
      for (int e = tid; e < FPW * m; e += nt) {
        const int qq = e % FPW, c = e / FPW;
        Xs[e] = qq < qw ? B[rw[q0 + qq] + (long long)c * ldb] : T(0);
      }
      for (int e = tid; e < FPW * nc; e += nt) {
        const int qq = e % FPW, i = e / FPW;
        Ls[qq + i * L1] = qq < qw ? A[(q0 + qq) + (long long)i * nr] : T(0);
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < BW_ACC; ++k) {
        const int e = tid + k * nt;
        if (e < tot) {
          const int i = e % nc, c = e / nc;
          const T* li = Ls + i * L1;
          const T* xc = Xs + c * FPW;
          T s = acc[k];
#pragma unroll 8
          for (int qq = 0; qq < FPW; ++qq) s += li[qq] * xc[qq];
          acc[k] = s;
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < BW_ACC; ++k) {
      const int e = tid + k * nt;
      if (e < tot) Y[e] = B[(f + e % nc) + (long long)(e / nc) * ldb] - acc[k];
    }
  } else {
    for (int e = tid; e < tot; e += nt) {
      const int i = e % nc, c = e / nc;
      T a = B[(f + i) + (long long)c * ldb];
      const T* li = A + (long long)i * nr;
      for (int q = nc; q < nr; ++q) a -= li[q] * B[rw[q] + (long long)c * ldb];
      Y[e] = a;
    }
  }
  __syncthreads();
  for (int p = (nc - 1) / FPW; p >= 0; --p) {
    const int j0 = p * FPW, pw = min(FPW, nc - j0), cols = j0 + pw;
    for (int e = tid; e < pw * cols; e += nt) {
      const int jj = e % pw, i = e / pw;
      Lp[jj + i * L1] = A[(j0 + jj) + (long long)i * nr];
    }
    __syncthreads();
    for (int c = wid; c < m; c += nw) {
      T y = lane < pw ? Y[j0 + lane + c * nc] : T(0);
      for (int kk = pw - 1; kk >= 0; --kk) {
        if (lane == kk) y = y / Lp[kk + (j0 + kk) * L1];
        const T xk = __shfl_sync(0xffffffffu, y, kk);
        if (lane < kk) y -= Lp[kk + (j0 + lane) * L1] * xk;  // L^T(lane, kk) = L(kk, lane)
      }
      if (lane < pw) Y[j0 + lane + c * nc] = y;
    }
    __syncthreads();
    for (int e = tid; e < j0 * m; e += nt) {
      const int i = e % j0, c = e / j0;
      T acc = Y[i + c * nc];
#pragma unroll 8
      for (int jj = 0; jj < pw; ++jj) acc -= Lp[jj + i * L1] * Y[j0 + jj + c * nc];
      Y[i + c * nc] = acc;
    }
    __syncthreads();
  }
  for (int e = tid; e < nc * m; e += nt) B[(f + e % nc) + (long long)(e / nc) * ldb] = Y[e];
}

template <typename T>
static size_t front_smem(int ncmax, int m) {
  return ((size_t)ncmax * m + (size_t)(FPW + 1) * (ncmax + 1) + (size_t)FPW * m) * sizeof(T);
}

// Extend-add of one child into its (dense) parent: the child's contribution
// rows go to the parent's own rows of B or to its contribution block.
// Positions within one child are distinct, so a grid over the child's
// entries is race-free; children are added by successive launches.
template <typename T>
__global__ void gather_child_kernel(int nbc, int m, const T* __restrict__ Cc, const int* __restrict__ rp, int nc,
                                    int nbl, long long f, T* B, long long ldb, T* Cb) {
  const long long tot = (long long)nbc * m;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % nbc), c = (int)(e / nbc);
    const int pos = rp[i];
    const T v = Cc[i + (long long)c * nbc];
    if (pos < nc) B[(f + pos) + (long long)c * ldb] += v;
    else Cb[(pos - nc) + (long long)c * nbl] += v;
  }
}

template <typename T>
__global__ void gather_rows_kernel(int nbl, int m, const int* __restrict__ rw, const T* __restrict__ B,
                                   long long ldb, T* G) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)nbl * m;
       e += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(e % nbl), c = (int)(e / nbl);
    G[e] = B[rw[q] + (long long)c * ldb];
  }
}

// Y = L X for checks: column j of L is row (start..) of its block.
template <typename T>
__global__ void apply_L_kernel(int nblk, const T* __restrict__ F, const long long* __restrict__ fptr,
                               const int* __restrict__ ncols, const int* __restrict__ nrows,
                               const long long* __restrict__ start, const long long* __restrict__ rowptr,
                               const int* __restrict__ rows, const T* __restrict__ X, long long ldx,
                               T* Y, long long ldy, int m) {
  // one CTA per block, scatter with atomics is avoided: every output row is
  // reached from several blocks, so Y is accumulated column by column of L
  // in a fixed block order by a single CTA sweep (slow but only for checks)
  if (blockIdx.x != 0) return;
  for (int b = 0; b < nblk; ++b) {
    const int nc = ncols[b], nr = nrows[b];
    const T* A = F + fptr[b];
    const int* rw = rows + rowptr[b];
    for (long long e = threadIdx.x; e < (long long)nr * m; e += blockDim.x) {
      const int i = (int)(e % nr), c = (int)(e / nr);
      T acc = T(0);
      const int jmax = (i < nc) ? i : nc - 1;
      for (int j = 0; j <= jmax; ++j) acc += A[i + (long long)j * nr] * X[(start[b] + j) + (long long)c * ldx];
      Y[rw[i] + (long long)c * ldy] += acc;
    }
    __syncthreads();
  }
}

// ---- host ----------------------------------------------------------------
template <typename T>
SparseFactorSolve<T>::SparseFactorSolve(const SparseSymbolic& S, cudaStream_t st) : p_(new Impl) {
  Impl& I = *p_;
  I.n = S.n;
  I.nb = S.nblock;
  const long long nb = I.nb;
  I.start.assign(S.bk_start.begin(), S.bk_start.end());
  I.rowptr.assign(S.bk_rowptr.begin(), S.bk_rowptr.end());
  I.ncols.resize(nb);
  I.nrows.resize(nb);
  I.fptr.assign(nb + 1, 0);
  I.cptr.assign(nb + 1, 0);
  for (long long b = 0; b < nb; ++b) {
    I.ncols[b] = (int)(I.start[b + 1] - I.start[b]);
    I.nrows[b] = (int)(I.rowptr[b + 1] - I.rowptr[b]);
    I.fptr[b + 1] = I.fptr[b] + (long long)I.nrows[b] * I.nrows[b];
    I.cptr[b + 1] = I.cptr[b] + (I.nrows[b] - I.ncols[b]);
  }
  I.ftotal = I.fptr[nb];
  std::vector<long long> col2b(I.n);
  for (long long b = 0; b < nb; ++b)
    for (long long c = I.start[b]; c < I.start[b + 1]; ++c) col2b[c] = b;
  // relative positions in the parent's row list
  std::vector<int> rows32(S.bk_rows.size()), relpos(S.bk_rows.size(), -1);
  for (size_t q = 0; q < S.bk_rows.size(); ++q) rows32[q] = (int)S.bk_rows[q];
  I.children.assign(nb, {});
  for (long long b = 0; b < nb; ++b) {
    const long long p = S.bk_parent[b];
    if (p < 0) {
      if (I.nrows[b] != I.ncols[b]) throw MplError{MPL_EINVAL, "root block with rows below", b};
      continue;
    }
    I.children[p].push_back((int)b);
    const long long* pr = S.bk_rows.data() + I.rowptr[p];
    const long long plen = I.rowptr[p + 1] - I.rowptr[p];
    for (long long q = I.rowptr[b] + I.ncols[b]; q < I.rowptr[b + 1]; ++q) {
      const long long* it = std::lower_bound(pr, pr + plen, S.bk_rows[q]);
      if (it == pr + plen || *it != S.bk_rows[q])
        throw MplError{MPL_EINVAL, "block structure not contained in its parent", b};
      relpos[q] = (int)(it - pr);
    }
  }
  // assembly map of the lower triangle: entry B(j, i), i <= j -> block of i
  I.nnzl = (long long)S.b_colind.size();
  std::vector<long long> amap(I.nnzl), dmap(I.n);
  for (long long j = 0; j < I.n; ++j) {
    for (long long q = S.b_rowptr[j]; q < S.b_rowptr[j + 1]; ++q) {
      const long long i = S.b_colind[q];
      const long long b = col2b[i];
      const long long* pr = S.bk_rows.data() + I.rowptr[b];
      const long long plen = I.rowptr[b + 1] - I.rowptr[b];
      const long long* it = std::lower_bound(pr, pr + plen, j);
      if (it == pr + plen || *it != j) throw MplError{MPL_EINVAL, "matrix entry outside the symbolic structure", j};
      amap[q] = I.fptr[b] + (it - pr) + (i - I.start[b]) * I.nrows[b];
    }
    const long long b = col2b[j];
    const long long p = j - I.start[b];
    dmap[j] = I.fptr[b] + p + p * I.nrows[b];
  }
  // levels, schedules, extend-add rounds
  I.maxlevel = 0;
  for (long long b = 0; b < nb; ++b) I.maxlevel = std::max(I.maxlevel, (int)S.bk_level[b]);
  const int L = I.maxlevel + 1;
  I.small_lv.assign(L, {});
  I.big_lv.assign(L, {});
  I.small_nrmax.assign(L, 1);
  I.big_dinv.assign(nb, -1);
  long long dinv_total = 0;
  constexpr int NB = CholBlock<T>::NB;
  for (long long b = 0; b < nb; ++b) {
    const bool big = I.ncols[b] >= BIG_NCOLS || I.nrows[b] >= BIG_NROWS;
    if (big) {
      I.big_lv[S.bk_level[b]].push_back((int)b);
      I.big_dinv[b] = dinv_total;
      dinv_total += (long long)ceil_div(I.ncols[b], NB) * NB * NB;
    } else {
      I.small_lv[S.bk_level[b]].push_back((int)b);
      I.ncmax_small = std::max(I.ncmax_small, I.ncols[b]);
      I.small_nrmax[S.bk_level[b]] = std::max(I.small_nrmax[S.bk_level[b]], I.nrows[b]);
    }
  }
  std::vector<int> small_all;
  I.small_off.assign(L + 1, 0);
  for (int l = 0; l < L; ++l) {
    I.small_off[l] = (long long)small_all.size();
    small_all.insert(small_all.end(), I.small_lv[l].begin(), I.small_lv[l].end());
  }
  I.small_off[L] = (long long)small_all.size();
  std::vector<int2> pairs;
  I.rounds.assign(L, {});
  for (int l = 0; l < L; ++l) {
    std::vector<int> parents = I.small_lv[l];
    parents.insert(parents.end(), I.big_lv[l].begin(), I.big_lv[l].end());
    std::sort(parents.begin(), parents.end());
    for (int r = 0;; ++r) {
      typename Impl::Round rd{(long long)pairs.size(), 0, 0};
      for (int p : parents)
        if ((int)I.children[p].size() > r) {
          const int c = I.children[p][r];
          pairs.push_back(make_int2(c, p));
          ++rd.cnt;
          rd.maxchunks = std::max(rd.maxchunks, ceil_div(I.nrows[c] - I.ncols[c], EA_COLS));
        }
      if (rd.cnt == 0) break;
      I.rounds[l].push_back(rd);
    }
  }
  std::vector<int> chptr(nb + 1, 0), chlist;
  for (long long b = 0; b < nb; ++b) {
    chptr[b + 1] = chptr[b] + (int)I.children[b].size();
    chlist.insert(chlist.end(), I.children[b].begin(), I.children[b].end());
  }
  // device copies
  auto up = [&](DevMem& d, const void* h, size_t bytes) {
    d.alloc(bytes);
    if (bytes) MPL_CUDA(cudaMemcpyAsync(d.ptr(), h, bytes, cudaMemcpyHostToDevice, st));
  };
  I.F.alloc(sizeof(T) * (size_t)I.ftotal);
  up(I.d_rows, rows32.data(), sizeof(int) * rows32.size());
  up(I.d_relpos, relpos.data(), sizeof(int) * relpos.size());
  up(I.d_rowptr, I.rowptr.data(), sizeof(long long) * I.rowptr.size());
  up(I.d_fptr, I.fptr.data(), sizeof(long long) * I.fptr.size());
  up(I.d_cptr, I.cptr.data(), sizeof(long long) * I.cptr.size());
  up(I.d_amap, amap.data(), sizeof(long long) * amap.size());
  up(I.d_avals, S.b_vals.data(), sizeof(double) * S.b_vals.size());
  up(I.d_dmap, dmap.data(), sizeof(long long) * dmap.size());
  up(I.d_start, I.start.data(), sizeof(long long) * I.start.size());
  up(I.d_ncols, I.ncols.data(), sizeof(int) * I.ncols.size());
  up(I.d_nrows, I.nrows.data(), sizeof(int) * I.nrows.size());
  up(I.d_chptr, chptr.data(), sizeof(int) * chptr.size());
  up(I.d_chlist, chlist.data(), sizeof(int) * std::max<size_t>(chlist.size(), 1));
  up(I.d_small, small_all.data(), sizeof(int) * std::max<size_t>(small_all.size(), 1));
  up(I.d_pairs, pairs.data(), sizeof(int2) * std::max<size_t>(pairs.size(), 1));
  I.dinv.alloc(sizeof(T) * (size_t)std::max<long long>(dinv_total, 1));
  int maxnr = 1;
  for (long long b = 0; b < nb; ++b) maxnr = std::max(maxnr, I.nrows[b]);
  I.tmp.alloc(sizeof(T) * (size_t)maxnr * NB);
  I.tmp_elems = (size_t)maxnr * NB;
  I.info.alloc(16);
  I.scr_mem.alloc((size_t)32 << 20);
  I.scr.ptr = I.scr_mem.ptr();
  I.scr.bytes = I.scr_mem.bytes();
  MPL_CUDA(cudaStreamSynchronize(st));
}

template <typename T>
SparseFactorSolve<T>::~SparseFactorSolve() { delete p_; }

template <typename T>
int SparseFactorSolve<T>::factorize(cudaStream_t st, double sigma) {
  Impl& I = *p_;
  MPL_CUDA(cudaMemsetAsync(I.F.ptr(), 0, sizeof(T) * (size_t)I.ftotal, st));
  MPL_CUDA(cudaMemsetAsync(I.info.ptr(), 0, sizeof(int), st));
  {
    int blocks = (int)std::min<long long>((I.nnzl + 255) / 256, 16 * NUM_SMS);
    count_launch();
    assemble_kernel<T><<<std::max(blocks, 1), 256, 0, st>>>(I.nnzl, I.d_amap.template as<long long>(),
                                                             I.d_avals.template as<double>(), I.F.template as<T>());
    if (sigma != 0.0) {
      int b2 = (int)std::min<long long>((I.n + 255) / 256, 16 * NUM_SMS);
      count_launch();
      add_sigma_kernel<T><<<b2, 256, 0, st>>>(I.n, I.d_dmap.template as<long long>(), I.F.template as<T>(), sigma);
    }
  }
  for (int l = 0; l <= I.maxlevel; ++l) {
    for (const auto& rd : I.rounds[l]) {
      count_launch();
      extend_add_kernel<T><<<dim3(rd.cnt, std::max(rd.maxchunks, 1)), 256, 0, st>>>(
          I.d_pairs.template as<int2>() + rd.off, I.F.template as<T>(), I.d_fptr.template as<long long>(), I.d_rowptr.template as<long long>(),
          I.d_relpos.template as<int>(), I.d_ncols.template as<int>(), I.d_nrows.template as<int>());
    }
    const long long ns = I.small_off[l + 1] - I.small_off[l];
    constexpr int PW = FrontPanel<T>::PW;
    const size_t psm = (size_t)(I.small_nrmax[l] + 1) * PW * sizeof(T);
    if (ns > 0 && psm <= 200 * 1024) {
      auto kern = factor_front_kernel<T, PW>;
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm);
      count_launch();
      kern<<<(int)ns, 256, psm, st>>>(I.d_small.template as<int>() + I.small_off[l], I.F.template as<T>(),
                                      I.d_fptr.template as<long long>(), I.d_ncols.template as<int>(),
                                      I.d_nrows.template as<int>(), I.d_start.template as<long long>(),
                                      I.info.template as<int>(), I.small_nrmax[l]);
    } else if (ns > 0) {
      count_launch();
      factor_small_kernel<T><<<(int)ns, 256, 0, st>>>(I.d_small.template as<int>() + I.small_off[l], I.F.template as<T>(),
                                                       I.d_fptr.template as<long long>(), I.d_ncols.template as<int>(),
                                                       I.d_nrows.template as<int>(), I.d_start.template as<long long>(),
                                                       I.info.template as<int>());
    }
    // dense fronts of the level: independent, concurrent on the auxiliary
    // streams (own panel buffer and split-K scratch each; the pivot status
    // word is updated with atomics)
    const auto& bl = I.big_lv[l];
    const bool par = bl.size() > 1;
    if (par) {
      I.ensure_aux();
      if (I.aux_tmp.bytes() < sizeof(T) * I.tmp_elems * Impl::NAUX) I.aux_tmp.alloc(sizeof(T) * I.tmp_elems * Impl::NAUX);
      I.fork_aux(st);
    }
    for (size_t idx = 0; idx < bl.size(); ++idx) {
      const int b = bl[idx];
      const int si = (int)(idx % Impl::NAUX);
      cudaStream_t s = par ? I.aux[si] : st;
      DenseFactor<T> D;
      D.L = I.F.template as<T>() + I.fptr[b];
      D.ldl = I.nrows[b];
      D.n = I.nrows[b];
      D.Dinv = I.dinv.template as<T>() + I.big_dinv[b];
      T* tmp = par ? I.aux_tmp.template as<T>() + (size_t)si * I.tmp_elems : I.tmp.template as<T>();
      dense_cholesky<T>(s, D, tmp, I.info.template as<int>(), par ? I.aux_scratch(si) : I.scr, I.ncols[b],
                        I.start[b], false);
    }
    if (par) I.join_aux(st, (int)bl.size());
  }
  check_launch("sparse factorize");
  int info = 0;
  MPL_CUDA(cudaMemcpyAsync(&info, I.info.ptr(), sizeof(int), cudaMemcpyDeviceToHost, st));
  MPL_CUDA(cudaStreamSynchronize(st));
  return info;
}

template <typename T>
void SparseFactorSolve<T>::solve(cudaStream_t st, T* B, long long ldb, int m) {
  Impl& I = *p_;
  if (m > I.mcap) {
    I.contrib.alloc(sizeof(T) * (size_t)std::max<long long>(I.cptr[I.nb], 1) * m);
    int maxnbl = 1;
    for (long long b = 0; b < I.nb; ++b) maxnbl = std::max(maxnbl, I.nrows[b] - I.ncols[b]);
    I.maxnbl = maxnbl;
    I.gbuf.alloc(sizeof(T) * (size_t)maxnbl * m);
    I.aux_gbuf.alloc(sizeof(T) * (size_t)maxnbl * m * Impl::NAUX);
    I.mcap = m;
  }
  I.ensure_aux();
  auto fork_aux = [&](cudaStream_t main) { I.fork_aux(main); };
  auto join_aux = [&](cudaStream_t main, int used) { I.join_aux(main, used); };
  auto aux_scratch = [&](int i) { return I.aux_scratch(i); };
  T* C = I.contrib.template as<T>();
  // the shared-memory front kernels when the largest small front fits
  const size_t fsm = front_smem<T>(I.ncmax_small, m);
  const bool use_front = fsm <= 200 * 1024;
  if (use_front) {
    cudaFuncSetAttribute(fwd_front_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm);
    cudaFuncSetAttribute(bwd_front_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm);
  }
  // forward
  for (int l = 0; l <= I.maxlevel; ++l) {
    const long long ns = I.small_off[l + 1] - I.small_off[l];
    if (ns > 0 && use_front) {
      count_launch();
      fwd_front_kernel<T><<<(int)ns, 256, fsm, st>>>(
          I.d_small.template as<int>() + I.small_off[l], I.F.template as<T>(), I.d_fptr.template as<long long>(),
          I.d_ncols.template as<int>(), I.d_nrows.template as<int>(), I.d_start.template as<long long>(),
          I.d_rowptr.template as<long long>(), I.d_relpos.template as<int>(), I.d_chptr.template as<int>(),
          I.d_chlist.template as<int>(), I.d_cptr.template as<long long>(), C, B, ldb, m, I.ncmax_small);
    } else if (ns > 0) {
      count_launch();
      fwd_small_kernel<T><<<(int)ns, 256, 0, st>>>(
          I.d_small.template as<int>() + I.small_off[l], -1, I.F.template as<T>(), I.d_fptr.template as<long long>(), I.d_ncols.template as<int>(),
          I.d_nrows.template as<int>(), I.d_start.template as<long long>(), I.d_rowptr.template as<long long>(), I.d_relpos.template as<int>(),
          I.d_chptr.template as<int>(), I.d_chlist.template as<int>(), I.d_cptr.template as<long long>(), C, B, ldb, m, 0);
    }
    const auto& bl = I.big_lv[l];
    const bool par = bl.size() > 1;
    if (par) fork_aux(st);
    for (size_t idx = 0; idx < bl.size(); ++idx) {
      const int b = bl[idx];
      cudaStream_t s = par ? I.aux[idx % Impl::NAUX] : st;
      Scratch sc = par ? aux_scratch((int)(idx % Impl::NAUX)) : I.scr;
      // gather children into B / C_b: zero C_b, then one grid-wide launch per child
      {
        const int nblb = I.nrows[b] - I.ncols[b];
        if (nblb > 0) MPL_CUDA(cudaMemsetAsync(C + I.cptr[b] * m, 0, sizeof(T) * (size_t)nblb * m, s));
        for (int ch : I.children[b]) {
          const int ncc = I.ncols[ch], nbc = I.nrows[ch] - ncc;
          if (nbc <= 0) continue;
          const int gb = (int)std::min<long long>(((long long)nbc * m + 255) / 256, 8 * NUM_SMS);
          count_launch();
          gather_child_kernel<T><<<gb, 256, 0, s>>>(nbc, m, C + I.cptr[ch] * m,
                                                    I.d_relpos.template as<int>() + I.rowptr[ch] + ncc, I.ncols[b],
                                                    nblb, I.start[b], B, ldb, C + I.cptr[b] * m);
        }
      }
      DenseFactor<T> D;
      D.L = I.F.template as<T>() + I.fptr[b];
      D.ldl = I.nrows[b];
      D.n = I.ncols[b];
      D.nb = CholBlock<T>::NB;
      D.nblk = ceil_div(I.ncols[b], D.nb);
      D.Dinv = I.dinv.template as<T>() + I.big_dinv[b];
      T* top = B + I.start[b];
      dense_trsm_fwd<T>(s, D, top, ldb, m);
      const int nbl = I.nrows[b] - I.ncols[b];
      if (nbl > 0)
        gemm<T>(s, false, false, nbl, m, I.ncols[b], T(-1), D.L + I.ncols[b], D.ldl, top, ldb, T(1),
                C + I.cptr[b] * m, nbl, false, sc);
    }
    if (par) join_aux(st, (int)bl.size());
  }
  // backward
  for (int l = I.maxlevel; l >= 0; --l) {
    const auto& bl = I.big_lv[l];
    const bool par = bl.size() > 1;
    if (par) fork_aux(st);
    for (size_t idx = 0; idx < bl.size(); ++idx) {
      const int b = bl[idx];
      const int si = (int)(idx % Impl::NAUX);
      cudaStream_t s = par ? I.aux[si] : st;
      Scratch sc = par ? aux_scratch(si) : I.scr;
      T* gb_buf = par ? I.aux_gbuf.template as<T>() + (size_t)si * I.maxnbl * m : I.gbuf.template as<T>();
      DenseFactor<T> D;
      D.L = I.F.template as<T>() + I.fptr[b];
      D.ldl = I.nrows[b];
      D.n = I.ncols[b];
      D.nb = CholBlock<T>::NB;
      D.nblk = ceil_div(I.ncols[b], D.nb);
      D.Dinv = I.dinv.template as<T>() + I.big_dinv[b];
      T* top = B + I.start[b];
      const int nbl = I.nrows[b] - I.ncols[b];
      if (nbl > 0) {
        int gb = (int)std::min<long long>(((long long)nbl * m + 255) / 256, 8 * NUM_SMS);
        count_launch();
        gather_rows_kernel<T><<<gb, 256, 0, s>>>(nbl, m, I.d_rows.template as<int>() + I.rowptr[b] + I.ncols[b], B, ldb,
                                                 gb_buf);
        gemm<T>(s, true, false, I.ncols[b], m, nbl, T(-1), D.L + I.ncols[b], D.ldl, gb_buf, nbl, T(1), top, ldb,
                false, sc);
      }
      dense_trsm_bwd<T>(s, D, top, ldb, m);
    }
    if (par) join_aux(st, (int)bl.size());
    const long long ns = I.small_off[l + 1] - I.small_off[l];
    if (ns > 0 && use_front) {
      count_launch();
      bwd_front_kernel<T><<<(int)ns, 256, fsm, st>>>(
          I.d_small.template as<int>() + I.small_off[l], I.F.template as<T>(), I.d_fptr.template as<long long>(),
          I.d_ncols.template as<int>(), I.d_nrows.template as<int>(), I.d_start.template as<long long>(),
          I.d_rowptr.template as<long long>(), I.d_rows.template as<int>(), B, ldb, m, I.ncmax_small);
    } else if (ns > 0) {
      count_launch();
      bwd_small_kernel<T><<<(int)ns, 256, 0, st>>>(
          I.d_small.template as<int>() + I.small_off[l], I.F.template as<T>(), I.d_fptr.template as<long long>(), I.d_ncols.template as<int>(),
          I.d_nrows.template as<int>(), I.d_start.template as<long long>(), I.d_rowptr.template as<long long>(), I.d_rows.template as<int>(), B,
          ldb, m);
    }
  }
  check_launch("sparse solve");
}

template <typename T>
void SparseFactorSolve<T>::apply_L(cudaStream_t st, const T* X, T* Y, int m) {
  Impl& I = *p_;
  MPL_CUDA(cudaMemsetAsync(Y, 0, sizeof(T) * (size_t)I.n * m, st));
  count_launch();
  apply_L_kernel<T><<<1, 256, 0, st>>>((int)I.nb, I.F.template as<T>(), I.d_fptr.template as<long long>(), I.d_ncols.template as<int>(),
                                       I.d_nrows.template as<int>(), I.d_start.template as<long long>(), I.d_rowptr.template as<long long>(),
                                       I.d_rows.template as<int>(), X, I.n, Y, I.n, m);
  check_launch("apply_L");
}

template class SparseFactorSolve<float>;
template class SparseFactorSolve<double>;

}  // namespace mpl
