// Algorithm 1 on the device: reorder (Algorithm 2) -> SVD of the A11 blocks
// (Eq. 1) -> row incremental update with A21 (Eq. 2) -> column incremental
// update with T = [A12; A22] (Eq. 3); plus the pseudoinverse apply of
// Problem 1 / Application 1 and the residual of Application 1.
//
// Both incremental updates are the same operation on a thin SVD
// X = Uc diag(sigma) W^T (Uc: p x k orthonormal, W: q x k): append c sparse
// columns D and keep `target` triplets.  The row update (Eq. 2) runs it on the
// transpose [V1 Sigma1, A21^T] (Uc = V1, the appended columns are rows of A21,
// W gives U_row = bdiag(U1, I) W); the column update (Eq. 3) runs it on
// [U_row Sigma_row, T] (Uc = U_row, W gives V = [[V_row W_top], [W_bot]]).
// One append step (the incremental SVD the paper cites for Eqs. 2 and 3):
//   P = Uc^T D (sparse x dense) ; R = D - Uc P ; second pass P2 = Uc^T R,
//   R -= Uc P2, P += P2 ; CholeskyQR2 of R with dependent directions dropped
//   (R = Q R_R, zero rows of R_R / zero columns of Q for dropped directions) ;
//   core K = [[diag(sigma), P], [0, R_R]] ; K = Ut diag(s) Vt^T (Jacobi) ;
//   keep kk = min(target, k + rank) ; Uc <- [Uc, Q] Ut[:, :kk] ;
//   W <- [[W, 0], [0, I_c]] Vt[:, :kk].
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <functional>
#include <string>
#include <thread>
#include <mutex>
#include <condition_variable>
#include <type_traits>

#include "cholqr.cuh"
#include "dense.cuh"
#include "factor.cuh"
#include "jacobi.cuh"
#include "tuning.cuh"

namespace fastpi {
namespace {

constexpr double DROP_TOL_FP64 = 1e-7;    // relative to the largest appended column norm
constexpr double DROP_TOL_MIXED = 1e-5;   // FP32 residuals: rounding floor near 1e-6
constexpr double DROP_ABS_PASS2 = 0.25;   // second CholeskyQR pass: kept columns have norm ~1
constexpr int64_t DEFAULT_CHUNK = 256;    // border rows / columns per append step when the caller passes 0

inline unsigned g1(int64_t n, int bs = 256) { return n > 0 ? unsigned((n + bs - 1) / bs) : 1u; }

// Dense products of the updates: FP64 SIMT in the FP64 form; in the mixed
// form the FP32 products go to the TF32 tensor cores (split hi + lo passes)
// when the shape has enough work.
template <typename T>
inline void gemm_t(cudaStream_t st, bool ta, bool tb, int64_t M, int64_t N, int64_t K, T alpha, const T* A,
                   int64_t lda, const T* B, int64_t ldb, T beta, T* C, int64_t ldc) {
  if constexpr (std::is_same<T, float>::value)
    gemm_f32(st, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  else
    gemm<T>(st, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
}

struct BlkDesc {
  int64_t m_b, n_b, s_b, ro, co, soff, data_off, v_off, u_off, sig_off;
};

// ----------------------------------------------------------------- blocks (Eq. 1)
template <typename T>
__global__ void k_block_out(const BlkDesc* __restrict__ d, const T* __restrict__ data, const T* __restrict__ vbuf,
                            const double* __restrict__ sig, const int32_t* __restrict__ perm,
                            const int32_t* __restrict__ pos, int64_t ldv, T* V1, T* U1, double* Sig1) {
  const BlkDesc b = d[blockIdx.x];
  const bool tall = b.m_b >= b.n_b;
  const int64_t p = tall ? b.m_b : b.n_b, q = tall ? b.n_b : b.m_b;
  const T* B = data + b.data_off;
  const T* J = vbuf + b.v_off;
  for (int64_t t = 0; t < b.s_b; ++t) {
    const int32_t src = perm[b.sig_off + t];
    const double s = sig[b.sig_off + t];
    const T inv = s > 0 ? T(1.0 / s) : T(0);
    const int32_t g = pos[b.soff + t];   // column of this triplet in the row-phase state, -1: not kept
    for (int64_t li = threadIdx.x; li < b.m_b; li += blockDim.x)
      U1[b.u_off + li * b.s_b + t] = tall ? B[int64_t(src) * p + li] * inv : J[int64_t(src) * q + li];
    if (g < 0) continue;
    if (threadIdx.x == 0) Sig1[g] = s;
    for (int64_t j = threadIdx.x; j < b.n_b; j += blockDim.x)
      V1[(b.co + j) * ldv + g] = tall ? J[int64_t(src) * q + j] : B[int64_t(src) * p + j] * inv;
  }
}

// W[g, pos[g]] = 1 for the kept block triplets (W zeroed before).
template <typename T>
__global__ void k_select_w(const int32_t* __restrict__ pos, int64_t S, T* W, int64_t ldw) {
  const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (g < S && pos[g] >= 0) W[g * ldw + pos[g]] = T(1);
}

__global__ void k_blk_of_row(const int64_t* off, int64_t B, int32_t* blk_of) {
  int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (b >= B) return;
  for (int64_t i = off[b]; i < off[b + 1]; ++i) blk_of[i] = int32_t(b);
}

// U_row = [[U1 W_top], [W_bot]] (Eq. 2): U1 block diagonal, packed per block.
template <typename T>
__global__ void k_urow(int64_t m, int64_t m1, int64_t s, int64_t S, const int32_t* __restrict__ blk_of_row,
                       const BlkDesc* __restrict__ bd, const T* __restrict__ U1, const T* __restrict__ W,
                       int64_t ldw, T* __restrict__ Urow, int64_t ldo) {
  const int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= m) return;
  if (i >= m1) {
    const T* src = W + (S + i - m1) * ldw;
    for (int64_t j = lane; j < s; j += 32) Urow[i * ldo + j] = src[j];
    return;
  }
  const BlkDesc b = bd[blk_of_row[i]];
  const int64_t li = i - b.ro;
  for (int64_t j = lane; j < s; j += 32) {
    T acc = 0;
    for (int64_t t = 0; t < b.s_b; ++t) acc = fma(U1[b.u_off + li * b.s_b + t], W[(b.soff + t) * ldw + j], acc);
    Urow[i * ldo + j] = acc;
  }
}

// ----------------------------------------------------------------- append step
// D (p x c, ld c) <- dense copy of sparse columns [a, a + c); dn[t] = |d_t|^2
template <typename T>
__global__ void k_scatter_cols(const int64_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                               const double* __restrict__ val, int64_t a, int64_t c, T* D, double* dn) {
  const int64_t t = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= c) return;
  double s = 0;
  for (int64_t e = ptr[a + t] + lane; e < ptr[a + t + 1]; e += 32) {
    double v = val[e];
    D[int64_t(idx[e]) * c + t] = T(v);
    s += v * v;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) dn[t] = s;
}

// Pt[t, :] = sum_e val_e * Uc[idx_e, :]  (P^T = D^T Uc for sparse D)
template <typename T>
__global__ void k_spmm_t(const int64_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                         const double* __restrict__ val, int64_t a, int64_t k, const T* __restrict__ Uc,
                         int64_t ldu, T* __restrict__ Pt, int64_t ldp) {
  const int64_t t = blockIdx.x;
  const int64_t e0 = ptr[a + t], e1 = ptr[a + t + 1];
  for (int64_t j = threadIdx.x; j < k; j += blockDim.x) {
    T acc = 0;
    for (int64_t e = e0; e < e1; ++e) acc = fma(T(val[e]), Uc[int64_t(idx[e]) * ldu + j], acc);
    Pt[t * ldp + j] = acc;
  }
}

// The same product with a column's nonzeros split over the CTA's 8 warps (a
// hub row or column has hundreds of them, and one thread walking them all is
// a chain of dependent gathers): warp w sums the nonzeros of its contiguous
// share, lane l the entries j = l + 32 u, u < SP_U (k <= 32 SP_U), and the 8
// partial sums are added in warp order through shared memory.
constexpr int SP_WARPS = 8, SP_U = 32;
template <typename T>
__global__ void __launch_bounds__(SP_WARPS * 32) k_spmm_t_split(const int64_t* __restrict__ ptr,
                                                                const int32_t* __restrict__ idx,
                                                                const double* __restrict__ val, int64_t a, int k,
                                                                const T* __restrict__ Uc, int64_t ldu,
                                                                T* __restrict__ Pt, int64_t ldp) {
  extern __shared__ unsigned char sp_raw[];
  T* part = reinterpret_cast<T*>(sp_raw);   // [SP_WARPS][k]
  const int64_t t = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t e0 = ptr[a + t], e1 = ptr[a + t + 1];
  const int64_t per = (e1 - e0 + SP_WARPS - 1) / SP_WARPS;
  const int64_t b0 = min(e1, e0 + w * per), b1 = min(e1, b0 + per);
  T acc[SP_U];
#pragma unroll
  for (int u = 0; u < SP_U; ++u) acc[u] = T(0);
  for (int64_t e = b0; e < b1; ++e) {
    const T v = T(val[e]);
    const T* row = Uc + int64_t(idx[e]) * ldu;
#pragma unroll
    for (int u = 0; u < SP_U; ++u) {
      const int j = lane + 32 * u;
      if (j < k) acc[u] = fma(v, row[j], acc[u]);
    }
  }
#pragma unroll
  for (int u = 0; u < SP_U; ++u) {
    const int j = lane + 32 * u;
    if (j < k) part[w * k + j] = acc[u];
  }
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += SP_WARPS * 32) {
    T s = part[j];
    for (int q = 1; q < SP_WARPS; ++q) s += part[q * k + j];
    Pt[t * ldp + j] = s;
  }
}

template <typename T>
__global__ void k_axpy2d(int64_t rows, int64_t cols, const T* X, int64_t ldx, T* Y, int64_t ldy) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= rows * cols) return;
  int64_t i = t / cols, j = t % cols;
  Y[i * ldy + j] += X[i * ldx + j];
}

template <typename Td, typename Ts>
__global__ void k_convert(int64_t n, const Ts* s, Td* d) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < n) d[t] = Td(s[t]);
}

// Cholesky of the c x c Gram G (row-major, lower triangle used) in the
// precision of T, right-looking, one CTA.  A pivot d_j <= thr marks column j
// as dependent: its column of L is zero (the direction is dropped).
// thr = (tol * max_t dn[t]) when dn != null, else tol (absolute).  On exit G
// holds L (upper part zero), kept[j] in {0,1}, *rank = number kept.
template <typename T>
__global__ void k_chol_drop(T* G, int c, const double* dn, double tol, int32_t* kept, int32_t* rank) {
  __shared__ double s_thr;
  __shared__ int s_keep;
  __shared__ double s_ljj;
  if (threadIdx.x == 0) {
    double thr = tol;
    if (dn) {
      double mx = 0;
      for (int t = 0; t < c; ++t) mx = fmax(mx, dn[t]);
      thr = tol * tol * mx;
    }
    s_thr = thr;
  }
  __syncthreads();
  int nk = 0;
  for (int j = 0; j < c; ++j) {
    if (threadIdx.x == 0) {
      double d = double(G[int64_t(j) * c + j]);
      s_keep = d > s_thr;
      s_ljj = s_keep ? sqrt(d) : 0.0;
      G[int64_t(j) * c + j] = T(s_ljj);
      kept[j] = s_keep;
    }
    __syncthreads();
    const int keep = s_keep;
    const T inv = keep ? T(1.0 / s_ljj) : T(0);
    nk += keep;
    for (int i = j + 1 + threadIdx.x; i < c; i += blockDim.x) G[int64_t(i) * c + j] *= inv;
    __syncthreads();
    if (keep) {
      const int nrem = c - j - 1;
      for (int64_t e = threadIdx.x; e < int64_t(nrem) * nrem; e += blockDim.x) {
        int i = j + 1 + int(e / nrem), l = j + 1 + int(e % nrem);
        if (l <= i) G[int64_t(i) * c + l] -= G[int64_t(i) * c + j] * G[int64_t(l) * c + j];
      }
    }
    __syncthreads();
  }
  for (int64_t e = threadIdx.x; e < int64_t(c) * c; e += blockDim.x) {
    int i = int(e / c), l = int(e % c);
    if (l > i) G[e] = T(0);
  }
  if (threadIdx.x == 0) *rank = nk;
}

// Same result as k_chol_drop, with the lower triangle of G held packed in
// shared memory for the whole factorization (row i starts at i (i + 1) / 2),
// so that each of the c sequential steps costs shared-memory latency only.
template <typename T>
__global__ void k_chol_drop_smem(T* G, int c, double tol, int32_t* kept, int32_t* rank) {
  extern __shared__ unsigned char craw[];
  T* P = reinterpret_cast<T*>(craw);
  T* colj = P + (int64_t(c) * (c + 1)) / 2;   // c entries
  __shared__ int s_keep;
  __shared__ T s_inv;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = w; i < c; i += nw)
    for (int l = lane; l <= i; l += 32) P[(int64_t(i) * (i + 1)) / 2 + l] = G[int64_t(i) * c + l];
  __syncthreads();
  int nk = 0;
  for (int j = 0; j < c; ++j) {
    const int64_t dj = (int64_t(j) * (j + 1)) / 2 + j;
    if (threadIdx.x == 0) {
      const double d = double(P[dj]);
      s_keep = d > tol;
      const double ljj = s_keep ? sqrt(d) : 0.0;
      P[dj] = T(ljj);
      s_inv = s_keep ? T(1.0 / ljj) : T(0);
      kept[j] = s_keep;
    }
    __syncthreads();
    const int keep = s_keep;
    nk += keep;
    const T inv = s_inv;
    // column j scaled in place and copied to a contiguous buffer: the update
    // below reads it by row index, which in the packed triangle lands on
    // scattered banks
    for (int i = j + 1 + threadIdx.x; i < c; i += blockDim.x) {
      const T v = P[(int64_t(i) * (i + 1)) / 2 + j] * inv;
      P[(int64_t(i) * (i + 1)) / 2 + j] = v;
      colj[i] = v;
    }
    __syncthreads();
    if (keep) {
      for (int i = j + 1 + w; i < c; i += nw) {
        const int64_t ri = (int64_t(i) * (i + 1)) / 2;
        const T lij = colj[i];
        for (int l = j + 1 + lane; l <= i; l += 32) P[ri + l] -= lij * colj[l];
      }
    }
    __syncthreads();
  }
  for (int i = w; i < c; i += nw)
    for (int l = lane; l < c; l += 32) G[int64_t(i) * c + l] = l <= i ? P[(int64_t(i) * (i + 1)) / 2 + l] : T(0);
  if (threadIdx.x == 0) *rank = nk;
}

// Cholesky with diagonal pivoting of the c x c Gram G = R^T R (full symmetric,
// row-major, FP64), one CTA; the pivot rule (largest remaining diagonal, ties
// to the lower index) is the one of QR with column pivoting on R.  Step t
// takes the column piv[t] with the largest Schur-complement diagonal d; when
// that d <= thr = (tol^2 max_t dn[t]) the remaining columns are dependent and
// the factorization stops at rank = t.  Output, in ORIGINAL column indexing:
//   Lo (c x c, row-major): Lo[i, t] = L[i, t] for t < rank (zero beyond), so
//   that G ~ Lo Lo^T and R = Q1 Lo^T with Q1 = R[:, piv[:rank]] L_pp^-T;
//   Lp (c x c): the rank x rank triangle L_pp[a, b] = Lo[piv[a], b] (zero
//   elsewhere); kept[a] = (a < rank); piv[t].
__global__ void k_pchol(const double* G, int c, const double* dn, double tol, double* Lo, double* Lp,
                        int32_t* kept, int32_t* piv, int32_t* rank_out) {
  extern __shared__ double psm[];
  double* d = psm;                                   // c
  int* used = reinterpret_cast<int*>(psm + c);       // c
  __shared__ double s_thr, s_best;
  __shared__ int s_arg, s_rank;
  __shared__ double red_v[32];
  __shared__ int red_i[32];
  for (int i = threadIdx.x; i < c; i += blockDim.x) {
    d[i] = G[int64_t(i) * c + i];
    used[i] = 0;
    kept[i] = 0;
    piv[i] = -1;
  }
  for (int64_t e = threadIdx.x; e < int64_t(c) * c; e += blockDim.x) {
    Lo[e] = 0.0;
    Lp[e] = 0.0;
  }
  if (threadIdx.x == 0) {
    double mx = 0;
    for (int t = 0; t < c; ++t) mx = fmax(mx, dn[t]);
    s_thr = tol * tol * mx;
    s_rank = 0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int t = 0; t < c; ++t) {
    // argmax of d over unused columns (ties: lower index)
    double bv = -1.0;
    int bi = c;
    for (int i = threadIdx.x; i < c; i += blockDim.x)
      if (!used[i] && (d[i] > bv || (d[i] == bv && i < bi))) {
        bv = d[i];
        bi = i;
      }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) {
        bv = ov;
        bi = oi;
      }
    }
    if (lane == 0) {
      red_v[w] = bv;
      red_i[w] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double v = red_v[0];
      int ii = red_i[0];
      for (int q = 1; q < nw; ++q)
        if (red_v[q] > v || (red_v[q] == v && red_i[q] < ii)) {
          v = red_v[q];
          ii = red_i[q];
        }
      s_best = v;
      s_arg = ii;
    }
    __syncthreads();
    if (!(s_best > s_thr) || s_arg >= c) break;   // every remaining column is dependent
    const int j = s_arg;
    const double ljj = sqrt(s_best);
    if (threadIdx.x == 0) {
      used[j] = 1;
      piv[t] = j;
      kept[t] = 1;
      Lo[int64_t(j) * c + t] = ljj;
      s_rank = t + 1;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < c; i += blockDim.x) {
      if (used[i]) continue;
      double s = G[int64_t(i) * c + j];
      for (int q = 0; q < t; ++q) s -= Lo[int64_t(i) * c + q] * Lo[int64_t(j) * c + q];
      const double lit = s / ljj;
      Lo[int64_t(i) * c + t] = lit;
      d[i] -= lit * lit;
    }
    __syncthreads();
  }
  __syncthreads();
  const int rank = s_rank;
  for (int64_t e = threadIdx.x; e < int64_t(rank) * rank; e += blockDim.x) {
    const int a = int(e / rank), b = int(e % rank);
    if (b <= a) Lp[int64_t(a) * c + b] = Lo[int64_t(piv[a]) * c + b];
  }
  if (threadIdx.x == 0) *rank_out = rank;
}

// Blocked form of k_pchol.  G (c x c, FP64, full symmetric) holds the Schur
// complement of the columns factored so far (earlier panels are removed from
// it by k_pchol_trailing after each panel); d / used / Lo / piv / kept / rank
// persist in global memory across the panels (Lo zero before the first).  One
// CTA factors the panel columns [t0, t0 + nb) with the same pivot rule and
// drop test as k_pchol: the pivot is the unused column with the largest
// remaining diagonal (ties to the lower index); when it is <= thr the
// factorization stops (state[0] = 1).  The panel's columns of Lo are staged
// in shared memory.
//
// A step is a chain of dependent parts, so each is kept off GB300's slow FP64
// pipe where it can be: the pivot search compares order-preserving integer
// images of the FP64 diagonal with warp reductions (value descending, index
// ascending; no FP64 compare), one thread takes the square root and the
// reciprocal and hands them to the others, and the row update splits its dot
// product over four independent accumulators, issued before the load of the
// pivot's row of G that it ends with.  (Loading every thread's entries of all
// eight warp winners' rows while the last reduction runs was measured slower.)
constexpr int PCHOL_NB = 32;
constexpr int PCHOL_PS = PCHOL_NB + 1;   // panel row stride: odd, so a warp's rows fall in different banks
constexpr int PCHOL_THREADS = 256;
#ifdef FASTPI_PHASE_CLOCKS
// clock64 per phase of the panel kernel, thread 0: 0 set-up, 1 pivot search
// (with the square root and reciprocal), 4 row update, 5 CTA barrier,
// 6 write-back, 7 steps
__device__ long long g_pc1_clk[8];
#define PC1_MARK(k)                          \
  do {                                       \
    if (threadIdx.x == 0) {                  \
      const long long t_ = clock64();        \
      g_pc1_clk[k] += t_ - t_mark;           \
      t_mark = t_;                           \
    }                                        \
  } while (0)
#else
#define PC1_MARK(k) \
  do {              \
  } while (0)
#endif

// Within a warp: the largest key, ties to the lowest index (idx = UINT_MAX
// for lanes without a candidate); every lane gets the result.
__device__ __forceinline__ void warp_argmax_key(unsigned long long& key, unsigned& idx) {
  const unsigned hi = unsigned(key >> 32), lo = unsigned(key);
  const unsigned mhi = __reduce_max_sync(0xffffffffu, hi);
  const unsigned mlo = __reduce_max_sync(0xffffffffu, hi == mhi ? lo : 0u);
  idx = __reduce_min_sync(0xffffffffu, (hi == mhi && lo == mlo) ? idx : 0xffffffffu);
  key = (static_cast<unsigned long long>(mhi) << 32) | mlo;
}

__global__ void __launch_bounds__(PCHOL_THREADS) k_pchol_panel(const double* __restrict__ G, int c, int t0,
                                                               const double* dn, double tol, double* d,
                                                               int32_t* used, double* Lo, int32_t* piv,
                                                               int32_t* kept, int32_t* state) {
  extern __shared__ double pan[];   // c x PCHOL_PS: Lo[:, t0 + k]; then d_s[c]; then used_s[c]
  double* d_s = pan + size_t(c) * PCHOL_PS;
  int* used_s = reinterpret_cast<int*>(d_s + c);
  __shared__ unsigned long long red_k[PCHOL_THREADS / 32];
  __shared__ unsigned red_i[PCHOL_THREADS / 32];
  __shared__ double red_v[PCHOL_THREADS / 32];
  __shared__ double s_thr, s_ljj, s_rljj;
  __shared__ int s_arg, s_stop;
#ifdef FASTPI_PHASE_CLOCKS
  long long t_mark = clock64();
#endif
  if (state[0]) return;   // an earlier panel stopped the factorization
  const int nb = min(PCHOL_NB, c - t0);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  constexpr int NW = PCHOL_THREADS / 32;
  // state of the pivoting (diagonal of the Schur complement, used columns) in
  // shared memory for the whole panel; the drop threshold from the largest
  // appended column norm (block reduction)
  double mx = 0.0;
  for (int i = tid; i < c; i += PCHOL_THREADS) {
    if (t0 == 0) {
      d_s[i] = G[int64_t(i) * c + i];
      used_s[i] = 0;
      kept[i] = 0;
      piv[i] = -1;
    } else {
      d_s[i] = d[i];
      used_s[i] = used[i];
    }
    mx = fmax(mx, dn[i]);
  }
  for (int e = tid; e < c * PCHOL_PS; e += PCHOL_THREADS) pan[e] = 0.0;
#pragma unroll
  for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) red_v[w] = mx;
  __syncthreads();
  if (tid == 0) {
    double m2 = 0.0;
    for (int q = 0; q < NW; ++q) m2 = fmax(m2, red_v[q]);
    s_thr = tol * tol * m2;
  }
  __syncthreads();
  int stop = 0;
  PC1_MARK(0);
  for (int k = 0; k < nb; ++k) {
    const int t = t0 + k;
    // pivot: the unused column with the largest remaining diagonal (ties: lower index)
    unsigned long long bk = 0;
    unsigned bi = 0xffffffffu;
    for (int i = tid; i < c; i += PCHOL_THREADS)
      if (!used_s[i]) {
        const unsigned long long kk = order_key(d_s[i]);
        if (bi == 0xffffffffu || kk > bk) {   // rows ascend per thread: ties keep the first
          bk = kk;
          bi = unsigned(i);
        }
      }
    warp_argmax_key(bk, bi);
    if (lane == 0) {
      red_k[w] = bk;
      red_i[w] = bi;
    }
    __syncthreads();
    if (w == 0) {
      bk = lane < NW ? red_k[lane] : 0ull;
      bi = lane < NW ? red_i[lane] : 0xffffffffu;
      warp_argmax_key(bk, bi);
      if (lane == 0) {
        const double best = order_value(bk);
        const bool st = bi >= unsigned(c) || !(best > s_thr);
        s_stop = st ? 1 : 0;
        s_arg = int(bi);
        if (!st) {
          const double ljj = sqrt(best);
          s_ljj = ljj;
          // one reciprocal instead of a division per row
          s_rljj = 1.0 / ljj;
        }
      }
    }
    __syncthreads();
    PC1_MARK(1);
    if (s_stop) {
      stop = 1;
      break;
    }
    const int j = s_arg;
    const double ljj = s_ljj, rljj = s_rljj;
    // column t for every unused row other than the pivot: the Schur complement
    // column of pivot j (row j of G, by symmetry) minus this panel's earlier columns
    const double* pj = pan + j * PCHOL_PS;
    for (int i = tid; i < c; i += PCHOL_THREADS) {
      if (i == j) {
        pan[j * PCHOL_PS + k] = ljj;
        used_s[j] = 1;
        continue;
      }
      if (used_s[i]) continue;
      const double* pi = pan + i * PCHOL_PS;
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      int q = 0;
      for (; q + 4 <= k; q += 4) {
        a0 = fma(pi[q], pj[q], a0);
        a1 = fma(pi[q + 1], pj[q + 1], a1);
        a2 = fma(pi[q + 2], pj[q + 2], a2);
        a3 = fma(pi[q + 3], pj[q + 3], a3);
      }
      for (; q < k; ++q) a0 = fma(pi[q], pj[q], a0);
      const double lit = (G[int64_t(j) * c + i] - ((a0 + a1) + (a2 + a3))) * rljj;
      pan[i * PCHOL_PS + k] = lit;
      d_s[i] -= lit * lit;
    }
    if (tid == 0) {
      piv[t] = j;
      kept[t] = 1;
      state[1] = t + 1;   // rank so far
    }
    PC1_MARK(4);
    __syncthreads();
    PC1_MARK(5);
#ifdef FASTPI_PHASE_CLOCKS
    if (tid == 0) g_pc1_clk[7] += 1;
#endif
  }
  for (int e = tid; e < c * nb; e += PCHOL_THREADS) {
    const int i = e / nb, k = e % nb;
    Lo[int64_t(i) * c + t0 + k] = pan[i * PCHOL_PS + k];
  }
  for (int i = tid; i < c; i += PCHOL_THREADS) {
    d[i] = d_s[i];
    used[i] = used_s[i];
  }
  if (tid == 0 && stop) state[0] = 1;
  PC1_MARK(6);
}

// G[i, l] -= sum_{q in [t0, t0 + nb)} Lo[i, q] Lo[l, q] for all i, l < c: the
// Schur-complement update after a panel of k_pchol_panel, one thread per entry
// so that the FP64 work spreads over every SM (a tiled GEMM of this c x c x 32
// shape has too few tiles to do so).  Skipped once the factorization stopped.
__global__ void k_pchol_trailing(double* __restrict__ G, int c, int t0, int nb, const double* __restrict__ Lo,
                                 const int32_t* __restrict__ state) {
  if (state[0]) return;
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= int64_t(c) * c) return;
  const int i = int(e / c), l = int(e % c);
  const double* Li = Lo + int64_t(i) * c + t0;
  const double* Ll = Lo + int64_t(l) * c + t0;
  double s = 0.0;
  for (int q = 0; q < nb; ++q) s = fma(Li[q], Ll[q], s);
  G[e] -= s;
}

// Instrumented builds: the panel kernel's phase clocks to stderr (per step).
void pchol_phase_report(const char* tag) {
#ifdef FASTPI_PHASE_CLOCKS
  long long clk[8] = {0};
  CK(cudaMemcpyFromSymbol(clk, g_pc1_clk, sizeof clk));
  const long long st = std::max<long long>(1, clk[7]);
  fprintf(stderr, "pchol %s: steps %lld, per step clk: pivot %lld rows %lld sync %lld; set-up total %lld "
          "write-back total %lld\n", tag, clk[7], clk[1] / st, clk[4] / st, clk[5] / st, clk[0], clk[6]);
  const long long z[8] = {0};
  CK(cudaMemcpyToSymbol(g_pc1_clk, z, sizeof z));
#else
  (void)tag;
#endif
}

// Whether the core SVD runs on K^T, i.e. one-sided Jacobi orthogonalises the
// rows of K = [[diag(sigma), P], [0, R_R]] rather than its columns (default;
// FASTPI_CORE_TRANSPOSE=0 takes the columns).  Two rows i, i' < k of K meet
// only through P (their inner product is P_i . P_i', against norms that
// include sigma_i and sigma_i'), while a column of the border has its full
// projection P[:, t] against the sigma_j e_j columns; so the rows start much
// closer to orthogonal and the iteration needs fewer sweeps (the strategy of
// running Jacobi on R^T after a QR; here K is already upper triangular).
// Measured on the 20 000 x 5 000 workload: core SVD time per step 189 ->
// 158 ms (mixed), FP64 form 4.70 -> 4.38 s.
bool core_transposed() {
  const char* e = std::getenv("FASTPI_CORE_TRANSPOSE");
  return !(e && e[0] == '0' && e[1] == 0);
}

// Lp[a, b] = Lo[piv[a], b] for b <= a < rank (zero elsewhere); rank = state[1].
__global__ void k_gather_lp(const double* Lo, const int32_t* piv, const int32_t* state, int c, double* Lp,
                            int32_t* rank_out) {
  const int rank = state[1];
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < int64_t(c) * c;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int a = int(e / c), b = int(e % c);
    Lp[e] = (a < rank && b <= a) ? Lo[int64_t(piv[a]) * c + b] : 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *rank_out = rank;
}

// Lio[a, piv[b]] = X[a, b] for a, b < rank: the inverse of the kept triangle
// in the original column order, the map that turns R (p x c) into
// Q1 = R Lio^T; one thread per entry (the caller clears Lio first).
template <typename E>
__global__ void k_scatter_inv(const E* X, const int32_t* piv, const int32_t* rank_p, int c, E* Lio) {
  const int rank = *rank_p;
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= int64_t(rank) * rank) return;
  const int a = int(e / rank), b = int(e % rank);
  Lio[int64_t(a) * c + piv[b]] = X[int64_t(a) * c + b];
}

// X = inverse of L restricted to the kept indices (zero rows / columns for
// dropped ones).  One warp per column j of X solves L x = e_j by forward
// substitution; the lanes split each dot product, so the FP64 work of the
// c columns runs on c different SMs.
template <typename T>
__global__ void k_trinv_cols(const T* __restrict__ L, int c, const int32_t* __restrict__ kept, T* X) {
  extern __shared__ unsigned char xraw[];
  T* xcol = reinterpret_cast<T*>(xraw);   // c
  const int j = blockIdx.x, lane = threadIdx.x;
  for (int i = lane; i < c; i += 32) xcol[i] = T(0);
  __syncwarp();
  if (kept[j]) {
    for (int i = j; i < c; ++i) {
      T s = T(0);
      for (int l = j + lane; l < i; l += 32) s = fma(L[int64_t(i) * c + l], xcol[l], s);
#pragma unroll
      for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) xcol[i] = kept[i] ? (((i == j) ? T(1) : T(0)) - s) / L[int64_t(i) * c + i] : T(0);
      __syncwarp();
    }
  }
  for (int i = lane; i < c; i += 32) X[int64_t(i) * c + j] = xcol[i];
}

// K ((k + c) x (k + c), COLUMN-major) = [[diag(sig), P], [0, R_R]] with
// P = Pt^T (Pt: c x k, ld ldp) and R_R = M^T (M: c x c row-major, FP64);
// trans: K^T instead (K stored row-major).
template <typename T, typename TM>
__global__ void k_build_core(int64_t k, int64_t c, const double* __restrict__ sig, const T* __restrict__ Pt,
                             int64_t ldp, const TM* __restrict__ M, T* __restrict__ K, bool trans) {
  const int64_t n = k + c;
  int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  const int64_t a = e / n, b = e % n;
  const int64_t col = trans ? b : a, row = trans ? a : b;
  T v = 0;
  if (col < k) {
    if (row == col) v = T(sig[col]);
  } else {
    const int64_t t = col - k;
    if (row < k)
      v = Pt[t * ldp + row];
    else
      v = T(M[t * c + (row - k)]);
  }
  K[e] = v;
}

// Ut[i, t] = K[:, perm[t]] / sig[t] ; Vt[i, t] = J[i, perm[t]]   (n x kk, ld kk)
template <typename T>
__global__ void k_core_vectors(int64_t n, int64_t kk, const T* __restrict__ Kb, const T* __restrict__ J,
                               const double* __restrict__ sig, const int32_t* __restrict__ perm, T* Ut, T* Vt) {
  int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= n * kk) return;
  const int64_t i = e / kk, t = e % kk;
  const int64_t src = perm[t];
  const double s = sig[t];
  Ut[e] = s > 0 ? T(double(Kb[src * n + i]) / s) : T(0);
  Vt[e] = J[src * n + i];
}

// G <- (3 I - G) / 2 for a cols x cols matrix (one Newton-Schulz coefficient).
__global__ void k_ns_coef(float* G, int64_t cols) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= cols * cols) return;
  const int64_t i = e / cols, j = e % cols;
  G[e] = (i == j ? 1.5f : 0.f) - 0.5f * G[e];
}

// One Newton-Schulz step towards the nearest matrix with orthonormal columns,
// X <- X (3 I - X^T X) / 2, for X rows x cols (row-major, ld cols) in FP32.
// The FP32 core SVD's V is a product of thousands of FP32 rotations per
// column, orthonormal to ~1e-5 per core; the incremental update multiplies
// these factors into the basis append after append, so without this step the
// deviation of U^T U and V^T V from I grows with the number of appends.  One
// step brings it to the rounding level of the products (~1e-6).
void ns_orthonormalize(cudaStream_t st, int64_t rows, int64_t cols, float* X) {
  if (rows <= 0 || cols <= 0) return;
  DArr<float> G(cols * cols, st), Y(rows * cols, st);
  gemm_f32(st, true, false, cols, cols, rows, 1.f, X, cols, X, cols, 0.f, G.get(), cols);
  k_ns_coef<<<g1(cols * cols), 256, 0, st>>>(G.get(), cols);
  CK_LAUNCH();
  gemm_f32(st, false, false, rows, cols, cols, 1.f, X, cols, G.get(), cols, 0.f, Y.get(), cols);
  CK(cudaMemcpyAsync(X, Y.get(), size_t(rows * cols) * sizeof(float), cudaMemcpyDeviceToDevice, st));
}

// Single-CTA descending sort of sig[0..k) (ties: lower index first) -> perm.
__global__ void k_sort_desc(const double* sig, int k, int nq, int32_t* perm, double* sorted) {
  extern __shared__ unsigned char sm[];
  double* key = reinterpret_cast<double*>(sm);
  int* idx = reinterpret_cast<int*>(key + nq);
  for (int t = threadIdx.x; t < nq; t += blockDim.x) {
    key[t] = t < k ? sig[t] : -1.0;
    idx[t] = t;
  }
  __syncthreads();
  for (int size = 2; size <= nq; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < nq; t += blockDim.x) {
        int u = t ^ stride;
        if (u > t) {
          bool up = (t & size) == 0;
          double ka = key[t], kb = key[u];
          int ia = idx[t], ib = idx[u];
          bool a_first = (ka > kb) || (ka == kb && ia < ib);
          if (a_first != up) {
            key[t] = kb;
            key[u] = ka;
            idx[t] = ib;
            idx[u] = ia;
          }
        }
      }
      __syncthreads();
    }
  for (int t = threadIdx.x; t < k; t += blockDim.x) {
    perm[t] = idx[t];
    sorted[t] = key[t];
  }
}

template <typename T>
__global__ void k_gather_cols(int64_t rows, int64_t kk, const int32_t* perm, const T* src, int64_t lds, T* dst,
                              int64_t ldd) {
  int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= rows * kk) return;
  int64_t i = e / kk, t = e % kk;
  dst[i * ldd + t] = src[i * lds + perm[t]];
}

// ----------------------------------------------------------------- phase
template <typename T>
struct Phase {
  fastpi_ctx* h;
  cudaStream_t st;
  int64_t p, kmax, qmax, cmax;
  DArr<T> Uc[2], W[2];
  DArr<double> sig[2];
  int cur = 0;
  int64_t k = 0, q = 0;
  double drop_tol;
  // statistics
  int64_t steps = 0, dropped = 0;
  int sweeps_max = 0;
  double min_gap = INFINITY;

  Phase(fastpi_ctx* hh, int64_t p_, int64_t kmax_, int64_t qmax_, int64_t cmax_, double tol)
      : h(hh), st(hh->stream), p(p_), kmax(kmax_), qmax(qmax_), cmax(cmax_), drop_tol(tol) {
    for (int i = 0; i < 2; ++i) {
      Uc[i] = DArr<T>(p * kmax, st);
      W[i] = DArr<T>(qmax * kmax, st);
      sig[i] = DArr<double>(kmax + cmax, st);
    }
  }
  T* U() { return Uc[cur].get(); }
  T* Wm() { return W[cur].get(); }
  double* S() { return sig[cur].get(); }

  void append(const SparseCols& sc, int64_t a, int64_t c, int64_t target) {
    const int64_t n = k + c;
    T* Ucur = U();
    DArr<T> D(p * c, st), Pt(c * std::max<int64_t>(k, 1), st), P2t(c * std::max<int64_t>(k, 1), st);
    DArr<double> dn(c, st);
    set_zero<T>(st, p, c, D.get(), c);
    k_scatter_cols<T><<<g1(c * 32), 256, 0, st>>>(sc.ptr, sc.idx, sc.val, a, c, D.get(), dn.get());
    CK_LAUNCH();
    const int64_t ldp = std::max<int64_t>(k, 1);
    if (k > 0) {
      if (k <= 32 * SP_U) {
        const size_t sm = size_t(SP_WARPS) * k * sizeof(T);
        if (sm > 48 * 1024) allow_max_dynamic_smem((const void*)k_spmm_t_split<T>);
        k_spmm_t_split<T><<<unsigned(c), SP_WARPS * 32, sm, st>>>(sc.ptr, sc.idx, sc.val, a, int(k), Ucur, kmax,
                                                                   Pt.get(), ldp);
      } else {
        k_spmm_t<T><<<unsigned(c), 256, 0, st>>>(sc.ptr, sc.idx, sc.val, a, k, Ucur, kmax, Pt.get(), ldp);
      }
      CK_LAUNCH();
      // R = D - Uc P ; second projection pass
      gemm_t<T>(st, false, true, p, c, k, T(-1), Ucur, kmax, Pt.get(), ldp, T(1), D.get(), c);
      gemm_t<T>(st, true, false, c, k, p, T(1), D.get(), c, Ucur, kmax, T(0), P2t.get(), ldp);
      gemm_t<T>(st, false, true, p, c, k, T(-1), Ucur, kmax, P2t.get(), ldp, T(1), D.get(), c);
      k_axpy2d<T><<<g1(c * k), 256, 0, st>>>(c, k, P2t.get(), ldp, Pt.get(), ldp);
      CK_LAUNCH();
    }
    // CholeskyQR2 with dependent directions dropped
    DArr<T> GT(c * c, st), Q1(p * c, st), Q(p * c, st), LinvT(c * c, st);
    DArr<double> G(c * c, st), Linv(c * c, st), G2(c * c, st), L2inv(c * c, st), M(c * c, st);
    DArr<double> Lo(c * c, st), Lp(c * c, st), X(c * c, st);
    DArr<int32_t> kept(c, st), kept2(c, st), piv(c, st), rk(2, st);
    // FP64 Gram of the residual: in the mixed mode from FP32 data, each
    // product split exactly and summed in FP32 pairs (about 48 bits), so that
    // its rounding floor sits far below the drop tolerance
    auto gram = [&](const T* X, double* Gd) {
      if constexpr (sizeof(T) == 8)
        gemm<double>(st, true, false, c, c, p, 1.0, X, c, X, c, 0.0, Gd, c);
      else
        gram_ff(st, p, c, X, c, Gd);
    };
    auto trinv = [&](auto* L, const int32_t* kp, auto* Xo) {
      using E = std::remove_pointer_t<decltype(L)>;
      int max_smem = 0;
      CK(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
      if (trinv_blocked_smem(int(c), sizeof(E)) + 1024 <= size_t(max_smem)) {
        trinv_blocked<E>(st, L, int(c), kp, Xo);   // 32-column blocks
      } else {
        const size_t sm = size_t(c) * sizeof(E);
        if (sm > 48 * 1024)
          allow_max_dynamic_smem((const void*)k_trinv_cols<E>);
        k_trinv_cols<E><<<unsigned(c), 32, sm, st>>>(L, int(c), kp, Xo);
        CK_LAUNCH();
      }
    };
    auto to_T = [&](const double* src, T* dst) {
      if (sizeof(T) == 8) {
        CK(cudaMemcpyAsync(dst, src, size_t(c * c) * 8, cudaMemcpyDeviceToDevice, st));
      } else {
        k_convert<T, double><<<g1(c * c), 256, 0, st>>>(c * c, src, dst);
        CK_LAUNCH();
      }
    };
    gram(D.get(), G.get());
    const size_t pan_bytes = size_t(c) * PCHOL_PS * sizeof(double) + size_t(c) * (sizeof(double) + sizeof(int));
    if (pan_bytes <= 200 * 1024) {
      // blocked: panels of PCHOL_NB columns in one CTA, each followed by the
      // Schur-complement update of the columns after it over every SM
      DArr<double> dd(c, st);
      DArr<int32_t> used(c, st), pstate(2, st);
      CK(cudaMemsetAsync(pstate.get(), 0, 8, st));
      CK(cudaMemsetAsync(Lo.get(), 0, size_t(c * c) * sizeof(double), st));
      if (pan_bytes > 48 * 1024)
        allow_max_dynamic_smem((const void*)k_pchol_panel);
      for (int64_t t0 = 0; t0 < c; t0 += PCHOL_NB) {
        k_pchol_panel<<<1, PCHOL_THREADS, pan_bytes, st>>>(G.get(), int(c), int(t0), dn.get(), drop_tol, dd.get(),
                                                  used.get(), Lo.get(), piv.get(), kept.get(), pstate.get());
        CK_LAUNCH();
        const int64_t nbp = std::min<int64_t>(PCHOL_NB, c - t0);
        if (t0 + nbp < c) {
          k_pchol_trailing<<<g1(c * c), 256, 0, st>>>(G.get(), int(c), int(t0), int(nbp), Lo.get(), pstate.get());
          CK_LAUNCH();
        }
      }
      k_gather_lp<<<g1(c * c), 256, 0, st>>>(Lo.get(), piv.get(), pstate.get(), int(c), Lp.get(), rk.get());
      CK_LAUNCH();
    } else {
      k_pchol<<<1, 1024, size_t(c) * 12, st>>>(G.get(), int(c), dn.get(), drop_tol, Lo.get(), Lp.get(), kept.get(),
                                               piv.get(), rk.get());
      CK_LAUNCH();
    }
    if constexpr (sizeof(T) == 8) {
      trinv(Lp.get(), kept.get(), X.get());
      CK(cudaMemsetAsync(Linv.get(), 0, size_t(c * c) * sizeof(double), st));
      k_scatter_inv<double><<<g1(c * c), 256, 0, st>>>(X.get(), piv.get(), rk.get(), int(c), Linv.get());
      CK_LAUNCH();
      to_T(Linv.get(), LinvT.get());
    } else {
      // mixed: the inverse of the kept triangle in FP32 -- its error, like that
      // of the FP32 product below, only perturbs the orthogonality of Q1, which
      // the second pass restores
      DArr<float> Lp32(c * c, st), X32(c * c, st);
      k_convert<float, double><<<g1(c * c), 256, 0, st>>>(c * c, Lp.get(), Lp32.get());
      CK_LAUNCH();
      trinv(Lp32.get(), kept.get(), X32.get());
      CK(cudaMemsetAsync(LinvT.get(), 0, size_t(c * c) * sizeof(float), st));
      k_scatter_inv<float><<<g1(c * c), 256, 0, st>>>(X32.get(), piv.get(), rk.get(), int(c), LinvT.get());
      CK_LAUNCH();
    }
    gemm_t<T>(st, false, true, p, c, c, T(1), D.get(), c, LinvT.get(), c, T(0), Q1.get(), c);
    // second pass: Q1 is orthonormal up to rounding, its Gram ~ I is well
    // conditioned, so this Cholesky runs in the storage precision
    gemm_t<T>(st, true, false, c, c, p, T(1), Q1.get(), c, Q1.get(), c, T(0), GT.get(), c);
    const size_t packed = (size_t(c) * (c + 1) / 2 + size_t(c)) * sizeof(T);
    int max_smem_b = 0;
    CK(cudaDeviceGetAttribute(&max_smem_b, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    if (sizeof(T) == 4 && chol_drop_blocked_smem(int(c)) + 16 * 1024 <= size_t(max_smem_b)) {
      // blocked by 32 columns, the packed triangle in shared memory
      chol_drop_blocked(st, reinterpret_cast<float*>(GT.get()), int(c), float(DROP_ABS_PASS2), kept2.get(),
                        rk.get() + 1);
    } else if (packed <= 200 * 1024) {
      if (packed > 48 * 1024)
        allow_max_dynamic_smem((const void*)k_chol_drop_smem<T>);
      k_chol_drop_smem<T><<<1, 1024, packed, st>>>(GT.get(), int(c), DROP_ABS_PASS2, kept2.get(), rk.get() + 1);
      CK_LAUNCH();
    } else {
      k_chol_drop<T><<<1, 1024, 0, st>>>(GT.get(), int(c), nullptr, DROP_ABS_PASS2, kept2.get(), rk.get() + 1);
      CK_LAUNCH();
    }
    trinv(GT.get(), kept2.get(), LinvT.get());
    gemm_t<T>(st, false, true, p, c, c, T(1), Q1.get(), c, LinvT.get(), c, T(0), Q.get(), c);
    // R_R = (Lo L2)^T : M = Lo * L2 (FP64 in the FP64 form; in the mixed form
    // in FP32 on the tensor cores, the precision of the core it feeds)
    DArr<T> K(n * n, st), J(n * n, st);
    const bool ktrans = core_transposed();
    if constexpr (sizeof(T) == 8) {
      CK(cudaMemcpyAsync(G2.get(), GT.get(), size_t(c * c) * 8, cudaMemcpyDeviceToDevice, st));
      gemm<double>(st, false, false, c, c, c, 1.0, Lo.get(), c, G2.get(), c, 0.0, M.get(), c);
      k_build_core<T, double><<<g1(n * n), 256, 0, st>>>(k, c, S(), Pt.get(), ldp, M.get(), K.get(), ktrans);
      CK_LAUNCH();
    } else {
      DArr<float> Lo32(c * c, st), M32(c * c, st);
      k_convert<float, double><<<g1(c * c), 256, 0, st>>>(c * c, Lo.get(), Lo32.get());
      CK_LAUNCH();
      gemm_f32(st, false, false, c, c, c, 1.f, Lo32.get(), c, GT.get(), c, 0.f, M32.get(), c);
      k_build_core<T, float><<<g1(n * n), 256, 0, st>>>(k, c, S(), Pt.get(), ldp, M32.get(), K.get(), ktrans);
      CK_LAUNCH();
    }
    // core SVD
    DArr<double> jsig(n, st);
    DArr<int32_t> jperm(n, st);
    JacobiStats js;
    bool done = false;
    if constexpr (sizeof(T) == 4) {
      done = jacobi_svd_block(h, K.get(), J.get(), int(n), jsig.get(), jperm.get(), &js);
    }
    if (!done) {
      std::vector<JacobiProblem<T>> pr(1);
      pr[0] = JacobiProblem<T>{K.get(), J.get(), n, n, int(n), int(n)};
      js = jacobi_svd_batched<T>(h, pr, jsig.get(), jperm.get(), sizeof(T) == 8 ? SVD_CORE64 : SVD_CORE32);
    }
    sweeps_max = std::max(sweeps_max, js.max_sweeps_used);
    int32_t rks[2];
    d2h_sync(rks, rk.get(), 8, st);
    const int64_t rank = std::min<int64_t>(rks[0], rks[1]);
    dropped += c - rank;
    int64_t kk = std::min<int64_t>(target, k + rank);
    std::vector<double> hs(n);
    d2h_sync(hs.data(), jsig.get(), size_t(n) * 8, st);
    if constexpr (sizeof(T) == 4) {
      // The FP32 Jacobi leaves columns below (n eps) |K|_F unrotated as noise;
      // their singular vectors are not orthogonal to the rest, so such
      // directions are never kept.
      double f2 = 0;
      for (double v : hs) f2 += v * v;
      const double floor_ = 2.0 * double(n) * 1.1920928955078125e-07 * std::sqrt(f2);
      int64_t live = 0;
      while (live < n && hs[live] > floor_) ++live;
      kk = std::min(kk, live);
    }
    if (kk > kmax) fail(FASTPI_ERR_ARG, "internal: basis exceeds its capacity");
    if (kk < n && kk > 0 && hs[0] > 0) min_gap = std::min(min_gap, (hs[kk - 1] - hs[kk]) / hs[0]);
    // rotations
    DArr<T> Ut(n * std::max<int64_t>(kk, 1), st), Vt(n * std::max<int64_t>(kk, 1), st);
    if (kk > 0) {
      // K^T J has orthogonal columns when the SVD ran on K^T: then J holds
      // K's left singular vectors and the normalised columns its right ones
      k_core_vectors<T><<<g1(n * kk), 256, 0, st>>>(n, kk, K.get(), J.get(), jsig.get(), jperm.get(),
                                                     ktrans ? Vt.get() : Ut.get(), ktrans ? Ut.get() : Vt.get());
      CK_LAUNCH();
      if constexpr (sizeof(T) == 4) {
        ns_orthonormalize(st, n, kk, Ut.get());
        ns_orthonormalize(st, n, kk, Vt.get());
      }
    }
    const int nx = cur ^ 1;
    T* Unew = Uc[nx].get();
    T* Wnew = W[nx].get();
    gemm_t<T>(st, false, false, p, kk, k, T(1), Ucur, kmax, Ut.get(), kk, T(0), Unew, kmax);
    gemm_t<T>(st, false, false, p, kk, c, T(1), Q.get(), c, Ut.get() + k * kk, kk, T(1), Unew, kmax);
    gemm_t<T>(st, false, false, q, kk, k, T(1), Wm(), kmax, Vt.get(), kk, T(0), Wnew, kmax);
    copy2d<T, T>(st, c, kk, Vt.get() + k * kk, kk, Wnew + q * kmax, kmax);
    CK(cudaMemcpyAsync(sig[nx].get(), jsig.get(), size_t(std::max<int64_t>(kk, 1)) * 8, cudaMemcpyDeviceToDevice,
                       st));
    cur = nx;
    k = kk;
    q += c;
    ++steps;
  }

  // Keep the `target` largest triplets when no append step ran.
  void truncate(int64_t target) {
    if (k <= target) return;
    int nq = 1;
    while (nq < k) nq <<= 1;
    if (nq > 16384) fail(FASTPI_ERR_ARG, "truncate: too many columns");
    DArr<int32_t> perm(k, st);
    DArr<double> sorted(k, st);
    size_t smem = size_t(nq) * 12;
    if (smem > 48 * 1024) allow_max_dynamic_smem((const void*)k_sort_desc);
    k_sort_desc<<<1, 1024, smem, st>>>(S(), int(k), nq, perm.get(), sorted.get());
    CK_LAUNCH();
    const int nx = cur ^ 1;
    k_gather_cols<T><<<g1(p * target), 256, 0, st>>>(p, target, perm.get(), U(), kmax, Uc[nx].get(), kmax);
    CK_LAUNCH();
    k_gather_cols<T><<<g1(q * target), 256, 0, st>>>(q, target, perm.get(), Wm(), kmax, W[nx].get(), kmax);
    CK_LAUNCH();
    CK(cudaMemcpyAsync(sig[nx].get(), sorted.get(), size_t(target) * 8, cudaMemcpyDeviceToDevice, st));
    cur = nx;
    k = target;
  }
};

template <typename T>
void run_phase(Phase<T>& ph, const SparseCols& sc, int64_t chunk, int64_t target) {
  const int64_t total = sc.ncols;
  for (int64_t a = 0; a < total; a += chunk) {
    int64_t c = std::min(chunk, total - a);
    ph.append(sc, a, c, target);
  }
  ph.truncate(target);
}

struct Timer {
  cudaStream_t st;
  cudaEvent_t a, b;
  explicit Timer(cudaStream_t s) : st(s) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
  void start() { cudaEventRecord(a, st); }
  double stop() {
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
  }
};

// The batched SVD of the A11 blocks (Eq. 1) is a parameter: one instance runs
// it on its own problems; a batch of instances hands them to a rendezvous that
// runs one launch over the blocks of every instance.  block_svd(probs, sig,
// perm) may redirect sig / perm to where it wrote the results.
template <typename T>
using BlockSvdFn = std::function<JacobiStats(const std::vector<JacobiProblem<T>>&, double*&, int32_t*&)>;

// Eq. 1 for the blocks of A11: dense copies in the working precision, one
// batched Jacobi SVD over all blocks, and the kept singular values on the host
// (sig_all[g] for block triplet g: blocks in order, descending within a block).
template <typename T>
struct BlockStage {
  std::vector<BlkDesc> bd;
  DArr<T> bdata, vbuf;
  DArr<double> bsig_own;
  DArr<int32_t> bperm_own;
  double* bsig = nullptr;
  int32_t* bperm = nullptr;
  int64_t utot = 0, vtot = 0, sigtot = 0;
  JacobiStats js;
  std::vector<double> sig_all;
};

template <typename T>
void run_block_stage(fastpi_ctx* h, const Reordering& R, const A11Blocks& blk, const BlockSvdFn<T>& block_svd,
                     BlockStage<T>& out) {
  cudaStream_t st = h->stream;
  const int64_t S = blk.S;
  std::vector<BlkDesc>& bd = out.bd;
  bd.resize(blk.B);
  std::vector<JacobiProblem<T>> probs;
  int64_t vtot = 0, utot = 0, sigtot = 0;
  for (int64_t b = 0; b < blk.B; ++b) {
    BlkDesc& d = bd[b];
    d.m_b = blk.m_b[b];
    d.n_b = blk.n_b[b];
    d.s_b = blk.s_b[b];
    d.ro = R.row_off[b];
    d.co = R.col_off[b];
    d.soff = blk.s_off[b];
    d.data_off = blk.data_off[b];
    d.u_off = utot;
    utot += d.m_b * d.s_b;
    if (d.s_b > 0) {
      int64_t q = std::min(d.m_b, d.n_b);
      d.v_off = vtot;
      d.sig_off = sigtot;
      vtot += q * q;
      sigtot += q;
    } else {
      d.v_off = d.sig_off = 0;
    }
  }
  out.bdata = DArr<T>(std::max<int64_t>(blk.total, 1), st);
  out.vbuf = DArr<T>(std::max<int64_t>(vtot, 1), st);
  if (blk.total > 0) {
    if (sizeof(T) == 8)
      CK(cudaMemcpyAsync(out.bdata.get(), blk.data.get(), size_t(blk.total) * 8, cudaMemcpyDeviceToDevice, st));
    else {
      k_convert<T, double><<<g1(blk.total), 256, 0, st>>>(blk.total, blk.data.get(), out.bdata.get());
      CK_LAUNCH();
    }
  }
  for (int64_t b = 0; b < blk.B; ++b) {
    const BlkDesc& d = bd[b];
    if (d.s_b == 0) continue;
    int64_t p = std::max(d.m_b, d.n_b), q = std::min(d.m_b, d.n_b);
    probs.push_back(
        JacobiProblem<T>{out.bdata.get() + d.data_off, out.vbuf.get() + d.v_off, p, q, int(p), int(q)});
  }
  out.bsig_own = DArr<double>(std::max<int64_t>(sigtot, 1), st);
  out.bperm_own = DArr<int32_t>(std::max<int64_t>(sigtot, 1), st);
  out.bsig = out.bsig_own.get();
  out.bperm = out.bperm_own.get();
  out.js = block_svd(probs, out.bsig, out.bperm);
  out.utot = utot;
  out.vtot = vtot;
  out.sigtot = sigtot;
  std::vector<double> hsig(std::max<int64_t>(sigtot, 1));
  out.sig_all.assign(std::max<int64_t>(S, 1), 0.0);
  if (sigtot > 0) d2h_sync(hsig.data(), out.bsig, size_t(sigtot) * 8, st);
  for (const BlkDesc& d : bd)
    for (int64_t t = 0; t < d.s_b; ++t) out.sig_all[d.soff + t] = hsig[d.sig_off + t];
}

template <typename T>
void factor_impl(fastpi_ctx* h, Factors& F, int64_t r, double kratio, int64_t chunk_row, int64_t chunk_col,
                 const BlockSvdFn<T>& block_svd) {
  cudaStream_t st = h->stream;
  const int64_t m = h->m, n = h->n;
  fastpi_info& info = h->info;
  Timer tm(st);
  // ---- Algorithm 2 + split
  tm.start();
  Reordering& R = F.R;
  run_reorder(h, kratio, R);
  SparseCols A21, Tc;
  split_border(h, R, A21, Tc);
  A11Blocks blk;
  extract_blocks(h, R, r, blk);
  info.ms_reorder = tm.stop();
  const int64_t m1 = R.m1, n1 = R.n1, m2 = m - m1, n2 = n - n1, S = blk.S;

  // ---- Eq. 1: batched SVD of the A11 blocks
  tm.start();
  BlockStage<T> bs;
  run_block_stage<T>(h, R, blk, block_svd, bs);
  std::vector<BlkDesc>& bd = bs.bd;
  double* bsig = bs.bsig;
  int32_t* bperm = bs.bperm;
  const int64_t utot = bs.utot;
  JacobiStats bjs = bs.js;
  // Row phase basis: V1 (n1 x k0); U1 packed per block (all S); Sigma1
  const int64_t s_row = std::min<int64_t>({(r * n1 + n - 1) / n, S + m2, n1});
  const int prec_id = sizeof(T) == 8 ? 0 : 1;
  const int64_t cr = chunk_row > 0 ? chunk_row : tuned_chunk(prec_id, 0, s_row, DEFAULT_CHUNK);
  // Block triplet g (blocks in order, descending within a block) goes to
  // state column pos[g].  With several appends the running SVD of Eq. 2 holds
  // rank s_row between appends and the block SVD is its initial state, so only
  // the s_row largest block triplets are kept (descending; equal values: lower
  // index first); with one append all S enter the single merge of Eq. 2.
  std::vector<int32_t> pos(std::max<int64_t>(S, 1));
  int64_t k0 = S;
  {
    const std::vector<double>& sig_all = bs.sig_all;
    for (int64_t g = 0; g < S; ++g) pos[g] = int32_t(g);
    if (cr < m2 && S > s_row) {
      std::vector<int32_t> idx(S);
      for (int64_t g = 0; g < S; ++g) idx[g] = int32_t(g);
      std::stable_sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) { return sig_all[a] > sig_all[b]; });
      k0 = s_row;
      for (int64_t g = 0; g < S; ++g) pos[g] = -1;
      for (int64_t j = 0; j < k0; ++j) pos[idx[j]] = int32_t(j);
    }
  }
  const int64_t kmax_r = std::max<int64_t>({k0, s_row, 1});
  Phase<T> rowp(h, std::max<int64_t>(n1, 1), kmax_r, S + m2, std::min(cr, std::max<int64_t>(m2, 1)),
                sizeof(T) == 8 ? DROP_TOL_FP64 : DROP_TOL_MIXED);
  DArr<T> U1(std::max<int64_t>(utot, 1), st);
  DArr<BlkDesc> d_bd(std::max<int64_t>(blk.B, 1), st);
  if (blk.B > 0) CK(cudaMemcpyAsync(d_bd.get(), bd.data(), sizeof(BlkDesc) * blk.B, cudaMemcpyHostToDevice, st));
  set_zero<T>(st, n1, k0, rowp.U(), kmax_r);
  set_zero<T>(st, S, k0, rowp.Wm(), kmax_r);
  if (S > 0) {
    DArr<int32_t> d_pos(S, st);
    CK(cudaMemcpyAsync(d_pos.get(), pos.data(), size_t(S) * 4, cudaMemcpyHostToDevice, st));
    std::vector<BlkDesc> act;
    for (auto& d : bd)
      if (d.s_b > 0) act.push_back(d);
    DArr<BlkDesc> d_act(int64_t(act.size()), st);
    CK(cudaMemcpyAsync(d_act.get(), act.data(), sizeof(BlkDesc) * act.size(), cudaMemcpyHostToDevice, st));
    k_block_out<T><<<unsigned(act.size()), 128, 0, st>>>(d_act.get(), bs.bdata.get(), bs.vbuf.get(), bsig,
                                                         bperm, d_pos.get(), kmax_r, rowp.U(), U1.get(),
                                                         rowp.S());
    CK_LAUNCH();
    k_select_w<T><<<g1(S), 256, 0, st>>>(d_pos.get(), S, rowp.Wm(), kmax_r);
    CK_LAUNCH();
  }
  rowp.k = k0;
  rowp.q = S;
  info.ms_block_svd = tm.stop();

  // ---- Eq. 2: row incremental update with A21
  tm.start();
  run_phase(rowp, A21, cr, s_row);
  // U_row = [[U1 W_top], [W_bot]]  (m x s_row, new row order)
  DArr<T> Urow(m * std::max<int64_t>(s_row, 1), st);
  {
    DArr<int32_t> blk_of_row(std::max<int64_t>(m1, 1), st);
    DArr<int64_t> d_ro(blk.B + 1, st);
    CK(cudaMemcpyAsync(d_ro.get(), R.row_off.data(), size_t(blk.B + 1) * 8, cudaMemcpyHostToDevice, st));
    if (blk.B > 0) {
      k_blk_of_row<<<g1(blk.B), 256, 0, st>>>(d_ro.get(), blk.B, blk_of_row.get());
      CK_LAUNCH();
    }
    k_urow<T><<<g1(m * 32), 256, 0, st>>>(m, m1, rowp.k, S, blk_of_row.get(), d_bd.get(), U1.get(), rowp.Wm(),
                                          kmax_r, Urow.get(), std::max<int64_t>(s_row, 1));
    CK_LAUNCH();
  }
  info.ms_row_update = tm.stop();

  // ---- Eq. 3: column incremental update with T
  tm.start();
  const int64_t s = rowp.k;
  const int64_t rr = std::min<int64_t>({r, m, s + n2});
  const int64_t cc = chunk_col > 0 ? chunk_col : tuned_chunk(prec_id, 1, rr, DEFAULT_CHUNK);
  const int64_t kmax_c = std::max<int64_t>({s, rr, 1});
  Phase<T> colp(h, m, kmax_c, s + n2, std::min(cc, std::max<int64_t>(n2, 1)),
                sizeof(T) == 8 ? DROP_TOL_FP64 : DROP_TOL_MIXED);
  copy2d<T, T>(st, m, s, Urow.get(), std::max<int64_t>(s_row, 1), colp.U(), kmax_c);
  CK(cudaMemcpyAsync(colp.S(), rowp.S(), size_t(std::max<int64_t>(s, 1)) * 8, cudaMemcpyDeviceToDevice, st));
  set_identity<T>(st, s, s, colp.Wm(), kmax_c);
  colp.k = s;
  colp.q = s;
  run_phase(colp, Tc, cc, rr);
  info.ms_col_update = tm.stop();
#ifdef FASTPI_PHASE_CLOCKS
  CK(cudaStreamSynchronize(st));
  pchol_phase_report("factor");
  chol_drop_phase_report("factor");
#endif

  // ---- V = [[V_row W_top], [W_bot]]; back to the caller's order
  tm.start();
  const int64_t rank = colp.k;
  DArr<T> Vnew(n * std::max<int64_t>(rank, 1), st);
  gemm_t<T>(st, false, false, n1, rank, s, T(1), rowp.U(), kmax_r, colp.Wm(), kmax_c, T(0), Vnew.get(),
          std::max<int64_t>(rank, 1));
  copy2d<T, T>(st, n2, rank, colp.Wm() + s * kmax_c, kmax_c, Vnew.get() + n1 * std::max<int64_t>(rank, 1),
               std::max<int64_t>(rank, 1));
  const int64_t ldr = std::max<int64_t>(rank, 1);
  if (sizeof(T) == 8) {
    F.U64 = DArr<double>(m * ldr, st);
    F.V64 = DArr<double>(n * ldr, st);
    gather_rows<double, double>(st, m, rank, R.row_pos, (const double*)colp.U(), kmax_c, F.U64.get(), ldr);
    gather_rows<double, double>(st, n, rank, R.col_pos, (const double*)Vnew.get(), ldr, F.V64.get(), ldr);
  } else {
    F.U32 = DArr<float>(m * ldr, st);
    F.V32 = DArr<float>(n * ldr, st);
    gather_rows<float, float>(st, m, rank, R.row_pos, (const float*)colp.U(), kmax_c, F.U32.get(), ldr);
    gather_rows<float, float>(st, n, rank, R.col_pos, (const float*)Vnew.get(), ldr, F.V32.get(), ldr);
  }
  F.S.resize(rank);
  F.S_d = DArr<double>(ldr, st);
  if (rank > 0) {
    CK(cudaMemcpyAsync(F.S_d.get(), colp.S(), size_t(rank) * 8, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(F.S.data(), colp.S(), size_t(rank) * 8, cudaMemcpyDeviceToHost, st));
  }
  CK(cudaStreamSynchronize(st));
  info.ms_finalize = tm.stop();
  if (gemm_tc_status(st, true) != 0) fail(FASTPI_ERR_CUDA, "tensor-core GEMM: a bounded wait ran out");
  F.m = m;
  F.n = n;
  F.rank = rank;
  info.m = m;
  info.n = n;
  info.nnz = h->nnz;
  info.m1 = m1;
  info.n1 = n1;
  info.m2 = m2;
  info.n2 = n2;
  info.num_blocks = R.num_blocks;
  info.iterations = R.iterations;
  info.S = S;
  info.s_row = s;
  info.rank = rank;
  info.chunk_row = cr;
  info.chunk_col = cc;
  info.row_chunks = rowp.steps;
  info.col_chunks = colp.steps;
  info.dropped_directions = rowp.dropped + colp.dropped;
  info.jacobi_sweeps_max = std::max({bjs.max_sweeps_used, rowp.sweeps_max, colp.sweeps_max});
  double g = std::min(rowp.min_gap, colp.min_gap);
  info.min_trunc_gap = std::isfinite(g) ? g : -1.0;
}

// ----------------------------------------------------------------- apply
template <typename T>
__global__ void k_scale_rows(int64_t rows, int64_t cols, const double* sig, double tau, T* X, int64_t ldx) {
  int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  int64_t i = e / cols, j = e % cols;
  double s = sig[i];
  X[i * ldx + j] = s > tau ? T(double(X[i * ldx + j]) / s) : T(0);
}

// WtT[l, :] = sum over nonzeros y_il of y_il * U[i, :]   (CSC of Y by label)
template <typename T>
__global__ void k_spmm_labels(const int64_t* __restrict__ cptr, const int32_t* __restrict__ rows,
                              const double* __restrict__ vals, int64_t r, const T* __restrict__ U, int64_t ldu,
                              T* __restrict__ WtT) {
  const int64_t l = blockIdx.x;
  for (int64_t j = threadIdx.x; j < r; j += blockDim.x) {
    T acc = 0;
    for (int64_t e = cptr[l]; e < cptr[l + 1]; ++e) acc = fma(T(vals[e]), U[int64_t(rows[e]) * ldu + j], acc);
    WtT[l * r + j] = acc;
  }
}

template <typename T>
__global__ void k_scale_cols(int64_t rows, int64_t cols, const double* sig, double tau, T* X) {
  int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  int64_t j = e % cols;
  double s = sig[j];
  X[e] = s > tau ? T(double(X[e]) / s) : T(0);
}

// One warp per row i of A: ||(A Z - Y)[i, :]||^2.  Lane l owns the columns
// l, l + 32, ... of a pass of RP * 32 columns, with their partial sums in
// registers, so each nonzero of the row (index and value) is read once per
// pass and the Z row it selects is read coalesced.
constexpr int RES_RP = 8;   // columns per lane per pass
__global__ void k_residual_rows(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                const double* __restrict__ val, int64_t m, int64_t L, const double* __restrict__ Y,
                                int64_t ldy, const double* __restrict__ Z, int64_t ldz, double* out) {
  const int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= m) return;
  const int64_t e0 = rowptr[i], e1 = rowptr[i + 1];
  double acc2 = 0;
  for (int64_t l0 = 0; l0 < L; l0 += 32 * RES_RP) {
    double s[RES_RP];
#pragma unroll
    for (int u = 0; u < RES_RP; ++u) {
      const int64_t l = l0 + lane + 32 * u;
      s[u] = l < L ? -Y[i * ldy + l] : 0.0;
    }
    for (int64_t e = e0; e < e1; ++e) {
      const double v = val[e];
      const double* zr = Z + int64_t(col[e]) * ldz;
#pragma unroll
      for (int u = 0; u < RES_RP; ++u) {
        const int64_t l = l0 + lane + 32 * u;
        if (l < L) s[u] = fma(v, zr[l], s[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < RES_RP; ++u) acc2 = fma(s[u], s[u], acc2);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) acc2 += __shfl_xor_sync(0xffffffffu, acc2, o);
  if (lane == 0) out[i] = acc2;
}

__global__ void k_sum(const double* x, int64_t n, double* out) {
  __shared__ double ws[32];
  double s = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) t += ws[w];
    *out = t;
  }
}

// out (m x L, ld ldo) = A X for A in CSR and X (n x L, ld ldx), FP64.  One
// warp per row; lane l owns the columns l, l + 32, ... of a pass of RES_RP * 32
// columns, so each nonzero of the row is read once per pass.
__global__ void k_spmm_rows(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            const double* __restrict__ val, int64_t m, int64_t L, const double* __restrict__ X,
                            int64_t ldx, double* __restrict__ out, int64_t ldo) {
  const int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= m) return;
  const int64_t e0 = rowptr[i], e1 = rowptr[i + 1];
  for (int64_t l0 = 0; l0 < L; l0 += 32 * RES_RP) {
    double s[RES_RP];
#pragma unroll
    for (int u = 0; u < RES_RP; ++u) s[u] = 0.0;
    for (int64_t e = e0; e < e1; ++e) {
      const double v = val[e];
      const double* xr = X + int64_t(col[e]) * ldx;
#pragma unroll
      for (int u = 0; u < RES_RP; ++u) {
        const int64_t l = l0 + lane + 32 * u;
        if (l < L) s[u] = fma(v, xr[l], s[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < RES_RP; ++u) {
      const int64_t l = l0 + lane + 32 * u;
      if (l < L) out[i * ldo + l] = s[u];
    }
  }
}

// cross[j] = sum_i U[i, j] AV[i, j] (one CTA per column j, fixed order).
__global__ void k_col_dots(int64_t m, int64_t r, const double* __restrict__ U, const double* __restrict__ AV,
                           double* cross) {
  __shared__ double ws[32];
  const int64_t j = blockIdx.x;
  double s = 0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) s = fma(U[i * r + j], AV[i * r + j], s);
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) t += ws[w];
    cross[j] = t;
  }
}

// out[0] = |A|_F^2 - 2 sum_j s_j cross_j + sum_{i,j} s_i s_j Gu_ij Gv_ij, one CTA.
__global__ void k_recon_total(int64_t nnz, const double* __restrict__ val, int64_t r, const double* __restrict__ S,
                              const double* __restrict__ cross, const double* __restrict__ Gu,
                              const double* __restrict__ Gv, double* out) {
  __shared__ double ws[3][32];
  double a2 = 0, cr = 0, q = 0;
  for (int64_t e = threadIdx.x; e < nnz; e += blockDim.x) a2 = fma(val[e], val[e], a2);
  for (int64_t j = threadIdx.x; j < r; j += blockDim.x) cr = fma(S[j], cross[j], cr);
  for (int64_t e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int64_t i = e / r, j = e % r;
    q = fma(S[i] * S[j], Gu[e] * Gv[e], q);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    cr += __shfl_xor_sync(0xffffffffu, cr, o);
    q += __shfl_xor_sync(0xffffffffu, q, o);
  }
  if ((threadIdx.x & 31) == 0) {
    ws[0][threadIdx.x >> 5] = a2;
    ws[1][threadIdx.x >> 5] = cr;
    ws[2][threadIdx.x >> 5] = q;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0, t1 = 0, t2 = 0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) {
      t0 += ws[0][w];
      t1 += ws[1][w];
      t2 += ws[2][w];
    }
    out[0] = t0;
    out[1] = t0 - 2.0 * t1 + t2;
  }
}

template <typename T>
BlockSvdFn<T> own_block_svd(fastpi_ctx* h) {
  return [h](const std::vector<JacobiProblem<T>>& probs, double*& sig, int32_t*& perm) {
    return jacobi_svd_batched<T>(h, probs, sig, perm);
  };
}

double pinv_tau(const Factors& F) {
  if (F.S.empty()) return 0.0;
  double s1 = *std::max_element(F.S.begin(), F.S.end());
  return double(std::max(F.m, F.n)) * 2.220446049250313e-16 * s1;
}

}  // namespace

namespace {

template <typename T>
void factor_into(fastpi_ctx* h, int64_t r, double k, fastpi_precision prec, int64_t chunk_row, int64_t chunk_col,
                 const BlockSvdFn<T>& block_svd) {
  Factors* F = new Factors();
  F->prec = int(prec);
  h->info = fastpi_info{};
  h->info.precision = int(prec);
  h->factored = false;
  h->reordered = false;
  try {
    factor_impl<T>(h, *F, r, k, chunk_row, chunk_col, block_svd);
  } catch (...) {
    delete F;
    throw;
  }
  delete h->fac;
  h->fac = F;
  h->factored = true;
  h->reordered = true;
}

// Counting semaphore (bounds how many instances of a batch are in a
// GPU-heavy stage at once).
class Gate {
 public:
  explicit Gate(int n) : free_(n > 0 ? n : 1) {}
  void acquire() {
    std::unique_lock<std::mutex> lk(mu_);
    cv_.wait(lk, [&] { return free_ > 0; });
    --free_;
  }
  void release() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      ++free_;
    }
    cv_.notify_one();
  }

 private:
  std::mutex mu_;
  std::condition_variable cv_;
  int free_;
};

// Rendezvous of the block SVDs (Eq. 1) of a batch of instances: every
// instance deposits its A11 block problems; the last one to arrive runs ONE
// persistent batched Jacobi launch over the blocks of all instances (the
// kernel picks its register tile from the largest block and walks the
// problems of every instance in one cooperative grid), then every instance
// reads its singular values / orders from its slice of the combined output.
template <typename T>
struct BlockRendezvous {
  std::mutex mu;
  std::condition_variable cv;
  int expected = 0, arrived = 0;
  bool done = false;
  struct Entry {
    const std::vector<JacobiProblem<T>>* probs = nullptr;
    double** sig = nullptr;
    int32_t** perm = nullptr;
  };
  std::vector<Entry> entries;
  JacobiStats stats;
  bool failed = false;
  Error error{FASTPI_OK, ""};
  DArr<double> sig_all;
  DArr<int32_t> perm_all;

  explicit BlockRendezvous(int count) : expected(count), entries(count) {}

  // Instance i arrives (probs == nullptr: it failed before its block SVD).
  JacobiStats arrive(int i, fastpi_ctx* h, const std::vector<JacobiProblem<T>>* probs, double** sig,
                     int32_t** perm) {
    // its blocks must be ready before another stream reads them; a failure
    // here still registers the instance (without problems), so that the
    // others are not left waiting
    bool own_fail = false;
    Error own_err{FASTPI_OK, ""};
    if (probs) {
      const cudaError_t e = cudaStreamSynchronize(h->stream);
      if (e != cudaSuccess) {
        own_fail = true;
        own_err = Error{FASTPI_ERR_CUDA, std::string("cudaStreamSynchronize: ") + cudaGetErrorString(e)};
        probs = nullptr;
      }
    }
    std::unique_lock<std::mutex> lk(mu);
    entries[i] = Entry{probs, sig, perm};
    if (++arrived == expected) {
      run(h);
      done = true;
      lk.unlock();
      cv.notify_all();
      lk.lock();
    } else {
      cv.wait(lk, [&] { return done; });
    }
    if (own_fail) throw own_err;
    if (failed && probs) throw error;
    return stats;
  }

  // Registers instance i as taking no part (its thread could not be started)
  // without waiting for the others.
  void absent(int i, fastpi_ctx* h) {
    std::unique_lock<std::mutex> lk(mu);
    entries[i] = Entry{};
    if (++arrived == expected) {
      run(h);
      done = true;
      lk.unlock();
      cv.notify_all();
    }
  }

  // Never throws: a failure is recorded in `failed` / `error` for every
  // instance that took part.
  void run(fastpi_ctx* h) {
    std::vector<JacobiProblem<T>> all;
    std::vector<int64_t> off(entries.size(), 0);
    int64_t tot = 0;
    try {
      for (size_t i = 0; i < entries.size(); ++i) {
        off[i] = tot;
        if (!entries[i].probs) continue;
        for (const auto& pr : *entries[i].probs) {
          all.push_back(pr);
          tot += pr.q;
        }
      }
    } catch (const std::exception& e) {
      failed = true;
      error = Error{FASTPI_ERR_OOM, e.what()};
      return;
    }
    try {
      sig_all = DArr<double>(std::max<int64_t>(tot, 1), h->stream);
      perm_all = DArr<int32_t>(std::max<int64_t>(tot, 1), h->stream);
      stats = jacobi_svd_batched<T>(h, all, sig_all.get(), perm_all.get());
      CK(cudaStreamSynchronize(h->stream));
    } catch (const Error& e) {
      failed = true;
      error = e;
      return;
    } catch (const std::exception& e) {   // never leave the waiting instances without `done`
      failed = true;
      error = Error{FASTPI_ERR_CUDA, e.what()};
      return;
    }
    for (size_t i = 0; i < entries.size(); ++i) {
      if (!entries[i].probs) continue;
      *entries[i].sig = sig_all.get() + off[i];
      *entries[i].perm = perm_all.get() + off[i];
    }
  }
};

template <typename T>
void factor_batched_impl(fastpi_ctx* const* hs, int count, const int64_t* r, double k, fastpi_precision prec,
                         int64_t chunk_row, int64_t chunk_col, int concurrency, fastpi_status* status,
                         std::string* msgs) {
  BlockRendezvous<T> rv(count);
  Gate pre(concurrency), post(concurrency);
  std::vector<std::thread> th;
  th.reserve(count);
  auto body = [&](int i) {
      fastpi_ctx* h = hs[i];
      bool arrived = false;
      bool in_pre = true, in_post = false;
      pre.acquire();
      try {
        CK(cudaSetDevice(h->device));
        BlockSvdFn<T> bs = [&](const std::vector<JacobiProblem<T>>& probs, double*& sig, int32_t*& perm) {
          pre.release();
          in_pre = false;
          arrived = true;
          JacobiStats js = rv.arrive(i, h, &probs, &sig, &perm);
          post.acquire();
          in_post = true;
          return js;
        };
        factor_into<T>(h, r[i], k, prec, chunk_row, chunk_col, bs);
        status[i] = FASTPI_OK;
      } catch (const Error& e) {
        status[i] = e.status;
        msgs[i] = e.msg;
      } catch (const std::exception& e) {
        status[i] = FASTPI_ERR_CUDA;
        msgs[i] = e.what();
      }
      if (in_pre) pre.release();
      if (in_post) post.release();
      if (!arrived) {
        try {
          rv.arrive(i, h, nullptr, nullptr, nullptr);
        } catch (...) {
        }
      }
  };
  for (int i = 0; i < count; ++i) {
    try {
      th.emplace_back(body, i);
    } catch (const std::exception& e) {
      status[i] = FASTPI_ERR_CUDA;
      msgs[i] = std::string("could not start a host thread: ") + e.what();
      rv.absent(i, hs[i]);
    }
  }
  for (auto& t : th) t.join();
}

}  // namespace

void factor(fastpi_ctx* h, int64_t r, double k, fastpi_precision prec, int64_t chunk_row, int64_t chunk_col) {
  if (prec == FASTPI_FP64)
    factor_into<double>(h, r, k, prec, chunk_row, chunk_col, own_block_svd<double>(h));
  else
    factor_into<float>(h, r, k, prec, chunk_row, chunk_col, own_block_svd<float>(h));
}

void factor_batched(fastpi_ctx* const* hs, int count, const int64_t* r, double k, fastpi_precision prec,
                    int64_t chunk_row, int64_t chunk_col, int concurrency, fastpi_status* status,
                    std::string* msgs) {
  if (prec == FASTPI_FP64)
    factor_batched_impl<double>(hs, count, r, k, prec, chunk_row, chunk_col, concurrency, status, msgs);
  else
    factor_batched_impl<float>(hs, count, r, k, prec, chunk_row, chunk_col, concurrency, status, msgs);
}

void load_factors(fastpi_ctx* h, int64_t r, const double* S, const double* U, int64_t ldu, const double* V,
                  int64_t ldv, fastpi_precision prec, bool on_device) {
  cudaStream_t st = h->stream;
  Factors* F = new Factors();
  try {
    F->prec = int(prec);
    F->m = h->m;
    F->n = h->n;
    F->rank = r;
    F->S.assign(S, S + r);
    const int64_t ldr = std::max<int64_t>(r, 1);
    F->S_d = DArr<double>(ldr, st);
    if (r > 0) CK(cudaMemcpyAsync(F->S_d.get(), S, size_t(r) * 8, cudaMemcpyHostToDevice, st));
    // stage host inputs on the device, then copy / convert into the packed layout
    DArr<double> Ud, Vd;
    const double* Us = U;
    const double* Vs = V;
    int64_t lu = ldu, lv = ldv;
    if (!on_device && r > 0) {
      Ud = DArr<double>(h->m * r, st);
      Vd = DArr<double>(h->n * r, st);
      CK(cudaMemcpy2DAsync(Ud.get(), size_t(r) * 8, U, size_t(ldu) * 8, size_t(r) * 8, size_t(h->m),
                           cudaMemcpyHostToDevice, st));
      CK(cudaMemcpy2DAsync(Vd.get(), size_t(r) * 8, V, size_t(ldv) * 8, size_t(r) * 8, size_t(h->n),
                           cudaMemcpyHostToDevice, st));
      Us = Ud.get();
      Vs = Vd.get();
      lu = lv = r;
    }
    if (prec == FASTPI_FP64) {
      F->U64 = DArr<double>(h->m * ldr, st);
      F->V64 = DArr<double>(h->n * ldr, st);
      copy2d<double, double>(st, h->m, r, Us, lu, F->U64.get(), ldr);
      copy2d<double, double>(st, h->n, r, Vs, lv, F->V64.get(), ldr);
    } else {
      F->U32 = DArr<float>(h->m * ldr, st);
      F->V32 = DArr<float>(h->n * ldr, st);
      copy2d<float, double>(st, h->m, r, Us, lu, F->U32.get(), ldr);
      copy2d<float, double>(st, h->n, r, Vs, lv, F->V32.get(), ldr);
    }
    CK(cudaStreamSynchronize(st));
  } catch (...) {
    delete F;
    throw;
  }
  delete h->fac;
  h->fac = F;
  h->factored = true;
  h->reordered = false;
  h->info = fastpi_info{};
  h->info.m = h->m;
  h->info.n = h->n;
  h->info.rank = r;
  h->info.precision = int(prec);
}

void truncate_factors(fastpi_ctx* h, int64_t r) {
  Factors& F = *h->fac;
  if (r >= F.rank) return;
  cudaStream_t st = h->stream;
  const int64_t ldo = std::max<int64_t>(F.rank, 1), ldr = std::max<int64_t>(r, 1);
  if (F.prec == FASTPI_FP64) {
    DArr<double> U(F.m * ldr, st), V(F.n * ldr, st);
    copy2d<double, double>(st, F.m, r, F.U64.get(), ldo, U.get(), ldr);
    copy2d<double, double>(st, F.n, r, F.V64.get(), ldo, V.get(), ldr);
    F.U64 = std::move(U);
    F.V64 = std::move(V);
  } else {
    DArr<float> U(F.m * ldr, st), V(F.n * ldr, st);
    copy2d<float, float>(st, F.m, r, F.U32.get(), ldo, U.get(), ldr);
    copy2d<float, float>(st, F.n, r, F.V32.get(), ldo, V.get(), ldr);
    F.U32 = std::move(U);
    F.V32 = std::move(V);
  }
  F.S.resize(r);
  F.rank = r;
  h->info.rank = r;
  CK(cudaStreamSynchronize(st));
}

// Algorithm 2 and Eq. 1 only: the kept singular values of every A11 block.
template <typename T>
void block_stage_only(fastpi_ctx* h, int64_t r, double kratio, std::vector<double>& sig_out) {
  Factors* F = new Factors();
  h->info = fastpi_info{};
  h->factored = false;
  h->reordered = false;
  int64_t S = 0;
  try {
    Timer tm(h->stream);
    tm.start();
    run_reorder(h, kratio, F->R);
    A11Blocks blk;
    extract_blocks(h, F->R, r, blk);
    h->info.ms_reorder = tm.stop();
    tm.start();
    BlockStage<T> bs;
    run_block_stage<T>(h, F->R, blk, own_block_svd<T>(h), bs);
    h->info.ms_block_svd = tm.stop();
    S = blk.S;
    sig_out.assign(bs.sig_all.begin(), bs.sig_all.begin() + S);
    h->info.jacobi_sweeps_max = bs.js.max_sweeps_used;
  } catch (...) {
    delete F;
    throw;
  }
  const Reordering& R = F->R;
  h->info.m = h->m;
  h->info.n = h->n;
  h->info.nnz = h->nnz;
  h->info.m1 = R.m1;
  h->info.n1 = R.n1;
  h->info.m2 = h->m - R.m1;
  h->info.n2 = h->n - R.n1;
  h->info.num_blocks = R.num_blocks;
  h->info.iterations = R.iterations;
  h->info.S = S;
  delete h->fac;
  h->fac = F;
  h->reordered = true;
}

void block_svd_only(fastpi_ctx* h, int64_t r, double k, fastpi_precision prec, std::vector<double>& sig) {
  if (prec == FASTPI_FP64)
    block_stage_only<double>(h, r, k, sig);
  else
    block_stage_only<float>(h, r, k, sig);
}

void reorder_only(fastpi_ctx* h, double k) {
  Factors* F = new Factors();
  h->info = fastpi_info{};
  try {
    Timer tm(h->stream);
    tm.start();
    run_reorder(h, k, F->R);
    h->info.ms_reorder = tm.stop();
  } catch (...) {
    delete F;
    throw;
  }
  const Reordering& R = F->R;
  h->info.m = h->m;
  h->info.n = h->n;
  h->info.nnz = h->nnz;
  h->info.m1 = R.m1;
  h->info.n1 = R.n1;
  h->info.m2 = h->m - R.m1;
  h->info.n2 = h->n - R.n1;
  h->info.num_blocks = R.num_blocks;
  h->info.iterations = R.iterations;
  delete h->fac;
  h->fac = F;
  h->factored = false;
  h->reordered = true;
}

void apply_dense(fastpi_ctx* h, const double* Y, int64_t L, int64_t ldy, double* Z, int64_t ldz) {
  Factors& F = *h->fac;
  cudaStream_t st = h->stream;
  const int64_t m = F.m, n = F.n, r = F.rank;
  const double tau = pinv_tau(F);
  if (L <= 0) return;
  if (F.prec == FASTPI_FP64) {
    DArr<double> Wt(std::max<int64_t>(r, 1) * L, st);
    gemm<double>(st, true, false, r, L, m, 1.0, F.U64.get(), std::max<int64_t>(r, 1), Y, ldy, 0.0, Wt.get(), L);
    k_scale_rows<double><<<g1(r * L), 256, 0, st>>>(r, L, F.S_d.get(), tau, Wt.get(), L);
    CK_LAUNCH();
    gemm<double>(st, false, false, n, L, r, 1.0, F.V64.get(), std::max<int64_t>(r, 1), Wt.get(), L, 0.0, Z, ldz);
  } else {
    DArr<float> Yf(m * L, st), Wt(std::max<int64_t>(r, 1) * L, st), Zf(n * L, st);
    copy2d<float, double>(st, m, L, Y, ldy, Yf.get(), L);
    gemm_f32(st, true, false, r, L, m, 1.f, F.U32.get(), std::max<int64_t>(r, 1), Yf.get(), L, 0.f, Wt.get(), L);
    k_scale_rows<float><<<g1(r * L), 256, 0, st>>>(r, L, F.S_d.get(), tau, Wt.get(), L);
    CK_LAUNCH();
    gemm_f32(st, false, false, n, L, r, 1.f, F.V32.get(), std::max<int64_t>(r, 1), Wt.get(), L, 0.f, Zf.get(), L);
    copy2d<double, float>(st, n, L, Zf.get(), L, Z, ldz);
  }
}

void apply_csr(fastpi_ctx* h, int64_t L, int64_t nnz_y, const int64_t* yrowptr, const int32_t* ycol,
               const double* yval, double* Z, int64_t ldz) {
  Factors& F = *h->fac;
  cudaStream_t st = h->stream;
  const int64_t m = F.m, n = F.n, r = F.rank;
  const double tau = pinv_tau(F);
  if (L <= 0) return;
  // CSC of Y by label: stable radix sort of the nonzeros by label
  DArr<int64_t> cptr(L + 1, st);
  DArr<int32_t> crow(std::max<int64_t>(nnz_y, 1), st);
  DArr<double> cval(std::max<int64_t>(nnz_y, 1), st);
  {
    fastpi_ctx tmp_ctx;   // scratch handle to reuse the CSC builder on Y
    tmp_ctx.stream = st;
    tmp_ctx.m = m;
    tmp_ctx.n = L;
    tmp_ctx.nnz = nnz_y;
    tmp_ctx.rowptr.n = m + 1;
    // borrow the caller's arrays without ownership
    tmp_ctx.rowptr.b.p = const_cast<int64_t*>(yrowptr);
    tmp_ctx.col.b.p = const_cast<int32_t*>(ycol);
    tmp_ctx.val.b.p = const_cast<double*>(yval);
    tmp_ctx.dstatus = DArr<unsigned>(1, st);
    try {
      // the CSC build indexes by label and row: check Y first, as A is
      // checked when the handle is made
      validate_csr(&tmp_ctx);
      build_csc(&tmp_ctx);
    } catch (...) {
      tmp_ctx.rowptr.b.p = nullptr;
      tmp_ctx.col.b.p = nullptr;
      tmp_ctx.val.b.p = nullptr;
      throw;
    }
    tmp_ctx.rowptr.b.p = nullptr;
    tmp_ctx.col.b.p = nullptr;
    tmp_ctx.val.b.p = nullptr;
    cptr = static_cast<DArr<int64_t>&&>(tmp_ctx.colptr);
    crow = static_cast<DArr<int32_t>&&>(tmp_ctx.csc_row);
    cval = static_cast<DArr<double>&&>(tmp_ctx.csc_val);
  }
  const int64_t ldr = std::max<int64_t>(r, 1);
  if (F.prec == FASTPI_FP64) {
    DArr<double> WtT(L * ldr, st);
    k_spmm_labels<double><<<unsigned(L), 256, 0, st>>>(cptr.get(), crow.get(), cval.get(), r, F.U64.get(), ldr,
                                                       WtT.get());
    CK_LAUNCH();
    k_scale_cols<double><<<g1(L * r), 256, 0, st>>>(L, r, F.S_d.get(), tau, WtT.get());
    CK_LAUNCH();
    gemm<double>(st, false, true, n, L, r, 1.0, F.V64.get(), ldr, WtT.get(), ldr, 0.0, Z, ldz);
  } else {
    DArr<float> WtT(L * ldr, st), Zf(n * L, st);
    k_spmm_labels<float><<<unsigned(L), 256, 0, st>>>(cptr.get(), crow.get(), cval.get(), r, F.U32.get(), ldr,
                                                      WtT.get());
    CK_LAUNCH();
    k_scale_cols<float><<<g1(L * r), 256, 0, st>>>(L, r, F.S_d.get(), tau, WtT.get());
    CK_LAUNCH();
    gemm_f32(st, false, true, n, L, r, 1.f, F.V32.get(), ldr, WtT.get(), ldr, 0.f, Zf.get(), L);
    copy2d<double, float>(st, n, L, Zf.get(), L, Z, ldz);
  }
}

void spmm(fastpi_ctx* h, const double* X, int64_t L, int64_t ldx, double* out, int64_t ldo) {
  cudaStream_t st = h->stream;
  if (h->m <= 0 || L <= 0) return;
  k_spmm_rows<<<g1(h->m * 32), 256, 0, st>>>(h->rowptr, h->col, h->val, h->m, L, X, ldx, out, ldo);
  CK_LAUNCH();
}

double recon_error(fastpi_ctx* h) {
  Factors& F = *h->fac;
  cudaStream_t st = h->stream;
  const int64_t m = F.m, n = F.n, r = F.rank;
  const int64_t ldr = std::max<int64_t>(r, 1);
  DArr<double> Ud, Vd;
  const double* U = F.U64.get();
  const double* V = F.V64.get();
  if (F.prec != FASTPI_FP64) {
    Ud = DArr<double>(m * ldr, st);
    Vd = DArr<double>(n * ldr, st);
    copy2d<double, float>(st, m, r, F.U32.get(), ldr, Ud.get(), ldr);
    copy2d<double, float>(st, n, r, F.V32.get(), ldr, Vd.get(), ldr);
    U = Ud.get();
    V = Vd.get();
  }
  DArr<double> AV(m * ldr, st), cross(ldr, st), Gu(ldr * ldr, st), Gv(ldr * ldr, st), tot(2, st);
  if (r > 0) {
    spmm(h, V, r, ldr, AV.get(), ldr);
    k_col_dots<<<unsigned(r), 256, 0, st>>>(m, r, U, AV.get(), cross.get());
    CK_LAUNCH();
    gemm<double>(st, true, false, r, r, m, 1.0, U, ldr, U, ldr, 0.0, Gu.get(), ldr);
    gemm<double>(st, true, false, r, r, n, 1.0, V, ldr, V, ldr, 0.0, Gv.get(), ldr);
  }
  k_recon_total<<<1, 1024, 0, st>>>(h->nnz, h->val, r, F.S_d.get(), cross.get(), Gu.get(), Gv.get(), tot.get());
  CK_LAUNCH();
  double t[2] = {0, 0};
  d2h_sync(t, tot.get(), sizeof t, st);
  if (!(t[0] > 0)) return 0.0;
  return std::sqrt(std::max(t[1], 0.0) / t[0]);
}

double residual(fastpi_ctx* h, const double* Y, int64_t L, int64_t ldy, const double* Z, int64_t ldz) {
  cudaStream_t st = h->stream;
  const int64_t m = h->m;
  DArr<double> part(std::max<int64_t>(m, 1), st), tot(1, st);
  if (m > 0 && L > 0) {
    k_residual_rows<<<g1(m * 32), 256, 0, st>>>(h->rowptr, h->col, h->val, m, L, Y, ldy, Z, ldz, part.get());
    CK_LAUNCH();
  } else {
    CK(cudaMemsetAsync(part.get(), 0, 8, st));
  }
  k_sum<<<1, 1024, 0, st>>>(part.get(), m > 0 && L > 0 ? m : 1, tot.get());
  CK_LAUNCH();
  double out = 0;
  d2h_sync(&out, tot.get(), 8, st);
  return std::sqrt(out);
}

}  // namespace fastpi
