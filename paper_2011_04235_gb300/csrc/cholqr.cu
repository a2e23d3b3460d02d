// Blocked kernels of the CholeskyQR2 orthogonalisation of an appended residual
// (the incremental update of Eqs. 2 / 3): the inverse of a lower-triangular
// factor restricted to its kept indices, and the Cholesky factorization of the
// second pass's Gram matrix with dependent directions dropped.  Both replace
// column-at-a-time kernels whose c dependent steps each cost a CTA barrier or a
// warp reduction: here the dependent chain is c / 32 block steps, each a
// 32-step chain inside one warp followed by work spread over the CTA.
#include <algorithm>
#include <cstdlib>
#include <cstdio>

#include "cholqr.cuh"

namespace fastpi {
namespace {

constexpr int NB = 32;   // block edge

// By one warp (lane j = column j): Linv = inverse of the lower-triangular
// NB x NB block Lb (shared memory, row stride NB + 1) restricted to the
// indices with keep[i] != 0 (zero rows and columns elsewhere), by forward
// substitution with the column held in registers (unrolled: the loads of Lb
// are broadcasts independent of the running sums, so only the multiply-add
// chain of each row is serial); bs = rows / columns in use.
template <typename T>
__device__ __forceinline__ void warp_trinv_block(const T* Lb, const int* keep, int bs, int lane, T* Linv) {
  const int j = lane;
  const bool colk = j < bs && keep[j];
  T x[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    T s = (i == j) ? T(1) : T(0);
    // x[l] = 0 for l < j, so the sum is the one over l = j .. i-1
#pragma unroll
    for (int l = 0; l < i; ++l) s = fma(-Lb[i * (NB + 1) + l], x[l], s);
    x[i] = (colk && i < bs && keep[i] && i >= j) ? s / Lb[i * (NB + 1) + i] : T(0);
  }
#pragma unroll
  for (int i = 0; i < NB; ++i) Linv[i * (NB + 1) + j] = x[i];
  __syncwarp();
}

// By one warp: Cholesky of the symmetric NB x NB block Ab (shared memory, row
// stride NB + 1, lower triangle used) in place, columns j < bw, with the drop
// rule (a pivot d_j <= tol gives a zero column); lane l holds row l in
// registers and takes the entries of other rows by warp shuffles.  Returns
// the bit mask of kept columns.
__device__ __forceinline__ unsigned warp_chol_block(float* Ab, int bw, float tol, int lane) {
  float a[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i) a[i] = (i <= lane && lane < bw && i < bw) ? Ab[lane * (NB + 1) + i] : 0.f;
  unsigned keepmask = 0;
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    const float d = __shfl_sync(0xffffffffu, a[j], j);
    const bool keep = j < bw && d > tol;
    const float ljj = keep ? sqrtf(d) : 0.f;
    const float inv = keep ? 1.f / ljj : 0.f;
    if (lane == j)
      a[j] = ljj;
    else if (lane > j)
      a[j] *= inv;
    if (keep) {
      keepmask |= 1u << j;
#pragma unroll
      for (int i = j + 1; i < NB; ++i) {
        const float lij = __shfl_sync(0xffffffffu, a[j], i);   // L[i, j]
        if (lane >= i) a[i] = fmaf(-a[j], lij, a[i]);
      }
    }
  }
  __syncwarp();
#pragma unroll
  for (int i = 0; i < NB; ++i) Ab[lane * (NB + 1) + i] = (i <= lane && lane < bw) ? a[i] : 0.f;
  __syncwarp();
  return keepmask;
}

// Dinv (nb blocks of NB x NB, row-major) <- inverse of each diagonal block of
// L (c x c, row-major, ld c) restricted to the kept indices; one warp per block.
constexpr int TD_WARPS = 2;   // warps (diagonal blocks) per CTA of k_trinv_diag
template <typename T>
__global__ void k_trinv_diag(const T* __restrict__ L, int c, const int32_t* __restrict__ kept, T* __restrict__ Dinv) {
  __shared__ T Lb[TD_WARPS][NB * (NB + 1)];
  __shared__ T Li[TD_WARPS][NB * (NB + 1)];
  __shared__ int kp[TD_WARPS][NB];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = int(blockIdx.x) * TD_WARPS + w;
  const int nb = (c + NB - 1) / NB;
  if (b >= nb) return;
  const int r0 = b * NB, bs = min(NB, c - r0);
  for (int i = 0; i < NB; ++i) Lb[w][i * (NB + 1) + lane] = (i < bs && lane < bs) ? L[int64_t(r0 + i) * c + r0 + lane] : T(0);
  kp[w][lane] = lane < bs ? kept[r0 + lane] : 0;
  __syncwarp();
  warp_trinv_block<T>(Lb[w], kp[w], bs, lane, Li[w]);
  T* D = Dinv + int64_t(b) * NB * NB;
  for (int i = 0; i < NB; ++i) D[i * NB + lane] = Li[w][i * (NB + 1) + lane];
}

// X (c x c, row-major) <- L^-1 restricted to the kept indices, one CTA per
// block column jb: X_jj = Dinv_j and, block row after block row,
// X_ij = -Dinv_i (sum_{k = j .. i-1} L_ik X_kj); the block column of X stays in
// shared memory, and L_ik is staged through shared memory TI_KC columns at a
// time (coalesced copies instead of a chain of dependent L2 loads per dot
// product).  Entries above the diagonal are zero.  256 threads: thread
// (warp w, lane s) owns the entries (w + 8 q, s), q = 0..3, of a block.
constexpr int TI_KC = 64;
constexpr int TI_THREADS = 256;
template <typename T>
__global__ void __launch_bounds__(TI_THREADS) k_trinv_cols_blocked(const T* __restrict__ L, int c,
                                                                   const T* __restrict__ Dinv, T* __restrict__ X) {
  extern __shared__ unsigned char xs_raw[];
  const int nb = (c + NB - 1) / NB, jb = blockIdx.x, tid = threadIdx.x;
  const int w = tid >> 5, lane = tid & 31;
  T* Xc = reinterpret_cast<T*>(xs_raw);          // [nb * NB][NB]: block column jb of X
  T* Tb = Xc + int64_t(nb) * NB * NB;            // [NB][NB] scratch
  T* Ls = Tb + NB * NB;                          // [NB][TI_KC]: staged columns of L's block row
  T* Ds = Ls + NB * TI_KC;                       // [NB][NB]: Dinv of the block row
  const int c0 = jb * NB;
  for (int e = tid; e < nb * NB * NB; e += TI_THREADS) Xc[e] = T(0);
  __syncthreads();
  for (int e = tid; e < NB * NB; e += TI_THREADS) Xc[int64_t(jb) * NB * NB + e] = Dinv[int64_t(jb) * NB * NB + e];
  __syncthreads();
  for (int ib = jb + 1; ib < nb; ++ib) {
    const int r0 = ib * NB, bh = min(NB, c - r0);
    for (int e = tid; e < NB * NB; e += TI_THREADS) Ds[e] = Dinv[int64_t(ib) * NB * NB + e];
    // T = sum over the block rows jb .. ib-1 of L[ib, k] X[k, jb]
    T acc[4] = {T(0), T(0), T(0), T(0)};
    for (int k0 = c0; k0 < r0; k0 += TI_KC) {
      const int kc = min(TI_KC, r0 - k0);
      for (int e = tid; e < NB * TI_KC; e += TI_THREADS) {
        const int r = e / TI_KC, k = e % TI_KC;
        Ls[e] = (r < bh && k < kc) ? L[int64_t(r0 + r) * c + k0 + k] : T(0);
      }
      __syncthreads();
      for (int k = 0; k < kc; ++k) {
        const T x = Xc[int64_t(k0 + k) * NB + lane];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = fma(Ls[(w + 8 * q) * TI_KC + k], x, acc[q]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) Tb[(w + 8 * q) * NB + lane] = acc[q];
    __syncthreads();
    // X[ib, jb] = -Dinv_ib T
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = w + 8 * q;
      T o = T(0);
      for (int k = 0; k < NB; ++k) o = fma(Ds[r * NB + k], Tb[k * NB + lane], o);
      Xc[int64_t(r0 + r) * NB + lane] = -o;
    }
    __syncthreads();
  }
  const int bw = min(NB, c - c0);
  for (int e = tid; e < c * NB; e += TI_THREADS) {
    const int r = e / NB, s = e % NB;
    if (s < bw) X[int64_t(r) * c + c0 + s] = Xc[e];
  }
}

// Cholesky of the c x c Gram G (row-major, lower triangle used, FP32) in one
// CTA, blocked by 32 columns, with the drop rule of the column kernel: a pivot
// d_j <= tol marks column j dependent (zero column of L, kept[j] = 0).  The
// lower triangle is held packed in shared memory (row i at i (i + 1) / 2).
// Per block column: one warp factors the diagonal block and inverts the
// factor, the panel below is G_21 Linv_kk^T (independent dot products), and
// the trailing lower triangle takes the panel's rank-32 update in 4 x 4 tiles.
// On exit G holds L (upper part zero), kept[j] in {0, 1}, *rank = number kept.
#ifdef FASTPI_PHASE_CLOCKS
// clock64 per block step of k_chol_drop_blocked, thread 0: 0 diagonal block
// (factor and inverse by warp 0), 1 panel, 2 trailing update, 3 block steps
__device__ long long g_cd_clk[4];
#define CD_MARK(k)                        \
  do {                                    \
    if (threadIdx.x == 0) {               \
      const long long t_ = clock64();     \
      g_cd_clk[k] += t_ - t_mark;         \
      t_mark = t_;                        \
    }                                     \
  } while (0)
#else
#define CD_MARK(k) \
  do {             \
  } while (0)
#endif

__global__ void __launch_bounds__(1024) k_chol_drop_blocked(float* G, int c, float tol, int32_t* kept,
                                                            int32_t* rank) {
  extern __shared__ float Pk[];                  // packed lower triangle of G
  __shared__ float Ab[NB * (NB + 1)];            // diagonal block, then its factor
  __shared__ float Ai[NB * (NB + 1)];            // inverse of the factor
  __shared__ float Xp[NB][NB + 1];               // scratch for one row block of the panel
  __shared__ int s_keep[NB];
  __shared__ int s_nk;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nth = blockDim.x;
  auto pk = [](int i, int l) { return (int64_t(i) * (i + 1)) / 2 + l; };
  for (int i = warp; i < c; i += nth / 32)
    for (int l = lane; l <= i; l += 32) Pk[pk(i, l)] = G[int64_t(i) * c + l];
  if (tid == 0) s_nk = 0;
  __syncthreads();
  const int nb = (c + NB - 1) / NB;
#ifdef FASTPI_PHASE_CLOCKS
  long long t_mark = clock64();
#endif
  for (int kb = 0; kb < nb; ++kb) {
    const int k0 = kb * NB, bw = min(NB, c - k0);
    // 1. diagonal block: Cholesky with drops, then the inverse (warp 0)
    if (warp == 0) {
      for (int i = 0; i < NB; ++i) Ab[i * (NB + 1) + lane] = (i < bw && lane <= i) ? Pk[pk(k0 + i, k0 + lane)] : 0.f;
      __syncwarp();
      const unsigned km = warp_chol_block(Ab, bw, tol, lane);
      s_keep[lane] = int((km >> lane) & 1u);
      if (lane == 0) s_nk += __popc(km);
      __syncwarp();
      warp_trinv_block<float>(Ab, s_keep, bw, lane, Ai);
      for (int i = 0; i < bw; ++i)
        if (lane <= i) Pk[pk(k0 + i, k0 + lane)] = Ab[i * (NB + 1) + lane];
      if (lane < bw) kept[k0 + lane] = s_keep[lane];
    }
    __syncthreads();
    CD_MARK(0);
    // 2. panel below, 32 rows at a time: L_21 = G_21 Linv^T
    for (int r0 = k0 + bw; r0 < c; r0 += NB) {
      const int rh = min(NB, c - r0);
      for (int e = tid; e < NB * NB; e += nth) {
        const int r = e / NB, j = e % NB;
        float s = 0.f;
        if (r < rh && j < bw) {
          const float* g = Pk + pk(r0 + r, k0);
          for (int l = 0; l <= j; ++l) s = fmaf(g[l], Ai[j * (NB + 1) + l], s);
        }
        Xp[r][j] = s;
      }
      __syncthreads();
      for (int e = tid; e < NB * NB; e += nth) {
        const int r = e / NB, j = e % NB;
        if (r < rh && j < bw) Pk[pk(r0 + r, k0 + j)] = Xp[r][j];
      }
      __syncthreads();
    }
    CD_MARK(1);
    // 3. trailing lower triangle in 4 x 4 tiles: G[i, l] -= L[i, k] . L[l, k]
    const int t0 = k0 + bw, nt = c - t0;
    const int nt4 = (nt + 3) / 4;
    const int64_t tiles = int64_t(nt4) * (nt4 + 1) / 2;
    for (int64_t e = tid; e < tiles; e += nth) {
      int ti = int((sqrtf(8.f * float(e) + 1.f) - 1.f) * 0.5f);
      while (int64_t(ti) * (ti + 1) / 2 > e) --ti;
      while (int64_t(ti + 1) * (ti + 2) / 2 <= e) ++ti;
      const int tl = int(e - int64_t(ti) * (ti + 1) / 2);
      const int i0 = t0 + 4 * ti, l0 = t0 + 4 * tl;
      float acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
      for (int j = 0; j < bw; ++j) {
        float u[4], v[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          u[a] = (i0 + a < c) ? Pk[pk(i0 + a, k0 + j)] : 0.f;
          v[a] = (l0 + a < c) ? Pk[pk(l0 + a, k0 + j)] : 0.f;
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(u[a], v[b], acc[a][b]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int i = i0 + a, l = l0 + b;
          if (i < c && l <= i) Pk[pk(i, l)] -= acc[a][b];
        }
    }
    __syncthreads();
    CD_MARK(2);
#ifdef FASTPI_PHASE_CLOCKS
    if (threadIdx.x == 0) g_cd_clk[3] += 1;
#endif
  }
  for (int i = warp; i < c; i += nth / 32)
    for (int l = lane; l < c; l += 32) G[int64_t(i) * c + l] = l <= i ? Pk[pk(i, l)] : 0.f;
  if (tid == 0) *rank = s_nk;
}


}  // namespace

template <typename T>
void trinv_blocked(cudaStream_t st, const T* L, int c, const int32_t* kept, T* X) {
  if (c <= 0) return;
  const int nb = (c + NB - 1) / NB;
  DArr<T> Dinv(int64_t(nb) * NB * NB, st);
  k_trinv_diag<T><<<unsigned((nb + TD_WARPS - 1) / TD_WARPS), 32 * TD_WARPS, 0, st>>>(L, c, kept, Dinv.get());
  CK_LAUNCH();
  const size_t smem = trinv_blocked_smem(c, sizeof(T));
  if (smem > 48 * 1024) allow_max_dynamic_smem((const void*)k_trinv_cols_blocked<T>);
  k_trinv_cols_blocked<T><<<unsigned(nb), TI_THREADS, smem, st>>>(L, c, Dinv.get(), X);
  CK_LAUNCH();
}

size_t trinv_blocked_smem(int c, size_t elem) {
  const int nb = (c + NB - 1) / NB;
  return (size_t(nb) * NB * NB + 2 * NB * NB + NB * TI_KC) * elem;
}

size_t chol_drop_blocked_smem(int c) { return size_t(int64_t(c) * (c + 1) / 2) * sizeof(float); }

void chol_drop_blocked(cudaStream_t st, float* G, int c, float tol, int32_t* kept, int32_t* rank) {
  if (c <= 0) return;
  const size_t smem = chol_drop_blocked_smem(c);
  if (smem > 48 * 1024) allow_max_dynamic_smem((const void*)k_chol_drop_blocked);
  k_chol_drop_blocked<<<1, 1024, smem, st>>>(G, c, tol, kept, rank);
  CK_LAUNCH();
}

void chol_drop_phase_report(const char* tag) {
#ifdef FASTPI_PHASE_CLOCKS
  long long clk[4] = {0};
  CK(cudaMemcpyFromSymbol(clk, g_cd_clk, sizeof clk));
  const long long b = clk[3] > 0 ? clk[3] : 1;
  fprintf(stderr, "chol_drop %s: block steps %lld, per step clk: diagonal %lld panel %lld trailing %lld\n", tag,
          clk[3], clk[0] / b, clk[1] / b, clk[2] / b);
  const long long z[4] = {0};
  CK(cudaMemcpyToSymbol(g_cd_clk, z, sizeof z));
#else
  (void)tag;
#endif
}

template void trinv_blocked<float>(cudaStream_t, const float*, int, const int32_t*, float*);
template void trinv_blocked<double>(cudaStream_t, const double*, int, const int32_t*, double*);

}  // namespace fastpi
