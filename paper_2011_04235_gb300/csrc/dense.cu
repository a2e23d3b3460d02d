// SIMT GEMM (FP64 / FP32) and small dense helpers.
//
// The FP64 path of GB300 has a low arithmetic rate relative to its memory
// bandwidth, so an FP64 GEMM here is bound by the FP64 pipe, not by HBM: a
// 64 x 64 output tile per CTA with a 4 x 4 register block per thread and
// 16-deep shared-memory K slices keeps the FP64 units busy.  When the output
// has too few tiles to fill the 152 SMs the K dimension is split across CTAs
// and the partial tiles are summed afterwards in a fixed order (so results do
// not depend on scheduling).
#include <algorithm>

#include <cstdlib>

#include "dense.cuh"
#include "tuning.cuh"

namespace fastpi {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

// TI: element type of A and B; T: accumulation and output type (products of
// two FP32 inputs are exact in FP64, so TI = float, T = double accumulates an
// FP32 product to FP64 accuracy).
template <typename TI, typename T, bool TA, bool TB>
__global__ void __launch_bounds__(NT) k_gemm(int64_t M, int64_t N, int64_t K, int64_t kchunk, T alpha,
                                             const TI* __restrict__ A, int64_t lda, const TI* __restrict__ B,
                                             int64_t ldb, T beta, T* __restrict__ C, int64_t ldc, T* __restrict__ W) {
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = int64_t(blockIdx.y) * BM, n0 = int64_t(blockIdx.x) * BN;
  const int64_t k_begin = int64_t(blockIdx.z) * kchunk;
  const int64_t k_end = (k_begin + kchunk < K) ? k_begin + kchunk : K;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

  // the next K-slice is read into registers while the current one is
  // multiplied out of shared memory (the global loads' latency overlaps the
  // multiply-adds; the arithmetic and its order are unchanged)
  constexpr int EA = (BM * BK) / NT, EB = (BN * BK) / NT;
  T ra[EA], rb[EB];
  auto load = [&](int64_t k0) {
#pragma unroll
    for (int e = 0; e < EA; ++e) {
      int lin = tid + NT * e;
      int i, kk;
      if (TA) {
        i = lin % BM;
        kk = lin / BM;
      } else {
        kk = lin % BK;
        i = lin / BK;
      }
      int64_t gi = m0 + i, gk = k0 + kk;
      ra[e] = (gi < M && gk < k_end) ? T(TA ? A[gk * lda + gi] : A[gi * lda + gk]) : T(0);
    }
#pragma unroll
    for (int e = 0; e < EB; ++e) {
      int lin = tid + NT * e;
      int j, kk;
      if (TB) {
        kk = lin % BK;
        j = lin / BK;
      } else {
        j = lin % BN;
        kk = lin / BN;
      }
      int64_t gj = n0 + j, gk = k0 + kk;
      rb[e] = (gj < N && gk < k_end) ? T(TB ? B[gj * ldb + gk] : B[gk * ldb + gj]) : T(0);
    }
  };
  auto store = [&] {
#pragma unroll
    for (int e = 0; e < EA; ++e) {
      int lin = tid + NT * e;
      if (TA)
        As[lin / BM][lin % BM] = ra[e];
      else
        As[lin % BK][lin / BK] = ra[e];
    }
#pragma unroll
    for (int e = 0; e < EB; ++e) {
      int lin = tid + NT * e;
      if (TB)
        Bs[lin % BK][lin / BK] = rb[e];
      else
        Bs[lin / BN][lin % BN] = rb[e];
    }
  };
  if (k_begin < k_end) load(k_begin);
  for (int64_t k0 = k_begin; k0 < k_end; k0 += BK) {
    store();
    __syncthreads();
    if (k0 + BK < k_end) load(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int64_t gi = m0 + ty + 16 * i;
    if (gi >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int64_t gj = n0 + tx + 16 * j;
      if (gj >= N) continue;
      if (W) {
        W[(int64_t(blockIdx.z) * M + gi) * N + gj] = alpha * acc[i][j];
      } else {
        T v = alpha * acc[i][j];
        if (beta != T(0)) v += beta * C[gi * ldc + gj];
        C[gi * ldc + gj] = v;
      }
    }
  }
}

template <typename T>
__global__ void k_splitk_reduce(int64_t M, int64_t N, int splits, const T* __restrict__ W, T beta, T* C,
                                int64_t ldc) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= M * N) return;
  int64_t i = t / N, j = t % N;
  T s = T(0);
  for (int z = 0; z < splits; ++z) s += W[int64_t(z) * M * N + t];
  if (beta != T(0)) s += beta * C[i * ldc + j];
  C[i * ldc + j] = s;
}

template <typename Td, typename Ts>
__global__ void k_copy2d(int64_t rows, int64_t cols, const Ts* src, int64_t lds, Td* dst, int64_t ldd) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= rows * cols) return;
  int64_t i = t / cols, j = t % cols;
  dst[i * ldd + j] = Td(src[i * lds + j]);
}

template <typename Td, typename Ts>
__global__ void k_gather_rows(int64_t rows, int64_t cols, const int32_t* idx, const Ts* src, int64_t lds, Td* dst,
                              int64_t ldd) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= rows * cols) return;
  int64_t i = t / cols, j = t % cols;
  dst[i * ldd + j] = Td(src[int64_t(idx[i]) * lds + j]);
}

template <typename T>
__global__ void k_set(int64_t rows, int64_t cols, T* a, int64_t ld, int ident) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= rows * cols) return;
  int64_t i = t / cols, j = t % cols;
  a[i * ld + j] = (ident && i == j) ? T(1) : T(0);
}

// Gram matrix G = X^T X (c x c, FP64) of an FP32 matrix X (p x c, row-major,
// ld) on the FP32 pipe with about 48 significand bits: every product is split
// exactly (x y = h + e with h = rn(x y) and e = fma(x, y, -h)), the sum of the
// h is carried as an unevaluated pair hi + lo (TwoSum: the rounding error of
// each addition goes to lo) and the e are added to lo.  Explicitly rounded
// operations keep the compiler from fusing a product into an addition, which
// would break the error terms.  Only the 64 x 64 tiles on or above the
// diagonal are formed (blockIdx.x enumerates them), each written with its
// mirror; K is split over blockIdx.z into partial tiles W[z] (c x c) that a
// fixed-order reduction sums.
constexpr int GTILE = 64;
__global__ void __launch_bounds__(NT) k_gram_ff(int64_t p, int c, const float* __restrict__ X, int64_t ld,
                                                int64_t kchunk, double* __restrict__ W) {
  __shared__ float As[BK][GTILE + 1];
  __shared__ float Bs[BK][GTILE + 1];
  const int nt = (c + GTILE - 1) / GTILE;
  int idx = int(blockIdx.x), ti = 0;
  while (idx >= nt - ti) {
    idx -= nt - ti;
    ++ti;
  }
  const int tj = ti + idx;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = ti * GTILE, j0 = tj * GTILE;
  const int64_t k_begin = int64_t(blockIdx.z) * kchunk;
  const int64_t k_end = (k_begin + kchunk < p) ? k_begin + kchunk : p;
  float hi[4][4], lo[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) hi[i][j] = lo[i][j] = 0.f;
  for (int64_t k0 = k_begin; k0 < k_end; k0 += BK) {
#pragma unroll
    for (int e = 0; e < (GTILE * BK) / NT; ++e) {
      const int lin = tid + NT * e;
      const int kk = lin / GTILE, i = lin % GTILE;
      const int64_t gk = k0 + kk;
      const bool krow = gk < k_end;
      As[kk][i] = (krow && i0 + i < c) ? X[gk * ld + i0 + i] : 0.f;
      Bs[kk][i] = (krow && j0 + i < c) ? X[gk * ld + j0 + i] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float h = __fmul_rn(a[i], b[j]);
          const float e = fmaf(a[i], b[j], -h);
          const float s = __fadd_rn(hi[i][j], h);
          const float bb = __fsub_rn(s, hi[i][j]);
          const float err = __fadd_rn(__fsub_rn(hi[i][j], __fsub_rn(s, bb)), __fsub_rn(h, bb));
          hi[i][j] = s;
          lo[i][j] = __fadd_rn(lo[i][j], __fadd_rn(err, e));
        }
    }
    __syncthreads();
  }
  double* Wz = W + int64_t(blockIdx.z) * c * c;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gi = i0 + ty + 16 * i;
    if (gi >= c) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gj = j0 + tx + 16 * j;
      if (gj >= c) continue;
      const double v = double(hi[i][j]) + double(lo[i][j]);
      Wz[int64_t(gi) * c + gj] = v;
      Wz[int64_t(gj) * c + gi] = v;
    }
  }
}

int g_num_sms = 0;
int num_sms() {
  if (!g_num_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  return g_num_sms;
}

inline unsigned grid1(int64_t n) { return unsigned((n + 255) / 256); }

}  // namespace

template <typename TI, typename T>
void gemm_mixed(cudaStream_t st, bool ta, bool tb, int64_t M, int64_t N, int64_t K, T alpha, const TI* A,
                int64_t lda, const TI* B, int64_t ldb, T beta, T* C, int64_t ldc) {
  if (M <= 0 || N <= 0) return;
  if (K <= 0) {
    // C = beta * C
    if (beta == T(0)) {
      set_zero<T>(st, M, N, C, ldc);
    } else if (beta != T(1)) {
      fail(FASTPI_ERR_ARG, "gemm: K == 0 with beta not in {0, 1}");
    }
    return;
  }
  const int64_t tm = (M + BM - 1) / BM, tn = (N + BN - 1) / BN;
  if (tm > 65535) fail(FASTPI_ERR_ARG, "gemm: M too large for the tile grid");
  int splits = 1;
  const int64_t tiles = tm * tn, target = 2 * int64_t(num_sms());
  if (tiles < target && K > 4 * BK * 8) {
    int64_t s = (target + tiles - 1) / tiles;
    int64_t smax = K / (BK * 8);
    if (s > smax) s = smax;
    if (s > 128) s = 128;
    if (s > 1) splits = int(s);
  }
  int64_t kchunk = (K + splits - 1) / splits;
  kchunk = (kchunk + BK - 1) / BK * BK;
  splits = int((K + kchunk - 1) / kchunk);
  DArr<T> work;
  if (splits > 1) work = DArr<T>(int64_t(splits) * M * N, st);
  const dim3 grid{unsigned(tn), unsigned(tm), unsigned(splits)};
  T* W = splits > 1 ? work.get() : nullptr;
  if (!ta && !tb)
    k_gemm<TI, T, false, false><<<grid, NT, 0, st>>>(M, N, K, kchunk, alpha, A, lda, B, ldb, beta, C, ldc, W);
  else if (ta && !tb)
    k_gemm<TI, T, true, false><<<grid, NT, 0, st>>>(M, N, K, kchunk, alpha, A, lda, B, ldb, beta, C, ldc, W);
  else if (!ta && tb)
    k_gemm<TI, T, false, true><<<grid, NT, 0, st>>>(M, N, K, kchunk, alpha, A, lda, B, ldb, beta, C, ldc, W);
  else
    k_gemm<TI, T, true, true><<<grid, NT, 0, st>>>(M, N, K, kchunk, alpha, A, lda, B, ldb, beta, C, ldc, W);
  CK_LAUNCH();
  if (splits > 1) {
    k_splitk_reduce<T><<<grid1(M * N), 256, 0, st>>>(M, N, splits, W, beta, C, ldc);
    CK_LAUNCH();
  }
}

template <typename T>
void gemm(cudaStream_t st, bool ta, bool tb, int64_t M, int64_t N, int64_t K, T alpha, const T* A, int64_t lda,
          const T* B, int64_t ldb, T beta, T* C, int64_t ldc) {
  gemm_mixed<T, T>(st, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
}

// Smallest product (2 M N K flops) sent to the tensor cores: the tuning
// table's value (below it the SIMT kernel's shorter start-up wins; measured
// on the 20 000 x 5 000 workload's step), else 2^24; FASTPI_TC_MIN_FLOPS
// overrides both.
static double tc_min_flops() {
  const char* e = std::getenv("FASTPI_TC_MIN_FLOPS");
  const double x = e && *e ? std::atof(e) : 0.0;
  return x > 0 ? x : tuned_tc_min_flops(double(1 << 24));
}

void gemm_f32(cudaStream_t st, bool ta, bool tb, int64_t M, int64_t N, int64_t K, float alpha, const float* A,
              int64_t lda, const float* B, int64_t ldb, float beta, float* C, int64_t ldc) {
  const double work = 2.0 * double(M) * double(N) * double(K);
  if (M >= 64 && work >= tc_min_flops() && gemm_tf32_supported(ta, tb, M, N, K, lda, ldb, ldc, A, B, C))
    gemm_tf32(st, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, 3);
  else
    gemm<float>(st, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
}

void gram_ff(cudaStream_t st, int64_t p, int64_t c, const float* X, int64_t ld, double* G) {
  if (c <= 0) return;
  if (p <= 0) {
    set_zero<double>(st, c, c, G, c);
    return;
  }
  const int64_t nt = (c + GTILE - 1) / GTILE, tiles = nt * (nt + 1) / 2;
  if (tiles > 65535) fail(FASTPI_ERR_ARG, "gram: too many columns");
  const int64_t target = 2 * int64_t(num_sms());
  int64_t splits = std::max<int64_t>(1, (target + tiles - 1) / tiles);
  splits = std::min<int64_t>(splits, std::max<int64_t>(1, p / (BK * 8)));
  splits = std::min<int64_t>(splits, 128);
  int64_t kchunk = (p + splits - 1) / splits;
  kchunk = (kchunk + BK - 1) / BK * BK;
  splits = (p + kchunk - 1) / kchunk;
  DArr<double> work(splits > 1 ? splits * c * c : 1, st);
  double* W = splits > 1 ? work.get() : G;
  k_gram_ff<<<dim3(unsigned(tiles), 1, unsigned(splits)), NT, 0, st>>>(p, int(c), X, ld, kchunk, W);
  CK_LAUNCH();
  if (splits > 1) {
    k_splitk_reduce<double><<<grid1(c * c), 256, 0, st>>>(c, c, int(splits), W, 0.0, G, c);
    CK_LAUNCH();
  }
}

template void gemm_mixed<float, double>(cudaStream_t, bool, bool, int64_t, int64_t, int64_t, double, const float*,
                                        int64_t, const float*, int64_t, double, double*, int64_t);

template <typename Td, typename Ts>
void copy2d(cudaStream_t st, int64_t rows, int64_t cols, const Ts* src, int64_t lds, Td* dst, int64_t ldd) {
  if (rows <= 0 || cols <= 0) return;
  k_copy2d<Td, Ts><<<grid1(rows * cols), 256, 0, st>>>(rows, cols, src, lds, dst, ldd);
  CK_LAUNCH();
}

template <typename Td, typename Ts>
void gather_rows(cudaStream_t st, int64_t rows, int64_t cols, const int32_t* idx, const Ts* src, int64_t lds,
                 Td* dst, int64_t ldd) {
  if (rows <= 0 || cols <= 0) return;
  k_gather_rows<Td, Ts><<<grid1(rows * cols), 256, 0, st>>>(rows, cols, idx, src, lds, dst, ldd);
  CK_LAUNCH();
}

template <typename T> void set_zero(cudaStream_t st, int64_t rows, int64_t cols, T* a, int64_t ld) {
  if (rows <= 0 || cols <= 0) return;
  k_set<T><<<grid1(rows * cols), 256, 0, st>>>(rows, cols, a, ld, 0);
  CK_LAUNCH();
}
template <typename T> void set_identity(cudaStream_t st, int64_t rows, int64_t cols, T* a, int64_t ld) {
  if (rows <= 0 || cols <= 0) return;
  k_set<T><<<grid1(rows * cols), 256, 0, st>>>(rows, cols, a, ld, 1);
  CK_LAUNCH();
}

template void gemm<double>(cudaStream_t, bool, bool, int64_t, int64_t, int64_t, double, const double*, int64_t,
                           const double*, int64_t, double, double*, int64_t);
template void gemm<float>(cudaStream_t, bool, bool, int64_t, int64_t, int64_t, float, const float*, int64_t,
                          const float*, int64_t, float, float*, int64_t);
template void copy2d<double, double>(cudaStream_t, int64_t, int64_t, const double*, int64_t, double*, int64_t);
template void copy2d<float, float>(cudaStream_t, int64_t, int64_t, const float*, int64_t, float*, int64_t);
template void copy2d<float, double>(cudaStream_t, int64_t, int64_t, const double*, int64_t, float*, int64_t);
template void copy2d<double, float>(cudaStream_t, int64_t, int64_t, const float*, int64_t, double*, int64_t);
template void gather_rows<double, double>(cudaStream_t, int64_t, int64_t, const int32_t*, const double*, int64_t,
                                          double*, int64_t);
template void gather_rows<double, float>(cudaStream_t, int64_t, int64_t, const int32_t*, const float*, int64_t,
                                         double*, int64_t);
template void gather_rows<float, float>(cudaStream_t, int64_t, int64_t, const int32_t*, const float*, int64_t,
                                        float*, int64_t);
template void set_zero<double>(cudaStream_t, int64_t, int64_t, double*, int64_t);
template void set_zero<float>(cudaStream_t, int64_t, int64_t, float*, int64_t);
template void set_identity<double>(cudaStream_t, int64_t, int64_t, double*, int64_t);
template void set_identity<float>(cudaStream_t, int64_t, int64_t, float*, int64_t);

}  // namespace fastpi
