// Dense linear-algebra kernels used by the incremental SVD updates.
// All matrices are row-major with a leading dimension unless stated.
#pragma once

#include "common.cuh"

namespace fastpi {

// C (M x N) = alpha * op(A) * op(B) + beta * C.  op(A) is M x K: A is M x K
// (ta = false) or K x M (ta = true); op(B) is K x N: B is K x N (tb = false)
// or N x K (tb = true).  beta == 0 never reads C.  Deterministic (split-K
// partials are reduced in a fixed order).
template <typename T>
void gemm(cudaStream_t st, bool ta, bool tb, int64_t M, int64_t N, int64_t K, T alpha, const T* A, int64_t lda,
          const T* B, int64_t ldb, T beta, T* C, int64_t ldc);

// Same contract with inputs of type TI and accumulation / output in T
// (instantiated for TI = float, T = double: FP32 data, FP64-accurate sums).
template <typename TI, typename T>
void gemm_mixed(cudaStream_t st, bool ta, bool tb, int64_t M, int64_t N, int64_t K, T alpha, const TI* A,
                int64_t lda, const TI* B, int64_t ldb, T beta, T* C, int64_t ldc);

// G (c x c, FP64, row-major) = X^T X for X (p x c, FP32, row-major, ld): the
// products split exactly and summed as FP32 pairs (about 48 significand bits)
// on the FP32 pipe; symmetric tiles formed once.
void gram_ff(cudaStream_t st, int64_t p, int64_t c, const float* X, int64_t ld, double* G);

// Same contract with FP32 storage on the TF32 tensor cores (tcgen05.mma,
// kind::tf32, FP32 accumulation in tensor memory, TMA-staged operands).
// passes = 1: operands rounded to TF32; passes = 3: split hi + lo TF32
// products (FP32-level accuracy).  gemm_tf32_supported says whether the
// device and the sizes allow the tensor path.
bool gemm_tf32_supported(bool ta, bool tb, int64_t M, int64_t N, int64_t K, int64_t lda, int64_t ldb,
                         int64_t ldc, const void* A, const void* B, const void* C);
void gemm_tf32(cudaStream_t st, bool ta, bool tb, int64_t M, int64_t N, int64_t K, float alpha, const float* A,
               int64_t lda, const float* B, int64_t ldb, float beta, float* C, int64_t ldc, int passes);
// Status bits raised by the tensor-core GEMM kernels since the last clear
// (synchronizes the stream).
unsigned gemm_tc_status(cudaStream_t st, bool clear);

// FP32 GEMM of the mixed-precision form: the tensor-core path for shapes with
// enough work to fill it (2 M N K >= 2^24 and M >= 64), SIMT FP32 otherwise.
void gemm_f32(cudaStream_t st, bool ta, bool tb, int64_t M, int64_t N, int64_t K, float alpha, const float* A,
              int64_t lda, const float* B, int64_t ldb, float beta, float* C, int64_t ldc);

// dst[i*ldd + j] = (T)src[i*lds + j] for a rows x cols block.
template <typename Td, typename Ts>
void copy2d(cudaStream_t st, int64_t rows, int64_t cols, const Ts* src, int64_t lds, Td* dst, int64_t ldd);

// Gather rows: dst[i, :] = src[idx[i], :] (rows x cols).
template <typename Td, typename Ts>
void gather_rows(cudaStream_t st, int64_t rows, int64_t cols, const int32_t* idx, const Ts* src, int64_t lds,
                 Td* dst, int64_t ldd);

// Set a rows x cols block to zero / the identity (row-major, ld).
template <typename T> void set_zero(cudaStream_t st, int64_t rows, int64_t cols, T* a, int64_t ld);
template <typename T> void set_identity(cudaStream_t st, int64_t rows, int64_t cols, T* a, int64_t ld);

}  // namespace fastpi
