// Blocked kernels of the CholeskyQR2 orthogonalisation (cholqr.cu).
#pragma once

#include "common.cuh"

namespace fastpi {

// X (c x c, row-major) <- the inverse of the lower-triangular L (c x c,
// row-major) restricted to the indices with kept[i] != 0 (zero rows and
// columns elsewhere).  Shared memory: trinv_blocked_smem(c, sizeof(T)) bytes
// per CTA.
template <typename T>
void trinv_blocked(cudaStream_t st, const T* L, int c, const int32_t* kept, T* X);
size_t trinv_blocked_smem(int c, size_t elem);

// Cholesky of the c x c FP32 Gram G (row-major, lower triangle used) with
// dependent directions dropped (a pivot <= tol gives a zero column,
// kept[j] = 0); on exit G holds L (upper part zero) and *rank the number kept.
// One CTA holding the packed lower triangle in shared memory:
// chol_drop_blocked_smem(c) bytes plus 13 KB of static shared memory.
void chol_drop_blocked(cudaStream_t st, float* G, int c, float tol, int32_t* kept, int32_t* rank);
size_t chol_drop_blocked_smem(int c);
// Instrumented builds (FASTPI_PHASE_CLOCKS): prints the accumulated phase
// clocks of chol_drop_blocked to stderr and resets them; no-op otherwise.
void chol_drop_phase_report(const char* tag);

}  // namespace fastpi
