// Batched one-sided (Hestenes) Jacobi SVD.
#pragma once

#include "common.cuh"

namespace fastpi {

// One problem: A (p x q, COLUMN-major, leading dimension lda) is overwritten
// by B = A J with mutually orthogonal columns; V (q x q, column-major, ldv)
// receives J.  Then sigma_j = |b_j|, A = (B diag(1/sigma)) diag(sigma) J^T.
template <typename T>
struct JacobiProblem {
  T* A;
  T* V;
  int64_t lda, ldv;
  int p, q;
};

struct JacobiStats {
  int max_sweeps_used = 0;
  bool hit_cap = false;
};

// Runs every problem to convergence in one persistent cooperative launch and
// writes, per problem b, the singular values in descending order (ties: lower
// column index first) to sig[sig_off_b .. + q_b) and the column index of each
// to perm[...], where sig_off_b = sum of q over earlier problems.
template <typename T>
JacobiStats jacobi_svd_batched(fastpi_ctx* h, const std::vector<JacobiProblem<T>>& probs, double* sig,
                               int32_t* perm, int kind = SVD_BLOCKS);

// Only the last step of jacobi_svd_batched: column norms of each (already
// orthogonalised) A and the descending sort, into sig / perm.
template <typename T>
void jacobi_sort_columns(fastpi_ctx* h, const std::vector<JacobiProblem<T>>& probs, double* sig, int32_t* perm);

// FP32 core SVD of one square n x n column-major K (ld n) by block one-sided
// Jacobi on the whole GPU (column blocks of 4 or 8 columns; one CTA per block
// pair and round).  Same outputs as jacobi_svd_batched for a single problem
// (V = J, n x n col-major, ld n); returns false, having
// done nothing, when a block pair's panels do not fit in one CTA's shared
// memory or the block pairs of a round exceed the co-resident CTAs.
struct CoreTiling;
bool jacobi_svd_block(fastpi_ctx* h, float* K, float* V, int n, double* sig, int32_t* perm, JacobiStats* stats,
                      const CoreTiling* tiling = nullptr, float* ms_out = nullptr, int* sweeps_out = nullptr);

// Tiling of the FP32 core SVD: panel = P (two column blocks of P / 2), parts
// = CTAs of a cluster sharing a block pair's rows (0: as many as keep one
// round's clusters on the SMs, at most 8), resident = the resident-block
// schedule, fast_solve = the P x P Gram sweep with one CTA barrier per inner
// round and fast rotations (false: two barriers and IEEE rotations).
struct CoreTiling {
  int panel = 16;
  int parts = 0;
  bool resident = false;
  bool fast_solve = true;   // the Gram sweep with one barrier per inner round and fast rotations
  bool single_cta = false;  // the single-CTA block kernel instead of the cluster form
  bool strict = false;      // no fallback to the single-CTA kernel when the cluster form does not fit
  // a sweep whose rotations all stay below this (|g| / sqrt(al be)) is the
  // last: measured on the 20 000 x 5 000 workload (mixed factor, 40 cores),
  // 1e-3 -> 399 ms, residual gap to the oracle 1.1e-8, sigma error 1.1e-5,
  // |U^T U - I| 3.9e-5; 5e-3 -> 376 ms, 6.8e-7, 1.4e-5, 3.8e-5; 1e-2 -> 359 ms,
  // 3.4e-7, 1.2e-4, 1.6e-4 (orthonormality starts to degrade beyond 5e-3)
  float early_exit = 5e-3f;
};
// U[:, t] = K[:, perm[t]] / sig[t] (zero when sig[t] = 0), Vs[:, t] = V[:, perm[t]]
// for the outputs of jacobi_svd_block (n x n column-major, ld n).
void core_vectors_f32(fastpi_ctx* h, int n, const float* K, const float* V, const double* sig, const int32_t* perm,
                      float* U, float* Vs);
// The cluster form of block one-sided Jacobi (jacobi_cluster.cu) on a p x n
// FP32 problem (p >= n, column-major, ld lda): K <- K J with mutually
// orthogonal columns and V (n x n, ld ldv) <- J, as jacobi_svd_block computes
// them before the final sort.  false, having done nothing, when the tiling
// does not fit (shared memory, co-resident clusters) or the launch form is
// refused.
bool jacobi_svd_cluster(fastpi_ctx* h, float* K, int64_t lda, float* V, int64_t ldv, int p, int n,
                        const CoreTiling& tiling, JacobiStats* stats, float* ms, int* sweeps, bool* used_res);

}  // namespace fastpi
