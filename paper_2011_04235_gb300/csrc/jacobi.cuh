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
bool jacobi_svd_block(fastpi_ctx* h, float* K, float* V, int n, double* sig, int32_t* perm, JacobiStats* stats);

}  // namespace fastpi
