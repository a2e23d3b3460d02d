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
                               int32_t* perm);

}  // namespace fastpi
