// Factorization state kept in a handle after fastpi_factor.
#pragma once

#include <string>

#include "internal.cuh"

namespace fastpi {

struct Factors {
  int prec = 0;
  int64_t m = 0, n = 0, rank = 0;
  // U (m x rank) and V (n x rank), row-major, ORIGINAL row order; FP64 mode
  // fills U64/V64, the mixed mode U32/V32.
  DArr<double> U64, V64;
  DArr<float> U32, V32;
  std::vector<double> S;   // host, descending
  DArr<double> S_d;        // device copy
  Reordering R;
};

void factor(fastpi_ctx* h, int64_t r, double k, fastpi_precision prec, int64_t chunk_row, int64_t chunk_col);
// Independent factorizations of count handles (same device, same precision,
// one stream each): one host thread per handle, at most `concurrency` of them
// in the stages before / after the block SVDs at a time, and the A11 block
// SVDs of all handles in one batched launch.  status[i] / msgs[i] per handle.
void factor_batched(fastpi_ctx* const* hs, int count, const int64_t* r, double k, fastpi_precision prec,
                    int64_t chunk_row, int64_t chunk_col, int concurrency, fastpi_status* status,
                    std::string* msgs);
// Factors given by the caller (U m x r, V n x r row-major FP64, host or device;
// S host, r values): the handle serves fastpi_apply* as if fastpi_factor had
// produced them (the mixed form stores U, V in FP32).
void load_factors(fastpi_ctx* h, int64_t r, const double* S, const double* U, int64_t ldu, const double* V,
                  int64_t ldv, fastpi_precision prec, bool on_device);
// Keep the r largest triplets of the current factors.
void truncate_factors(fastpi_ctx* h, int64_t r);
// Algorithm 2 and Eq. 1 alone: the kept singular values of the A11 blocks
// (block order, descending within a block); the reordering is kept for the
// permutation / block getters.
void block_svd_only(fastpi_ctx* h, int64_t r, double k, fastpi_precision prec, std::vector<double>& sig);
// Algorithm 2 alone: the reordering is kept for the permutation / block getters.
void reorder_only(fastpi_ctx* h, double k);
void apply_dense(fastpi_ctx* h, const double* Y, int64_t L, int64_t ldy, double* Z, int64_t ldz);
void apply_csr(fastpi_ctx* h, int64_t L, int64_t nnz_y, const int64_t* yrowptr, const int32_t* ycol,
               const double* yval, double* Z, int64_t ldz);
double residual(fastpi_ctx* h, const double* Y, int64_t L, int64_t ldy, const double* Z, int64_t ldz);
// out (m x L) = A X (X: n x L), FP64, device buffers.
void spmm(fastpi_ctx* h, const double* X, int64_t L, int64_t ldx, double* out, int64_t ldo);
// |A - U diag(S) V^T|_F / |A|_F from the stored factors.
double recon_error(fastpi_ctx* h);

}  // namespace fastpi
