// Internal data structures passed between the stages of fastpi_factor.
#pragma once

#include "common.cuh"

namespace fastpi {

// Result of the hub-and-spoke reordering (Algorithm 2) plus the split of the
// reordered A into A11 blocks, A21 and T = [A12; A22] (Section 3.3).
struct Reordering {
  int64_t m = 0, n = 0, m1 = 0, n1 = 0, iterations = 0, num_blocks = 0;
  std::vector<int64_t> row_off, col_off;      // host, B+1 entries each
  DArr<int32_t> row_order, col_order;         // new position -> original id
  DArr<int32_t> row_pos, col_pos;             // original id -> new position
};

// "Sparse columns" of a border matrix: column t holds entries
// (idx[e], val[e]) for e in [ptr[t], ptr[t+1]); idx is a new-order position.
struct SparseCols {
  int64_t ncols = 0, nrows = 0, nnz = 0;
  DArr<int64_t> ptr;
  DArr<int32_t> idx;
  DArr<double> val;
  std::vector<int64_t> ptr_h;   // host copy of ptr (chunk boundaries)
};

// Dense copies of the A11 diagonal blocks for Eq. 1.  Block b is stored
// column-major in its "tall" orientation: p_b = max(m_b, n_b) rows and
// q_b = min(m_b, n_b) columns (the transpose when m_b < n_b), at offset
// data_off[b].  Blocks with s_b = 0 store nothing.
struct A11Blocks {
  int64_t B = 0, S = 0, total = 0;
  std::vector<int64_t> m_b, n_b, s_b, data_off, s_off;   // host
  DArr<double> data;
};

void run_reorder(fastpi_ctx* h, double k, Reordering& R);
void split_border(fastpi_ctx* h, const Reordering& R, SparseCols& A21rows, SparseCols& Tcols);
void extract_blocks(fastpi_ctx* h, const Reordering& R, int64_t r, A11Blocks& blk);

// CSC build and CSR validation at create time.
void build_csc(fastpi_ctx* h);
void validate_csr(fastpi_ctx* h);

}  // namespace fastpi
