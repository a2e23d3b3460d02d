/*
 * fastpi.h -- C ABI of libfastpi, a single-GPU (sm_103a) implementation of
 * FastPI: approximate Moore-Penrose pseudoinverse of a sparse feature matrix by
 * hub-and-spoke reordering and incremental low-rank SVD (Jung and Sael,
 * "Fast and Accurate Pseudoinverse with Sparse Matrix Reordering and
 * Incremental Approach").
 *
 * Conventions (all entry points):
 *   - Every call returns a fastpi_status and never aborts the process.  On an
 *     error, fastpi_last_error(h) returns a human-readable message.
 *   - Dense matrices are ROW-MAJOR with an explicit leading dimension (the
 *     distance in elements between consecutive rows, >= the row length).
 *   - "device" pointers are CUDA device (or managed) addresses on the device
 *     that was current when fastpi_create ran; "host" pointers are ordinary
 *     host memory.  Each argument below says which one it takes.
 *   - The library owns every allocation it makes; the caller keeps ownership of
 *     its inputs (they are copied) and of its output buffers.
 *   - Work is issued on the CUDA stream given to fastpi_create.  Calls that
 *     return host-visible results synchronise that stream (never the device).
 *   - Indices are 0-based.  "new" positions refer to the reordered matrix of
 *     Algorithm 2; "original" to the caller's row / column numbering.
 */
#ifndef FASTPI_H
#define FASTPI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fastpi_ctx* fastpi_t;

typedef enum {
  FASTPI_OK = 0,
  FASTPI_ERR_ARG = 1,            /* invalid argument (null handle, bad size, k outside (0,1), ...) */
  FASTPI_ERR_CSR = 2,            /* malformed CSR: rowptr not monotone, column out of range,
                                    unsorted or duplicate columns in a row */
  FASTPI_ERR_OOM = 3,            /* device allocation failed */
  FASTPI_ERR_CUDA = 4,           /* a CUDA runtime call failed */
  FASTPI_ERR_NO_CONVERGENCE = 5, /* an iteration cap was reached on the device (Jacobi sweeps,
                                    union-find retries, a bounded device-wide barrier) */
  FASTPI_ERR_STATE = 6           /* call out of order (e.g. a getter before fastpi_factor) */
} fastpi_status;

typedef enum {
  FASTPI_FP64 = 0,        /* every floating-point step in FP64 */
  FASTPI_MIXED_TF32 = 1   /* FP32 storage; dense products on TF32 tensor cores with FP32
                             accumulation; Gram Cholesky and singular values in FP64 */
} fastpi_precision;

/* Summary of the last factorization (host struct filled by fastpi_get_info). */
typedef struct {
  int64_t m, n, nnz;
  int64_t m1, n1, m2, n2;    /* A11 is m1 x n1; hubs are the trailing m2 rows / n2 columns */
  int64_t num_blocks;        /* B: diagonal blocks of A11, including empty ones */
  int64_t iterations;        /* T: iterations of the reordering loop */
  int64_t S;                 /* columns kept by the block SVD (sum of s_i) */
  int64_t s_row;             /* rank after the row update */
  int64_t rank;              /* r' = rank after the column update */
  int64_t chunk_row, chunk_col;        /* border rows / columns appended per incremental step */
  int64_t row_chunks, col_chunks;      /* number of incremental steps of each phase */
  int64_t dropped_directions;          /* residual directions dropped as dependent */
  int64_t jacobi_sweeps_max;           /* most sweeps any Jacobi SVD needed */
  double min_trunc_gap;      /* min over truncations of (sigma_keep_last - sigma_drop_first)/sigma_1 */
  double ms_reorder, ms_block_svd, ms_row_update, ms_col_update, ms_finalize;  /* stage times */
  int precision;
} fastpi_info;

/*
 * fastpi_create -- upload a sparse feature matrix A (m x n, CSR) and build the
 * handle.  A is the feature matrix of Application 1 (instances = rows,
 * features = columns); its bipartite network is Definition 1.
 *   rowptr: int64[m+1], monotone, rowptr[0] = 0, rowptr[m] = nnz
 *   colind: int32[nnz], strictly increasing within each row, in [0, n)
 *   val:    float64[nnz]
 *   ptrs_on_device: 0 -> the three arrays are host pointers; 1 -> device pointers.
 *   cuda_stream: a cudaStream_t (NULL = legacy default stream) used by every
 *   later call on this handle.
 * The arrays are validated (FASTPI_ERR_CSR on failure) and copied; the caller
 * may free them on return.  *out is set to NULL on any error.
 */
fastpi_status fastpi_create(fastpi_t* out, int64_t m, int64_t n, int64_t nnz,
                            const int64_t* rowptr, const int32_t* colind, const double* val,
                            int ptrs_on_device, void* cuda_stream);

/*
 * fastpi_factor -- Algorithm 1 up to the solve: reorder A by Algorithm 2 (hub ratio
 * k in (0,1)), SVD of the block-diagonal A11 (Eq. 1, per-block rank
 * s_i = min(ceil(alpha n_1i), m_1i, n_1i)), row incremental update with A21
 * (Eq. 2, rank s = min(ceil(alpha n1), S + m2, n1)) and column incremental
 * update with T = [A12; A22] (Eq. 3, rank r' = min(r, m, s + n2)), where the
 * target rank ratio is alpha = r / n (Table 1).
 *   r:     target rank, 1 <= r.
 *   k:     hub selection ratio, 0 < k < 1.
 *   prec:  FASTPI_FP64 or FASTPI_MIXED_TF32.
 *   chunk_row, chunk_col: border rows of A21 / columns of T appended per
 *          incremental step (0 = autotuned: the tuning table's value for the
 *          phase's target rank, 256 without a table; >= the border size gives
 *          the single-shot form of Eqs. 2 and 3).  Each step truncates to the
 *          phase's target rank; fastpi_get_info reports the chunks used.
 * Re-factoring a handle replaces the previous factors.
 */
fastpi_status fastpi_factor(fastpi_t h, int64_t r, double k, fastpi_precision prec,
                            int64_t chunk_row, int64_t chunk_col);

/*
 * fastpi_apply -- Problem 1 / Application 1: Z = V Sigma^+ U^T Y for a dense
 * label matrix.  Sigma^+_ii = 1/sigma_i if sigma_i > tau, else 0, with
 * tau = max(m, n) * 2^-52 * sigma_1.
 *   Y: device float64, m x L row-major (ldy >= L), rows in ORIGINAL order.
 *   Z: device float64, n x L row-major (ldz >= L), rows in ORIGINAL order; overwritten.
 * FASTPI_ERR_STATE before a successful fastpi_factor.
 * The apply synchronises nothing on the host and allocates only
 * stream-ordered memory on the handle's stream, so it may be recorded into a
 * CUDA graph (capture on that stream) and replayed for new Y of the same
 * shape. */
fastpi_status fastpi_apply(fastpi_t h, const double* Y, int64_t L, int64_t ldy,
                           double* Z, int64_t ldz);

/* fastpi_apply_host -- as fastpi_apply, with Y and Z in HOST memory; the
 * host<->device copies run on the handle's stream and the call returns when Z
 * is written. */
fastpi_status fastpi_apply_host(fastpi_t h, const double* Y, int64_t L, int64_t ldy,
                                double* Z, int64_t ldz);

/*
 * fastpi_apply_csr -- as fastpi_apply for a sparse label matrix Y (m x L, CSR,
 * device pointers: yrowptr int64[m+1], ycol int32[nnz_y] in [0, L), yval
 * float64[nnz_y]).  Z: device float64 n x L row-major (ldz >= L), rows in
 * ORIGINAL order; overwritten.  Y is checked as fastpi_create checks A:
 * FASTPI_ERR_CSR when yrowptr does not run from 0 to nnz_y without
 * decreasing, or a row's labels are not strictly increasing within [0, L)
 * (Z is then untouched).  FASTPI_ERR_ARG for L or nnz_y of 2^31 - 1 or more;
 * FASTPI_ERR_STATE before a successful fastpi_factor.  The check reads Y back,
 * so the call synchronises the handle's stream.
 */
fastpi_status fastpi_apply_csr(fastpi_t h, int64_t L, int64_t nnz_y, const int64_t* yrowptr,
                               const int32_t* ycol, const double* yval, double* Z, int64_t ldz);

/* fastpi_residual -- ||A Z - Y||_F in FP64 (Application 1's objective).
 * Y: device m x L (ldy), Z: device n x L (ldz), both rows in ORIGINAL order.
 * *out: host double; the call synchronises the handle's stream.  Errors:
 * FASTPI_ERR_ARG (null pointers, ldy or ldz < L), FASTPI_ERR_STATE (a handle
 * made from factors has no matrix). */
fastpi_status fastpi_residual(fastpi_t h, const double* Y, int64_t L, int64_t ldy,
                              const double* Z, int64_t ldz, double* out);

/* fastpi_spmm -- out = A X (m x L) for the handle's sparse matrix A: the
 * scores of Application 1's multi-label regression when X = Z and A holds
 * held-out instances.  X: device float64 n x L row-major (ldx >= L); out:
 * device float64 m x L row-major (ldo >= L), overwritten.  The call returns
 * when out is written.  Errors: FASTPI_ERR_ARG (sizes, null pointers),
 * FASTPI_ERR_STATE (a handle made from factors has no matrix). */
fastpi_status fastpi_spmm(fastpi_t h, const double* X, int64_t L, int64_t ldx, double* out, int64_t ldo);

/* fastpi_recon_error -- |A - U Sigma V^T|_F / |A|_F, the reconstruction error
 * of the low-rank approximation behind the pseudoinverse (Section 4), from the
 * stored factors, in FP64: |A|^2 - 2 sum_i sigma_i u_i^T A v_i +
 * sigma^T ((U^T U) o (V^T V)) sigma (exact also when U and V are orthonormal
 * only to rounding), so an error below about 1e-7 is resolved only to
 * rounding.  *out: host double.  Errors: FASTPI_ERR_STATE (before
 * fastpi_factor, or a handle made from factors). */
fastpi_status fastpi_recon_error(fastpi_t h, double* out);

/*
 * fastpi_residual_noalloc -- |A Z - Y|_F in FP64, like fastpi_residual, but
 * without a handle and without allocating anything.  The paper has no
 * counterpart: this serves callers that cannot allocate device memory when
 * they need the residual -- code under a fixed memory budget with the
 * allocator locked, allocation-free real-time loops.  Its scratch is a static device array of
 * FASTPI_NOALLOC_MAX_ROWS + 1 doubles (8 MiB) that every GPU loading the
 * library keeps until the process exits.
 *   A: device CSR (rowptr int64[m+1], colind int32[nnz], val float64[nnz]), m x n;
 *      not checked here (that would be a second pass over A on every call):
 *      it must pass the checks fastpi_create makes, else the result is
 *      undefined.
 *   Y: device m x L (ldy), Z: device n x L (ldz), row-major.  *out: host double.
 *   cuda_stream: the stream to run on (NULL = legacy default stream of the
 *   current device).  The call runs on the stream's device, whatever device
 *   is current; A, Y and Z must be on that device.  The caller's current
 *   device is restored on return.
 * FASTPI_ERR_ARG when m > FASTPI_NOALLOC_MAX_ROWS or an argument is invalid.
 * The first call on each device is its set-up: it looks up the scratch
 * address on that device and, under CUDA's lazy module loading, loads this
 * entry point's kernels and the scratch array there, which takes device
 * memory once.  Make one call on each device (m = 0 is enough) before the
 * memory budget is locked; later calls allocate nothing.  A cudaDeviceReset
 * invalidates that set-up like every other resource of the process on the
 * device: do not call this entry point on a device after resetting it.
 * All calls share the scratch, so calls that overlap on the GPU race; each
 * call overwrites all the scratch it reads.
 * The call synchronises the stream to return the value.
 */
#define FASTPI_NOALLOC_MAX_ROWS (1 << 20)
fastpi_status fastpi_residual_noalloc(int64_t m, int64_t n, const int64_t* rowptr, const int32_t* colind,
                                      const double* val, const double* Y, int64_t L, int64_t ldy,
                                      const double* Z, int64_t ldz, double* out, void* cuda_stream);

/* Many independent factorizations (Algorithm 1 up to the solve, once per handle):
 * handle i is factored at target rank r[i] with the common hub ratio k,
 * precision and chunk sizes, exactly as fastpi_factor would (same results).
 * The A11 block SVDs (Eq. 1) of ALL handles run in one persistent batched
 * launch; the reorderings and the incremental updates of different handles
 * run concurrently, one host thread per handle, at most `concurrency` (<= 0:
 * 4) of them in those stages at a time.  Requirements: count >= 1 distinct
 * handles created on one device; give each handle its own stream, or they
 * serialise.  The call returns when every factorization has finished (or
 * failed): FASTPI_OK, or the status of the first failing handle (its message
 * in fastpi_last_error of that handle, and of NULL); status_out (host,
 * count entries, may be NULL) receives each handle's status.  Argument errors
 * (FASTPI_ERR_ARG) are reported before any work starts. */
fastpi_status fastpi_factor_batched(fastpi_t* hs, int count, const int64_t* r, double k, fastpi_precision prec,
                                    int64_t chunk_row, int64_t chunk_col, int concurrency,
                                    fastpi_status* status_out);

/* Factor reuse (serving the apply of Application 1 from stored factors):
 * a handle that holds the given rank-r factors of an m x n matrix -- S (host,
 * r values, descending, >= 0), U (m x r) and V (n x r), row-major FP64 with
 * leading dimensions ldu, ldv >= r, in the caller's original row / column
 * order (as fastpi_get_U / _V return them), on the device when
 * ptrs_on_device != 0, else on the host.  The inputs are copied; the mixed
 * precision stores U and V in FP32 as fastpi_factor would.  The handle
 * serves fastpi_apply, fastpi_apply_host, fastpi_apply_csr and the factor
 * getters; it has no matrix, so fastpi_factor, fastpi_reorder and
 * fastpi_residual return FASTPI_ERR_STATE.  Errors: FASTPI_ERR_ARG (sizes,
 * null arrays, unsorted or negative S), FASTPI_ERR_OOM, FASTPI_ERR_CUDA. */
fastpi_status fastpi_create_from_factors(fastpi_t* out, int64_t m, int64_t n, int64_t r, const double* S,
                                        const double* U, int64_t ldu, const double* V, int64_t ldv,
                                        fastpi_precision prec, int ptrs_on_device, void* cuda_stream);

/* Keep the r largest triplets of the current factors (a sweep over smaller
 * target ranks -- alpha = r / n -- from one factorization; an approximation
 * of fastpi_factor at rank r, whose appends truncate at r along the way).
 * r >= the current rank leaves the factors unchanged.  Errors:
 * FASTPI_ERR_ARG (r < 1), FASTPI_ERR_STATE (no factors). */
fastpi_status fastpi_truncate(fastpi_t h, int64_t r);

/* Algorithm 2 (Section 3.2) alone: the hub-and-spoke reordering of A for hub
 * ratio k in (0, 1), without any factorization.  Afterwards fastpi_get_perm,
 * fastpi_get_blocks and fastpi_get_info (reordering fields; the factorization
 * fields are zero) are valid and the factor getters return FASTPI_ERR_STATE
 * until fastpi_factor runs.  Gives the same permutation as fastpi_factor with
 * the same k.  Errors: FASTPI_ERR_ARG (k outside (0, 1)), FASTPI_ERR_CUDA. */
fastpi_status fastpi_reorder(fastpi_t h, double k);

/* Eq. 1 (Section 3.3) alone: Algorithm 2 with hub ratio k, then the SVD of
 * every diagonal block A11^(i) of A11, keeping its s_i = min(ceil(alpha n_1i),
 * m_1i, n_1i) largest singular values, alpha = r / n -- the first stage of
 * fastpi_factor with the same r, k and precision, stopped there.
 *   sigma: host float64[cap]; receives the S = sum of s_i kept values, block by
 *          block in the block order of fastpi_get_blocks, descending within a
 *          block (ties: lower column of the block's Jacobi result first).
 *   S_out: host int64, receives S (also when cap is too small).
 * Afterwards fastpi_get_perm, fastpi_get_blocks and fastpi_get_info (the
 * reordering fields and S) are valid; the factor getters return
 * FASTPI_ERR_STATE.  Errors: FASTPI_ERR_ARG (r < 1, k outside (0, 1), unknown
 * precision, S_out NULL, or cap < S: the values are then not written),
 * FASTPI_ERR_STATE (a handle made from factors), FASTPI_ERR_CUDA,
 * FASTPI_ERR_NO_CONVERGENCE. */
fastpi_status fastpi_block_svd(fastpi_t h, int64_t r, double k, fastpi_precision prec, double* sigma,
                               int64_t cap, int64_t* S_out);

/* Getters (valid after fastpi_factor; FASTPI_ERR_STATE before; fastpi_get_perm,
 * fastpi_get_blocks and fastpi_get_info also after fastpi_reorder). */
fastpi_status fastpi_get_rank(fastpi_t h, int64_t* r_out);            /* host int64 */
fastpi_status fastpi_get_S(fastpi_t h, double* S);                    /* host float64[r'], descending */
/* U: device float64 m x r' row-major (ldu >= r'), rows in ORIGINAL order. */
fastpi_status fastpi_get_U(fastpi_t h, double* U, int64_t ldu);
/* V: device float64 n x r' row-major (ldv >= r'), rows in ORIGINAL order. */
fastpi_status fastpi_get_V(fastpi_t h, double* V, int64_t ldv);
/* Reordering of Algorithm 2 (host arrays): row_order[new] = original row,
 * col_order[new] = original column; m2 / n2 hub counts (the trailing rows /
 * columns).  Any output pointer may be NULL. */
fastpi_status fastpi_get_perm(fastpi_t h, int32_t* row_order, int32_t* col_order,
                              int64_t* m2, int64_t* n2);
/* Diagonal blocks of A11 (host arrays of B+1 entries): block b covers new rows
 * [row_off[b], row_off[b+1]) and new columns [col_off[b], col_off[b+1]).
 * Pass NULL offsets to query *B only. */
fastpi_status fastpi_get_blocks(fastpi_t h, int64_t* B, int64_t* row_off, int64_t* col_off);
fastpi_status fastpi_get_info(fastpi_t h, fastpi_info* info);          /* host struct */

/* Process-wide diagnostic counters (no citation: instrumentation of this
 * library, not a step of the method).  kernel_launches counts every kernel
 * this library launched.  The svd_* arrays cover the SVD launches, indexed
 * [0] batched Jacobi of the A11 blocks (Eq. 1), [1] FP32 block-Jacobi SVD of
 * an update core (Eqs. 2 / 3, mixed form), [2] FP64 SVD of an update core
 * (FP64 form): launches; summed device time from CUDA events recorded on the
 * launching stream; the dense-SVD flop model 4 p q^2 + 8 q^3 per p x q problem
 * (12 n^3 for an n x n core); and the rotation work done, sweeps x q(q-1)/2
 * pair visits x (12 p + 6 q).  core_resident_launches: core SVD launches that
 * used the resident-block schedule. */
typedef struct {
  uint64_t kernel_launches;
  uint64_t svd_launches[3];
  double svd_ms[3];
  double svd_flops[3];
  double svd_flops_rot[3];
  uint64_t core_resident_launches;
} fastpi_counters;
fastpi_status fastpi_get_counters(fastpi_counters* out);   /* host struct */
void fastpi_reset_counters(void);

/* Diagnostic entry point (no citation: it exposes the library's internal
 * FP32 dense kernel so that it can be checked on its own).
 * C (M x N) = alpha * op(A) op(B) + beta * C on device float32 row-major
 * arrays: op(A) = A (M x K, lda) or, with ta != 0, A^T of a K x M array;
 * op(B) = B (K x N, ldb) or, with tb != 0, B^T of an N x K array.
 * engine 0: SIMT FP32 kernel; 1: tcgen05 TF32 kernel with operands rounded
 * to TF32 (one tensor pass); 3: tcgen05 TF32 kernel with split hi + lo
 * operands (three tensor passes, FP32-level accuracy).  The tensor engines
 * return FASTPI_ERR_ARG on devices other than sm_103, for M, N or K of 2^31
 * or more, for M above 8 388 480 (65 535 tiles of 128 rows), and for M (with
 * ta) or N (without tb) above 2 097 120 (the operand re-layout's grid).  Scratch is allocated on the stream; the call returns
 * after the stream has finished (it checks the kernels' status word). */
fastpi_status fastpi_gemm_f32(int ta, int tb, int64_t M, int64_t N, int64_t K, float alpha, const float* A,
                              int64_t lda, const float* B, int64_t ldb, float beta, float* C, int64_t ldc,
                              int engine, void* cuda_stream);

/* Diagnostic entry point (no citation: it exposes the FP32 SVD of the
 * incremental-update cores of Eqs. 2 and 3 -- block one-sided Jacobi -- so
 * that it can be checked and tuned on its own).  K: device float32 n x n,
 * COLUMN-major (ld n), the matrix; overwritten (scratch).  On return S (host
 * float64[n]) holds the singular values in descending order, U and V (device
 * float32 n x n, column-major) the left and right singular vectors in that
 * order (a column of U is zero where its value is zero).  Tiling: panel = 16
 * or 32 columns per block pair, parts = CTAs of a thread-block cluster that
 * share a block pair's rows (1..8; 0 picks the largest that keeps one round's
 * clusters on the SMs); flags: 1 = resident-block schedule, 2 = the Gram
 * sweep in its IEEE form (two CTA barriers per inner round) instead of the
 * fast one (one barrier, fast rotations), 4 = the single-CTA kernel
 * (panel 16, no clusters).  *sweeps and *ms (may be NULL) receive the sweeps
 * and the CUDA-event time of the Jacobi kernel.  Errors: FASTPI_ERR_ARG
 * (sizes, flags, or a tiling that does not fit: shared memory or co-resident
 * clusters), FASTPI_ERR_NO_CONVERGENCE (sweep cap, or a bounded wait ran
 * out).  The call synchronises the stream. */
fastpi_status fastpi_core_svd_f32(int n, float* K, float* U, double* S, float* V, int panel, int parts, int flags,
                                  int* sweeps, float* ms, void* cuda_stream);

/* Tuning table (no citation: parameters of this implementation, picked on the
 * GPU by the package's autotuner, python -m paper_2011_04235_gb300.autotune).
 * A plain-text file of lines
 *   core   <n_max> <panel> <parts> <resident> <fast>   FP32 core-SVD tiling for n <= n_max
 *   chunk  <prec> <phase> <k_max> <c>                  appends of c border rows (phase 0) /
 *                                                      columns (phase 1) when fastpi_factor
 *                                                      gets chunk 0; prec 0 FP64, 1 mixed
 *   bucket <prec> <dim_max> <class>                    register-tile class of the batched
 *                                                      Jacobi of the A11 blocks
 * The library reads it on first use from $FASTPI_TUNING, else from tuning.txt
 * beside libfastpi.so, else uses built-in defaults (chunk 256).
 * fastpi_load_tuning replaces the table with the file at path (NULL: the
 * built-in defaults), for every handle of the process.  FASTPI_ERR_ARG (and
 * the reason in fastpi_last_error(NULL)) when the file cannot be read or a
 * line is malformed; the table is then unchanged. */
fastpi_status fastpi_load_tuning(const char* path);

/* Message of the last failed call on h (or of the last failed fastpi_create
 * when h is NULL).  Never NULL; valid until the next call on h. */
const char* fastpi_last_error(fastpi_t h);

/* Release every device and host resource of h (NULL is a no-op). */
void fastpi_destroy(fastpi_t h);

#ifdef __cplusplus
}
#endif
#endif /* FASTPI_H */
