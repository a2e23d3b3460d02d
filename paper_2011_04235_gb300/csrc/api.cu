// C ABI of libfastpi (declared in include/fastpi.h).  Every entry point
// converts internal errors into a status code and a message.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "dense.cuh"
#include "factor.cuh"
#include "jacobi.cuh"
#include "tuning.cuh"

using namespace fastpi;

namespace {

thread_local std::string g_create_error;

fastpi_status handle_error(fastpi_t h, const Error& e) {
  if (h)
    h->last_error = e.msg;
  else
    g_create_error = e.msg;
  return e.status;
}

#define API_BEGIN try {
#define API_END(h)                                        \
  }                                                       \
  catch (const Error& e) {                                \
    return handle_error(h, e);                            \
  }                                                       \
  catch (const std::exception& e) {                       \
    return handle_error(h, Error{FASTPI_ERR_CUDA, e.what()}); \
  }                                                       \
  return FASTPI_OK;

void require(bool ok, fastpi_status s, const char* msg) {
  if (!ok) fail(s, msg);
}

void require_factored(fastpi_t h) { require(h->factored && h->fac, FASTPI_ERR_STATE, "call fastpi_factor first"); }
void require_reordered(fastpi_t h) {
  require(h->reordered && h->fac, FASTPI_ERR_STATE, "call fastpi_reorder or fastpi_factor first");
}

void use_device(fastpi_t h) { CK(cudaSetDevice(h->device)); }

}  // namespace

extern "C" {

fastpi_status fastpi_create(fastpi_t* out, int64_t m, int64_t n, int64_t nnz, const int64_t* rowptr,
                            const int32_t* colind, const double* val, int ptrs_on_device, void* cuda_stream) {
  if (out) *out = nullptr;
  fastpi_ctx* h = nullptr;
  try {
    require(out != nullptr, FASTPI_ERR_ARG, "out is NULL");
    require(m >= 1 && n >= 1 && nnz >= 0, FASTPI_ERR_ARG, "need m >= 1, n >= 1, nnz >= 0");
    require(m + n < (int64_t(1) << 31) - 1, FASTPI_ERR_ARG, "m + n must fit in int32");
    require(nnz <= int64_t(m) * int64_t(n), FASTPI_ERR_ARG, "nnz exceeds m * n");
    require(nnz < (int64_t(1) << 31) - 1, FASTPI_ERR_ARG, "nnz must fit in int32");
    require(rowptr && (nnz == 0 || (colind && val)), FASTPI_ERR_ARG, "null CSR array");
    h = new fastpi_ctx();
    CK(cudaGetDevice(&h->device));
    CK(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    {
      // keep freed stream-ordered memory in the pool between calls
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, h->device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
      }
      (void)cudaGetLastError();
    }
    h->m = m;
    h->n = n;
    h->nnz = nnz;
    cudaStream_t st = h->stream;
    h->rowptr = DArr<int64_t>(m + 1, st);
    h->col = DArr<int32_t>(nnz, st);
    h->val = DArr<double>(nnz, st);
    h->dstatus = DArr<unsigned>(1, st);
    cudaMemcpyKind kind = ptrs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(h->rowptr.get(), rowptr, size_t(m + 1) * 8, kind, st));
    if (nnz > 0) {
      CK(cudaMemcpyAsync(h->col.get(), colind, size_t(nnz) * 4, kind, st));
      CK(cudaMemcpyAsync(h->val.get(), val, size_t(nnz) * 8, kind, st));
    }
    validate_csr(h);
    build_csc(h);
    *out = h;
    return FASTPI_OK;
  } catch (const Error& e) {
    g_create_error = e.msg;
    delete h;
    return e.status;
  } catch (const std::exception& e) {
    g_create_error = e.what();
    delete h;
    return FASTPI_ERR_CUDA;
  }
}

fastpi_status fastpi_factor(fastpi_t h, int64_t r, double k, fastpi_precision prec, int64_t chunk_row,
                            int64_t chunk_col) {
  if (!h) return FASTPI_ERR_ARG;
  API_BEGIN
  use_device(h);
  require(r >= 1, FASTPI_ERR_ARG, "target rank r must be >= 1");
  require(k > 0.0 && k < 1.0 && std::isfinite(k), FASTPI_ERR_ARG, "hub ratio k must lie in (0, 1)");
  require(prec == FASTPI_FP64 || prec == FASTPI_MIXED_TF32, FASTPI_ERR_ARG, "unknown precision");
  require(chunk_row >= 0 && chunk_col >= 0, FASTPI_ERR_ARG, "chunk sizes must be >= 0");
  require(h->has_matrix, FASTPI_ERR_STATE, "handle made from factors has no matrix");
  h->factored = false;
  h->reordered = false;
  fastpi::factor(h, r, k, prec, chunk_row, chunk_col);
  API_END(h)
}

fastpi_status fastpi_factor_batched(fastpi_t* hs, int count, const int64_t* r, double k, fastpi_precision prec,
                                    int64_t chunk_row, int64_t chunk_col, int concurrency,
                                    fastpi_status* status_out) {
  try {
    require(hs != nullptr && r != nullptr && count >= 1, FASTPI_ERR_ARG, "need count >= 1 handles and ranks");
    require(k > 0.0 && k < 1.0 && std::isfinite(k), FASTPI_ERR_ARG, "hub ratio k must lie in (0, 1)");
    require(prec == FASTPI_FP64 || prec == FASTPI_MIXED_TF32, FASTPI_ERR_ARG, "unknown precision");
    require(chunk_row >= 0 && chunk_col >= 0, FASTPI_ERR_ARG, "chunk sizes must be >= 0");
    for (int i = 0; i < count; ++i) {
      require(hs[i] != nullptr, FASTPI_ERR_ARG, "null handle in the batch");
      require(r[i] >= 1, FASTPI_ERR_ARG, "every target rank must be >= 1");
      require(hs[i]->device == hs[0]->device, FASTPI_ERR_ARG, "all handles of a batch must be on one device");
      require(hs[i]->has_matrix, FASTPI_ERR_ARG, "a handle made from factors has no matrix");
      for (int j = 0; j < i; ++j) require(hs[j] != hs[i], FASTPI_ERR_ARG, "a handle appears twice in the batch");
    }
  } catch (const Error& e) {
    g_create_error = e.msg;
    return e.status;
  }
  std::vector<fastpi_status> st;
  std::vector<std::string> msg;
  try {
    st.assign(count, FASTPI_OK);
    msg.resize(count);
    CK(cudaSetDevice(hs[0]->device));
    fastpi::factor_batched(hs, count, r, k, prec, chunk_row, chunk_col, concurrency > 0 ? concurrency : 4,
                           st.data(), msg.data());
  } catch (const Error& e) {
    g_create_error = e.msg;
    return e.status;
  } catch (const std::exception& e) {   // e.g. a host thread that could not start
    g_create_error = e.what();
    return FASTPI_ERR_CUDA;
  }
  fastpi_status first = FASTPI_OK;
  for (int i = 0; i < count; ++i) {
    if (status_out) status_out[i] = st[i];
    if (st[i] != FASTPI_OK) {
      hs[i]->last_error = msg[i];
      if (first == FASTPI_OK) {
        first = st[i];
        g_create_error = "batch member " + std::to_string(i) + ": " + msg[i];
      }
    }
  }
  return first;
}

fastpi_status fastpi_create_from_factors(fastpi_t* out, int64_t m, int64_t n, int64_t r, const double* S,
                                        const double* U, int64_t ldu, const double* V, int64_t ldv,
                                        fastpi_precision prec, int ptrs_on_device, void* cuda_stream) {
  if (out) *out = nullptr;
  fastpi_ctx* h = nullptr;
  try {
    require(out != nullptr, FASTPI_ERR_ARG, "out is NULL");
    require(m >= 1 && n >= 1 && r >= 0 && r <= std::min(m, n), FASTPI_ERR_ARG, "need m, n >= 1, 0 <= r <= min(m, n)");
    require(prec == FASTPI_FP64 || prec == FASTPI_MIXED_TF32, FASTPI_ERR_ARG, "unknown precision");
    require(r == 0 || (S && U && V), FASTPI_ERR_ARG, "null factor array");
    require(ldu >= r && ldv >= r, FASTPI_ERR_ARG, "leading dimension smaller than r");
    for (int64_t i = 0; i < r; ++i) {
      require(std::isfinite(S[i]) && S[i] >= 0.0, FASTPI_ERR_ARG, "singular values must be finite and >= 0");
      require(i == 0 || S[i] <= S[i - 1], FASTPI_ERR_ARG, "singular values must be in descending order");
    }
    h = new fastpi_ctx();
    CK(cudaGetDevice(&h->device));
    CK(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    h->m = m;
    h->n = n;
    h->nnz = 0;
    h->has_matrix = false;
    h->dstatus = DArr<unsigned>(1, h->stream);
    fastpi::load_factors(h, r, S, U, ldu, V, ldv, prec, ptrs_on_device != 0);
    *out = h;
    return FASTPI_OK;
  } catch (const Error& e) {
    g_create_error = e.msg;
    delete h;
    return e.status;
  } catch (const std::exception& e) {
    g_create_error = e.what();
    delete h;
    return FASTPI_ERR_CUDA;
  }
}

fastpi_status fastpi_truncate(fastpi_t h, int64_t r) {
  if (!h) return FASTPI_ERR_ARG;
  API_BEGIN
  use_device(h);
  require_factored(h);
  require(r >= 1, FASTPI_ERR_ARG, "rank must be >= 1");
  fastpi::truncate_factors(h, r);
  API_END(h)
}

fastpi_status fastpi_reorder(fastpi_t h, double k) {
  if (!h) return FASTPI_ERR_ARG;
  API_BEGIN
  use_device(h);
  require(k > 0.0 && k < 1.0 && std::isfinite(k), FASTPI_ERR_ARG, "hub ratio k must lie in (0, 1)");
  require(h->has_matrix, FASTPI_ERR_STATE, "handle made from factors has no matrix");
  h->factored = false;
  h->reordered = false;
  fastpi::reorder_only(h, k);
  API_END(h)
}

fastpi_status fastpi_block_svd(fastpi_t h, int64_t r, double k, fastpi_precision prec, double* sigma, int64_t cap,
                               int64_t* S_out) {
  if (!h) return FASTPI_ERR_ARG;
  API_BEGIN
  use_device(h);
  require(r >= 1, FASTPI_ERR_ARG, "target rank r must be >= 1");
  require(k > 0.0 && k < 1.0 && std::isfinite(k), FASTPI_ERR_ARG, "hub ratio k must lie in (0, 1)");
  require(prec == FASTPI_FP64 || prec == FASTPI_MIXED_TF32, FASTPI_ERR_ARG, "unknown precision");
  require(S_out != nullptr && cap >= 0 && (cap == 0 || sigma != nullptr), FASTPI_ERR_ARG,
          "need S_out, and sigma when cap > 0");
  require(h->has_matrix, FASTPI_ERR_STATE, "handle made from factors has no matrix");
  h->factored = false;
  h->reordered = false;
  std::vector<double> sig;
  fastpi::block_svd_only(h, r, k, prec, sig);
  *S_out = int64_t(sig.size());
  require(int64_t(sig.size()) <= cap, FASTPI_ERR_ARG, "sigma holds fewer than S values (S returned in S_out)");
  if (!sig.empty()) std::memcpy(sigma, sig.data(), sig.size() * sizeof(double));
  API_END(h)
}

fastpi_status fastpi_apply(fastpi_t h, const double* Y, int64_t L, int64_t ldy, double* Z, int64_t ldz) {
  if (!h) return FASTPI_ERR_ARG;
  API_BEGIN
  use_device(h);
  require_factored(h);
  require(L >= 0 && ldy >= L && ldz >= L, FASTPI_ERR_ARG, "need L >= 0, ldy >= L, ldz >= L");
  require(L == 0 || (Y && Z), FASTPI_ERR_ARG, "null Y or Z");
  apply_dense(h, Y, L, ldy, Z, ldz);
  API_END(h)
}

fastpi_status fastpi_apply_host(fastpi_t h, const double* Y, int64_t L, int64_t ldy, double* Z, int64_t ldz) {
  if (!h) return FASTPI_ERR_ARG;
  API_BEGIN
  use_device(h);
  require_factored(h);
  require(L >= 0 && ldy >= L && ldz >= L, FASTPI_ERR_ARG, "need L >= 0, ldy >= L, ldz >= L");
  require(L == 0 || (Y && Z), FASTPI_ERR_ARG, "null Y or Z");
  if (L == 0) return FASTPI_OK;
  cudaStream_t st = h->stream;
  DArr<double> dY(h->m * L, st), dZ(h->n * L, st);
  CK(cudaMemcpy2DAsync(dY.get(), size_t(L) * 8, Y, size_t(ldy) * 8, size_t(L) * 8, size_t(h->m),
                       cudaMemcpyHostToDevice, st));
  apply_dense(h, dY.get(), L, L, dZ.get(), L);
  CK(cudaMemcpy2DAsync(Z, size_t(ldz) * 8, dZ.get(), size_t(L) * 8, size_t(L) * 8, size_t(h->n),
                       cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  API_END(h)
}

fastpi_status fastpi_apply_csr(fastpi_t h, int64_t L, int64_t nnz_y, const int64_t* yrowptr, const int32_t* ycol,
                               const double* yval, double* Z, int64_t ldz) {
  if (!h) return FASTPI_ERR_ARG;
  API_BEGIN
  use_device(h);
  require_factored(h);
  require(L >= 0 && ldz >= L && nnz_y >= 0, FASTPI_ERR_ARG, "need L >= 0, ldz >= L, nnz_y >= 0");
  require(L < (int64_t(1) << 31) - 1 && nnz_y < (int64_t(1) << 31) - 1, FASTPI_ERR_ARG,
          "L and nnz_y must fit in int32");
  require(L == 0 || (yrowptr && Z && (nnz_y == 0 || (ycol && yval))), FASTPI_ERR_ARG, "null pointer");
  apply_csr(h, L, nnz_y, yrowptr, ycol, yval, Z, ldz);
  API_END(h)
}

fastpi_status fastpi_residual(fastpi_t h, const double* Y, int64_t L, int64_t ldy, const double* Z, int64_t ldz,
                              double* out) {
  if (!h) return FASTPI_ERR_ARG;
  API_BEGIN
  use_device(h);
  require(out != nullptr, FASTPI_ERR_ARG, "out is NULL");
  require(L >= 0 && ldy >= L && ldz >= L, FASTPI_ERR_ARG, "need L >= 0, ldy >= L, ldz >= L");
  require(L == 0 || (Y && Z), FASTPI_ERR_ARG, "null Y or Z");
  require(h->has_matrix, FASTPI_ERR_STATE, "handle made from factors has no matrix");
  *out = residual(h, Y, L, ldy, Z, ldz);
  API_END(h)
}

fastpi_status fastpi_spmm(fastpi_t h, const double* X, int64_t L, int64_t ldx, double* out, int64_t ldo) {
  if (!h) return FASTPI_ERR_ARG;
  API_BEGIN
  use_device(h);
  require(L >= 0 && ldx >= L && ldo >= L, FASTPI_ERR_ARG, "need L >= 0, ldx >= L, ldo >= L");
  require(L == 0 || (X && out), FASTPI_ERR_ARG, "null X or out");
  require(h->has_matrix, FASTPI_ERR_STATE, "handle made from factors has no matrix");
  spmm(h, X, L, ldx, out, ldo);
  CK(cudaStreamSynchronize(h->stream));
  API_END(h)
}

fastpi_status fastpi_recon_error(fastpi_t h, double* out) {
  if (!h) return FASTPI_ERR_ARG;
  API_BEGIN
  use_device(h);
  require(out != nullptr, FASTPI_ERR_ARG, "out is NULL");
  require_factored(h);
  require(h->has_matrix, FASTPI_ERR_STATE, "handle made from factors has no matrix");
  *out = recon_error(h);
  API_END(h)
}

fastpi_status fastpi_get_rank(fastpi_t h, int64_t* r_out) {
  if (!h) return FASTPI_ERR_ARG;
  API_BEGIN
  require_factored(h);
  require(r_out != nullptr, FASTPI_ERR_ARG, "r_out is NULL");
  *r_out = h->fac->rank;
  API_END(h)
}

fastpi_status fastpi_get_S(fastpi_t h, double* S) {
  if (!h) return FASTPI_ERR_ARG;
  API_BEGIN
  require_factored(h);
  require(S != nullptr || h->fac->rank == 0, FASTPI_ERR_ARG, "S is NULL");
  if (h->fac->rank > 0) std::memcpy(S, h->fac->S.data(), size_t(h->fac->rank) * 8);
  API_END(h)
}

static void get_factor(fastpi_t h, bool isU, double* out, int64_t ld) {
  Factors& F = *h->fac;
  const int64_t rows = isU ? F.m : F.n, r = F.rank, ldr = r > 0 ? r : 1;
  require(ld >= r, FASTPI_ERR_ARG, "leading dimension smaller than the rank");
  require(out != nullptr || r == 0, FASTPI_ERR_ARG, "output is NULL");
  if (r == 0) return;
  cudaStream_t st = h->stream;
  if (F.prec == FASTPI_FP64)
    copy2d<double, double>(st, rows, r, isU ? F.U64.get() : F.V64.get(), ldr, out, ld);
  else
    copy2d<double, float>(st, rows, r, isU ? F.U32.get() : F.V32.get(), ldr, out, ld);
  CK(cudaStreamSynchronize(st));
}

fastpi_status fastpi_get_U(fastpi_t h, double* U, int64_t ldu) {
  if (!h) return FASTPI_ERR_ARG;
  API_BEGIN
  use_device(h);
  require_factored(h);
  get_factor(h, true, U, ldu);
  API_END(h)
}

fastpi_status fastpi_get_V(fastpi_t h, double* V, int64_t ldv) {
  if (!h) return FASTPI_ERR_ARG;
  API_BEGIN
  use_device(h);
  require_factored(h);
  get_factor(h, false, V, ldv);
  API_END(h)
}

fastpi_status fastpi_get_perm(fastpi_t h, int32_t* row_order, int32_t* col_order, int64_t* m2, int64_t* n2) {
  if (!h) return FASTPI_ERR_ARG;
  API_BEGIN
  use_device(h);
  require_reordered(h);
  const Reordering& R = h->fac->R;
  cudaStream_t st = h->stream;
  if (row_order) CK(cudaMemcpyAsync(row_order, R.row_order.get(), size_t(R.m) * 4, cudaMemcpyDeviceToHost, st));
  if (col_order) CK(cudaMemcpyAsync(col_order, R.col_order.get(), size_t(R.n) * 4, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (m2) *m2 = R.m - R.m1;
  if (n2) *n2 = R.n - R.n1;
  API_END(h)
}

fastpi_status fastpi_get_blocks(fastpi_t h, int64_t* B, int64_t* row_off, int64_t* col_off) {
  if (!h) return FASTPI_ERR_ARG;
  API_BEGIN
  require_reordered(h);
  const Reordering& R = h->fac->R;
  if (B) *B = R.num_blocks;
  if (row_off) std::memcpy(row_off, R.row_off.data(), R.row_off.size() * 8);
  if (col_off) std::memcpy(col_off, R.col_off.data(), R.col_off.size() * 8);
  API_END(h)
}

fastpi_status fastpi_get_info(fastpi_t h, fastpi_info* info) {
  if (!h) return FASTPI_ERR_ARG;
  API_BEGIN
  require((h->reordered || h->factored) && h->fac, FASTPI_ERR_STATE, "call fastpi_reorder or fastpi_factor first");
  require(info != nullptr, FASTPI_ERR_ARG, "info is NULL");
  *info = h->info;
  API_END(h)
}

fastpi_status fastpi_get_counters(fastpi_counters* out) {
  if (!out) return FASTPI_ERR_ARG;
  read_counters(out);
  return FASTPI_OK;
}

void fastpi_reset_counters(void) { reset_counters(); }

fastpi_status fastpi_gemm_f32(int ta, int tb, int64_t M, int64_t N, int64_t K, float alpha, const float* A,
                              int64_t lda, const float* B, int64_t ldb, float beta, float* C, int64_t ldc,
                              int engine, void* cuda_stream) {
  try {
    require(M >= 0 && N >= 0 && K >= 0, FASTPI_ERR_ARG, "negative size");
    require(engine == 0 || engine == 1 || engine == 3, FASTPI_ERR_ARG, "engine must be 0, 1 or 3");
    require(ldc >= N && lda >= (ta ? M : K) && ldb >= (tb ? K : N), FASTPI_ERR_ARG, "leading dimension too small");
    require(M * N == 0 || C != nullptr, FASTPI_ERR_ARG, "C is NULL");
    require(M * N * K == 0 || (A != nullptr && B != nullptr), FASTPI_ERR_ARG, "A or B is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (engine == 0) {
      gemm<float>(st, ta != 0, tb != 0, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    } else {
      require(M * N == 0 || K == 0 || gemm_tf32_supported(ta != 0, tb != 0, M, N, K, lda, ldb, ldc, A, B, C),
              FASTPI_ERR_ARG, "the tensor-core GEMM needs an sm_103 device and sizes within its grid limits");
      gemm_tf32(st, ta != 0, tb != 0, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, engine);
    }
    CK(cudaStreamSynchronize(st));
    const unsigned stat = gemm_tc_status(st, true);
    require(stat == 0, FASTPI_ERR_CUDA, "tensor-core GEMM: a bounded wait ran out");
  } catch (const Error& e) {
    g_create_error = e.msg;
    return e.status;
  } catch (const std::exception& e) {
    g_create_error = e.what();
    return FASTPI_ERR_CUDA;
  }
  return FASTPI_OK;
}

fastpi_status fastpi_core_svd_f32(int n, float* K, float* U, double* S, float* V, int panel, int parts, int flags,
                                  int* sweeps, float* ms, void* cuda_stream) {
  try {
    require(n >= 2 && n <= 8192, FASTPI_ERR_ARG, "need 2 <= n <= 8192");
    require(K && U && S && V, FASTPI_ERR_ARG, "null pointer");
    require(panel == 16 || panel == 32, FASTPI_ERR_ARG, "panel must be 16 or 32");
    require(parts >= 0 && parts <= 8, FASTPI_ERR_ARG, "parts must lie in [0, 8]");
    require((flags & ~7) == 0, FASTPI_ERR_ARG, "unknown flag");
    require(!((flags & 4) && panel != 16), FASTPI_ERR_ARG, "the single-CTA kernel has panel 16");
    fastpi_ctx ctx;
    CK(cudaGetDevice(&ctx.device));
    CK(cudaDeviceGetAttribute(&ctx.num_sms, cudaDevAttrMultiProcessorCount, ctx.device));
    ctx.stream = static_cast<cudaStream_t>(cuda_stream);
    ctx.has_matrix = false;
    ctx.dstatus = DArr<unsigned>(1, ctx.stream);
    CoreTiling tl;
    tl.panel = panel;
    tl.parts = parts;
    tl.resident = (flags & 1) != 0;
    tl.fast_solve = (flags & 2) == 0;
    tl.single_cta = (flags & 4) != 0;
    tl.strict = true;
    DArr<float> J(int64_t(n) * n, ctx.stream);
    DArr<double> sig(n, ctx.stream);
    DArr<int32_t> perm(n, ctx.stream);
    JacobiStats js;
    float t = 0;
    int sw = 0;
    require(jacobi_svd_block(&ctx, K, J.get(), n, sig.get(), perm.get(), &js, &tl, &t, &sw), FASTPI_ERR_ARG,
            "this tiling does not fit the core (shared memory or co-resident clusters)");
    core_vectors_f32(&ctx, n, K, J.get(), sig.get(), perm.get(), U, V);
    CK(cudaMemcpyAsync(S, sig.get(), size_t(n) * 8, cudaMemcpyDeviceToHost, ctx.stream));
    CK(cudaStreamSynchronize(ctx.stream));
    if (sweeps) *sweeps = sw;
    if (ms) *ms = t;
    require(!js.hit_cap, FASTPI_ERR_NO_CONVERGENCE, "core SVD: sweep cap reached");
  } catch (const Error& e) {
    g_create_error = e.msg;
    return e.status;
  } catch (const std::exception& e) {
    g_create_error = e.what();
    return FASTPI_ERR_CUDA;
  }
  return FASTPI_OK;
}

fastpi_status fastpi_load_tuning(const char* path) {
  std::string why;
  if (!load_tuning(path, &why)) {
    g_create_error = why;
    return FASTPI_ERR_ARG;
  }
  return FASTPI_OK;
}

const char* fastpi_last_error(fastpi_t h) {
  if (!h) return g_create_error.c_str();
  return h->last_error.c_str();
}

void fastpi_destroy(fastpi_t h) {
  if (!h) return;
  cudaSetDevice(h->device);
  cudaStreamSynchronize(h->stream);
  delete h->fac;
  h->fac = nullptr;
  cudaStream_t st = h->stream;
  delete h;
  cudaStreamSynchronize(st);
}

}  // extern "C"
