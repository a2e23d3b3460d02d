// Internal declarations shared by the libfastpi translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/fastpi.h"

namespace fastpi {

// ---------------------------------------------------------------- errors
struct Error {
  fastpi_status status;
  std::string msg;
};

[[noreturn]] void fail(fastpi_status s, const std::string& msg);
void check_cuda(cudaError_t e, const char* what, const char* file, int line);
// Checks the launch that precedes it and counts it (every kernel launch in
// this library is followed by exactly one CK_LAUNCH).
void note_launch(const char* file, int line);
#define CK(x) ::fastpi::check_cuda((x), #x, __FILE__, __LINE__)
#define CK_LAUNCH() ::fastpi::note_launch(__FILE__, __LINE__)
// Adds one event-timed SVD launch to the process counters: kind SVD_BLOCKS
// (batched Jacobi of the A11 blocks, Eq. 1), SVD_CORE32 (FP32 block-Jacobi
// core SVD) or SVD_CORE64 (FP64 core SVD); flops_model = 4 p q^2 + 8 q^3 per
// p x q problem, flops_rot = sweeps x q (q - 1) / 2 x (12 p + 6 q).
enum { SVD_BLOCKS = 0, SVD_CORE32 = 1, SVD_CORE64 = 2 };
void note_svd(int kind, double ms, double flops_model, double flops_rot, bool resident = false);
void read_counters(fastpi_counters* out);
void reset_counters();

// Device-side status bits (a word in device memory, read at sync points).
enum : unsigned {
  ST_BARRIER_TIMEOUT = 1u,   // a bounded device-wide barrier gave up
  ST_UF_RETRY_CAP = 2u,      // union-find hooking exceeded its retry cap
  ST_JACOBI_SWEEPS = 4u,     // a Jacobi SVD hit its sweep cap
  ST_BAD_INDEX = 8u          // an index check failed inside a kernel
};

// ---------------------------------------------------------------- memory
// Stream-ordered device buffer (cudaMallocAsync / cudaFreeAsync on the owner's
// stream).  Move-only.
struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t st = nullptr;
  DBuf() = default;
  DBuf(size_t nbytes, cudaStream_t s);
  ~DBuf();
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept { *this = static_cast<DBuf&&>(o); }
  DBuf& operator=(DBuf&& o) noexcept;
  void reset();
  template <typename T> T* as() const { return static_cast<T*>(p); }
};

template <typename T>
struct DArr {
  DBuf b;
  int64_t n = 0;
  DArr() = default;
  DArr(int64_t count, cudaStream_t s) : b(size_t(count > 0 ? count : 1) * sizeof(T), s), n(count) {}
  T* get() const { return b.as<T>(); }
  operator T*() const { return get(); }
};

// ---------------------------------------------------------------- context
struct Factors;   // defined in factor.cu

}  // namespace fastpi

struct fastpi_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  int64_t m = 0, n = 0, nnz = 0;
  // A in CSR (device) and its CSC transpose (rows ascending within a column)
  fastpi::DArr<int64_t> rowptr, colptr;
  fastpi::DArr<int32_t> col, csc_row;
  fastpi::DArr<double> val, csc_val;
  fastpi::DArr<unsigned> dstatus;   // device status word
  // results
  bool factored = false;
  bool reordered = false;   // fac->R holds Algorithm 2's result (after fastpi_reorder or fastpi_factor)
  bool has_matrix = true;   // false for a handle made from given factors (apply only)
  fastpi::Factors* fac = nullptr;
  fastpi_info info{};
  std::string last_error;
};

namespace fastpi {

// ---------------------------------------------------------------- primitives
// Exclusive prefix sum of n values (out may alias in).  Returns nothing; the
// total is out[n-1] + in[n-1] (callers that need it pass n+1 with a trailing 0).
void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t st);
void exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, cudaStream_t st);

// Stable LSD radix sort of (key, value) pairs by the low `bits` bits of key.
// keys/vals are sorted in place (scratch buffers allocated internally).
void radix_sort_pairs(uint32_t* keys, uint32_t* vals, int64_t n, int bits, cudaStream_t st);

// Number of bits needed to represent values in [0, maxval].
int bits_for(uint64_t maxval);

// Lets `func` launch with up to the device's opt-in maximum of dynamic shared
// memory.  The attribute belongs to the function for the whole process, so it
// is always raised to the maximum, never set to one launch's size (a
// concurrent launch from another host thread could be left below its need).
void allow_max_dynamic_smem(const void* func);

// Copy device->host of a small POD value / array on the stream and wait.
void d2h_sync(void* dst, const void* src, size_t bytes, cudaStream_t st);

int ceil_div_i(int64_t a, int64_t b);

// An unsigned image of a double whose order is the order of the values
// (non-NaN): the sign bit flipped for non-negative values, all bits flipped
// for negative ones.  Comparing these on the integer pipe replaces FP64
// compares, which GB300 runs on its narrow FP64 pipe.
__device__ __forceinline__ unsigned long long order_key(double v) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double order_value(unsigned long long k) {
  return __longlong_as_double(static_cast<long long>((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k));
}

}  // namespace fastpi
