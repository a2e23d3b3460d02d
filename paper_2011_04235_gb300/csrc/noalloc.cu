// fastpi_residual_noalloc: |A Z - Y|_F without any device allocation.
//
// Some callers cannot call cudaMalloc (or anything that allocates) at the
// moment they need this number: code that works under a fixed, pre-reserved
// memory budget with the allocator locked, and allocation-free real-time loops
// that must not touch the allocator.  For them this entry point keeps its scratch (one FP64
// partial sum per row of A, plus the total) in a file-scope __device__ array of
// FASTPI_NOALLOC_MAX_ROWS + 1 doubles (8 MiB).  Every GPU that loads the
// library holds that array until the process exits.
//
// The array's host-side name is only a stand-in for the symbol, not a device
// address, so the host never passes it to a kernel.  Every call runs on the
// device of the caller's stream (made current for the call).  The first call
// on each device is its set-up: with that device current it looks the address
// up with cudaGetSymbolAddress, checks the result and caches it for that
// device; every call passes the cached address to the kernels.  With CUDA's
// lazy module loading that first call is also the one that loads this file's
// kernels and the array onto the device, which takes device memory once: make
// one call (m = 0 is enough) before the memory budget is locked.  A
// cudaDeviceReset invalidates the cached address together with everything else
// the process held on that device; do not call this entry point on a device
// after resetting it.  All calls share the array: calls that overlap on the
// GPU (for example on two streams) race on it.  Every call overwrites all the
// entries it reads, so nothing has to be cleared between calls.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "common.cuh"

namespace {

constexpr int64_t kMaxRows = FASTPI_NOALLOC_MAX_ROWS;

static __device__ __align__(256) double g_residual_scratch[kMaxRows + 1];

constexpr int kMaxDevices = 64;
double* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Restores the caller's current device when the call returns.
struct DeviceGuard {
  int saved = -1;
  ~DeviceGuard() {
    if (saved >= 0) (void)cudaSetDevice(saved);
  }
};

// per-row squared residual of A Z - Y (warp per row)
__global__ void k_rows(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                       const double* __restrict__ val, int64_t m, int64_t L, const double* __restrict__ Y, int64_t ldy,
                       const double* __restrict__ Z, int64_t ldz, double* __restrict__ part) {
  const int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= m) return;
  double acc2 = 0;
  for (int64_t l = lane; l < L; l += 32) {
    double s = -Y[i * ldy + l];
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) s = fma(val[e], Z[int64_t(col[e]) * ldz + l], s);
    acc2 = fma(s, s, acc2);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) acc2 += __shfl_xor_sync(0xffffffffu, acc2, o);
  if (lane == 0) part[i] = acc2;
}

// total = sum of part[0..m) in a fixed order (one CTA), written to part[kMaxRows]
__global__ void k_total(double* part, int64_t m) {
  __shared__ double ws[32];
  double s = 0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) s += part[i];
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) t += ws[w];
    part[kMaxRows] = t;
  }
}

}  // namespace

extern "C" fastpi_status fastpi_residual_noalloc(int64_t m, int64_t n, const int64_t* rowptr, const int32_t* colind,
                                                 const double* val, const double* Y, int64_t L, int64_t ldy,
                                                 const double* Z, int64_t ldz, double* out, void* cuda_stream) {
  if (!out || !rowptr || m < 0 || n < 0 || L < 0 || ldy < L || ldz < L) return FASTPI_ERR_ARG;
  if (m > kMaxRows) return FASTPI_ERR_ARG;   // more rows than the static scratch holds
  if (m > 0 && L > 0 && (!Y || !Z || !colind || !val)) return FASTPI_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // the stream's own device (the legacy default stream belongs to the current one)
  DeviceGuard guard;
  int cur = 0, dev = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) return FASTPI_ERR_CUDA;
  if (st == nullptr) {
    dev = cur;
  } else if (cudaStreamGetDevice(st, &dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return FASTPI_ERR_ARG;
  }
  if (dev != cur) {
    if (cudaSetDevice(dev) != cudaSuccess) return FASTPI_ERR_CUDA;
    guard.saved = cur;
  }
  if (dev < 0 || dev >= kMaxDevices) return FASTPI_ERR_CUDA;
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_residual_scratch) != cudaSuccess || !p) {
        (void)cudaGetLastError();
        return FASTPI_ERR_CUDA;
      }
      g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_scratch_ptr[dev];
  }
  const int64_t rows = (m > 0 && L > 0) ? m : 0;
  if (rows > 0) {
    const unsigned grid = unsigned((rows * 32 + 255) / 256);
    k_rows<<<grid, 256, 0, st>>>(rowptr, colind, val, rows, L, Y, ldy, Z, ldz, scratch);
    if (cudaGetLastError() != cudaSuccess) return FASTPI_ERR_CUDA;
  }
  k_total<<<1, 1024, 0, st>>>(scratch, rows);
  if (cudaGetLastError() != cudaSuccess) return FASTPI_ERR_CUDA;
  double tot = 0;
  if (cudaMemcpyAsync(&tot, scratch + kMaxRows, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return FASTPI_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return FASTPI_ERR_CUDA;
  *out = sqrt(tot);
  return FASTPI_OK;
}
