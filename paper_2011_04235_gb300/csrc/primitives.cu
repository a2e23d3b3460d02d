// Runtime support and data-parallel primitives: errors, stream-ordered
// buffers, exclusive scans and a stable LSD radix sort.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "common.cuh"

namespace fastpi {

void fail(fastpi_status s, const std::string& msg) { throw Error{s, msg}; }

namespace {
std::atomic<uint64_t> g_launches{0};
std::mutex g_prof_mu;
uint64_t g_svd_launches[3] = {0, 0, 0};
double g_svd_ms[3] = {0, 0, 0}, g_svd_flops[3] = {0, 0, 0}, g_svd_flops_rot[3] = {0, 0, 0};
uint64_t g_core_resident = 0;
}  // namespace

void note_launch(const char* file, int line) {
  check_cuda(cudaGetLastError(), "kernel launch", file, line);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void note_svd(int kind, double ms, double flops_model, double flops_rot, bool resident) {
  if (kind < 0 || kind > 2) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  ++g_svd_launches[kind];
  g_svd_ms[kind] += ms;
  g_svd_flops[kind] += flops_model;
  g_svd_flops_rot[kind] += flops_rot;
  if (resident) ++g_core_resident;
}

void read_counters(fastpi_counters* out) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  out->kernel_launches = g_launches.load();
  for (int k = 0; k < 3; ++k) {
    out->svd_launches[k] = g_svd_launches[k];
    out->svd_ms[k] = g_svd_ms[k];
    out->svd_flops[k] = g_svd_flops[k];
    out->svd_flops_rot[k] = g_svd_flops_rot[k];
  }
  out->core_resident_launches = g_core_resident;
}

void reset_counters() {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_launches.store(0);
  for (int k = 0; k < 3; ++k) {
    g_svd_launches[k] = 0;
    g_svd_ms[k] = g_svd_flops[k] = g_svd_flops_rot[k] = 0;
  }
  g_core_resident = 0;
}

void allow_max_dynamic_smem(const void* func) {
  int dev = 0, mx = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa;
  CK(cudaFuncGetAttributes(&fa, func));
  // the opt-in limit covers static and dynamic shared memory together
  CK(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, mx - int(fa.sharedSizeBytes)));
}

void check_cuda(cudaError_t e, const char* what, const char* file, int line) {
  if (e == cudaSuccess) return;
  fastpi_status s = (e == cudaErrorMemoryAllocation) ? FASTPI_ERR_OOM : FASTPI_ERR_CUDA;
  char buf[512];
  snprintf(buf, sizeof buf, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  throw Error{s, buf};
}

DBuf::DBuf(size_t nbytes, cudaStream_t s) : bytes(nbytes), st(s) {
  if (nbytes == 0) nbytes = 1;
  cudaError_t e = cudaMallocAsync(&p, nbytes, s);
  if (e != cudaSuccess) {
    p = nullptr;
    (void)cudaGetLastError();
    char buf[160];
    snprintf(buf, sizeof buf, "device allocation of %zu bytes failed: %s", nbytes, cudaGetErrorString(e));
    throw Error{FASTPI_ERR_OOM, buf};
  }
}

void DBuf::reset() {
  if (p) cudaFreeAsync(p, st);
  p = nullptr;
  bytes = 0;
}

DBuf::~DBuf() { reset(); }

DBuf& DBuf::operator=(DBuf&& o) noexcept {
  if (this != &o) {
    reset();
    p = o.p;
    bytes = o.bytes;
    st = o.st;
    o.p = nullptr;
    o.bytes = 0;
  }
  return *this;
}

void d2h_sync(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
}

int ceil_div_i(int64_t a, int64_t b) { return int((a + b - 1) / b); }

int bits_for(uint64_t maxval) {
  int b = 0;
  while (b < 64 && (maxval >> b) != 0) ++b;
  return b;
}

// ------------------------------------------------------------------ scan
namespace {

constexpr int SCAN_BS = 1024;
constexpr int SCAN_IPT = 4;
constexpr int SCAN_TILE = SCAN_BS * SCAN_IPT;

template <typename T>
__device__ T warp_inclusive(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Block-wide exclusive scan of one value per thread; returns the block total in *total.
template <typename T>
__device__ T block_exclusive(T v, T* total) {
  __shared__ T wsum[33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T inc = warp_inclusive(v);
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x >> 5;
    T x = lane < nw ? wsum[lane] : T(0);
    T xi = warp_inclusive(x);
    if (lane < nw) wsum[lane] = xi - x;
    if (lane == nw - 1) wsum[32] = xi;
  }
  __syncthreads();
  T res = wsum[w] + inc - v;
  if (total) *total = wsum[32];
  __syncthreads();
  return res;
}

template <typename T>
__global__ void k_tile_sums(const T* in, int64_t n, T* sums) {
  int64_t base = int64_t(blockIdx.x) * SCAN_TILE;
  T s = 0;
  for (int i = 0; i < SCAN_IPT; ++i) {
    int64_t idx = base + int64_t(i) * SCAN_BS + threadIdx.x;
    if (idx < n) s += in[idx];
  }
  T tot;
  block_exclusive(s, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

template <typename T>
__global__ void k_tile_scan(const T* in, T* out, int64_t n, const T* offs) {
  int64_t base = int64_t(blockIdx.x) * SCAN_TILE + int64_t(threadIdx.x) * SCAN_IPT;
  T v[SCAN_IPT];
  T s = 0;
  for (int i = 0; i < SCAN_IPT; ++i) {
    int64_t idx = base + i;
    v[i] = idx < n ? in[idx] : T(0);
    s += v[i];
  }
  T pre = block_exclusive(s, (T*)nullptr);
  T run = pre + (offs ? offs[blockIdx.x] : T(0));
  for (int i = 0; i < SCAN_IPT; ++i) {
    int64_t idx = base + i;
    if (idx < n) out[idx] = run;
    run += v[i];
  }
}

template <typename T>
void scan_impl(const T* in, T* out, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (tiles == 1) {
    k_tile_scan<T><<<1, SCAN_BS, 0, st>>>(in, out, n, nullptr);
    CK_LAUNCH();
    return;
  }
  DArr<T> sums(tiles, st);
  k_tile_sums<T><<<unsigned(tiles), SCAN_BS, 0, st>>>(in, n, sums);
  CK_LAUNCH();
  scan_impl<T>(sums, sums, tiles, st);
  k_tile_scan<T><<<unsigned(tiles), SCAN_BS, 0, st>>>(in, out, n, sums);
  CK_LAUNCH();
}

}  // namespace

void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t st) {
  scan_impl<int64_t>(in, out, n, st);
}
void exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, cudaStream_t st) {
  scan_impl<int32_t>(in, out, n, st);
}

// ------------------------------------------------------------------ radix sort
// Stable LSD radix sort, 8 bits per pass.  Each CTA owns a tile of
// RS_TILE = 8 warps x 8 steps x 32 lanes consecutive elements.  Per pass:
//   1. histogram of each tile's digits  -> counts[digit * ntiles + tile]
//   2. exclusive scan of counts (digit-major) -> global start of (digit, tile)
//   3. scatter: each warp walks its 256 consecutive elements 32 at a time;
//      peers with the same digit are ranked by lane (match.any), and a
//      per-warp running count per digit plus the exclusive sum over earlier
//      warps of the tile keep the order of equal digits (stability).
namespace {

constexpr int RS_WARPS = 8;
constexpr int RS_STEPS = 8;
constexpr int RS_TILE = RS_WARPS * RS_STEPS * 32;

__global__ void k_radix_hist(const uint32_t* keys, int64_t n, int shift, int ntiles, int32_t* counts) {
  __shared__ int32_t h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  int64_t base = int64_t(blockIdx.x) * RS_TILE;
  for (int i = threadIdx.x; i < RS_TILE; i += blockDim.x) {
    int64_t idx = base + i;
    if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += blockDim.x) counts[int64_t(d) * ntiles + blockIdx.x] = h[d];
}

__global__ void k_radix_scatter(const uint32_t* kin, const uint32_t* vin, uint32_t* kout, uint32_t* vout,
                                int64_t n, int shift, int ntiles, const int32_t* offs) {
  __shared__ int32_t wcnt[RS_WARPS][256];
  __shared__ int32_t toff[256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < RS_WARPS * 256; i += blockDim.x) (&wcnt[0][0])[i] = 0;
  for (int d = threadIdx.x; d < 256; d += blockDim.x) toff[d] = offs[int64_t(d) * ntiles + blockIdx.x];
  __syncthreads();
  const int64_t base = int64_t(blockIdx.x) * RS_TILE + int64_t(w) * RS_STEPS * 32;
  uint32_t key[RS_STEPS], val[RS_STEPS];
  int32_t rank[RS_STEPS];
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int s = 0; s < RS_STEPS; ++s) {
    int64_t idx = base + s * 32 + lane;
    bool valid = idx < n;
    key[s] = valid ? kin[idx] : 0u;
    val[s] = valid ? vin[idx] : 0u;
    unsigned d = valid ? ((key[s] >> shift) & 255u) : 0x100u;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    int pre = valid ? wcnt[w][d] : 0;
    __syncwarp();
    int leader = 31 - __clz(peers);
    if (valid && lane == leader) wcnt[w][d] = pre + __popc(peers);
    __syncwarp();
    rank[s] = pre + __popc(peers & lt);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += blockDim.x) {
    int run = 0;
    for (int ww = 0; ww < RS_WARPS; ++ww) {
      int t = wcnt[ww][d];
      wcnt[ww][d] = run;
      run += t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int s = 0; s < RS_STEPS; ++s) {
    int64_t idx = base + s * 32 + lane;
    if (idx < n) {
      unsigned d = (key[s] >> shift) & 255u;
      int64_t pos = int64_t(toff[d]) + wcnt[w][d] + rank[s];
      kout[pos] = key[s];
      vout[pos] = val[s];
    }
  }
}

}  // namespace

void radix_sort_pairs(uint32_t* keys, uint32_t* vals, int64_t n, int bits, cudaStream_t st) {
  if (n <= 1 || bits <= 0) return;
  if (n > (int64_t(1) << 31) - 1) fail(FASTPI_ERR_ARG, "radix sort: too many elements");
  int ntiles = ceil_div_i(n, RS_TILE);
  DArr<uint32_t> k2(n, st), v2(n, st);
  DArr<int32_t> counts(int64_t(ntiles) * 256, st);
  uint32_t *ka = keys, *va = vals, *kb = k2, *vb = v2;
  int passes = (bits + 7) / 8;
  for (int p = 0; p < passes; ++p) {
    int shift = 8 * p;
    k_radix_hist<<<ntiles, 256, 0, st>>>(ka, n, shift, ntiles, counts);
    CK_LAUNCH();
    exclusive_scan_i32(counts, counts, int64_t(ntiles) * 256, st);
    k_radix_scatter<<<ntiles, RS_WARPS * 32, 0, st>>>(ka, va, kb, vb, n, shift, ntiles, counts);
    CK_LAUNCH();
    uint32_t* t = ka; ka = kb; kb = t;
    t = va; va = vb; vb = t;
  }
  if (ka != keys) {
    CK(cudaMemcpyAsync(keys, ka, size_t(n) * 4, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(vals, va, size_t(n) * 4, cudaMemcpyDeviceToDevice, st));
  }
}

}  // namespace fastpi
