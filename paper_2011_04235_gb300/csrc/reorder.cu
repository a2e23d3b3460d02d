// Hub-and-spoke reordering (Algorithm 2, Section 3.2), the split of the
// reordered matrix (Section 3.3), and the create-time CSC build.
//
// Node ids: instance (row) i -> i, feature (column) j -> m + j.  One
// iteration on the active graph G:
//   degrees in G -> hubs = the first ceil(k|V|) active nodes of each side in
//   (degree desc, id asc) order, placed at the back with the first hub last ->
//   connected components of G minus hubs by union-find (roots always link to
//   the smaller id, so a component's root is its minimum id = its label) ->
//   GCC = most nodes, ties to the smallest label -> non-giant components take
//   the front positions in (label asc, id asc) order, one A11 block each ->
//   G := GCC; stop when |I_GCC| < m_hub or |F_GCC| < n_hub or G is empty.
// The final GCC fills the middle positions (ascending ids) as the last block.
// Every decision is integer, so the permutation is bit-exact and
// deterministic: all orderings come from stable radix sorts of keys in id order.
#include <cmath>
#include <cstdio>

#include "internal.cuh"

namespace fastpi {
namespace {

constexpr int BS = 256;
inline unsigned nblk(int64_t n, int bs = BS) { return n > 0 ? unsigned((n + bs - 1) / bs) : 1u; }

// ------------------------------------------------------------ create-time
__global__ void k_validate(const int64_t* rowptr, const int32_t* col, int64_t m, int64_t n, int64_t nnz,
                           unsigned* bad) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i > m) return;
  if (i == 0 && rowptr[0] != 0) atomicOr(bad, 1u);
  if (i == m) {
    if (rowptr[m] != nnz) atomicOr(bad, 1u);
    return;
  }
  int64_t a = rowptr[i], b = rowptr[i + 1];
  if (b < a || a < 0 || b > nnz) {
    atomicOr(bad, 1u);
    return;
  }
  int32_t prev = -1;
  for (int64_t e = a; e < b; ++e) {
    int32_t c = col[e];
    if (c < 0 || c >= n || c <= prev) {
      atomicOr(bad, 2u);
      return;
    }
    prev = c;
  }
}

__global__ void k_row_of_nz(const int64_t* rowptr, int64_t m, int32_t* nz_row) {
  int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (w >= m) return;
  for (int64_t e = rowptr[w] + lane; e < rowptr[w + 1]; e += 32) nz_row[e] = int32_t(w);
}

__global__ void k_col_count(const int32_t* col, int64_t nnz, int64_t* cnt) {
  int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e < nnz) atomicAdd((unsigned long long*)&cnt[col[e]], 1ull);
}

__global__ void k_iota_u32(uint32_t* a, int64_t n) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) a[i] = uint32_t(i);
}

__global__ void k_keys_from_col(const int32_t* col, int64_t nnz, uint32_t* keys) {
  int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e < nnz) keys[e] = uint32_t(col[e]);
}

__global__ void k_csc_fill(const uint32_t* perm, const int32_t* nz_row, const double* val, int64_t nnz,
                           int32_t* csc_row, double* csc_val) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < nnz) {
    uint32_t e = perm[t];
    csc_row[t] = nz_row[e];
    csc_val[t] = val[e];
  }
}

// ------------------------------------------------------------ iteration
__global__ void k_deg_rows(const int64_t* rowptr, const int32_t* col, const uint8_t* act, int64_t m,
                           int32_t* deg) {
  int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (w >= m) return;
  int cnt = 0;
  if (act[w]) {
    for (int64_t e = rowptr[w] + lane; e < rowptr[w + 1]; e += 32) cnt += act[m + col[e]];
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (lane == 0) deg[w] = cnt;
}

__global__ void k_deg_cols(const int64_t* colptr, const int32_t* row, const uint8_t* act, int64_t m, int64_t n,
                           int32_t* deg) {
  int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (w >= n) return;
  int cnt = 0;
  if (act[m + w]) {
    for (int64_t e = colptr[w] + lane; e < colptr[w + 1]; e += 32) cnt += act[row[e]];
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (lane == 0) deg[m + w] = cnt;
}

// flags[i] = act[base + i] (and, when label != null, label[base+i] != gcc)
__global__ void k_flags_active(const uint8_t* act, const int32_t* label, int32_t gcc, int64_t base, int64_t cnt,
                               int32_t* flags) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= cnt) return;
  int f = act[base + i] != 0;
  if (label && f) f = label[base + i] != gcc;
  flags[i] = f;
}

// One CTA for a small compaction (cnt <= CS_MAX): the flags of
// k_flags_active (roots = 1: those of k_flags_roots instead), a block-wide
// prefix sum and the scatter of k_compact, in one launch.  Thread t owns the
// consecutive indices [t E, (t + 1) E), so the output keeps the ascending
// order of i, as the three-launch form does.
constexpr int CS_THREADS = 1024;
constexpr int CS_PER = 32;
constexpr int64_t CS_MAX = int64_t(CS_THREADS) * CS_PER;
__global__ void __launch_bounds__(CS_THREADS) k_compact_small(const uint8_t* act, const int32_t* label, int32_t gcc,
                                                              int roots, int64_t base, int64_t cnt,
                                                              const int32_t* keysrc, int32_t key_bias, int key_neg,
                                                              uint32_t* out_ids, uint32_t* out_keys) {
  __shared__ int wsum[CS_THREADS / 32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int E = int((cnt + CS_THREADS - 1) / CS_THREADS);
  const int64_t i0 = int64_t(tid) * E;
  unsigned bits = 0;   // E <= 32
  for (int e = 0; e < E; ++e) {
    const int64_t i = i0 + e;
    if (i >= cnt) break;
    const int64_t v = base + i;
    int f;
    if (roots)
      f = act[v] && label[v] == int32_t(v) && int32_t(v) != gcc;
    else {
      f = act[v] != 0;
      if (label && f) f = label[v] != gcc;
    }
    bits |= unsigned(f) << e;
  }
  const int own = __popc(bits);
  int inc = own;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  if (w == 0) {
    const int x = wsum[lane];
    int xi = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, xi, o);
      if (lane >= o) xi += t;
    }
    wsum[lane] = xi - x;
  }
  __syncthreads();
  int p = wsum[w] + inc - own;
  for (int e = 0; e < E; ++e) {
    if (!((bits >> e) & 1u)) continue;
    const int64_t i = i0 + e;
    out_ids[p] = uint32_t(i);
    if (out_keys) {
      const int32_t kv = keysrc[base + i];
      out_keys[p] = uint32_t(key_neg ? key_bias - kv : kv);
    }
    ++p;
  }
}

// One CTA: sorts n <= SS_MAX (key, id) pairs by key, then id, with a bitonic
// network on the 64-bit words (key << 32 | id) in shared memory.  Where the
// ids arrive in ascending order (every caller here: they come from an
// ascending compaction) and are distinct, this is exactly the stable sort by
// key that radix_sort_pairs computes.
constexpr int SS_THREADS = 1024;
constexpr int64_t SS_MAX = 2048;   // beyond it the network's n log^2 n shared-memory traffic loses to the radix passes
__global__ void __launch_bounds__(SS_THREADS) k_sort_small(uint32_t* keys, uint32_t* ids, int n, int np2) {
  extern __shared__ unsigned long long sk[];
  for (int i = threadIdx.x; i < np2; i += SS_THREADS)
    sk[i] = i < n ? ((static_cast<unsigned long long>(keys[i]) << 32) | ids[i]) : ~0ull;
  __syncthreads();
  for (int size = 2; size <= np2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < np2 / 2; t += SS_THREADS) {
        const int lo = 2 * t - (t & (stride - 1));   // index with bit `stride` clear
        const int hi = lo + stride;
        const bool up = (lo & size) == 0;
        const unsigned long long a = sk[lo], b = sk[hi];
        if ((a > b) == up) {
          sk[lo] = b;
          sk[hi] = a;
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += SS_THREADS) {
    keys[i] = uint32_t(sk[i] >> 32);
    ids[i] = uint32_t(sk[i]);
  }
}

// Sorts the (key, id) pairs of the reordering (ids ascending and distinct on
// entry): one CTA when they fit, else the multi-pass radix sort.
void sort_key_id(uint32_t* keys, uint32_t* ids, int64_t n, int bits, cudaStream_t st) {
  if (n <= 1) return;
  if (n <= SS_MAX) {
    int np2 = 2;
    while (np2 < n) np2 <<= 1;
    const size_t smem = size_t(np2) * 8;
    if (smem > 48 * 1024) allow_max_dynamic_smem((const void*)k_sort_small);
    k_sort_small<<<1, SS_THREADS, smem, st>>>(keys, ids, int(n), np2);
    CK_LAUNCH();
    return;
  }
  radix_sort_pairs(keys, ids, n, bits, st);
}

// roots of non-giant components: active v with label[v] == v and v != gcc
__global__ void k_flags_roots(const uint8_t* act, const int32_t* label, int32_t gcc, int64_t cnt, int32_t* flags) {
  int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (v >= cnt) return;
  flags[v] = (act[v] && label[v] == int32_t(v) && int32_t(v) != gcc) ? 1 : 0;
}

// scatter i (plus key) to position pos[i] where flags[i]; write count to *count
__global__ void k_compact(const int32_t* flags, const int32_t* pos, int64_t cnt, const int32_t* keysrc,
                          int64_t key_base, int32_t key_bias, int key_neg, uint32_t* out_ids, uint32_t* out_keys,
                          int32_t* count) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= cnt) return;
  if (i == cnt - 1) *count = pos[i] + flags[i];
  if (!flags[i]) return;
  int32_t p = pos[i];
  out_ids[p] = uint32_t(i);
  if (out_keys) {
    int32_t kv = keysrc[key_base + i];
    out_keys[p] = uint32_t(key_neg ? key_bias - kv : kv);
  }
}

__global__ void k_place_hubs(const uint32_t* sorted_ids, int64_t count, int64_t back, int64_t node_base,
                             int32_t* order, uint8_t* act) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= count) return;
  uint32_t id = sorted_ids[t];
  order[back - 1 - t] = int32_t(id);
  act[node_base + id] = 0;
}

__global__ void k_place_front(const uint32_t* sorted_ids, int64_t count, int64_t front, int32_t* order) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < count) order[front + t] = int32_t(sorted_ids[t]);
}

__device__ __forceinline__ int32_t uf_find(int32_t* parent, int32_t x) {
  // path halving; parents only ever decrease towards the root, so the racy
  // plain stores keep every pointer valid
  int32_t p = parent[x];
  while (p != x) {
    int32_t gp = parent[p];
    if (gp != p) parent[x] = gp;
    x = p;
    p = gp;
  }
  return x;
}

// Union-find hooking of the active edges, by rows: one warp per row i, the
// lanes over its nonzeros; the larger root is always linked under the smaller.
// A row that is no longer active (a hub or a component placed earlier) is
// skipped with one load instead of one per nonzero, which matters more with
// every iteration.  Whatever order the hooks land in, every component ends up
// rooted at its minimum id.
__global__ void k_cc_hook_rows(const int64_t* rowptr, const int32_t* col, const uint8_t* act, int64_t m,
                               int32_t* parent, unsigned* status) {
  const int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= m || !act[w]) return;
  const int32_t i = int32_t(w);
  for (int64_t e = rowptr[w] + lane; e < rowptr[w + 1]; e += 32) {
    const int32_t j = int32_t(m) + col[e];
    if (!act[j]) continue;
    int32_t ru = uf_find(parent, i), rv = uf_find(parent, j);
    int guard = 0;
    while (ru != rv) {
      if (ru > rv) {
        const int32_t t = ru;
        ru = rv;
        rv = t;
      }
      const int32_t old = atomicCAS(&parent[rv], rv, ru);
      if (old == rv) break;
      rv = uf_find(parent, old);
      ru = uf_find(parent, ru);
      if (++guard > (1 << 20)) {
        atomicOr(status, ST_UF_RETRY_CAP);
        break;
      }
    }
  }
}

__global__ void k_cc_label(const uint8_t* act, int64_t N, int32_t* parent, int32_t* label, int64_t m,
                           int32_t* cntT, int32_t* cntF) {
  int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (v >= N) return;
  if (!act[v]) {
    label[v] = -1;
    return;
  }
  int32_t r = uf_find(parent, int32_t(v));
  label[v] = r;
  atomicAdd(v < m ? &cntT[r] : &cntF[r], 1);
}

__global__ void k_gcc(const uint8_t* act, const int32_t* label, const int32_t* cntT, const int32_t* cntF,
                      int64_t N, unsigned long long* best, int32_t* nroots) {
  int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (v >= N) return;
  if (act[v] && label[v] == int32_t(v)) {
    unsigned long long size = unsigned(cntT[v] + cntF[v]);
    unsigned long long key = (size << 32) | (0xFFFFFFFFull - unsigned(v));
    atomicMax(best, key);
    atomicAdd(nroots, 1);
  }
}

__global__ void k_block_counts(const uint32_t* roots, int64_t nroots, const int32_t* cntT, const int32_t* cntF,
                               int64_t* bT, int64_t* bF) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= nroots) return;
  uint32_t v = roots[t];
  bT[t] = cntT[v];
  bF[t] = cntF[v];
}

// After the exclusive scans of bT / bF: block t spans rows
// [fT + bT[t], fT + bT[t] + cnt) -> write the END offsets at nb + 1 + t.
__global__ void k_block_offsets(const uint32_t* roots, int64_t nroots, const int32_t* cntT, const int32_t* cntF,
                                const int64_t* exT, const int64_t* exF, int64_t fT, int64_t fF, int64_t nb,
                                int64_t* row_off, int64_t* col_off) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= nroots) return;
  uint32_t v = roots[t];
  row_off[nb + 1 + t] = fT + exT[t] + cntT[v];
  col_off[nb + 1 + t] = fF + exF[t] + cntF[v];
}

__global__ void k_keep_gcc(uint8_t* act, const int32_t* label, int32_t gcc, int64_t N) {
  int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (v < N && act[v]) act[v] = (label[v] == gcc) ? 1 : 0;
}

// out = {GCC label (-1: G' empty), its instances, its features, the number of
// the other (non-giant) components}
__global__ void k_summary(const unsigned long long* best, const int32_t* cntT, const int32_t* cntF,
                          const int32_t* nroots, int64_t* out) {
  unsigned long long b = *best;
  int32_t gcc = b ? int32_t(0xFFFFFFFFull - (b & 0xFFFFFFFFull)) : -1;
  out[0] = gcc;
  out[1] = gcc >= 0 ? cntT[gcc] : 0;
  out[2] = gcc >= 0 ? cntF[gcc] : 0;
  out[3] = *nroots - (gcc >= 0 ? 1 : 0);
}

__global__ void k_inverse_perm(const int32_t* order, int64_t n, int32_t* pos) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < n) pos[order[t]] = int32_t(t);
}

// A second stream and two events for the parts of an iteration in which the
// rows and the columns are handled independently (fork: the side stream waits
// for the main one; join: the main one waits for the side one).  Destroyed
// with the object; a stream destroyed with work pending finishes that work.
struct SideStream {
  cudaStream_t st = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  SideStream() {
    CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
  }
  ~SideStream() {
    if (join) cudaEventDestroy(join);
    if (fork) cudaEventDestroy(fork);
    if (st) cudaStreamDestroy(st);
  }
  SideStream(const SideStream&) = delete;
  SideStream& operator=(const SideStream&) = delete;
  void start(cudaStream_t main) {
    CK(cudaEventRecord(fork, main));
    CK(cudaStreamWaitEvent(st, fork, 0));
  }
  void finish(cudaStream_t main) {
    CK(cudaEventRecord(join, st));
    CK(cudaStreamWaitEvent(main, join, 0));
  }
};

// Per-iteration reset of the component state: parent[v] = v and zero counts,
// the GCC key and the root count.
__global__ void k_cc_reset(int32_t* parent, int32_t* cntT, int32_t* cntF, int64_t N, unsigned long long* best,
                           int32_t* nroots) {
  int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (v == 0) {
    *best = 0ull;
    *nroots = 0;
  }
  if (v < N) {
    parent[v] = int32_t(v);
    cntT[v] = 0;
    cntF[v] = 0;
  }
}

}  // namespace

// ------------------------------------------------------------ public
void validate_csr(fastpi_ctx* h) {
  cudaStream_t st = h->stream;
  CK(cudaMemsetAsync(h->dstatus, 0, sizeof(unsigned), st));
  k_validate<<<nblk(h->m + 1), BS, 0, st>>>(h->rowptr, h->col, h->m, h->n, h->nnz, h->dstatus);
  CK_LAUNCH();
  unsigned bad = 0;
  d2h_sync(&bad, h->dstatus, sizeof bad, st);
  if (bad & 1u) fail(FASTPI_ERR_CSR, "malformed CSR: rowptr must start at 0, be non-decreasing and end at nnz");
  if (bad & 2u) fail(FASTPI_ERR_CSR, "malformed CSR: column index out of range, or columns not strictly increasing within a row");
}

void build_csc(fastpi_ctx* h) {
  cudaStream_t st = h->stream;
  const int64_t m = h->m, n = h->n, nnz = h->nnz;
  DArr<int32_t> nz_row(nnz, st);
  if (nnz > 0) {
    k_row_of_nz<<<nblk(m * 32), BS, 0, st>>>(h->rowptr, m, nz_row);
    CK_LAUNCH();
  }
  h->colptr = DArr<int64_t>(n + 1, st);
  CK(cudaMemsetAsync(h->colptr.get(), 0, size_t(n + 1) * 8, st));
  h->csc_row = DArr<int32_t>(nnz, st);
  h->csc_val = DArr<double>(nnz, st);
  if (nnz > 0) {
    k_col_count<<<nblk(nnz), BS, 0, st>>>(h->col, nnz, h->colptr);
    CK_LAUNCH();
  }
  exclusive_scan_i64(h->colptr, h->colptr, n + 1, st);
  if (nnz > 0) {
    DArr<uint32_t> keys(nnz, st), perm(nnz, st);
    k_keys_from_col<<<nblk(nnz), BS, 0, st>>>(h->col, nnz, keys);
    CK_LAUNCH();
    k_iota_u32<<<nblk(nnz), BS, 0, st>>>(perm, nnz);
    CK_LAUNCH();
    radix_sort_pairs(keys, perm, nnz, bits_for(uint64_t(n > 0 ? n - 1 : 0)), st);
    k_csc_fill<<<nblk(nnz), BS, 0, st>>>(perm, nz_row, h->val, nnz, h->csc_row, h->csc_val);
    CK_LAUNCH();
  }
  CK(cudaStreamSynchronize(st));
}

void run_reorder(fastpi_ctx* h, double k, Reordering& R) {
  cudaStream_t st = h->stream;
  const int64_t m = h->m, n = h->n, nnz = h->nnz, N = m + n;
  R.m = m;
  R.n = n;
  R.row_order = DArr<int32_t>(m, st);
  R.col_order = DArr<int32_t>(n, st);
  R.row_pos = DArr<int32_t>(m, st);
  R.col_pos = DArr<int32_t>(n, st);

  DArr<uint8_t> act(N, st);
  CK(cudaMemsetAsync(act.get(), 1, size_t(N), st));
  DArr<int32_t> deg(N, st), parent(N, st), label(N, st), cntT(N, st), cntF(N, st);
  const int64_t cap = N + 1;
  // scratch of the main stream (rows, components) and of the side stream (columns)
  DArr<int32_t> flags(cap, st), pos(cap, st), dcount(4, st);
  DArr<uint32_t> ids(cap, st), keys(cap, st);
  DArr<int32_t> flags2(cap, st), pos2(cap, st), dcount2(4, st);
  DArr<uint32_t> ids2(cap, st), keys2(cap, st);
  SideStream side;
  cudaStream_t st2 = side.st;
  DArr<int64_t> bT(cap, st), bF(cap, st), d_row_off(cap + 1, st), d_col_off(cap + 1, st), summ(4, st);
  DArr<unsigned long long> best(1, st);
  DArr<int32_t> dnroots(1, st);
  CK(cudaMemsetAsync(d_row_off.get(), 0, 8, st));
  CK(cudaMemsetAsync(d_col_off.get(), 0, 8, st));

  // compact the active nodes of one side (plus keys); `known` is the number
  // of nodes that pass, which the host always knows from the counts of the
  // iteration (active instances / features, the GCC's size), so no read-back
  // side 0: rows on the main stream, side 1: columns on the side stream
  auto compact = [&](int sd, int64_t base, int64_t cnt, const int32_t* lab, int32_t gcc, const int32_t* keysrc,
                     int32_t key_bias, int key_neg, int64_t known) -> int64_t {
    if (cnt == 0 || known == 0) return 0;
    cudaStream_t cs = sd ? st2 : st;
    if (cnt <= CS_MAX) {
      k_compact_small<<<1, CS_THREADS, 0, cs>>>(act, lab, gcc, 0, base, cnt, keysrc, key_bias, key_neg,
                                                sd ? ids2.get() : ids.get(),
                                                keysrc ? (sd ? keys2.get() : keys.get()) : nullptr);
      CK_LAUNCH();
      return known;
    }
    int32_t* fl = sd ? flags2.get() : flags.get();
    int32_t* ps = sd ? pos2.get() : pos.get();
    k_flags_active<<<nblk(cnt), BS, 0, cs>>>(act, lab, gcc, base, cnt, fl);
    CK_LAUNCH();
    exclusive_scan_i32(fl, ps, cnt, cs);
    k_compact<<<nblk(cnt), BS, 0, cs>>>(fl, ps, cnt, keysrc, base, key_bias, key_neg, sd ? ids2.get() : ids.get(),
                                        keysrc ? (sd ? keys2.get() : keys.get()) : nullptr,
                                        sd ? dcount2.get() : dcount.get());
    CK_LAUNCH();
    return known;
  };

  int64_t fT = 0, fF = 0, bTc = m, bFc = n, nb = 0, nI = m, nF = n, it = 0;
  int32_t gcc = -1;
  while (nI + nF > 0) {
    ++it;
    const int64_t m_hub = int64_t(std::ceil(k * double(nI)));
    const int64_t n_hub = int64_t(std::ceil(k * double(nF)));
    // degrees in the current graph
    k_deg_rows<<<nblk(m * 32), BS, 0, st>>>(h->rowptr, h->col, act, m, deg);
    CK_LAUNCH();
    k_deg_cols<<<nblk(n * 32), BS, 0, st>>>(h->colptr, h->csc_row, act, m, n, deg);
    CK_LAUNCH();
    // hubs (key = n - deg so that ascending key = degree descending): the
    // rows here, the columns on the side stream (each side reads and clears
    // only its own part of act and deg)
    side.start(st);
    if (m_hub > 0) {
      int64_t c = compact(0, 0, m, nullptr, 0, deg, int32_t(n), 1, nI);
      sort_key_id(keys, ids, c, bits_for(uint64_t(n)), st);
      k_place_hubs<<<nblk(m_hub), BS, 0, st>>>(ids, m_hub, bTc, 0, R.row_order, act);
      CK_LAUNCH();
      bTc -= m_hub;
    }
    if (n_hub > 0) {
      int64_t c = compact(1, m, n, nullptr, 0, deg, int32_t(m), 1, nF);
      sort_key_id(keys2, ids2, c, bits_for(uint64_t(m)), st2);
      k_place_hubs<<<nblk(n_hub), BS, 0, st2>>>(ids2, n_hub, bFc, m, R.col_order, act);
      CK_LAUNCH();
      bFc -= n_hub;
    }
    // connected components of G' (the reset overlaps the columns' hubs)
    k_cc_reset<<<nblk(N), BS, 0, st>>>(parent, cntT, cntF, N, best, dnroots);
    CK_LAUNCH();
    side.finish(st);
    if (nnz > 0) {
      k_cc_hook_rows<<<nblk(m * 32), BS, 0, st>>>(h->rowptr, h->col, act, m, parent, h->dstatus);
      CK_LAUNCH();
    }
    k_cc_label<<<nblk(N), BS, 0, st>>>(act, N, parent, label, m, cntT, cntF);
    CK_LAUNCH();
    k_gcc<<<nblk(N), BS, 0, st>>>(act, label, cntT, cntF, N, best, dnroots);
    CK_LAUNCH();
    k_summary<<<1, 1, 0, st>>>(best, cntT, cntF, dnroots, summ);
    CK_LAUNCH();
    int64_t sm[4];
    d2h_sync(sm, summ, sizeof sm, st);
    gcc = int32_t(sm[0]);
    if (gcc < 0) {   // G' is empty
      nI = nF = 0;
      break;
    }
    // non-giant components: front positions in (label asc, id asc)
    // rows of the non-giant components: the active rows less the hubs just
    // placed and the GCC's rows (likewise for the features)
    // (the columns on the side stream again)
    side.start(st);
    int64_t cT = compact(0, 0, m, label, gcc, label, 0, 0, nI - m_hub - sm[1]);
    if (cT > 0) {
      sort_key_id(keys, ids, cT, bits_for(uint64_t(N)), st);
      k_place_front<<<nblk(cT), BS, 0, st>>>(ids, cT, fT, R.row_order);
      CK_LAUNCH();
    }
    int64_t cF = compact(1, m, n, label, gcc, label, 0, 0, nF - n_hub - sm[2]);
    if (cF > 0) {
      sort_key_id(keys2, ids2, cF, bits_for(uint64_t(N)), st2);
      k_place_front<<<nblk(cF), BS, 0, st2>>>(ids2, cF, fF, R.col_order);
      CK_LAUNCH();
    }
    // one block per non-giant component, in ascending label (= root id) order
    const int64_t nroots = sm[3];
    if (nroots > 0) {
      if (N <= CS_MAX) {
        k_compact_small<<<1, CS_THREADS, 0, st>>>(act, label, gcc, 1, 0, N, nullptr, 0, 0, ids, nullptr);
        CK_LAUNCH();
      } else {
        k_flags_roots<<<nblk(N), BS, 0, st>>>(act, label, gcc, N, flags);
        CK_LAUNCH();
        exclusive_scan_i32(flags, pos, N, st);
        k_compact<<<nblk(N), BS, 0, st>>>(flags, pos, N, nullptr, 0, 0, 0, ids, nullptr, dcount);
        CK_LAUNCH();
      }
      k_block_counts<<<nblk(nroots), BS, 0, st>>>(ids, nroots, cntT, cntF, bT, bF);
      CK_LAUNCH();
      exclusive_scan_i64(bT, bT, nroots, st);
      exclusive_scan_i64(bF, bF, nroots, st);
      k_block_offsets<<<nblk(nroots), BS, 0, st>>>(ids, nroots, cntT, cntF, bT, bF, fT, fF, nb, d_row_off,
                                                   d_col_off);
      CK_LAUNCH();
    }
    nb += nroots;
    fT += cT;
    fF += cF;
    side.finish(st);
    // recurse on the GCC
    k_keep_gcc<<<nblk(N), BS, 0, st>>>(act, label, gcc, N);
    CK_LAUNCH();
    nI = sm[1];
    nF = sm[2];
    if (nI < m_hub || nF < n_hub) break;
  }
  // the final GCC fills the middle positions and forms the last A11 block
  if (nI + nF > 0) {
    int64_t c = compact(0, 0, m, nullptr, 0, nullptr, 0, 0, nI);
    if (c > 0) {
      k_place_front<<<nblk(c), BS, 0, st>>>(ids, c, fT, R.row_order);
      CK_LAUNCH();
    }
    fT += c;
    int64_t c2 = compact(0, m, n, nullptr, 0, nullptr, 0, 0, nF);
    if (c2 > 0) {
      k_place_front<<<nblk(c2), BS, 0, st>>>(ids, c2, fF, R.col_order);
      CK_LAUNCH();
    }
    fF += c2;
    int64_t offs[2] = {fT, fF};
    CK(cudaMemcpyAsync(d_row_off.get() + nb + 1, &offs[0], 8, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_col_off.get() + nb + 1, &offs[1], 8, cudaMemcpyHostToDevice, st));
    ++nb;
  }
  if (fT != bTc || fF != bFc) {
    char buf[200];
    snprintf(buf, sizeof buf, "reordering cursors did not meet (rows %lld/%lld, cols %lld/%lld)", (long long)fT,
             (long long)bTc, (long long)fF, (long long)bFc);
    fail(FASTPI_ERR_NO_CONVERGENCE, buf);
  }
  unsigned stat = 0;
  d2h_sync(&stat, h->dstatus, 4, st);
  if (stat & ST_UF_RETRY_CAP) fail(FASTPI_ERR_NO_CONVERGENCE, "union-find hooking exceeded its retry cap");
  R.m1 = fT;
  R.n1 = fF;
  R.iterations = it;
  R.num_blocks = nb;
  R.row_off.resize(nb + 1);
  R.col_off.resize(nb + 1);
  CK(cudaMemcpyAsync(R.row_off.data(), d_row_off, size_t(nb + 1) * 8, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(R.col_off.data(), d_col_off, size_t(nb + 1) * 8, cudaMemcpyDeviceToHost, st));
  if (m > 0) {
    k_inverse_perm<<<nblk(m), BS, 0, st>>>(R.row_order, m, R.row_pos);
    CK_LAUNCH();
  }
  if (n > 0) {
    k_inverse_perm<<<nblk(n), BS, 0, st>>>(R.col_order, n, R.col_pos);
    CK_LAUNCH();
  }
  CK_LAUNCH();
  CK(cudaStreamSynchronize(st));
}

// ------------------------------------------------------------ split
namespace {

// A21: new rows i' in [m1, m): entries with col_pos < n1, in CSR order.
__global__ void k_a21_count(const int64_t* rowptr, const int32_t* col, const int32_t* row_order,
                            const int32_t* col_pos, int64_t m1, int64_t m2, int64_t n1, int64_t* cnt) {
  int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (w >= m2) return;
  int32_t orig = row_order[m1 + w];
  int c = 0;
  for (int64_t e = rowptr[orig] + lane; e < rowptr[orig + 1]; e += 32) c += col_pos[col[e]] < n1;
#pragma unroll
  for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) cnt[w] = c;
}

__global__ void k_a21_fill(const int64_t* rowptr, const int32_t* col, const double* val, const int32_t* row_order,
                           const int32_t* col_pos, int64_t m1, int64_t m2, int64_t n1, const int64_t* ptr,
                           int32_t* idx, double* v) {
  int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (w >= m2) return;
  int32_t orig = row_order[m1 + w];
  int64_t out = ptr[w];
  const int64_t a = rowptr[orig], b = rowptr[orig + 1];
  for (int64_t e0 = a; e0 < b; e0 += 32) {
    int64_t e = e0 + lane;
    int32_t cp = e < b ? col_pos[col[e]] : INT32_MAX;
    bool keep = e < b && cp < n1;
    unsigned mask = __ballot_sync(0xffffffffu, keep);
    if (keep) {
      int64_t o = out + __popc(mask & ((1u << lane) - 1u));
      idx[o] = cp;
      v[o] = val[e];
    }
    out += __popc(mask);
  }
}

// T: new cols j' in [n1, n): all entries of the original column, rows mapped.
__global__ void k_t_count(const int64_t* colptr, const int32_t* col_order, int64_t n1, int64_t n2, int64_t* cnt) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n2) return;
  int32_t orig = col_order[n1 + t];
  cnt[t] = colptr[orig + 1] - colptr[orig];
}

__global__ void k_t_fill(const int64_t* colptr, const int32_t* csc_row, const double* csc_val,
                         const int32_t* col_order, const int32_t* row_pos, int64_t n1, int64_t n2,
                         const int64_t* ptr, int32_t* idx, double* v) {
  int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (w >= n2) return;
  int32_t orig = col_order[n1 + w];
  int64_t a = colptr[orig], b = colptr[orig + 1], o = ptr[w];
  for (int64_t e = a + lane; e < b; e += 32) {
    idx[o + (e - a)] = row_pos[csc_row[e]];
    v[o + (e - a)] = csc_val[e];
  }
}

__global__ void k_blk_of(const int64_t* off, int64_t B, int32_t* blk_of) {
  int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (b >= B) return;
  for (int64_t i = off[b]; i < off[b + 1]; ++i) blk_of[i] = int32_t(b);
}

__global__ void k_blocks_fill(const int32_t* nz_row, const int32_t* col, const double* val, int64_t nnz,
                              const int32_t* row_pos, const int32_t* col_pos, int64_t m1, int64_t n1,
                              const int32_t* blk_of_row, const int64_t* row_off, const int64_t* col_off,
                              const int64_t* data_off, double* data) {
  int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= nnz) return;
  int32_t i = row_pos[nz_row[e]], j = col_pos[col[e]];
  if (i >= m1 || j >= n1) return;
  int32_t b = blk_of_row[i];
  int64_t off = data_off[b];
  if (off < 0) return;   // s_b == 0: not stored
  int64_t mb = row_off[b + 1] - row_off[b], nbk = col_off[b + 1] - col_off[b];
  int64_t li = i - row_off[b], lj = j - col_off[b];
  if (mb >= nbk)
    data[off + li + lj * mb] = val[e];
  else
    data[off + lj + li * nbk] = val[e];
}

}  // namespace

void split_border(fastpi_ctx* h, const Reordering& R, SparseCols& A21, SparseCols& T) {
  cudaStream_t st = h->stream;
  const int64_t m = R.m, n = R.n, m1 = R.m1, n1 = R.n1, m2 = m - m1, n2 = n - n1;
  A21.ncols = m2;
  A21.nrows = n1;
  A21.ptr = DArr<int64_t>(m2 + 1, st);
  CK(cudaMemsetAsync(A21.ptr.get(), 0, size_t(m2 + 1) * 8, st));
  if (m2 > 0) {
    k_a21_count<<<nblk(m2 * 32), BS, 0, st>>>(h->rowptr, h->col, R.row_order, R.col_pos, m1, m2, n1, A21.ptr);
    CK_LAUNCH();
  }
  exclusive_scan_i64(A21.ptr, A21.ptr, m2 + 1, st);
  A21.ptr_h.resize(m2 + 1);
  CK(cudaMemcpyAsync(A21.ptr_h.data(), A21.ptr, size_t(m2 + 1) * 8, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  A21.nnz = A21.ptr_h[m2];
  A21.idx = DArr<int32_t>(A21.nnz, st);
  A21.val = DArr<double>(A21.nnz, st);
  if (m2 > 0 && A21.nnz > 0) {
    k_a21_fill<<<nblk(m2 * 32), BS, 0, st>>>(h->rowptr, h->col, h->val, R.row_order, R.col_pos, m1, m2, n1,
                                             A21.ptr, A21.idx, A21.val);
    CK_LAUNCH();
  }
  T.ncols = n2;
  T.nrows = m;
  T.ptr = DArr<int64_t>(n2 + 1, st);
  CK(cudaMemsetAsync(T.ptr.get(), 0, size_t(n2 + 1) * 8, st));
  if (n2 > 0) {
    k_t_count<<<nblk(n2), BS, 0, st>>>(h->colptr, R.col_order, n1, n2, T.ptr);
    CK_LAUNCH();
  }
  exclusive_scan_i64(T.ptr, T.ptr, n2 + 1, st);
  T.ptr_h.resize(n2 + 1);
  CK(cudaMemcpyAsync(T.ptr_h.data(), T.ptr, size_t(n2 + 1) * 8, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  T.nnz = T.ptr_h[n2];
  T.idx = DArr<int32_t>(T.nnz, st);
  T.val = DArr<double>(T.nnz, st);
  if (n2 > 0 && T.nnz > 0) {
    k_t_fill<<<nblk(n2 * 32), BS, 0, st>>>(h->colptr, h->csc_row, h->csc_val, R.col_order, R.row_pos, n1, n2,
                                           T.ptr, T.idx, T.val);
    CK_LAUNCH();
  }
}

void extract_blocks(fastpi_ctx* h, const Reordering& R, int64_t r, A11Blocks& blk) {
  cudaStream_t st = h->stream;
  const int64_t B = R.num_blocks, n = R.n;
  blk.B = B;
  blk.m_b.resize(B);
  blk.n_b.resize(B);
  blk.s_b.resize(B);
  blk.data_off.resize(B);
  blk.s_off.resize(B + 1);
  int64_t total = 0, S = 0;
  for (int64_t b = 0; b < B; ++b) {
    int64_t mb = R.row_off[b + 1] - R.row_off[b], nb = R.col_off[b + 1] - R.col_off[b];
    int64_t sa = (r * nb + n - 1) / n;   // ceil(alpha n_1i), alpha = r / n
    int64_t sb = sa < mb ? sa : mb;
    sb = sb < nb ? sb : nb;
    blk.m_b[b] = mb;
    blk.n_b[b] = nb;
    blk.s_b[b] = sb;
    blk.s_off[b] = S;
    S += sb;
    if (sb > 0) {
      blk.data_off[b] = total;
      total += mb * nb;
    } else {
      blk.data_off[b] = -1;
    }
  }
  blk.s_off[B] = S;
  blk.S = S;
  blk.total = total;
  blk.data = DArr<double>(total, st);
  if (total > 0) CK(cudaMemsetAsync(blk.data.get(), 0, size_t(total) * 8, st));
  if (R.m1 == 0 || total == 0) return;
  DArr<int64_t> d_row_off(B + 1, st), d_col_off(B + 1, st), d_data_off(B, st);
  CK(cudaMemcpyAsync(d_row_off.get(), R.row_off.data(), size_t(B + 1) * 8, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_col_off.get(), R.col_off.data(), size_t(B + 1) * 8, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_data_off.get(), blk.data_off.data(), size_t(B) * 8, cudaMemcpyHostToDevice, st));
  DArr<int32_t> blk_of_row(R.m1, st), nz_row(h->nnz, st);
  k_blk_of<<<nblk(B), BS, 0, st>>>(d_row_off, B, blk_of_row);
  CK_LAUNCH();
  k_row_of_nz<<<nblk(h->m * 32), BS, 0, st>>>(h->rowptr, h->m, nz_row);
  CK_LAUNCH();
  k_blocks_fill<<<nblk(h->nnz), BS, 0, st>>>(nz_row, h->col, h->val, h->nnz, R.row_pos, R.col_pos, R.m1, R.n1,
                                             blk_of_row, d_row_off, d_col_off, d_data_off, blk.data);
  CK_LAUNCH();
  CK(cudaStreamSynchronize(st));
}

}  // namespace fastpi
