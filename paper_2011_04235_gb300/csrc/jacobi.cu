// Batched one-sided Jacobi SVD (Hestenes' method) in one persistent
// cooperative launch.
//
// Parallel ordering: a problem with q columns (padded to an even qe) runs
// sweeps of qe - 1 rounds; round r pairs the columns by the circle method
// (qe - 1 with r, and (r + s, r - s) mod (qe - 1) for s = 1 .. qe/2 - 1), so the
// qe/2 pairs of a round are disjoint and a sweep visits every pair once.  All
// problems advance one round per global step; every pair of every active
// problem is one warp-sized work item; steps are separated by a device-wide
// barrier whose spin is bounded (on timeout the kernel records
// ST_BARRIER_TIMEOUT and returns).
//
// Rotation (one pair, warp-wide): alpha = |a_i|^2, beta = |a_j|^2,
// gamma = a_i . a_j; if |gamma| > tol sqrt(alpha beta):
//   zeta = (beta - alpha) / (2 gamma), t = sign(zeta) / (|zeta| + hypot(1, zeta)),
//   c = 1 / sqrt(1 + t^2), s = c t,  a_i' = c a_i - s a_j,  a_j' = s a_i + c a_j
// (the same on the columns of V).  A problem has converged when a whole sweep
// made no rotation; columns whose squared norm is below a tiny fraction of the
// problem's squared Frobenius norm are treated as zero (they stem from rank
// deficiency and are never rotated).
#include <algorithm>
#include <cmath>

#include "jacobi.cuh"
#include "tuning.cuh"

namespace fastpi {
namespace {

template <typename T>
struct DevProb {
  T* A;
  T* V;
  int64_t lda, ldv;
  int p, q, qe, R;
  int64_t pair_off;
  double tol_abs2;   // squared-norm threshold below which a column counts as zero
};

struct ProbState {
  unsigned long long offmax[3];
  int done;
  int sweeps;
};

struct GridBar {
  unsigned count;
  unsigned gen;
  int stop;
  int done_count;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Device-wide barrier for a cooperative launch.  The last CTA to arrive
// decides whether every problem is done (all increments of done_count of the
// step are complete by then) and publishes that decision with the new
// generation, so every CTA takes the same exit decision.
__device__ bool grid_barrier(GridBar* gb, int nprob, unsigned* status) {
  __shared__ int s_stop;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned gen = ld_acquire(&gb->gen);
    __threadfence();
    unsigned arrived = atomicAdd(&gb->count, 1u) + 1u;
    int stop;
    if (arrived == gridDim.x) {
      gb->count = 0;
      stop = (*(volatile int*)&gb->done_count >= nprob) ? 1 : 0;
      *(volatile int*)&gb->stop = stop;
      __threadfence();
      st_release(&gb->gen, gen + 1u);
    } else {
      long long spins = 0;
      stop = 0;
      while (ld_acquire(&gb->gen) == gen) {
        if (++spins > (1ll << 24)) {   // ~1-2 s
          atomicOr(status, ST_BARRIER_TIMEOUT);
          stop = 1;
          break;
        }
        __nanosleep(64);
      }
      if (!stop) stop = *(volatile int*)&gb->stop;
    }
    __threadfence();
    s_stop = stop;
  }
  __syncthreads();
  return s_stop != 0;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int find_prob(const int64_t* pair_off, int nprob, int64_t w) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (pair_off[mid] <= w)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

template <typename T>
__global__ void k_fro2(const DevProb<T>* probs, double* fro2) {
  const DevProb<T> pr = probs[blockIdx.x];
  double s = 0;
  for (int j = 0; j < pr.q; ++j)
    for (int r = threadIdx.x; r < pr.p; r += blockDim.x) {
      double x = double(pr.A[int64_t(j) * pr.lda + r]);
      s += x * x;
    }
  s = warp_sum(s);
  __shared__ double ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) t += ws[w];
    fro2[blockIdx.x] = t;
  }
}

template <typename T>
__global__ void k_init_v(const DevProb<T>* probs, int nprob) {
  // problems strided over grid.y (a batch may hold more than 65 535 problems)
  for (int b = blockIdx.y; b < nprob; b += gridDim.y) {
    const DevProb<T> pr = probs[b];
    const int64_t n = int64_t(pr.q) * pr.q;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n; t += int64_t(gridDim.x) * blockDim.x) {
      const int64_t c = t / pr.q, r = t % pr.q;
      pr.V[c * pr.ldv + r] = (r == c) ? T(1) : T(0);
    }
  }
}

__device__ __forceinline__ void team_bar(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Sum of three values over a team of NW warps (warp shuffles, then shared
// memory across the team's warps, synchronised by the team's named barrier).
template <typename T, int NW>
__device__ __forceinline__ void team_sum3(T& a, T& b, T& c, int tm, T* red) {
  a = warp_sum(a);
  b = warp_sum(b);
  c = warp_sum(c);
  if constexpr (NW > 1) {
    const int lane = threadIdx.x & 31, wi = (threadIdx.x >> 5) % NW;
    T* r = red + tm * NW * 3;
    if (lane == 0) {
      r[wi * 3] = a;
      r[wi * 3 + 1] = b;
      r[wi * 3 + 2] = c;
    }
    team_bar(1 + tm, 32 * NW);
    a = b = c = T(0);
#pragma unroll
    for (int q = 0; q < NW; ++q) {
      a += r[q * 3];
      b += r[q * 3 + 1];
      c += r[q * 3 + 2];
    }
    team_bar(1 + tm, 32 * NW);
  }
}

// One pair of columns per team of NW warps; team-lane tl owns rows
// tl, tl + 32 NW, ...  Every decision below depends only on values that are
// identical across the team, so the team's threads always take the same path.
template <typename T, int MAXV, int NW>
__global__ void __launch_bounds__(256) k_jacobi(const DevProb<T>* __restrict__ probs, const int64_t* __restrict__ pair_off,
                                                int nprob, int64_t total_pairs, ProbState* state, GridBar* gb,
                                                int max_sweeps, int64_t max_steps, double tol_rel,
                                                unsigned* status) {
  constexpr int TS = 32 * NW;
  __shared__ T red[(256 / TS) * NW * 3];
  const int tl = threadIdx.x % TS, tm = threadIdx.x / TS;
  const int64_t teams_per_cta = blockDim.x / TS;
  const int64_t gt = int64_t(blockIdx.x) * teams_per_cta + tm;
  const int64_t nteams = int64_t(gridDim.x) * teams_per_cta;
  for (int64_t t = 0; t < max_steps; ++t) {
    for (int64_t w = gt; w < total_pairs; w += nteams) {
      const int b = find_prob(pair_off, nprob, w);
      const DevProb<T> pr = probs[b];
      if (*(volatile int*)&state[b].done) continue;
      const int64_t slot = w - pr.pair_off;
      const int64_t sweep = t / pr.R;
      const int rr = int(t % pr.R);
      if (rr == 0 && sweep > 0) {
        // converged when the previous sweep made no rotation
        const bool conv = *(volatile unsigned long long*)&state[b].offmax[(sweep - 1) % 3] == 0ull;
        if (conv || sweep >= max_sweeps) {
          if (slot == 0 && tl == 0) {
            state[b].done = 1;
            state[b].sweeps = int(sweep);
            atomicAdd(&gb->done_count, 1);
            if (!conv) atomicOr(status, ST_JACOBI_SWEEPS);
          }
          continue;
        }
        if (slot == 0 && tl == 0) state[b].offmax[(sweep + 1) % 3] = 0ull;
      }
      const int qe = pr.qe;
      int i, j;
      if (slot == 0) {
        i = qe - 1;
        j = rr;
      } else {
        i = int((rr + slot) % (qe - 1));
        j = int((rr - slot + qe - 1) % (qe - 1));
      }
      if (i > j) {
        int tmp = i;
        i = j;
        j = tmp;
      }
      if (j >= pr.q) continue;   // paired with the padding column
      T* ai = pr.A + int64_t(i) * pr.lda;
      T* aj = pr.A + int64_t(j) * pr.lda;
      T* vi = pr.V + int64_t(i) * pr.ldv;
      T* vj = pr.V + int64_t(j) * pr.ldv;
      if (pr.p <= TS * MAXV && pr.q <= TS * MAXV) {
        // register-resident pair: every load of the two columns of A and of V
        // is issued before the first use, so a round costs one L2 round trip
        T xa[MAXV], ya[MAXV], xv[MAXV], yv[MAXV];
#pragma unroll
        for (int u = 0; u < MAXV; ++u) {
          const int r = tl + TS * u;
          const bool ok = r < pr.p, okv = r < pr.q;
          xa[u] = ok ? __ldcg(ai + r) : T(0);
          ya[u] = ok ? __ldcg(aj + r) : T(0);
          xv[u] = okv ? __ldcg(vi + r) : T(0);
          yv[u] = okv ? __ldcg(vj + r) : T(0);
        }
        T al = 0, be = 0, ga = 0;
#pragma unroll
        for (int u = 0; u < MAXV; ++u) {
          al = fma(xa[u], xa[u], al);
          be = fma(ya[u], ya[u], be);
          ga = fma(xa[u], ya[u], ga);
        }
        team_sum3<T, NW>(al, be, ga, tm, red);
        if (double(al) <= pr.tol_abs2 || double(be) <= pr.tol_abs2) continue;
        const double off = fabs(double(ga)) / (sqrt(double(al)) * sqrt(double(be)));
        if (!(off > tol_rel)) continue;
        if (tl == 0) *(volatile unsigned long long*)&state[b].offmax[sweep % 3] = 1ull;   // rotated
        const T zeta = (be - al) / (T(2) * ga);
        const T tt = copysign(T(1), zeta) / (fabs(zeta) + hypot(T(1), zeta));
        const T c = T(1) / sqrt(T(1) + tt * tt);
        const T s = c * tt;
#pragma unroll
        for (int u = 0; u < MAXV; ++u) {
          const int r = tl + TS * u;
          if (r < pr.p) {
            __stcg(ai + r, c * xa[u] - s * ya[u]);
            __stcg(aj + r, s * xa[u] + c * ya[u]);
          }
          if (r < pr.q) {
            __stcg(vi + r, c * xv[u] - s * yv[u]);
            __stcg(vj + r, s * xv[u] + c * yv[u]);
          }
        }
        continue;
      }
      // long columns: two passes over L2, loads unrolled four deep
      T al = 0, be = 0, ga = 0;
#pragma unroll 4
      for (int r = tl; r < pr.p; r += TS) {
        T x = __ldcg(ai + r), y = __ldcg(aj + r);
        al = fma(x, x, al);
        be = fma(y, y, be);
        ga = fma(x, y, ga);
      }
      team_sum3<T, NW>(al, be, ga, tm, red);
      if (double(al) <= pr.tol_abs2 || double(be) <= pr.tol_abs2) continue;
      double off = fabs(double(ga)) / (sqrt(double(al)) * sqrt(double(be)));
      if (!(off > tol_rel)) continue;
      if (tl == 0) *(volatile unsigned long long*)&state[b].offmax[sweep % 3] = 1ull;   // rotated
      T zeta = (be - al) / (T(2) * ga);
      T tt = copysign(T(1), zeta) / (fabs(zeta) + hypot(T(1), zeta));
      T c = T(1) / sqrt(T(1) + tt * tt);
      T s = c * tt;
#pragma unroll 4
      for (int r = tl; r < pr.p; r += TS) {
        T x = __ldcg(ai + r), y = __ldcg(aj + r);
        __stcg(ai + r, c * x - s * y);
        __stcg(aj + r, s * x + c * y);
      }
#pragma unroll 4
      for (int r = tl; r < pr.q; r += TS) {
        T x = __ldcg(vi + r), y = __ldcg(vj + r);
        __stcg(vi + r, c * x - s * y);
        __stcg(vj + r, s * x + c * y);
      }
    }
    if (grid_barrier(gb, nprob, status)) break;
  }
}

// Per problem: sigma_j = |b_j| and a descending sort (ties: lower index first).
template <typename T>
__global__ void k_finish(const DevProb<T>* probs, const int64_t* sig_off, double* sig, int32_t* perm, int nq_max,
                         const double* norms) {
  extern __shared__ unsigned char smem_raw[];
  const DevProb<T> pr = probs[blockIdx.x];
  int nq = 1;
  while (nq < pr.q) nq <<= 1;
  // the norms as order-preserving integers: the sort compares on the
  // integer pipe
  unsigned long long* key = reinterpret_cast<unsigned long long*>(smem_raw);
  int* idx = reinterpret_cast<int*>(key + nq_max);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  if (norms) {
    // column norms computed beforehand (a single large problem: k_colnorms)
    for (int j = threadIdx.x; j < nq; j += blockDim.x) {
      key[j] = order_key(j < pr.q ? norms[j] : -1.0);
      idx[j] = j;
    }
  } else {
    for (int j = w; j < nq; j += nwarp) {
      double s = 0;
      if (j < pr.q) {
        const T* col = pr.A + int64_t(j) * pr.lda;
        for (int r = lane; r < pr.p; r += 32) {
          double x = double(__ldcg(col + r));
          s += x * x;
        }
        s = warp_sum(s);
      }
      if (lane == 0) {
        key[j] = order_key(j < pr.q ? sqrt(s) : -1.0);
        idx[j] = j;
      }
    }
  }
  __syncthreads();
  // bitonic sort: descending key, ascending index on ties
  for (int size = 2; size <= nq; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < nq; t += blockDim.x) {
        int u = t ^ stride;
        if (u > t) {
          bool up = ((t & size) == 0);
          const unsigned long long ka = key[t], kb = key[u];
          int ia = idx[t], ib = idx[u];
          bool a_first = (ka > kb) || (ka == kb && ia < ib);
          if (a_first != up) {
            key[t] = kb;
            key[u] = ka;
            idx[t] = ib;
            idx[u] = ia;
          }
        }
      }
      __syncthreads();
    }
  }
  const int64_t o = sig_off[blockIdx.x];
  for (int t = threadIdx.x; t < pr.q; t += blockDim.x) {
    sig[o + t] = order_value(key[t]);
    perm[o + t] = idx[t];
  }
}

// |A[:, j]| for the q columns of one p x q problem, one warp per column (many
// CTAs: the norms of a single large problem off the sort's critical path).
template <typename T>
__global__ void k_colnorms(const T* __restrict__ A, int64_t lda, int p, int q, double* __restrict__ out) {
  const int j = int(blockIdx.x) * int(blockDim.x >> 5) + int(threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (j >= q) return;
  const T* col = A + int64_t(j) * lda;
  double s = 0;
  for (int r = lane; r < p; r += 32) {
    const double x = double(__ldcg(col + r));
    s += x * x;
  }
  s = warp_sum(s);
  if (lane == 0) out[j] = sqrt(s);
}

// FP32 problems with at least ROUTE_MIN_Q columns, the ROUTE_MAX largest,
// run in the cluster form of block Jacobi instead of a bucket.
constexpr int ROUTE_MIN_Q = 96;
constexpr int ROUTE_MAX = 16;

template <typename T> struct Eps;
template <> struct Eps<double> { static constexpr double v = 2.220446049250313e-16; };
template <> struct Eps<float> { static constexpr double v = 1.1920928955078125e-07; };


// One persistent cooperative launch over `probs`, problem b writing its
// outputs at sig / perm + out_off[b].
template <typename T>
JacobiStats run_bucket(fastpi_ctx* h, const std::vector<JacobiProblem<T>>& probs,
                       const std::vector<int64_t>& out_off, double* sig, int32_t* perm, int kind, int cls) {
  JacobiStats stats;
  const int nprob = int(probs.size());
  if (nprob == 0) return stats;
  cudaStream_t st = h->stream;
  std::vector<DevProb<T>> dp(nprob);
  std::vector<int64_t> pair_off(nprob), sig_off(nprob);
  int64_t pairs = 0;
  int maxR = 1, maxq = 1, maxp = 1;
  for (int b = 0; b < nprob; ++b) {
    const auto& P = probs[b];
    DevProb<T>& d = dp[b];
    d.A = P.A;
    d.V = P.V;
    d.lda = P.lda;
    d.ldv = P.ldv;
    d.p = P.p;
    d.q = P.q;
    d.qe = P.q + (P.q & 1);
    if (d.qe < 2) d.qe = 2;
    d.R = d.qe - 1;
    d.pair_off = pairs;
    d.tol_abs2 = 0;
    pair_off[b] = pairs;
    sig_off[b] = out_off[b];
    pairs += d.qe / 2;
    maxR = std::max(maxR, d.R);
    maxq = std::max(maxq, P.q);
    maxp = std::max(maxp, P.p);
  }
  if (maxq > 8192) fail(FASTPI_ERR_ARG, "Jacobi SVD: more than 8192 columns in one problem");
  DArr<DevProb<T>> d_probs(nprob, st);
  DArr<int64_t> d_pair_off(nprob, st), d_sig_off(nprob, st);
  DArr<double> fro2(nprob, st);
  CK(cudaMemcpyAsync(d_probs.get(), dp.data(), sizeof(DevProb<T>) * nprob, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_pair_off.get(), pair_off.data(), 8 * nprob, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_sig_off.get(), sig_off.data(), 8 * nprob, cudaMemcpyHostToDevice, st));
  // absolute column threshold: (q * eps)^2 * |A|_F^2
  k_fro2<T><<<nprob, 256, 0, st>>>(d_probs, fro2);
  CK_LAUNCH();
  std::vector<double> f2(nprob);
  d2h_sync(f2.data(), fro2.get(), 8 * nprob, st);
  for (int b = 0; b < nprob; ++b) {
    double e = double(std::max(dp[b].q, dp[b].p)) * Eps<T>::v;
    dp[b].tol_abs2 = e * e * f2[b];
  }
  CK(cudaMemcpyAsync(d_probs.get(), dp.data(), sizeof(DevProb<T>) * nprob, cudaMemcpyHostToDevice, st));
  {
    dim3 g(unsigned(std::min<int64_t>(64, (int64_t(maxq) * maxq + 255) / 256)), unsigned(std::min(nprob, 65535)));
    k_init_v<T><<<g, 256, 0, st>>>(d_probs, nprob);
    CK_LAUNCH();
  }
  DArr<ProbState> state(nprob, st);
  DArr<GridBar> gb(1, st);
  CK(cudaMemsetAsync(state.get(), 0, sizeof(ProbState) * nprob, st));
  CK(cudaMemsetAsync(gb.get(), 0, sizeof(GridBar), st));
  CK(cudaMemsetAsync(h->dstatus.get(), 0, 4, st));

  const int max_sweeps = sizeof(T) == 8 ? 40 : 30;
  const double tol_rel = std::sqrt(double(maxp)) * Eps<T>::v;
  // FP32: one warp per pair, eight pairs per CTA, registers per lane = the
  // smallest of {8, 16, 32, 44} that holds the longest column.  FP64: the
  // FP64 rate per SM is low, so a pair is shared by a team of 2 or 4 warps
  // (one team per CTA, spreading pairs over the SMs) holding 16 values per lane.
  // the kernel variant of the bucket's register-tile class (tile_class; the
  // tuning table may put small problems in a larger class)
  void* kern = nullptr;
  int bs = 256, pairs_per_cta = 8;
  if constexpr (sizeof(T) == 4) {
    kern = (void*)k_jacobi<T, 8, 1>;   // classes 0 and 4 (long columns: the two-pass path)
    if (cls == 1) kern = (void*)k_jacobi<T, 16, 1>;
    if (cls == 2) kern = (void*)k_jacobi<T, 32, 1>;
    if (cls == 3) kern = (void*)k_jacobi<T, 44, 1>;
  } else {
    pairs_per_cta = 1;
    if (cls == 0) {
      kern = (void*)k_jacobi<T, 8, 2>;
      bs = 64;
    } else if (cls == 1) {
      kern = (void*)k_jacobi<T, 16, 2>;
      bs = 64;
    } else {
      kern = (void*)k_jacobi<T, 16, 4>;   // register path up to 2048 rows, two-pass beyond
      bs = 128;
    }
  }
  int occ = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, bs, 0));
  if (occ < 1) occ = 1;
  int64_t want = (pairs + pairs_per_cta - 1) / pairs_per_cta;
  int64_t cap = int64_t(h->num_sms) * occ;
  int grid = int(std::max<int64_t>(1, std::min(want, cap)));
  int64_t max_steps = int64_t(max_sweeps + 2) * maxR + 2;
  int nprob_arg = nprob;
  int64_t pairs_arg = pairs;
  DevProb<T>* a0 = d_probs.get();
  int64_t* a1 = d_pair_off.get();
  ProbState* a4 = state.get();
  GridBar* a5 = gb.get();
  int a6 = max_sweeps;
  int64_t a7 = max_steps;
  double a8 = tol_rel;
  unsigned* a9 = h->dstatus.get();
  void* args[] = {&a0, &a1, &nprob_arg, &pairs_arg, &a4, &a5, &a6, &a7, &a8, &a9};
  cudaEvent_t ev0, ev1;
  CK(cudaEventCreate(&ev0));
  CK(cudaEventCreate(&ev1));
  CK(cudaEventRecord(ev0, st));
  CK(cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(bs), args, 0, st));
  CK_LAUNCH();
  CK(cudaEventRecord(ev1, st));

  int nq_max = 1;
  while (nq_max < maxq) nq_max <<= 1;
  size_t smem = size_t(nq_max) * (sizeof(double) + sizeof(int));
  if (smem > 48 * 1024) allow_max_dynamic_smem((const void*)k_finish<T>);
  DArr<double> norms;
  if (nprob == 1) {
    norms = DArr<double>(probs[0].q, st);
    k_colnorms<T><<<unsigned((probs[0].q + 7) / 8), 256, 0, st>>>(probs[0].A, probs[0].lda, probs[0].p, probs[0].q,
                                                                    norms.get());
    CK_LAUNCH();
  }
  k_finish<T><<<nprob, 512, smem, st>>>(d_probs, d_sig_off, sig, perm, nq_max, nprob == 1 ? norms.get() : nullptr);
  CK_LAUNCH();

  unsigned stat = 0;
  d2h_sync(&stat, h->dstatus.get(), 4, st);
  std::vector<ProbState> hs(nprob);
  d2h_sync(hs.data(), state.get(), sizeof(ProbState) * nprob, st);
  for (auto& s : hs) stats.max_sweeps_used = std::max(stats.max_sweeps_used, s.sweeps);
  {
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, ev0, ev1));
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    double flops = 0, model = 0;
    for (int b = 0; b < nprob; ++b) {
      const double p = dp[b].p, q = dp[b].q;
      flops += double(hs[b].sweeps) * (q * (q - 1) / 2) * (12 * p + 6 * q);
      model += 4 * p * q * q + 8 * q * q * q;
    }
    note_svd(kind, ms, model, flops);
  }
  if (stat & ST_BARRIER_TIMEOUT) fail(FASTPI_ERR_NO_CONVERGENCE, "Jacobi SVD: device-wide barrier timed out");
  stats.hit_cap = (stat & ST_JACOBI_SWEEPS) != 0;
  return stats;
}

// Register-tile class of a problem: the kernel variant that holds its longest
// column (FP32: 8 / 16 / 32 / 44 values per lane, beyond that the two-pass
// path; FP64: teams of two warps with 8 or 16 values per lane, or four warps).
template <typename T>
int tile_class(const JacobiProblem<T>& P) {
  const int maxdim = std::max(P.p, P.q);
  if constexpr (sizeof(T) == 4) {
    const int need = (maxdim + 31) / 32;
    return need <= 8 ? 0 : need <= 16 ? 1 : need <= 32 ? 2 : need <= 44 ? 3 : 4;
  } else {
    return maxdim <= 64 * 8 ? 0 : maxdim <= 64 * 16 ? 1 : 2;
  }
}

}  // namespace

// Size-bucketed: the problems are grouped by the register tile their longest
// column needs, and each group runs in its own persistent launch of the
// matching kernel variant (a single launch would give every problem the tile
// of the largest one, and its convergence threshold).
template <typename T>
JacobiStats jacobi_svd_batched(fastpi_ctx* h, const std::vector<JacobiProblem<T>>& probs, double* sig,
                               int32_t* perm, int kind) {
  JacobiStats stats;
  const int nprob = int(probs.size());
  if (nprob == 0) return stats;
  constexpr int NCLASS = 5;
  std::vector<JacobiProblem<T>> bucket[NCLASS];
  std::vector<int64_t> off[NCLASS];
  std::vector<char> routed(nprob, 0);
  if constexpr (sizeof(T) == 4) {
    // The largest FP32 problems go one by one to the cluster form of block
    // Jacobi: in a bucket a problem with q columns costs q - 1 device-wide
    // barriers per sweep (and sets the pace of every problem in its bucket),
    // in the cluster form about q / 8 rounds of one cluster each.
    std::vector<int> cand;
    for (int b = 0; b < nprob; ++b)
      if (probs[b].q >= ROUTE_MIN_Q && probs[b].p >= probs[b].q && probs[b].lda == probs[b].p &&
          probs[b].ldv == probs[b].q)
        cand.push_back(b);
    std::stable_sort(cand.begin(), cand.end(), [&](int a, int b) { return probs[a].q > probs[b].q; });
    if (int(cand.size()) > ROUTE_MAX) cand.resize(ROUTE_MAX);
    std::vector<int64_t> offs(nprob, 0);
    for (int b = 1; b < nprob; ++b) offs[b] = offs[b - 1] + probs[b - 1].q;
    for (int b : cand) {
      const JacobiProblem<T>& P = probs[b];
      CoreTiling tl;
      tuned_core_tiling(P.q, &tl);
      JacobiStats js;
      float ms = 0;
      int sw = 0;
      bool res = false;
      if (!jacobi_svd_cluster(h, reinterpret_cast<float*>(P.A), P.lda, reinterpret_cast<float*>(P.V), P.ldv, P.p,
                              P.q, tl, &js, &ms, &sw, &res))
        continue;   // stays in its bucket
      std::vector<JacobiProblem<T>> one(1, P);
      jacobi_sort_columns<T>(h, one, sig + offs[b], perm + offs[b]);
      routed[b] = 1;
      stats.max_sweeps_used = std::max(stats.max_sweeps_used, js.max_sweeps_used);
      stats.hit_cap = stats.hit_cap || js.hit_cap;
      const double p = P.p, q = P.q;
      note_svd(kind, ms, 4 * p * q * q + 8 * q * q * q, double(sw) * (q * (q - 1) / 2) * (12 * p + 6 * q));
    }
  }
  int64_t soff = 0;
  for (int b = 0; b < nprob; ++b) {
    if (routed[b]) {
      soff += probs[b].q;
      continue;
    }
    const int c = tuned_bucket_class(sizeof(T) == 8 ? 0 : 1, std::max(probs[b].p, probs[b].q),
                                     tile_class<T>(probs[b]));
    bucket[c].push_back(probs[b]);
    off[c].push_back(soff);
    soff += probs[b].q;
  }
  for (int c = 0; c < NCLASS; ++c) {
    if (bucket[c].empty()) continue;
    const JacobiStats js = run_bucket<T>(h, bucket[c], off[c], sig, perm, kind, c);
    stats.max_sweeps_used = std::max(stats.max_sweeps_used, js.max_sweeps_used);
    stats.hit_cap = stats.hit_cap || js.hit_cap;
  }
  return stats;
}


template <typename T>
void jacobi_sort_columns(fastpi_ctx* h, const std::vector<JacobiProblem<T>>& probs, double* sig, int32_t* perm) {
  const int nprob = int(probs.size());
  if (nprob == 0) return;
  cudaStream_t st = h->stream;
  std::vector<DevProb<T>> dp(nprob);
  std::vector<int64_t> sig_off(nprob);
  int64_t soff = 0;
  int maxq = 1;
  for (int b = 0; b < nprob; ++b) {
    dp[b] = DevProb<T>{probs[b].A, probs[b].V, probs[b].lda, probs[b].ldv, probs[b].p, probs[b].q, 0, 0, 0, 0.0};
    sig_off[b] = soff;
    soff += probs[b].q;
    maxq = std::max(maxq, probs[b].q);
  }
  if (maxq > 8192) fail(FASTPI_ERR_ARG, "Jacobi SVD: more than 8192 columns in one problem");
  DArr<DevProb<T>> d_probs(nprob, st);
  DArr<int64_t> d_sig_off(nprob, st);
  CK(cudaMemcpyAsync(d_probs.get(), dp.data(), sizeof(DevProb<T>) * nprob, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_sig_off.get(), sig_off.data(), 8 * nprob, cudaMemcpyHostToDevice, st));
  int nq_max = 1;
  while (nq_max < maxq) nq_max <<= 1;
  size_t smem = size_t(nq_max) * (sizeof(double) + sizeof(int));
  if (smem > 48 * 1024) allow_max_dynamic_smem((const void*)k_finish<T>);
  DArr<double> norms;
  if (nprob == 1) {
    norms = DArr<double>(probs[0].q, st);
    k_colnorms<T><<<unsigned((probs[0].q + 7) / 8), 256, 0, st>>>(probs[0].A, probs[0].lda, probs[0].p, probs[0].q,
                                                                    norms.get());
    CK_LAUNCH();
  }
  k_finish<T><<<nprob, 512, smem, st>>>(d_probs, d_sig_off, sig, perm, nq_max, nprob == 1 ? norms.get() : nullptr);
  CK_LAUNCH();
}

template void jacobi_sort_columns<double>(fastpi_ctx*, const std::vector<JacobiProblem<double>>&, double*, int32_t*);
template void jacobi_sort_columns<float>(fastpi_ctx*, const std::vector<JacobiProblem<float>>&, double*, int32_t*);

template JacobiStats jacobi_svd_batched<double>(fastpi_ctx*, const std::vector<JacobiProblem<double>>&, double*,
                                                int32_t*, int);
template JacobiStats jacobi_svd_batched<float>(fastpi_ctx*, const std::vector<JacobiProblem<float>>&, double*,
                                               int32_t*, int);

}  // namespace fastpi
