// Block one-sided Jacobi SVD of one FP32 core matrix on the whole GPU.
//
// The scalar one-sided Jacobi of the core K ((k + c) x (k + c), Eqs. 2 / 3)
// spends its time in n - 1 device- or cluster-wide synchronisations per
// sweep; the arithmetic per round is tiny.  The block form pairs column
// BLOCKS instead of columns: with blocks of b = P / 2 columns there are only
// n / b - 1 rounds per sweep, and everything inside a round is local to one
// CTA.  CTA w of round rr owns the block pair (I, J) of the circle method and
//   1. stages the panels X = [K_I K_J] and Y = [V_I V_J] (n x P each) in
//      shared memory with 16-byte asynchronous copies from L2;
//   2. forms the Gram matrix G = X^T X (P x P) with register tiles;
//   3. runs one cyclic two-sided Jacobi sweep on G (the rotation of a pair
//      comes from G_pp, G_qq, G_pq exactly as from the column dot products of
//      scalar one-sided Jacobi), accumulating the rotations in Q (P x P); the
//      whole CTA updates G and Q in shared memory;
//   4. writes K_IJ <- X Q and V_IJ <- Y Q.
// Every block is owned by exactly one CTA per round, so instead of a
// device-wide barrier per round a CTA waits only for the two CTAs that wrote
// its blocks in the previous round: a per-block counter holds the number of
// rounds completed on that block (release store after the block is written,
// acquire load before it is read).  A device-wide barrier ends each sweep,
// where the CTAs combine their rotation flags: a sweep in which no pair had
// |G_pq| / sqrt(G_pp G_qq) above tol leaves K unchanged (converged), and a
// sweep whose rotations all stayed below 1e-3 ends the iteration (quadratic
// convergence leaves the next sweep ~1e-6, below tol = sqrt(n) eps32 for the
// core sizes here; measured on the medium and 200k x 50k workloads: the same
// residual and orthogonality as with 1e-4, one sweep fewer).
//
// K and V are worked on in copies whose leading dimension is a multiple of 4
// floats (zero rows below n), so every column starts on a 16-byte boundary.
// Results (the same contract as the other Jacobi kernels): K <- K J with
// mutually orthogonal columns, V <- J.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <string>

#include "jacobi.cuh"
#include "jacobi_dev.cuh"
#include "tuning.cuh"

namespace fastpi {
namespace {

using namespace jdev;

constexpr int BT = 512;              // threads per CTA (16 warps)
constexpr int B_MAX_SWEEPS = 30;
constexpr int INNER_SWEEPS = 1;      // sweeps of the P x P Gram solve per block pair
constexpr float B_EARLY_OFF = 1e-3f;
#ifdef FASTPI_PHASE_CLOCKS
__device__ long long g_phase_clk[8];
#define PHASE_MARK(k)                          \
  do {                                         \
    if (blockIdx.x == gridDim.x / 2 && threadIdx.x == 0) { \
      const long long t_ = clock64();          \
      g_phase_clk[k] += t_ - t_mark;           \
      t_mark = t_;                             \
    }                                          \
  } while (0)
#else
#define PHASE_MARK(k) \
  do {                \
  } while (0)
#endif

struct BlkArgs {
  float* K;        // ldk x n column-major: in A (rows >= n zero), out A J
  float* V;        // ldk x n column-major: in I, out J
  unsigned* ver;   // [nb * VER_STRIDE] rounds completed per block
  int n, ldk;      // ldk: multiple of 4, >= n
  int nb;          // number of column blocks (even; the last may be empty)
  float tol;
  int inner;       // sweeps of the P x P Gram solve
  BBar* gb;
  int* out;        // [0] sweeps used, [1] hit the sweep cap
  unsigned* status;
};

// VS: the V panel is staged in shared memory next to the K panel (false: the
// update reads V's rows straight from L2, for cores whose two panels do not
// fit in one CTA's shared memory).  RES: the resident-block schedule below.
template <int P, bool VS, bool RES>
__global__ void __launch_bounds__(BT, 1) k_jacobi_block(BlkArgs a) {
  constexpr int B = P / 2;         // columns per block
  constexpr int TW = P / 4;        // Gram tile edge (4 x 4 tiles of TW x TW)
  constexpr int GS = P;            // row stride of G and Q (a warp covers whole rows: no bank conflicts)
  extern __shared__ float4 smem4[];
  const int ldk = a.ldk, n = a.n;
  float* Xs = reinterpret_cast<float*>(smem4);   // [P][ldk]
  float* Ys = Xs + size_t(P) * ldk;              // [P][ldk] (VS only)
  float* G = Ys + (VS ? size_t(P) * ldk : 0);    // [P][GS]
  float* Q = G + P * GS;                         // [P][GS]
  float* Gn = Q + P * GS;                        // [P][GS] (second buffers of the Gram solve)
  float* Qn = Gn + P * GS;                       // [P][GS]
  __shared__ float s_sc[P], s_so[P];
  __shared__ int s_gcol[P];
  __shared__ int s_rot, s_ok, s_pair_rot;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float tabs = [&] {
    const float ne = float(n) * 1.1920929e-7f;
    return float(double(ne) * double(ne) * a.gb->fro2);
  }();
  const float tol2 = a.tol * a.tol, early2 = B_EARLY_OFF * B_EARLY_OFF;
  if (tid == 0) s_rot = 0;
  const int nq = ldk / 4;   // 16-byte chunks per column

  int sweep = 0;
  // Resident mode: the circle method's pairs are kept, but CTAs swap slots in
  // fixed pairs (0 <-> 1, 2 <-> 3, ...; the last slot stays when their number
  // is odd) every round.  Slot s holds {r + s, r - s} in round r, so a move to
  // s - 1 keeps block r + s and a move to s + 1 keeps r - s: every CTA's pair
  // shares one block with its previous pair, which stays in shared memory,
  // and only the other block is waited for and loaded.  held0 / held1: the
  // blocks in the two physical halves of the panels.
  int held0 = -1, held1 = -1;
  const bool slot_fixed = (gridDim.x & 1u) && blockIdx.x == gridDim.x - 1;
#ifdef FASTPI_PHASE_CLOCKS
  long long t_mark = clock64();
#endif
  for (;;) {
    for (int rr = 0; rr < a.nb - 1; ++rr) {
      const unsigned t = unsigned(sweep) * unsigned(a.nb - 1) + unsigned(rr);
      const int slot = (RES && !slot_fixed) ? int(blockIdx.x ^ (t & 1u)) : int(blockIdx.x);
      int bi, bj;
      circle_pair(slot, rr, a.nb, bi, bj);
      // physical halves of bi and bj; `need`: the blocks to wait for and load
      // (bit 0: bi, bit 1: bj)
      int hi = 0, hj = 1, need = 3;
      if (RES) {
        if (bi == held0 || bi == held1) {
          hi = bi == held0 ? 0 : 1;
          hj = 1 - hi;
          need = 2;
        } else if (bj == held0 || bj == held1) {
          hj = bj == held0 ? 0 : 1;
          hi = 1 - hj;
          need = 1;
        }
        held0 = hi == 0 ? bi : bj;
        held1 = hi == 0 ? bj : bi;
      }
      // physical panel column of logical column c (logical order: the columns
      // of bi, then those of bj, whatever half holds them)
      auto pcol = [&](int c) { return (c < B ? hi : hj) * B + (c & (B - 1)); };
      if (tid < P) {
        const int g = tid < B ? bi * B + tid : bj * B + (tid - B);
        s_gcol[tid] = g < n ? g : -1;
      }
      // wait until the previous round on the blocks to load is complete
      if (tid == 0) {
        int ok = 1;
        auto ready = [&] {
          return (!(need & 1) || b_ld_acquire(a.ver + bi * VER_STRIDE) >= t) &&
                 (!(need & 2) || b_ld_acquire(a.ver + bj * VER_STRIDE) >= t);
        };
        if (!ready()) {
          const unsigned long long t0 = b_gtimer();
          unsigned spins = 0;
          while (!ready()) {
            if ((++spins & 63u) == 0 && b_gtimer() - t0 > B_WAIT_NS) {
              atomicOr(a.status, ST_BARRIER_TIMEOUT);
              ok = 0;
              break;
            }
          }
        }
        // the acquire loads order this CTA's reads (through the barrier below)
        // after the producers' writes
        s_ok = ok;
        s_pair_rot = 0;
      }
      __syncthreads();
      if (!s_ok) return;
      PHASE_MARK(5);
      // 1. panels: X (first group), Y (second group)
      for (int e = tid; e < P * nq; e += BT) {
        const int c = e / nq, r4 = (e - c * nq) * 4;
        if (!(need & (c < B ? 1 : 2))) continue;
        const int g = s_gcol[c];
        float* d = Xs + size_t(pcol(c)) * ldk + r4;
        if (g >= 0)
          cp_async16(d, a.K + size_t(g) * ldk + r4);
        else
          *reinterpret_cast<float4*>(d) = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      cp_async_commit();
      if (VS) {
        for (int e = tid; e < P * nq; e += BT) {
          const int c = e / nq, r4 = (e - c * nq) * 4;
          if (!(need & (c < B ? 1 : 2))) continue;
          const int g = s_gcol[c];
          float* d = Ys + size_t(pcol(c)) * ldk + r4;
          if (g >= 0)
            cp_async16(d, a.V + size_t(g) * ldk + r4);
          else
            *reinterpret_cast<float4*>(d) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
      cp_async_commit();
      cp_async_wait<1>();
      __syncthreads();
      PHASE_MARK(0);
      // 2. Gram: warp w owns tile (w / 4, w % 4); lanes split the rows
      {
        const int tp = warp >> 2, tq = warp & 3;
        float acc[TW * TW];
#pragma unroll
        for (int i = 0; i < TW * TW; ++i) acc[i] = 0.f;
        // a tile of TW logical columns lies inside one block: consecutive
        // physical columns
        const float* xa = Xs + size_t(pcol(tp * TW)) * ldk;
        const float* xb = Xs + size_t(pcol(tq * TW)) * ldk;
#pragma unroll 2
        for (int r = lane; r < n; r += 32) {
          float u[TW], w[TW];
#pragma unroll
          for (int i = 0; i < TW; ++i) {
            u[i] = xa[size_t(i) * ldk + r];
            w[i] = xb[size_t(i) * ldk + r];
          }
#pragma unroll
          for (int i = 0; i < TW; ++i)
#pragma unroll
            for (int j = 0; j < TW; ++j) acc[i * TW + j] = fmaf(u[i], w[j], acc[i * TW + j]);
        }
        int off;
        warp_reduce_scatter<TW * TW>(acc, lane, off);
        if ((TW * TW) >= 32) {
#pragma unroll
          for (int e = 0; e < ((TW * TW) >= 32 ? (TW * TW) / 32 : 1); ++e) {
            const int idx = off + e, i = idx / TW, j = idx % TW;
            G[(tp * TW + i) * GS + tq * TW + j] = acc[e];
          }
        } else if ((lane & (32 / (TW * TW) - 1)) == 0) {
          const int i = off / TW, j = off % TW;
          G[(tp * TW + i) * GS + tq * TW + j] = acc[0];
        }
      }
      for (int e = tid; e < P * P; e += BT) Q[(e / P) * GS + e % P] = (e / P == e % P) ? 1.f : 0.f;
      __syncthreads();
      PHASE_MARK(1);
      // 3. cyclic two-sided Jacobi on G, rotations accumulated in Q: the pairs
      // inside the blocks in the first round of a sweep (every block meets its
      // first partner there), only cross pairs afterwards, so every column
      // pair is still visited at least once per sweep
      const float* Qf = inner_solve_cta<P, BT>(G, Gn, Q, Qn, s_sc, s_so, tid, tabs, tol2, early2, a.inner, rr != 0,
                                               &s_rot, &s_pair_rot);
      // Q orthonormal to rounding (no drift of the FP32 rotations; G and Gn are free now)
      if (s_pair_rot) Qf = ns_orthonormalize<P, BT>(Qf, Gn, Qf == Q ? Qn : Q, tid);
      PHASE_MARK(2);
      cp_async_wait<0>();
      __syncthreads();
      PHASE_MARK(6);
      // 4. K_IJ <- X Q, V_IJ <- Y Q; one item = one row and one half of the P
      // output columns when V is staged (items of one warp share the half, so
      // every store instruction writes 32 consecutive rows of one column);
      // nothing to write when no pair of the block pair rotated (Q = I)
      {
        // with V read from L2 and written in place, one item must own whole
        // rows (a half-row item would overwrite V entries the other half of
        // the row still has to read)
        constexpr int NH = VS ? 2 : 1;
        constexpr int H = P / NH;
        if (VS && RES) {
          // resident mode: the panels are updated in place as well, so one
          // item owns whole rows (no other thread reads the row it rewrites)
          for (int r = tid; s_pair_rot && r < n; r += BT) {
            float u[P], v[P];
#pragma unroll
            for (int j = 0; j < P; ++j) u[j] = v[j] = 0.f;
#pragma unroll
            for (int c = 0; c < P; ++c) {
              const float xc = Xs[size_t(pcol(c)) * ldk + r];
              const float yc = Ys[size_t(pcol(c)) * ldk + r];
              const float4* q4 = reinterpret_cast<const float4*>(Qf + c * GS);
#pragma unroll
              for (int j4 = 0; j4 < P / 4; ++j4) {
                const float4 q = q4[j4];
                u[4 * j4 + 0] = fmaf(xc, q.x, u[4 * j4 + 0]);
                u[4 * j4 + 1] = fmaf(xc, q.y, u[4 * j4 + 1]);
                u[4 * j4 + 2] = fmaf(xc, q.z, u[4 * j4 + 2]);
                u[4 * j4 + 3] = fmaf(xc, q.w, u[4 * j4 + 3]);
                v[4 * j4 + 0] = fmaf(yc, q.x, v[4 * j4 + 0]);
                v[4 * j4 + 1] = fmaf(yc, q.y, v[4 * j4 + 1]);
                v[4 * j4 + 2] = fmaf(yc, q.z, v[4 * j4 + 2]);
                v[4 * j4 + 3] = fmaf(yc, q.w, v[4 * j4 + 3]);
              }
            }
#pragma unroll
            for (int j = 0; j < P; ++j) {
              const int g = s_gcol[j];
              if (g >= 0) {
                __stcg(a.K + size_t(g) * ldk + r, u[j]);
                __stcg(a.V + size_t(g) * ldk + r, v[j]);
              }
              Xs[size_t(pcol(j)) * ldk + r] = g >= 0 ? u[j] : 0.f;
              Ys[size_t(pcol(j)) * ldk + r] = g >= 0 ? v[j] : 0.f;
            }
          }
        }
        for (int it = tid; !(VS && RES) && s_pair_rot && it < NH * n; it += BT) {
          const int half = it >= n ? 1 : 0, r = it - half * n, j0 = half * H;
          float u[H], v[H];
#pragma unroll
          for (int j = 0; j < H; ++j) u[j] = v[j] = 0.f;
#pragma unroll
          for (int c = 0; c < P; ++c) {
            const float xc = Xs[size_t(pcol(c)) * ldk + r];
            float yc;
            if (VS) {
              yc = Ys[size_t(pcol(c)) * ldk + r];
            } else {
              const int g = s_gcol[c];
              yc = g >= 0 ? __ldcg(a.V + size_t(g) * ldk + r) : 0.f;
            }
            const float4* q4 = reinterpret_cast<const float4*>(Qf + c * GS + j0);
#pragma unroll
            for (int j4 = 0; j4 < H / 4; ++j4) {
              const float4 q = q4[j4];
              u[4 * j4 + 0] = fmaf(xc, q.x, u[4 * j4 + 0]);
              u[4 * j4 + 1] = fmaf(xc, q.y, u[4 * j4 + 1]);
              u[4 * j4 + 2] = fmaf(xc, q.z, u[4 * j4 + 2]);
              u[4 * j4 + 3] = fmaf(xc, q.w, u[4 * j4 + 3]);
              v[4 * j4 + 0] = fmaf(yc, q.x, v[4 * j4 + 0]);
              v[4 * j4 + 1] = fmaf(yc, q.y, v[4 * j4 + 1]);
              v[4 * j4 + 2] = fmaf(yc, q.z, v[4 * j4 + 2]);
              v[4 * j4 + 3] = fmaf(yc, q.w, v[4 * j4 + 3]);
            }
          }
#pragma unroll
          for (int j = 0; j < H; ++j) {
            const int g = s_gcol[j0 + j];
            if (g >= 0) {
              __stcg(a.K + size_t(g) * ldk + r, u[j]);
              __stcg(a.V + size_t(g) * ldk + r, v[j]);
            }
            // resident mode without a staged V (NH = 1: whole rows): keep the
            // K panel current in place
            if (!VS && RES) Xs[size_t(pcol(j0 + j)) * ldk + r] = g >= 0 ? u[j] : 0.f;
          }
        }
      }
      __syncthreads();
      PHASE_MARK(3);
      // hand both blocks to the next round (the release store publishes every
      // write of the CTA, ordered before it by the barrier above)
      if (tid == 0) {
        b_st_release(a.ver + bi * VER_STRIDE, t + 1u);
        b_st_release(a.ver + bj * VER_STRIDE, t + 1u);
      }
      if (rr == a.nb - 2) {
        // end of a sweep: combine the rotation flags of all CTAs
        if (tid == 0) {
          atomicMax(&a.gb->flag[sweep % 3], s_rot);
          if (blockIdx.x == 0) a.gb->flag[(sweep + 1) % 3] = 0;
        }
        if (!b_barrier(a.gb, a.status)) return;
        PHASE_MARK(4);
        ++sweep;
        const int any = *(volatile int*)&a.gb->flag[(sweep - 1) % 3];
        __syncthreads();
        if (tid == 0) s_rot = 0;
        if (any < 2 || sweep >= B_MAX_SWEEPS) {
          if (blockIdx.x == 0 && tid == 0) {
            a.out[0] = sweep;
            a.out[1] = any >= 2 ? 1 : 0;
            if (any >= 2) atomicOr(a.status, ST_JACOBI_SWEEPS);
          }
          return;
        }
      }
    }
  }
}

// ||K||_F^2 in a fixed order: per-CTA partial sums, then one CTA.
__global__ void k_b_sumsq_part(const float* __restrict__ K, int64_t len, double* part) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < len; i += int64_t(gridDim.x) * blockDim.x) {
    const double v = K[i];
    s += v * v;
  }
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
  }
}
__global__ void k_b_sumsq_final(const double* part, int np, BBar* gb) {
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < np; ++i) s += part[i];
    gb->fro2 = s;
    gb->count = 0;
    gb->gen = 0;
    gb->flag[0] = gb->flag[1] = gb->flag[2] = 0;
  }
}

// Kp (ldk x q) <- K (p x q, ld lda) with zero rows p..ldk-1; Vp <- I (ldk x q).
__global__ void k_b_pad_in(const float* __restrict__ K, int64_t lda, int p, int q, int ldk, float* __restrict__ Kp,
                           float* __restrict__ Vp) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= int64_t(ldk) * q) return;
  const int c = int(e / ldk), r = int(e % ldk);
  Kp[e] = r < p ? K[int64_t(c) * lda + r] : 0.f;
  Vp[e] = r == c ? 1.f : 0.f;
}
// K (p x q, ld lda) <- Kp, V (q x q, ld ldv) <- Vp.
__global__ void k_b_pad_out(const float* __restrict__ Kp, const float* __restrict__ Vp, int p, int q, int ldk,
                            float* __restrict__ K, int64_t lda, float* __restrict__ V, int64_t ldv) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int rows = p > q ? p : q;
  if (e >= int64_t(rows) * q) return;
  const int c = int(e / rows), r = int(e % rows);
  if (r < p) K[int64_t(c) * lda + r] = Kp[int64_t(c) * ldk + r];
  if (r < q) V[int64_t(c) * ldv + r] = Vp[int64_t(c) * ldk + r];
}

// FASTPI_JACOBI_RESIDENT=1 selects the resident-block schedule (same pairs,
// same arithmetic in the same order, so the same results; fewer loads and
// waits per round).
bool resident_schedule() {
  const char* e = std::getenv("FASTPI_JACOBI_RESIDENT");
  return e && e[0] == '1' && e[1] == 0;
}

template <int P, bool VS>
size_t block_smem(int ldk) {
  return ((VS ? 2 : 1) * size_t(P) * ldk + 4 * size_t(P) * P) * sizeof(float);
}

template <int P, bool VS>
bool launch_block(fastpi_ctx* hc, float* K, float* V, int n, JacobiStats* stats, float* ms_out, int* sweeps,
                  bool* used_res) {
  cudaStream_t st = hc->stream;
  constexpr int B = P / 2;
  int nb = (n + B - 1) / B;
  if (nb & 1) ++nb;
  if (nb < 2) nb = 2;
  const int ldk = (n + 3) / 4 * 4;
  const size_t smem = block_smem<P, VS>(ldk);
  int max_smem = 0;
  CK(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, hc->device));
  if (smem > size_t(max_smem)) return false;
  // the resident schedule is used with staged panels only (the form it has
  // been checked on); cores that stream V from L2 keep the default schedule
  const bool res = VS && resident_schedule();
  const void* kern = res ? (const void*)k_jacobi_block<P, VS, true> : (const void*)k_jacobi_block<P, VS, false>;
  allow_max_dynamic_smem(kern);
  int occ = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, BT, smem));
  const int grid = nb / 2;
  if (occ < 1 || int64_t(occ) * hc->num_sms < grid) return false;

  DArr<BBar> gb(1, st);
  constexpr int NPART = 128;
  DArr<double> part(NPART, st);
  DArr<int> out(2, st);
  DArr<unsigned> ver(int64_t(nb) * VER_STRIDE, st);
  DArr<float> Kp(int64_t(ldk) * n, st), Vp(int64_t(ldk) * n, st);
  core_prepare(hc, K, n, n, n, ldk, Kp.get(), Vp.get(), part.get(), NPART, gb.get());
  CK(cudaMemsetAsync(out.get(), 0, 2 * sizeof(int), st));
  CK(cudaMemsetAsync(ver.get(), 0, size_t(nb) * VER_STRIDE * sizeof(unsigned), st));
  CK(cudaMemsetAsync(hc->dstatus.get(), 0, 4, st));

  BlkArgs a;
  a.K = Kp.get();
  a.V = Vp.get();
  a.ver = ver.get();
  a.n = n;
  a.ldk = ldk;
  a.nb = nb;
  a.tol = float(std::sqrt(double(n)) * 1.1920928955078125e-07);
  a.inner = INNER_SWEEPS;
  a.gb = gb.get();
  a.out = out.get();
  a.status = hc->dstatus.get();
  void* args[] = {&a};
  cudaEvent_t ev0, ev1;
  CK(cudaEventCreate(&ev0));
  CK(cudaEventCreate(&ev1));
  CK(cudaEventRecord(ev0, st));
  CK(cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(BT), args, smem, st));
  CK_LAUNCH();
  CK(cudaEventRecord(ev1, st));
  core_finish(hc, Kp.get(), Vp.get(), n, n, ldk, K, n, V, n);
  int ho[2] = {0, 0};
  d2h_sync(ho, out.get(), sizeof ho, st);
  unsigned stat = 0;
  d2h_sync(&stat, hc->dstatus.get(), 4, st);
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, ev0, ev1));
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  if (stat & ST_BARRIER_TIMEOUT) fail(FASTPI_ERR_NO_CONVERGENCE, "block Jacobi SVD: a device-wide wait timed out");
#ifdef FASTPI_PHASE_CLOCKS
  {
    long long clk[8] = {0};
    CK(cudaMemcpyFromSymbol(clk, g_phase_clk, sizeof clk));
    const long long rounds = std::max<long long>(1, int64_t(ho[0]) * (nb - 1));
    fprintf(stderr,
            "block P=%d n=%d sweeps=%d ms=%.3f per-round clk: wait %lld load %lld gram %lld inner %lld ywait %lld "
            "apply %lld sweep-bar %lld\n",
            P, n, ho[0], ms, clk[5] / rounds, clk[0] / rounds, clk[1] / rounds, clk[2] / rounds, clk[6] / rounds,
            clk[3] / rounds, clk[4] / rounds);
    const long long z[8] = {0};
    CK(cudaMemcpyToSymbol(g_phase_clk, z, sizeof z));
  }
#endif
  *ms_out = ms;
  *sweeps = ho[0];
  *used_res = res;
  if (stats) {
    stats->max_sweeps_used = ho[0];
    stats->hit_cap = (stat & ST_JACOBI_SWEEPS) != 0;
  }
  return true;
}

}  // namespace

namespace jdev {

void core_prepare(fastpi_ctx* hc, const float* K, int64_t lda, int p, int q, int ldk, float* Kp, float* Vp,
                  double* part, int npart, BBar* gb) {
  cudaStream_t st = hc->stream;
  // |K|_F^2 over the p x q entries (K packed: lda == p, or a square core)
  k_b_sumsq_part<<<npart, 256, 0, st>>>(K, int64_t(lda) * q, part);
  CK_LAUNCH();
  k_b_sumsq_final<<<1, 32, 0, st>>>(part, npart, gb);
  CK_LAUNCH();
  k_b_pad_in<<<unsigned((int64_t(ldk) * q + 255) / 256), 256, 0, st>>>(K, lda, p, q, ldk, Kp, Vp);
  CK_LAUNCH();
}

void core_finish(fastpi_ctx* hc, const float* Kp, const float* Vp, int p, int q, int ldk, float* K, int64_t lda,
                 float* V, int64_t ldv) {
  const int rows = p > q ? p : q;
  k_b_pad_out<<<unsigned((int64_t(rows) * q + 255) / 256), 256, 0, hc->stream>>>(Kp, Vp, p, q, ldk, K, lda, V, ldv);
  CK_LAUNCH();
}

}  // namespace jdev

// Tiling of the core SVD from the environment (measurement switches):
// FASTPI_CORE_KERNEL=block selects the single-CTA kernel, FASTPI_CORE_P=16|32
// the panel, FASTPI_CORE_C=1..8 the CTAs per cluster, FASTPI_CORE_FAST=0 the
// IEEE Gram sweep, FASTPI_JACOBI_RESIDENT=1 the resident-block schedule,
// FASTPI_CORE_EARLY the early-exit threshold of the sweeps.
static bool env_int(const char* name, int* v) {
  const char* e = std::getenv(name);
  if (!e || !*e) return false;
  char* end = nullptr;
  const long x = std::strtol(e, &end, 10);
  if (*end) return false;
  *v = int(x);
  return true;
}

bool jacobi_svd_block(fastpi_ctx* hc, float* K, float* V, int n, double* sig, int32_t* perm, JacobiStats* stats,
                      const CoreTiling* tiling, float* ms_out, int* sweeps_out) {
  if (n < 2) return false;
  float ms = 0;
  int sweeps = 0;
  bool res = false;
  bool ok = false;
  CoreTiling tl;
  if (tiling) {
    tl = *tiling;
  } else {
    tuned_core_tiling(n, &tl);
    const char* kind = std::getenv("FASTPI_CORE_KERNEL");
    tl.single_cta = kind && std::string(kind) == "block";
    int v = 0;
    if (env_int("FASTPI_CORE_P", &v) && (v == 16 || v == 32)) tl.panel = v;
    if (env_int("FASTPI_CORE_C", &v) && v >= 1 && v <= 8) tl.parts = v;
    if (env_int("FASTPI_CORE_FAST", &v)) tl.fast_solve = v != 0;
    if (const char* e = std::getenv("FASTPI_CORE_EARLY")) {
      const double x = std::atof(e);
      if (x > 0 && x < 1) tl.early_exit = float(x);
    }
    if (std::getenv("FASTPI_JACOBI_RESIDENT")) tl.resident = resident_schedule();
  }
  if (!tl.single_cta) ok = jacobi_svd_cluster(hc, K, n, V, n, n, n, tl, stats, &ms, &sweeps, &res);
  if (!ok && !(tl.strict && !tl.single_cta)) {
    // the single-CTA kernel (its resident form from the environment only)
    ok = launch_block<16, true>(hc, K, V, n, stats, &ms, &sweeps, &res);
    if (!ok) ok = launch_block<16, false>(hc, K, V, n, stats, &ms, &sweeps, &res);
  }
  if (!ok) return false;
  if (ms_out) *ms_out = ms;
  if (sweeps_out) *sweeps_out = sweeps;
  std::vector<JacobiProblem<float>> pr(1);
  pr[0] = JacobiProblem<float>{K, V, n, n, n, n};
  jacobi_sort_columns<float>(hc, pr, sig, perm);
  const double dn = n;
  note_svd(SVD_CORE32, ms, 12 * dn * dn * dn, double(sweeps) * (dn * (dn - 1) / 2) * (12 * dn + 6 * dn), res);
  return true;
}


namespace {
__global__ void k_core_uv(int n, const float* __restrict__ K, const float* __restrict__ V,
                          const double* __restrict__ sig, const int32_t* __restrict__ perm, float* __restrict__ U,
                          float* __restrict__ Vs) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= int64_t(n) * n) return;
  const int t = int(e / n), i = int(e % n);
  const int src = perm[t];
  const double s = sig[t];
  U[e] = s > 0 ? float(double(K[int64_t(src) * n + i]) / s) : 0.f;
  Vs[e] = V[int64_t(src) * n + i];
}
}  // namespace

void core_vectors_f32(fastpi_ctx* h, int n, const float* K, const float* V, const double* sig, const int32_t* perm,
                      float* U, float* Vs) {
  k_core_uv<<<unsigned((int64_t(n) * n + 255) / 256), 256, 0, h->stream>>>(n, K, V, sig, perm, U, Vs);
  CK_LAUNCH();
}

}  // namespace fastpi
