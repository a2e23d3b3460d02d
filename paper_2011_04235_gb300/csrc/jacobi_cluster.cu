// Block one-sided Jacobi SVD of one FP32 core matrix with every block pair's
// rows split over a thread-block cluster.
//
// The schedule is the one of the single-CTA block kernel (jacobi_block.cu):
// column blocks of B = P / 2 columns paired by the circle method, n_b - 1
// rounds per sweep, one two-sided Jacobi sweep on the P x P Gram matrix of a
// block pair per round, K_IJ <- X Q and V_IJ <- Y Q.  What differs is who
// does a pair's work: a cluster of C CTAs, CTA `part` holding rows
// [part * rpc, (part + 1) * rpc) of the two panels.  Per round each CTA
//   1. waits for the CTAs that last wrote ITS rows of the two blocks
//      (per-(block, part) release / acquire round counters, bounded waits);
//   2. copies its rows of the K panel (and, overlapped, of the V panel) into
//      shared memory with 16-byte asynchronous copies;
//   3. forms its partial Gram matrix (P x P) and stores it into the shared
//      memory of every CTA of the cluster (distributed shared memory); one
//      cluster barrier later every CTA sums the C partials in rank order from
//      its own shared memory, so all C CTAs hold the same Gram matrix bit for
//      bit;
//   4. runs the same Jacobi sweep on it (the same rotations in every CTA),
//      takes one Newton-Schulz step on the accumulated rotation Q (so that it
//      is orthonormal to rounding, without the drift of FP32 rotations) and
//      applies Q to its own rows.
// Load, Gram and update shrink by C per CTA and C times more SMs work; the
// price is one cluster barrier and C remote stores per Gram entry per round.
//
// Cluster barriers cannot time out, so every CTA of a cluster executes the
// same sequence of them on every path: one per round, two at the end of each
// sweep (exchange of the stop decision), one before leaving.  A CTA whose
// bounded wait ran out does not leave on its own: it flags the failure in the
// header its peers read after the next barrier, and the whole cluster leaves
// together.  No CTA leaves while a peer may still read its shared memory.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include "jacobi.cuh"
#include "jacobi_dev.cuh"

namespace cg = cooperative_groups;

namespace fastpi {
namespace {

using namespace jdev;

constexpr int CT = 256;                 // threads per CTA (8 warps)
constexpr int C_MAX_SWEEPS = 30;

struct ClArgs {
  float* K;         // ldk x n column-major: in A (rows >= its row count zero), out A J
  float* V;         // ldk x n column-major: in I, out J
  unsigned* ver;    // [nb * C * VER_STRIDE]: rounds completed per (block, row part)
  int n, ldk, rpc;  // n columns; ldk = C * rpc rows (>= the row count); rpc a multiple of 4
  int len;          // the longer side of the problem (the absolute zero threshold scales with it)
  int nb;           // number of column blocks (even)
  int parts;        // C: CTAs per cluster the grid was laid out for
  float tol;
  float early;      // a sweep whose rotations all stay below this ends the iteration
  BBar* gb;
  int* out;         // [0] sweeps used, [1] hit the sweep cap
  unsigned* status;
};

#ifdef FASTPI_PHASE_CLOCKS
__device__ long long g_cphase_clk[8];
#define CPHASE_MARK(k)                                     \
  do {                                                     \
    if (blockIdx.x == gridDim.x / 2 && threadIdx.x == 0) { \
      const long long t_ = clock64();                      \
      g_cphase_clk[k] += t_ - t_mark;                      \
      t_mark = t_;                                         \
    }                                                      \
  } while (0)
#else
#define CPHASE_MARK(k) \
  do {                 \
  } while (0)
#endif

template <int P, bool RES, bool FAST>
__global__ void __launch_bounds__(CT) k_jacobi_cluster(ClArgs a) {
  constexpr int B = P / 2;    // columns per block
  constexpr int TW = P / 4;   // Gram tile edge (4 x 4 tiles of TW x TW)
  constexpr int PP = P * P;
  cg::cluster_group cl = cg::this_cluster();
  const int C = int(cl.num_blocks());
  const int part = int(cl.block_rank());
  // a launch whose clusters do not match the layout leaves at once, every CTA
  // alike, before any barrier
  if (C != a.parts || int(gridDim.x) % C != 0) {
    if (threadIdx.x == 0) atomicOr(a.status, ST_BAD_INDEX);
    return;
  }
  const int cid = int(blockIdx.x) / C;     // cluster = pair slot
  const int ncl = int(gridDim.x) / C;
  const int rpc = a.rpc, ldk = a.ldk, n = a.n;
  const int row0 = part * rpc;
  extern __shared__ float4 smem4[];
  float* Xs = reinterpret_cast<float*>(smem4);   // [P][rpc]: this part's rows of the K panel
  float* Ys = Xs + size_t(P) * rpc;              // [P][rpc]: of the V panel
  float* G = Ys + size_t(P) * rpc;               // [P][P]
  float* Q = G + PP;
  float* Gn = Q + PP;
  float* Qn = Gn + PP;
  float* Rx = Qn + PP;                           // [2][C][P][P]: the partial Grams of the cluster's CTAs,
                                                 // pushed here by their owners, by round parity
  __shared__ int s_hdr[2][8];                    // failure flags of the cluster's CTAs, by round parity
  __shared__ int s_dec;                          // stop decision at the end of a sweep
  __shared__ float s_sc[P], s_so[P];
  __shared__ int s_gcol[P];
  __shared__ int s_rot, s_ok, s_pair_rot;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float tabs = [&] {
    const float ne = float(a.len) * 1.1920929e-7f;
    return float(double(ne) * double(ne) * a.gb->fro2);
  }();
  const float tol2 = a.tol * a.tol, early2 = a.early * a.early;
  if (tid == 0) s_rot = 0;
  const int nq = rpc / 4;   // 16-byte chunks per column part
  int sweep = 0;
  // resident schedule (as in the single-CTA kernel): clusters swap slots in
  // fixed pairs every round, so each keeps one of its blocks in shared memory
  int held0 = -1, held1 = -1;
  const bool slot_fixed = (ncl & 1) && cid == ncl - 1;
#ifdef FASTPI_PHASE_CLOCKS
  long long t_mark = clock64();
#endif
  for (;;) {
    for (int rr = 0; rr < a.nb - 1; ++rr) {
      const unsigned t = unsigned(sweep) * unsigned(a.nb - 1) + unsigned(rr);
      const int buf = int(t & 1u);
      const int slot = (RES && !slot_fixed) ? (cid ^ int(t & 1u)) : cid;
      int bi, bj;
      circle_pair(slot, rr, a.nb, bi, bj);
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
      auto pcol = [&](int c) { return (c < B ? hi : hj) * B + (c & (B - 1)); };
      if (tid < P) {
        const int g = tid < B ? bi * B + tid : bj * B + (tid - B);
        s_gcol[tid] = g < n ? g : -1;
      }
      // 1. wait until the previous round on this part of both blocks is done:
      // lanes 0 and 1 poll the two counters with one load instruction, so the
      // two acquire latencies overlap
      if (tid < 2) {
        const bool needed = (need & (tid == 0 ? 1 : 2)) != 0;
        const unsigned* vp = a.ver + (size_t(tid == 0 ? bi : bj) * C + part) * VER_STRIDE;
        int ok = 1;
        bool rdy = !needed || b_ld_acquire(vp) >= t;
        if (!__all_sync(0x3u, rdy)) {
          const unsigned long long t0 = b_gtimer();
          unsigned spins = 0;
          for (;;) {
            if (!rdy) rdy = b_ld_acquire(vp) >= t;
            if (__all_sync(0x3u, rdy)) break;
            int late = 0;
            if ((++spins & 63u) == 0) late = (b_gtimer() - t0 > B_WAIT_NS) ? 1 : 0;
            if (__shfl_sync(0x3u, late, 0)) {   // lane 0 decides for both
              if (tid == 0) atomicOr(a.status, ST_BARRIER_TIMEOUT);
              ok = 0;
              break;
            }
          }
        }
        if (tid == 0) {
          s_ok = ok;
          s_pair_rot = 0;
        }
      }
      __syncthreads();
      const bool ok = s_ok != 0;
      CPHASE_MARK(5);
      if (ok) {
        // 2. this part's rows of the panels: K (first group), V (second group)
        for (int e = tid; e < P * nq; e += CT) {
          const int c = e / nq, r4 = (e - c * nq) * 4;
          if (!(need & (c < B ? 1 : 2))) continue;
          const int g = s_gcol[c];
          float* d = Xs + size_t(pcol(c)) * rpc + r4;
          if (g >= 0)
            cp_async16(d, a.K + size_t(g) * ldk + row0 + r4);
          else
            *reinterpret_cast<float4*>(d) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        cp_async_commit();
        for (int e = tid; e < P * nq; e += CT) {
          const int c = e / nq, r4 = (e - c * nq) * 4;
          if (!(need & (c < B ? 1 : 2))) continue;
          const int g = s_gcol[c];
          float* d = Ys + size_t(pcol(c)) * rpc + r4;
          if (g >= 0)
            cp_async16(d, a.V + size_t(g) * ldk + row0 + r4);
          else
            *reinterpret_cast<float4*>(d) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        CPHASE_MARK(0);
        // 3. partial Gram of this part's rows: warp w owns tiles w, w + 8 of
        // the 4 x 4 tiles; lanes split the rows.  Each sum is stored straight
        // into slot `part` of every CTA of the cluster (this one included),
        // so that after the barrier each CTA reads only its own shared memory
        float* gp = Rx + (size_t(buf) * C + part) * PP;
        for (int tile = warp; tile < 16; tile += CT / 32) {
          const int tp = tile >> 2, tq = tile & 3;
          float acc[TW * TW];
#pragma unroll
          for (int i = 0; i < TW * TW; ++i) acc[i] = 0.f;
          const float* xa = Xs + size_t(pcol(tp * TW)) * rpc;
          const float* xb = Xs + size_t(pcol(tq * TW)) * rpc;
#pragma unroll 2
          for (int r = lane; r < rpc; r += 32) {
            float u[TW], w[TW];
#pragma unroll
            for (int i = 0; i < TW; ++i) {
              u[i] = xa[size_t(i) * rpc + r];
              w[i] = xb[size_t(i) * rpc + r];
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
              for (int c = 0; c < C; ++c) cl.map_shared_rank(gp, c)[(tp * TW + i) * P + tq * TW + j] = acc[e];
            }
          } else if ((lane & (32 / (TW * TW) - 1)) == 0) {
            const int i = off / TW, j = off % TW;
            for (int c = 0; c < C; ++c) cl.map_shared_rank(gp, c)[(tp * TW + i) * P + tq * TW + j] = acc[0];
          }
        }
      }
      if (tid < C) cl.map_shared_rank(&s_hdr[buf][0], tid)[part] = ok ? 0 : 1;
      CPHASE_MARK(1);
      // the exchange: every CTA of the cluster has pushed its partial Gram and
      // its flag into every CTA's shared memory
      cl.sync();
      CPHASE_MARK(7);
      int anyerr = 0;
      for (int c = 0; c < C; ++c) anyerr |= s_hdr[buf][c];
      if (anyerr) {
        // leave together; nobody touches a peer's shared memory after this barrier
        cp_async_wait<0>();
        __syncthreads();
        cl.sync();
        return;
      }
      {
        const float* rx = Rx + size_t(buf) * C * PP;
        for (int e = tid; e < PP; e += CT) {
          float sum = 0.f;
          for (int c = 0; c < C; ++c) sum += rx[size_t(c) * PP + e];
          G[e] = sum;
          Q[e] = (e / P == e % P) ? 1.f : 0.f;
        }
      }
      __syncthreads();
      CPHASE_MARK(2);
      // 4. the Jacobi sweep on G (identical in every CTA of the cluster): with
      // one barrier per inner round and fast rotations, or the IEEE form with
      // two barriers per inner round
      float* Qf = Q;
      if constexpr (FAST) {
        inner_solve_fast<P, CT>(G, Gn, Q, tid, tabs, tol2, early2, rr != 0, &s_rot, &s_pair_rot);
        __syncthreads();
      } else {
        Qf = inner_solve_cta<P, CT>(G, Gn, Q, Qn, s_sc, s_so, tid, tabs, tol2, early2, 1, rr != 0, &s_rot,
                                    &s_pair_rot);
      }
      // Q orthonormal to rounding (G and Gn are free now)
      if (s_pair_rot) Qf = ns_orthonormalize<P, CT>(Qf, Gn, Qf == Q ? Qn : Q, tid);
      CPHASE_MARK(3);
      cp_async_wait<0>();
      __syncthreads();
      CPHASE_MARK(6);
      // K_IJ <- X Q, V_IJ <- Y Q on this part's rows (nothing to write when no
      // pair of the block pair rotated: Q = I)
      if (RES) {
        for (int r = tid; s_pair_rot && r < rpc; r += CT) {
          float u[P], v[P];
#pragma unroll
          for (int j = 0; j < P; ++j) u[j] = v[j] = 0.f;
#pragma unroll
          for (int c = 0; c < P; ++c) {
            const float xc = Xs[size_t(pcol(c)) * rpc + r];
            const float yc = Ys[size_t(pcol(c)) * rpc + r];
            const float4* q4 = reinterpret_cast<const float4*>(Qf + c * P);
#pragma unroll
            for (int j4 = 0; j4 < P / 4; ++j4) {
              const float4 qv = q4[j4];
              u[4 * j4 + 0] = fmaf(xc, qv.x, u[4 * j4 + 0]);
              u[4 * j4 + 1] = fmaf(xc, qv.y, u[4 * j4 + 1]);
              u[4 * j4 + 2] = fmaf(xc, qv.z, u[4 * j4 + 2]);
              u[4 * j4 + 3] = fmaf(xc, qv.w, u[4 * j4 + 3]);
              v[4 * j4 + 0] = fmaf(yc, qv.x, v[4 * j4 + 0]);
              v[4 * j4 + 1] = fmaf(yc, qv.y, v[4 * j4 + 1]);
              v[4 * j4 + 2] = fmaf(yc, qv.z, v[4 * j4 + 2]);
              v[4 * j4 + 3] = fmaf(yc, qv.w, v[4 * j4 + 3]);
            }
          }
#pragma unroll
          for (int j = 0; j < P; ++j) {
            const int g = s_gcol[j];
            if (g >= 0) {
              __stcg(a.K + size_t(g) * ldk + row0 + r, u[j]);
              __stcg(a.V + size_t(g) * ldk + row0 + r, v[j]);
            }
            Xs[size_t(pcol(j)) * rpc + r] = g >= 0 ? u[j] : 0.f;
            Ys[size_t(pcol(j)) * rpc + r] = g >= 0 ? v[j] : 0.f;
          }
        }
      } else {
        // one item = one row and one half of the P output columns (items of
        // one warp share the half: every store writes 32 consecutive rows)
        constexpr int H = P / 2;
        for (int it = tid; s_pair_rot && it < 2 * rpc; it += CT) {
          const int half = it >= rpc ? 1 : 0, r = it - half * rpc, j0 = half * H;
          float u[H], v[H];
#pragma unroll
          for (int j = 0; j < H; ++j) u[j] = v[j] = 0.f;
#pragma unroll
          for (int c = 0; c < P; ++c) {
            const float xc = Xs[size_t(pcol(c)) * rpc + r];
            const float yc = Ys[size_t(pcol(c)) * rpc + r];
            const float4* q4 = reinterpret_cast<const float4*>(Qf + c * P + j0);
#pragma unroll
            for (int j4 = 0; j4 < H / 4; ++j4) {
              const float4 qv = q4[j4];
              u[4 * j4 + 0] = fmaf(xc, qv.x, u[4 * j4 + 0]);
              u[4 * j4 + 1] = fmaf(xc, qv.y, u[4 * j4 + 1]);
              u[4 * j4 + 2] = fmaf(xc, qv.z, u[4 * j4 + 2]);
              u[4 * j4 + 3] = fmaf(xc, qv.w, u[4 * j4 + 3]);
              v[4 * j4 + 0] = fmaf(yc, qv.x, v[4 * j4 + 0]);
              v[4 * j4 + 1] = fmaf(yc, qv.y, v[4 * j4 + 1]);
              v[4 * j4 + 2] = fmaf(yc, qv.z, v[4 * j4 + 2]);
              v[4 * j4 + 3] = fmaf(yc, qv.w, v[4 * j4 + 3]);
            }
          }
#pragma unroll
          for (int j = 0; j < H; ++j) {
            const int g = s_gcol[j0 + j];
            if (g >= 0) {
              __stcg(a.K + size_t(g) * ldk + row0 + r, u[j]);
              __stcg(a.V + size_t(g) * ldk + row0 + r, v[j]);
            }
          }
        }
      }
      __syncthreads();
      CPHASE_MARK(4);
      // hand this part of both blocks to the next round (lanes 0 and 1: one
      // release instruction for the two counters)
      if (tid < 2) b_st_release(a.ver + (size_t(tid == 0 ? bi : bj) * C + part) * VER_STRIDE, t + 1u);
      if (rr == a.nb - 2) {
        // end of a sweep: combine the rotation flags of all CTAs (the flags
        // of the CTAs of one cluster are equal)
        if (tid == 0) {
          atomicMax(&a.gb->flag[sweep % 3], s_rot);
          if (blockIdx.x == 0) a.gb->flag[(sweep + 1) % 3] = 0;
        }
        const bool bok = b_barrier(a.gb, a.status);
        ++sweep;
        const int any = *(volatile int*)&a.gb->flag[(sweep - 1) % 3];
        __syncthreads();
        if (tid == 0) {
          s_rot = 0;
          s_dec = !bok ? 2 : ((any < 2 || sweep >= C_MAX_SWEEPS) ? 1 : 0);
        }
        // the same decision in every CTA of the cluster
        cl.sync();
        int dec = 0;
        for (int c = 0; c < C; ++c) dec = max(dec, *cl.map_shared_rank(&s_dec, c));
        cl.sync();
        if (dec) {
          if (dec == 1 && blockIdx.x == 0 && tid == 0) {
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

size_t cluster_smem(int P, int C, int rpc) {
  return (2 * size_t(P) * rpc + (4 + 2 * size_t(C)) * size_t(P) * P) * sizeof(float);
}

// C (CTAs per cluster) for an n-column core: as many row parts as keep the
// clusters of one round on the SMs once each, at most 8, unless the caller
// (autotuned table or environment) gives one.
int pick_parts(int slots, int num_sms, int want) {
  if (want >= 1 && want <= 8) return want;
  int c = num_sms / std::max(slots, 1);
  return std::max(1, std::min(8, c));
}

template <int P, bool RES, bool FAST>
bool launch_cluster(fastpi_ctx* hc, float* K, int64_t lda, float* V, int64_t ldv, int p, int n, int parts,
                    float early, JacobiStats* stats, float* ms_out, int* sweeps) {
  cudaStream_t st = hc->stream;
  constexpr int B = P / 2;
  int nb = (n + B - 1) / B;
  if (nb & 1) ++nb;
  if (nb < 2) nb = 2;
  const int slots = nb / 2;
  const int C = parts;
  const int len = std::max(p, n);
  int rpc = (len + C - 1) / C;
  rpc = (rpc + 3) / 4 * 4;
  const int ldk = C * rpc;
  const size_t smem = cluster_smem(P, C, rpc);
  int max_smem = 0;
  CK(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, hc->device));
  if (smem + 1024 > size_t(max_smem)) return false;
  const void* kern = (const void*)k_jacobi_cluster<P, RES, FAST>;
  allow_max_dynamic_smem(kern);

  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(slots * C));
  cfg.blockDim = dim3(CT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = unsigned(C);
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeCooperative;
  at[1].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  // every cluster of the grid must be resident at once (the CTAs wait on one
  // another)
  int ncl = 0;
  if (cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  if (ncl < slots) return false;
  // the CTAs wait on one another, so the launch is cooperative (all clusters
  // resident at once, also beside other instances' kernels on other streams);
  // FASTPI_CORE_NOCOOP=1 drops that attribute for profilers that do not pass
  // a cooperative cluster launch through (a single instance alone on the GPU
  // still finds every cluster resident: checked above)
  const char* nc = std::getenv("FASTPI_CORE_NOCOOP");
  cfg.numAttrs = (nc && nc[0] == '1' && nc[1] == 0) ? 1 : 2;

  DArr<BBar> gb(1, st);
  constexpr int NPART = 128;
  DArr<double> partsum(NPART, st);
  DArr<int> out(2, st);
  DArr<unsigned> ver(int64_t(nb) * C * VER_STRIDE, st);
  DArr<float> Kp(int64_t(ldk) * n, st), Vp(int64_t(ldk) * n, st);
  core_prepare(hc, K, lda, p, n, ldk, Kp.get(), Vp.get(), partsum.get(), NPART, gb.get());
  CK(cudaMemsetAsync(out.get(), 0, 2 * sizeof(int), st));
  CK(cudaMemsetAsync(ver.get(), 0, size_t(nb) * C * VER_STRIDE * sizeof(unsigned), st));
  CK(cudaMemsetAsync(hc->dstatus.get(), 0, 4, st));

  ClArgs a;
  a.K = Kp.get();
  a.V = Vp.get();
  a.ver = ver.get();
  a.n = n;
  a.len = len;
  a.ldk = ldk;
  a.rpc = rpc;
  a.nb = nb;
  a.parts = C;
  a.tol = float(std::sqrt(double(len)) * 1.1920928955078125e-07);
  a.early = early;
  a.gb = gb.get();
  a.out = out.get();
  a.status = hc->dstatus.get();
  cudaEvent_t ev0, ev1;
  CK(cudaEventCreate(&ev0));
  CK(cudaEventCreate(&ev1));
  CK(cudaEventRecord(ev0, st));
  const cudaError_t le = cudaLaunchKernelEx(&cfg, k_jacobi_cluster<P, RES, FAST>, a);
  if (le != cudaSuccess) {
    // not launchable in this form (for example a cooperative cluster launch
    // refused): nothing ran; the caller takes the single-CTA kernel
    (void)cudaGetLastError();
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    return false;
  }
  CK_LAUNCH();
  CK(cudaEventRecord(ev1, st));
  core_finish(hc, Kp.get(), Vp.get(), p, n, ldk, K, lda, V, ldv);
  int ho[2] = {0, 0};
  d2h_sync(ho, out.get(), sizeof ho, st);
  unsigned stat = 0;
  d2h_sync(&stat, hc->dstatus.get(), 4, st);
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, ev0, ev1));
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  if (stat & ST_BARRIER_TIMEOUT) fail(FASTPI_ERR_NO_CONVERGENCE, "cluster Jacobi SVD: a bounded wait timed out");
  if (stat & ST_BAD_INDEX) {
    // the launch did not get its clusters (the kernel left at once, before
    // touching K or V): the caller takes the single-CTA kernel
    CK(cudaMemsetAsync(hc->dstatus.get(), 0, 4, st));
    return false;
  }
#ifdef FASTPI_PHASE_CLOCKS
  {
    long long clk[8] = {0};
    CK(cudaMemcpyFromSymbol(clk, g_cphase_clk, sizeof clk));
    const long long rounds = std::max<long long>(1, int64_t(ho[0]) * (nb - 1));
    fprintf(stderr,
            "cluster P=%d C=%d n=%d sweeps=%d ms=%.3f per-round clk: wait %lld load %lld gram %lld xchg %lld "
            "sum %lld solve %lld ywait %lld update %lld\n",
            P, C, n, ho[0], ms, clk[5] / rounds, clk[0] / rounds, clk[1] / rounds, clk[7] / rounds,
            clk[2] / rounds, clk[3] / rounds, clk[6] / rounds, clk[4] / rounds);
    const long long z[8] = {0};
    CK(cudaMemcpyToSymbol(g_cphase_clk, z, sizeof z));
  }
#endif
  *ms_out = ms;
  *sweeps = ho[0];
  if (stats) {
    stats->max_sweeps_used = ho[0];
    stats->hit_cap = (stat & ST_JACOBI_SWEEPS) != 0;
  }
  return true;
}

}  // namespace

bool jacobi_svd_cluster(fastpi_ctx* hc, float* K, int64_t lda, float* V, int64_t ldv, int p, int n,
                        const CoreTiling& tiling, JacobiStats* stats, float* ms, int* sweeps, bool* used_res) {
  const int P = tiling.panel;
  const int B = P / 2;
  int nb = (n + B - 1) / B;
  if (nb & 1) ++nb;
  const int C = pick_parts(std::max(nb / 2, 1), hc->num_sms, tiling.parts);
  *used_res = tiling.resident;
#define FASTPI_CL(PV, RV, WV) \
  launch_cluster<PV, RV, WV>(hc, K, lda, V, ldv, p, n, C, tiling.early_exit, stats, ms, sweeps)
  const bool r = tiling.resident, w = tiling.fast_solve;
  if (P == 16) return r ? (w ? FASTPI_CL(16, true, true) : FASTPI_CL(16, true, false))
                        : (w ? FASTPI_CL(16, false, true) : FASTPI_CL(16, false, false));
  if (P == 32) return r ? (w ? FASTPI_CL(32, true, true) : FASTPI_CL(32, true, false))
                        : (w ? FASTPI_CL(32, false, true) : FASTPI_CL(32, false, false));
#undef FASTPI_CL
  return false;
}

}  // namespace fastpi
