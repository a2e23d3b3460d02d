// One-sided Jacobi SVD of one FP32 core matrix inside one thread-block
// cluster (16 CTAs), with the matrix resident in distributed shared memory.
//
// The rounds of a Jacobi sweep are sequential, so for the core sizes of the
// incremental update (n ~ 300-900) a sweep is bound by the latency of a round,
// not by arithmetic.  Keeping K on chip removes every global-memory round trip
// from a round: CTA q of the cluster holds rows [q h, (q+1) h) of K (and of
// V = J when it fits), column-major in its shared memory.  One round (the
// same circle-method pairing as the batched kernel):
//   1. every CTA: partial alpha, beta, gamma of every pair over its rows;
//   2. cluster barrier; CTA q reduces the pairs [q s, (q+1) s) over the 16
//      CTAs through DSMEM, decides each rotation (c, s) and writes it into the
//      shared memory of all 16 CTAs (and into a rotation log when V is not
//      kept on chip);
//   3. cluster barrier; every CTA rotates its rows of the pair columns.
// At the end of a sweep the CTAs exchange "did I rotate" flags; when no pair
// of a whole sweep rotated the matrix is converged.  When V does not fit, it
// is rebuilt afterwards by replaying the rotation log on blocks of rows of
// the identity, in parallel over the rows.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>

#include "jacobi.cuh"

namespace cg = cooperative_groups;

namespace fastpi {
namespace {

constexpr int CT = 512;      // threads per CTA
constexpr int MAXCL = 16;    // CTAs per cluster
constexpr int MAX_SWEEPS = 30;
constexpr float EARLY_OFF = 1e-4f;   // see the end-of-sweep test
constexpr int REPLAY_ROWS = 8;
constexpr int REPLAY_BATCH = 16;   // rounds of rotations staged in shared memory at once

// circle-method pair of `slot` in round rr (0 <= rr < qe - 1, 0 <= slot < qe/2)
__device__ __forceinline__ void pair_of(int slot, int rr, int qe, int& i, int& j) {
  const int m = qe - 1;
  if (slot == 0) {
    i = m;
    j = rr;
  } else {
    i = rr + slot;
    if (i >= m) i -= m;
    j = rr - slot;
    if (j < 0) j += m;
  }
  if (i > j) {
    const int t = i;
    i = j;
    j = t;
  }
}

// (x, y) <- (c x - s y, s x + c y) on 4 n4 consecutive floats of two columns
__device__ __forceinline__ void rotate4(float4* xi, float4* xj, int n4, float c, float s) {
#pragma unroll 2
  for (int u = 0; u < n4; ++u) {
    const float4 x = xi[u], y = xj[u];
    xi[u] = make_float4(c * x.x - s * y.x, c * x.y - s * y.y, c * x.z - s * y.z, c * x.w - s * y.w);
    xj[u] = make_float4(s * x.x + c * y.x, s * x.y + c * y.y, s * x.z + c * y.z, s * x.w + c * y.w);
  }
}

struct CArgs {
  float* K;          // n x n column-major (ld n): in A, out B = A J
  float* V;          // n x n column-major (ld n): out J (only when with_v)
  float2* rotlog;    // rotations, [round][slot] (only when !with_v)
  int n, qe, np, R, h, hp, with_v;
  float tol;
  int* out;          // [0] rounds, [1] sweeps
  unsigned* status;
};

__global__ void __launch_bounds__(CT, 1) k_jacobi_cluster(CArgs a) {
  cg::cluster_group cl = cg::this_cluster();
  const int CL = int(cl.num_blocks());
  const int rank = int(cl.block_rank());
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  extern __shared__ __align__(16) float smem[];
  const int n = a.n, qe = a.qe, np = a.np, R = a.R, h = a.h, hp = a.hp;
  const int hq = hp / 4;   // float4 per local column (hp is a multiple of 4)
  const size_t blk = size_t(qe) * hp;
  float* Ks = smem;
  float* Vs = Ks + blk;                       // only when with_v
  float4* part = reinterpret_cast<float4*>(Ks + (a.with_v ? 2 * blk : blk));   // (alpha, beta, gamma, -)
  float2* rot = reinterpret_cast<float2*>(part + np);                          // (c, s)
  float* fro = reinterpret_cast<float*>(rot + np);                             // [MAXCL]
  int* flg = reinterpret_cast<int*>(fro + MAXCL);   // [2][MAXCL]
  __shared__ int s_rot;
  __shared__ float s_red[CT / 32];
  const int r0 = rank * h;
  const int hh = max(0, min(h, n - r0));
  for (size_t e = tid; e < blk; e += CT) {
    const int j = int(e / hp), i = int(e % hp);
    Ks[e] = (j < n && i < hh) ? a.K[size_t(j) * n + r0 + i] : 0.f;
    if (a.with_v) Vs[e] = (j < n && i < hh && r0 + i == j) ? 1.f : 0.f;
  }
  for (int e = tid; e < 2 * MAXCL; e += CT) flg[e] = 0;
  if (tid == 0) s_rot = 0;
  float f = 0.f;
  for (size_t e = tid; e < blk; e += CT) f = fmaf(Ks[e], Ks[e], f);
#pragma unroll
  for (int o = 16; o; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
  if (lane == 0) s_red[warp] = f;
  __syncthreads();
  if (tid == 0) {
    float t = 0.f;
    for (int w = 0; w < CT / 32; ++w) t += s_red[w];
    s_red[0] = t;
  }
  __syncthreads();
  cl.sync();   // every CTA initialised before any remote write
  if (tid < CL) cl.map_shared_rank(fro, tid)[rank] = s_red[0];
  cl.sync();
  float fro2 = 0.f;
  for (int q = 0; q < CL; ++q) fro2 += fro[q];
  const float ne = float(n) * 1.1920929e-7f;
  const float tabs = ne * ne * fro2;   // columns below this squared norm count as zero
  const int share = (np + CL - 1) / CL;
  const int s0 = rank * share;
  int sweep = 0, rr = 0;
  long long t = 0;
  for (;;) {
    // 1. partial dot products over the local rows, one thread per pair, four
    //    rows per 128-bit shared-memory load (rows past hh are zero)
    for (int slot = tid; slot < np; slot += CT) {
      int i, j;
      pair_of(slot, rr, qe, i, j);
      float al = 0.f, be = 0.f, ga = 0.f;
      if (j < n) {
        const float4* xi = reinterpret_cast<const float4*>(Ks + size_t(i) * hp);
        const float4* xj = reinterpret_cast<const float4*>(Ks + size_t(j) * hp);
#pragma unroll 2
        for (int u = 0; u < hq; ++u) {
          const float4 x = xi[u], y = xj[u];
          al = fmaf(x.x, x.x, fmaf(x.y, x.y, fmaf(x.z, x.z, fmaf(x.w, x.w, al))));
          be = fmaf(y.x, y.x, fmaf(y.y, y.y, fmaf(y.z, y.z, fmaf(y.w, y.w, be))));
          ga = fmaf(x.x, y.x, fmaf(x.y, y.y, fmaf(x.z, y.z, fmaf(x.w, y.w, ga))));
        }
      }
      part[slot] = make_float4(al, be, ga, 0.f);
    }
    cl.sync();
    // 2. reduce this CTA's share of pairs over the cluster; decide; broadcast
    for (int base = 0; base < share; base += CT / 16) {
      const int g = base + (tid >> 4), src = tid & 15;
      const int slot = s0 + g;
      const bool valid = g < share && slot < np;
      float al = 0.f, be = 0.f, ga = 0.f;
      if (valid && src < CL) {
        const float4 pv = cl.map_shared_rank(part, src)[slot];   // one 128-bit DSMEM load
        al = pv.x;
        be = pv.y;
        ga = pv.z;
      }
#pragma unroll
      for (int o = 8; o; o >>= 1) {
        al += __shfl_xor_sync(0xffffffffu, al, o);
        be += __shfl_xor_sync(0xffffffffu, be, o);
        ga += __shfl_xor_sync(0xffffffffu, ga, o);
      }
      if (valid) {
        int i, j;
        pair_of(slot, rr, qe, i, j);
        float c = 1.f, s = 0.f;
        if (j < n && al > tabs && be > tabs) {
          const float off = fabsf(ga) / (sqrtf(al) * sqrtf(be));
          if (off > a.tol) {
            const float zeta = (be - al) / (2.f * ga);
            const float tt = copysignf(1.f, zeta) / (fabsf(zeta) + hypotf(1.f, zeta));
            c = 1.f / sqrtf(1.f + tt * tt);
            s = c * tt;
            if (src == 0) s_rot = off > EARLY_OFF ? 2 : max(s_rot, 1);
          }
        }
        if (src < CL) cl.map_shared_rank(rot, src)[slot] = make_float2(c, s);   // one 64-bit DSMEM store
        if (!a.with_v && src == 0) a.rotlog[t * np + slot] = make_float2(c, s);
      }
    }
    cl.sync();
    // 3. rotate the local rows of both columns of every pair
    for (int slot = tid; slot < np; slot += CT) {
      const float2 cs = rot[slot];
      const float c = cs.x, s = cs.y;
      if (s == 0.f) continue;
      int i, j;
      pair_of(slot, rr, qe, i, j);
      rotate4(reinterpret_cast<float4*>(Ks + size_t(i) * hp), reinterpret_cast<float4*>(Ks + size_t(j) * hp), hq,
              c, s);
      if (a.with_v)
        rotate4(reinterpret_cast<float4*>(Vs + size_t(i) * hp), reinterpret_cast<float4*>(Vs + size_t(j) * hp), hq,
                c, s);
    }
    __syncthreads();
    ++t;
    if (++rr == R) {
      rr = 0;
      const int par = sweep & 1;
      if (tid < CL) cl.map_shared_rank(flg, tid)[par * MAXCL + rank] = s_rot;
      cl.sync();
      int any = 0;
      for (int q = 0; q < CL; ++q) any = max(any, flg[par * MAXCL + q]);
      __syncthreads();
      if (tid == 0) s_rot = 0;
      ++sweep;
      // converged: no rotation at all in this sweep, or only rotations with
      // off <= EARLY_OFF -- in the quadratic phase of convergence the next
      // sweep would then meet off ~ EARLY_OFF^2 < tol and rotate nothing
      if (any < 2) break;
      if (sweep >= MAX_SWEEPS) {
        if (rank == 0 && tid == 0) atomicOr(a.status, ST_JACOBI_SWEEPS);
        break;
      }
    }
  }
  for (size_t e = tid; e < blk; e += CT) {
    const int j = int(e / hp), i = int(e % hp);
    if (j < n && i < hh) {
      a.K[size_t(j) * n + r0 + i] = Ks[e];
      if (a.with_v) a.V[size_t(j) * n + r0 + i] = Vs[e];
    }
  }
  if (rank == 0 && tid == 0) {
    a.out[0] = int(t);
    a.out[1] = sweep;
  }
  cl.sync();   // no CTA leaves while another may still address its shared memory
}

// V = J rebuilt from the rotation log: block b owns rows [b RB, (b+1) RB) of
// the identity and applies every logged rotation to its rows, round by round.
__global__ void k_replay(const float2* __restrict__ rotlog, const int* __restrict__ out, int n, int qe, int np,
                         int R, float* __restrict__ V) {
  extern __shared__ float sm_rep[];
  float* vs = sm_rep;                                                  // REPLAY_ROWS x qe
  float2* lg = reinterpret_cast<float2*>(sm_rep + REPLAY_ROWS * qe);  // REPLAY_BATCH x np
  const int row0 = blockIdx.x * REPLAY_ROWS;
  const int nr = min(REPLAY_ROWS, n - row0);
  for (int e = threadIdx.x; e < REPLAY_ROWS * qe; e += blockDim.x) {
    const int r = e / qe, c = e % qe;
    vs[e] = (r < nr && row0 + r == c) ? 1.f : 0.f;
  }
  const long long T = out[0];
  int rr = 0;
  for (long long t0 = 0; t0 < T; t0 += REPLAY_BATCH) {
    const int nb = int(min(static_cast<long long>(REPLAY_BATCH), T - t0));
    __syncthreads();   // the previous batch is consumed
    for (int e = threadIdx.x; e < nb * np; e += blockDim.x) lg[e] = rotlog[t0 * np + e];
    __syncthreads();
    // warp w owns row w of the block; its lanes take the slots lane, lane + 32, ...
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* row = vs + w * qe;
    for (int b = 0; b < nb; ++b) {
      if (w < nr) {
        for (int slot = lane; slot < np; slot += 32) {
          const float2 cs = lg[b * np + slot];
          if (cs.y == 0.f) continue;
          int i, j;
          pair_of(slot, rr, qe, i, j);
          const float x = row[i], y = row[j];
          row[i] = cs.x * x - cs.y * y;
          row[j] = cs.y * x + cs.x * y;
        }
      }
      __syncwarp();
      if (++rr == R) rr = 0;
    }
  }
  for (int e = threadIdx.x; e < nr * n; e += blockDim.x) {
    const int c = e / nr, r = e % nr;
    V[size_t(c) * n + row0 + r] = vs[r * qe + c];
  }
}

int g_cluster_ok[64];   // 0 unknown, 1 usable, -1 not usable (per device)

}  // namespace

bool jacobi_svd_cluster(fastpi_ctx* hc, float* K, float* V, int n, double* sig, int32_t* perm,
                        JacobiStats* stats) {
  if (n < 2 || hc->device < 0 || hc->device >= 64 || g_cluster_ok[hc->device] < 0) return false;
  cudaStream_t st = hc->stream;
  int max_smem = 0;
  CK(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, hc->device));
  const int CL = MAXCL;
  const int qe = n + (n & 1), np = qe / 2, R = qe - 1;
  const int h = (n + CL - 1) / CL;
  // column stride: a multiple of 4 floats for 128-bit accesses, with an odd
  // number of float4, so that the columns of different pairs start in
  // different bank groups
  const int hp = 4 * (((h + 3) / 4) | 1);
  const size_t blk = size_t(qe) * hp * sizeof(float);
  const size_t tail = size_t(np) * (sizeof(float4) + sizeof(float2)) + (MAXCL + 2 * MAXCL) * sizeof(float) + 64;
  int with_v = 1;
  size_t bytes = 2 * blk + tail;
  if (bytes > size_t(max_smem)) {
    with_v = 0;
    bytes = blk + tail;
  }
  if (bytes > size_t(max_smem)) return false;
  allow_max_dynamic_smem((const void*)k_jacobi_cluster);
  CK(cudaFuncSetAttribute(k_jacobi_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL);
  cfg.blockDim = dim3(CT);
  cfg.dynamicSmemBytes = bytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (g_cluster_ok[hc->device] == 0) {
    int nclusters = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, k_jacobi_cluster, &cfg);
    if (e != cudaSuccess || nclusters < 1) {
      (void)cudaGetLastError();
      g_cluster_ok[hc->device] = -1;
      return false;
    }
    g_cluster_ok[hc->device] = 1;
  }
  DArr<float2> rotlog;
  if (!with_v) rotlog = DArr<float2>(int64_t(MAX_SWEEPS) * R * np, st);
  DArr<int> out(2, st);
  CK(cudaMemsetAsync(hc->dstatus.get(), 0, 4, st));
  CArgs a;
  a.K = K;
  a.V = V;
  a.rotlog = with_v ? nullptr : rotlog.get();
  a.n = n;
  a.qe = qe;
  a.np = np;
  a.R = R;
  a.h = h;
  a.hp = hp;
  a.with_v = with_v;
  a.tol = float(std::sqrt(double(n)) * 1.1920928955078125e-07);
  a.out = out.get();
  a.status = hc->dstatus.get();

  cudaEvent_t ev0, ev1;
  CK(cudaEventCreate(&ev0));
  CK(cudaEventCreate(&ev1));
  CK(cudaEventRecord(ev0, st));
  CK(cudaLaunchKernelEx(&cfg, k_jacobi_cluster, a));
  CK_LAUNCH();
  if (!with_v) {
    const size_t rs = size_t(REPLAY_ROWS) * qe * sizeof(float) + size_t(REPLAY_BATCH) * np * sizeof(float2);
    if (rs > 48 * 1024) allow_max_dynamic_smem((const void*)k_replay);
    k_replay<<<(n + REPLAY_ROWS - 1) / REPLAY_ROWS, 256, rs, st>>>(rotlog.get(), out.get(), n, qe, np, R, V);
    CK_LAUNCH();
  }
  CK(cudaEventRecord(ev1, st));
  std::vector<JacobiProblem<float>> pr(1);
  pr[0] = JacobiProblem<float>{K, V, n, n, n, n};
  jacobi_sort_columns<float>(hc, pr, sig, perm);
  int ho[2] = {0, 0};
  d2h_sync(ho, out.get(), sizeof ho, st);
  unsigned stat = 0;
  d2h_sync(&stat, hc->dstatus.get(), 4, st);
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, ev0, ev1));
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  const double dn = n;
  note_jacobi(ms, double(ho[1]) * (dn * (dn - 1) / 2) * (12 * dn + 6 * dn));
  if (stats) {
    stats->max_sweeps_used = ho[1];
    stats->hit_cap = (stat & ST_JACOBI_SWEEPS) != 0;
  }
  return true;
}

}  // namespace fastpi
