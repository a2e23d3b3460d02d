// Device helpers shared by the block one-sided Jacobi kernels of the update
// cores (jacobi_block.cu: one CTA per block pair; jacobi_cluster.cu: a block
// pair's rows split over a thread-block cluster): bounded waits and the
// device-wide barrier, the circle-method pairings, the warp reduction of the
// Gram tiles, 16-byte asynchronous copies, and the Jacobi sweep on the small
// Gram matrix of a block pair.
#pragma once

#include "common.cuh"

namespace fastpi {
namespace jdev {

constexpr unsigned long long B_WAIT_NS = 2000000000ull;   // bound of every wait (2 s)
constexpr int VER_STRIDE = 32;   // one 128-byte line per block's round counter (no shared polling lines)

struct BBar {
  unsigned count;
  unsigned gen;
  int flag[3];
  double fro2;
};

__device__ __forceinline__ unsigned long long b_gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned b_ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void b_st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Device-wide barrier of a cooperative launch; false when the bounded wait
// ran out (status bit set).
static __device__ bool b_barrier(BBar* gb, unsigned* status) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned gen = b_ld_acquire(&gb->gen);
    __threadfence();
    const unsigned arrived = atomicAdd(&gb->count, 1u) + 1u;
    int ok = 1;
    if (arrived == gridDim.x) {
      gb->count = 0;
      __threadfence();
      b_st_release(&gb->gen, gen + 1u);
    } else {
      const unsigned long long t0 = b_gtimer();
      unsigned spins = 0;
      while (b_ld_acquire(&gb->gen) == gen) {
        if ((++spins & 63u) == 0 && b_gtimer() - t0 > B_WAIT_NS) {
          atomicOr(status, ST_BARRIER_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ void circle_pair(int slot, int rr, int qe, int& i, int& j) {
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

// Partner of column i in round rr of the circle method over qe columns.
__device__ __forceinline__ int circle_mate(int i, int rr, int qe) {
  const int m = qe - 1;
  if (i == m) return rr;
  if (i == rr) return m;
  int j = 2 * rr - i;
  if (j < 0) j += m;
  if (j >= m) j -= m;
  return j;
}

// Butterfly reduction of NV per-lane values over the 32 lanes of a warp.
// NV >= 32: afterwards lane L holds the sums of values [off, off + NV / 32),
// off built from the lane bits.  NV < 32: lanes that differ only in their
// lowest log2(32 / NV) bits hold the same single sum, index off.
template <int NV>
__device__ __forceinline__ void warp_reduce_scatter(float (&v)[NV], int lane, int& off) {
  off = 0;
  int len = NV;
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) {
    if (len > 1) {
      const int half = len / 2;
      const bool up = (lane & m) != 0;
#pragma unroll
      for (int i = 0; i < NV / 2; ++i) {
        if (i < half) {
          const float mine = up ? v[i + half] : v[i];
          const float other = up ? v[i] : v[i + half];
          v[i] = mine + __shfl_xor_sync(0xffffffffu, other, m);
        }
      }
      if (up) off += half;
      len = half;
    } else {
      v[0] += __shfl_xor_sync(0xffffffffu, v[0], m);
    }
  }
}

__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Whole CTA, any P: G and Q in shared memory, double-buffered.  Per round,
// threads 0..P/2-1 compute the rotations of the round's pairs, then all
// threads update the P x P entries of G <- J^T G J and Q <- Q J.  Returns
// the buffer that holds the final Q.  Runs `sweeps` sweeps.
// Pairs of one inner round.  Full rounds (cross = false): the circle method
// over all P columns, P - 1 rounds.  Cross rounds (cross = true): column i of
// the first block with column B + (i + ir) mod B of the second, B rounds.
template <int P>
__device__ __forceinline__ void inner_pair(bool cross, int k, int ir, int& p, int& q) {
  constexpr int B = P / 2;
  if (cross) {
    p = k;
    q = B + (k + ir) % B;
  } else {
    circle_pair(k, ir, P, p, q);
  }
}
template <int P>
__device__ __forceinline__ int inner_mate(bool cross, int i, int ir) {
  constexpr int B = P / 2;
  if (!cross) return circle_mate(i, ir, P);
  return i < B ? B + (i + ir) % B : ((i - B - ir) % B + B) % B;
}

// Whole CTA, any P: G and Q in shared memory, double-buffered.  Per round,
// threads 0..P/2-1 compute the rotations of the round's pairs, then all
// threads update the P x P entries of G <- J^T G J and Q <- Q J.  Returns
// the buffer that holds the final Q.  `cross`: only the pairs across the two
// blocks (the pairs inside each block were visited in the first round of
// the sweep).
template <int P, int NT>
__device__ __forceinline__ float* inner_solve_cta(float* G, float* Gn, float* Q, float* Qn, float* sc, float* so,
                                                  int tid, float tabs, float tol2, float early2, int sweeps,
                                                  bool cross, int* s_rot, int* s_pair_rot) {
  constexpr int GS = P;
  const int rounds = cross ? P / 2 : P - 1;
  for (int is = 0; is < sweeps; ++is) {
    for (int ir = 0; ir < rounds; ++ir) {
      if (tid < P / 2) {
        int p, q;
        inner_pair<P>(cross, tid, ir, p, q);
        const float al = G[p * GS + p], be = G[q * GS + q], ga = G[p * GS + q];
        float c = 1.f, s = 0.f;
        if (al > tabs && be > tabs && ga * ga > tol2 * al * be) {
          // t = 2 g sgn(d) / (|d| + sqrt(d^2 + 4 g^2)), d = be - al (smaller root)
          const float d = be - al;
          // IEEE square root and division: an approximate c (c^2 + s^2 != 1 by a
          // few ulp with a fixed sign) would scale V's columns a little on every
          // one of the thousands of rotations each column receives
          const float t = 2.f * (d < 0.f ? -ga : ga) / (fabsf(d) + sqrtf(fmaf(d, d, 4.f * ga * ga)));
          c = 1.f / sqrtf(fmaf(t, t, 1.f));
          s = c * t;
          *s_pair_rot = 1;
          atomicMax(s_rot, ga * ga > early2 * al * be ? 2 : 1);
        }
        // x_p' = c x_p - s x_q, x_q' = s x_p + c x_q
        sc[p] = c;
        so[p] = -s;
        sc[q] = c;
        so[q] = s;
      }
      __syncthreads();
      for (int e = tid; e < P * P; e += NT) {
        const int i = e / P, j = e % P;
        const int mi = inner_mate<P>(cross, i, ir), mj = inner_mate<P>(cross, j, ir);
        const float ci = sc[i], si = so[i], cj = sc[j], sj = so[j];
        Gn[i * GS + j] = ci * (cj * G[i * GS + j] + sj * G[i * GS + mj]) +
                         si * (cj * G[mi * GS + j] + sj * G[mi * GS + mj]);
        Qn[i * GS + j] = cj * Q[i * GS + j] + sj * Q[i * GS + mj];
      }
      __syncthreads();
      float* t = G;
      G = Gn;
      Gn = t;
      t = Q;
      Q = Qn;
      Qn = t;
    }
  }
  return Q;
}


// The same sweep on G by ONE warp (the caller's other warps wait at a CTA
// barrier afterwards): per inner round the lanes holding a pair compute its
// rotation, then every lane rotates whole 2 x 2 blocks of G (rows {i, mi},
// columns {j, mj}) and pairs of entries of Q's rows in place -- a block is
// read and written by one lane only -- with warp barriers instead of CTA
// barriers between the steps.  G and Q are P x P row-major in shared memory;
// sc / so receive the rotation of each column (x_i' = sc_i x_i + so_i
// x_mate(i)).  On return Q holds the accumulated rotations, *rot_flag the
// largest rotation class of the sweep (0 none, 1 above tol, 2 above the early
// exit threshold), *pair_rot whether any pair rotated (lane 0 writes both).
template <int P>
__device__ __forceinline__ void inner_solve_warp(float* G, float* Q, float* sc, float* so, int lane, float tabs,
                                                 float tol2, float early2, bool cross, int* rot_flag,
                                                 int* pair_rot) {
  constexpr int H = P / 2;
  const int rounds = cross ? H : P - 1;
  int rot = 0;
  for (int ir = 0; ir < rounds; ++ir) {
    if (lane < H) {
      int p, q;
      inner_pair<P>(cross, lane, ir, p, q);
      const float al = G[p * P + p], be = G[q * P + q], ga = G[p * P + q];
      float c = 1.f, s = 0.f;
      if (al > tabs && be > tabs && ga * ga > tol2 * al * be) {
        // t = 2 g sgn(d) / (|d| + sqrt(d^2 + 4 g^2)), d = be - al (the smaller
        // root); IEEE square root and division keep c^2 + s^2 = 1 unbiased
        const float d = be - al;
        const float t = 2.f * (d < 0.f ? -ga : ga) / (fabsf(d) + sqrtf(fmaf(d, d, 4.f * ga * ga)));
        c = 1.f / sqrtf(fmaf(t, t, 1.f));
        s = c * t;
        rot = max(rot, ga * ga > early2 * al * be ? 2 : 1);
      }
      sc[p] = c;
      so[p] = -s;
      sc[q] = c;
      so[q] = s;
    }
    __syncwarp();
    for (int idx = lane; idx < H * H; idx += 32) {
      const int a = idx / H, b = idx - (idx / H) * H;
      int i, mi, j, mj;
      inner_pair<P>(cross, a, ir, i, mi);
      inner_pair<P>(cross, b, ir, j, mj);
      const float g00 = G[i * P + j], g01 = G[i * P + mj], g10 = G[mi * P + j], g11 = G[mi * P + mj];
      const float ci = sc[i], si = so[i], cmi = sc[mi], smi = so[mi];
      const float cj = sc[j], sj = so[j], cmj = sc[mj], smj = so[mj];
      G[i * P + j] = ci * (cj * g00 + sj * g01) + si * (cj * g10 + sj * g11);
      G[i * P + mj] = ci * (cmj * g01 + smj * g00) + si * (cmj * g11 + smj * g10);
      G[mi * P + j] = cmi * (cj * g10 + sj * g11) + smi * (cj * g00 + sj * g01);
      G[mi * P + mj] = cmi * (cmj * g11 + smj * g10) + smi * (cmj * g01 + smj * g00);
    }
    for (int idx = lane; idx < P * H; idx += 32) {
      const int r = idx / H, b = idx - (idx / H) * H;
      int j, mj;
      inner_pair<P>(cross, b, ir, j, mj);
      const float q0 = Q[r * P + j], q1 = Q[r * P + mj];
      Q[r * P + j] = sc[j] * q0 + so[j] * q1;
      Q[r * P + mj] = sc[mj] * q1 + so[mj] * q0;
    }
    __syncwarp();
  }
  rot = __reduce_max_sync(0xffffffffu, rot);
  if (lane == 0) {
    *rot_flag = max(*rot_flag, rot);
    *pair_rot = rot > 0 ? 1 : 0;
  }
}

// Host side, shared by the two core kernels (defined in jacobi_block.cu):
// Kp (ldk x n, column-major) <- K (n x n, ld n) with zero rows n..ldk-1,
// Vp <- I; gb->fro2 = |K|_F^2 (fixed-order sum) and the barrier reset.
void core_prepare(fastpi_ctx* hc, const float* K, int n, int ldk, float* Kp, float* Vp, double* part, int npart,
                  BBar* gb);
// K (n x n) <- Kp, V (n x n) <- Vp.
void core_finish(fastpi_ctx* hc, const float* Kp, const float* Vp, int n, int ldk, float* K, float* V);

}  // namespace jdev
}  // namespace fastpi
