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


// Rotation of the pair (p, q) from the Gram entries al = G_pp, be = G_qq,
// ga = G_pq (row-major P x P): t = 2 g sgn(d) / (|d| + sqrt(d^2 + 4 g^2)),
// d = be - al (the smaller root), c = 1 / sqrt(1 + t^2), s = c t, with the
// fast reciprocal square root and division (the caller re-orthonormalises the
// accumulated rotation, so their last-ulp errors do not accumulate).  cls: 0
// no rotation, 1 above tol, 2 above the early-exit threshold.
template <int P>
__device__ __forceinline__ void rot_fast(const float* G, int p, int q, float tabs, float tol2, float early2, float& c,
                                         float& s, int& cls) {
  const float al = G[p * P + p], be = G[q * P + q], ga = G[p * P + q];
  c = 1.f;
  s = 0.f;
  cls = 0;
  if (al > tabs && be > tabs && ga * ga > tol2 * al * be) {
    const float d = be - al;
    const float h = fmaf(d, d, 4.f * ga * ga);
    const float t = __fdividef(2.f * (d < 0.f ? -ga : ga), fabsf(d) + h * rsqrtf(h));
    c = rsqrtf(fmaf(t, t, 1.f));
    s = c * t;
    cls = ga * ga > early2 * al * be ? 2 : 1;
  }
}

// The sweep on G with ONE CTA barrier per inner round: every work item --
// a 2 x 2 block of G (rows {i, mi}, columns {j, mj}) or a pair of entries of
// a row of Q -- computes the rotations it needs from the current G itself
// (the same inputs and code in every thread, so the same values), reads G
// from one buffer and writes the rotated block to the other, and rotates its
// entries of Q in place.  Returns the buffer that holds the final G; the
// largest rotation class goes to *rot_flag and whether any pair rotated to
// *pair_rot (both through shared-memory atomics).
template <int P, int NT>
__device__ __forceinline__ void inner_solve_fast(float* G, float* Gn, float* Q, int tid, float tabs, float tol2,
                                                 float early2, bool cross, int* rot_flag, int* pair_rot) {
  constexpr int H = P / 2;
  constexpr int NB = H * H, NQ = P * H;
  const int rounds = cross ? H : P - 1;
  int rot = 0;
  for (int ir = 0; ir < rounds; ++ir) {
    for (int item = tid; item < NB + NQ; item += NT) {
      if (item < NB) {
        const int a = item / H, b = item - (item / H) * H;
        int i, mi, j, mj;
        inner_pair<P>(cross, a, ir, i, mi);
        inner_pair<P>(cross, b, ir, j, mj);
        float ca, sa, cb, sb;
        int cla, clb;
        rot_fast<P>(G, i, mi, tabs, tol2, early2, ca, sa, cla);
        rot_fast<P>(G, j, mj, tabs, tol2, early2, cb, sb, clb);
        if (a == b) rot = max(rot, cla);
        // x_i' = c x_i - s x_mi, x_mi' = s x_i + c x_mi on both sides
        const float g00 = G[i * P + j], g01 = G[i * P + mj], g10 = G[mi * P + j], g11 = G[mi * P + mj];
        const float r0j = cb * g00 - sb * g01, r0m = sb * g00 + cb * g01;   // row i after the column rotation
        const float r1j = cb * g10 - sb * g11, r1m = sb * g10 + cb * g11;   // row mi
        Gn[i * P + j] = ca * r0j - sa * r1j;
        Gn[i * P + mj] = ca * r0m - sa * r1m;
        Gn[mi * P + j] = sa * r0j + ca * r1j;
        Gn[mi * P + mj] = sa * r0m + ca * r1m;
      } else {
        const int e = item - NB;
        const int r = e / H, b = e - (e / H) * H;
        int j, mj;
        inner_pair<P>(cross, b, ir, j, mj);
        float cb, sb;
        int clb;
        rot_fast<P>(G, j, mj, tabs, tol2, early2, cb, sb, clb);
        const float q0 = Q[r * P + j], q1 = Q[r * P + mj];
        Q[r * P + j] = cb * q0 - sb * q1;
        Q[r * P + mj] = sb * q0 + cb * q1;
      }
    }
    __syncthreads();
    float* t = G;
    G = Gn;
    Gn = t;
  }
  rot = __reduce_max_sync(0xffffffffu, rot);
  if ((tid & 31) == 0 && rot > 0) {
    atomicMax(rot_flag, rot);
    *pair_rot = 1;
  }
}

// One Newton-Schulz step on the accumulated rotation Q of a block pair
// (P x P, row-major, shared memory), by the whole CTA: W = Q^T Q, then
// Qo = Q (3 I - W) / 2.  Q is a product of FP32 rotations whose c^2 + s^2
// misses 1 by about an ulp, with a fixed sign for the small angles of the
// late sweeps (c rounds to 1), so without this step every round would scale
// the columns of K and V by that much and a column that takes part in
// thousands of rounds would drift by thousands of ulps; after it Q is
// orthonormal to rounding, whose error has no preferred sign.  Returns Qo.
template <int P, int NT>
__device__ __forceinline__ float* ns_orthonormalize(const float* Q, float* W, float* Qo, int tid) {
  for (int e = tid; e < P * P; e += NT) {
    const int i = e / P, j = e % P;
    float acc = 0.f;
#pragma unroll 4
    for (int r = 0; r < P; ++r) acc = fmaf(Q[r * P + i], Q[r * P + j], acc);
    W[e] = acc;
  }
  __syncthreads();
  for (int e = tid; e < P * P; e += NT) {
    const int r = e / P, j = e % P;
    float acc = 0.f;
#pragma unroll 4
    for (int c = 0; c < P; ++c) acc = fmaf(Q[r * P + c], W[c * P + j], acc);
    Qo[e] = fmaf(-0.5f, acc, 1.5f * Q[e]);
  }
  __syncthreads();
  return Qo;
}

// Host side, shared by the two core kernels (defined in jacobi_block.cu):
// Kp (ldk x q, column-major) <- K (p x q, ld lda; lda == p or a square core)
// with zero rows p..ldk-1, Vp <- I (ldk x q); gb->fro2 = |K|_F^2 (fixed-order
// sum) and the barrier reset.
void core_prepare(fastpi_ctx* hc, const float* K, int64_t lda, int p, int q, int ldk, float* Kp, float* Vp,
                  double* part, int npart, BBar* gb);
// K (p x q, ld lda) <- Kp, V (q x q, ld ldv) <- Vp.
void core_finish(fastpi_ctx* hc, const float* Kp, const float* Vp, int p, int q, int ldk, float* K, int64_t lda,
                 float* V, int64_t ldv);

}  // namespace jdev
}  // namespace fastpi
