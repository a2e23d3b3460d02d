// FP32-storage GEMM on the 5th-generation tensor cores (tcgen05.mma,
// kind::tf32, FP32 accumulation in tensor memory), with TMA tile loads.
//
// Used by the mixed-precision form for the dense contractions of the
// incremental updates (Eq. 2 / Eq. 3: the projection correction R = D - U P,
// the CholeskyQR products, the U / V rotations) and for the apply step
// (Problem 1: U^T Y and V W).
//
// C[M x N] (row-major) = alpha * A[M x K] * B[N x K]^T + beta * C, both
// operands K-major (row-major with K contiguous).  Operands stored the other
// way are first transposed into scratch by k_transpose (an HBM-bound pass;
// every such operand in the factorization is either small or read once).
//
// One CTA computes a 128 x BN tile of C (BN = 128) over a K range:
//   warp 0      one elected thread issues the TMA loads of the A and B
//               K-slices (32 FP32 = 128 bytes per row, 128-byte swizzle)
//               into a ring of NS stages;
//   warp 1      allocates BN tensor-memory columns and one elected thread
//               issues the MMAs (4 per stage: K = 8 each);
//   warps 2-5   round each landed stage to TF32 in place (round to nearest;
//               the tensor core itself would truncate the low 13 bits, a
//               bias that accumulates over the many rotations of the
//               updates) and, in the 3-pass form, write the remainders
//               lo = rn(x - hi) to a second buffer; then run the epilogue
//               (tcgen05.ld of the accumulator, alpha / beta, store).
// The 3-pass form accumulates hi*hi + hi*lo + lo*hi, which keeps about 21
// bits of every product: the result is as accurate as an FP32 SIMT GEMM at
// a third of the TF32 tensor rate.
//
// Every mbarrier wait is bounded (a wall-clock limit read from %globaltimer):
// a wait that runs out sets a status bit, the CTA stops issuing work, waits
// (again bounded) for the copies and MMAs it already issued, frees its
// tensor memory and returns.
#include <cuda.h>

#include "dense.cuh"

namespace fastpi {
namespace {

constexpr int TC_BM = 128, TC_BK = 32, TC_THREADS = 192;
constexpr unsigned long long TC_WAIT_NS = 2000000000ull;   // 2 s per wait

__device__ unsigned g_tc_status;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity to complete.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  for (unsigned it = 1;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 63u) == 0 && gtimer() - t0 > TC_WAIT_NS) {
      atomicOr(&g_tc_status, ST_BARRIER_TIMEOUT);
      return false;
    }
  }
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major tile whose rows are 128 bytes
// (32 FP32) with the 128-byte swizzle: 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= uint64_t((addr >> 4) & 0x3FFF);          // start address
  d |= uint64_t(1) << 16;                        // leading byte offset (unused by swizzled K-major)
  d |= uint64_t(1024 >> 4) << 32;                // stride byte offset: next 8-row group
  d |= uint64_t(1) << 46;                        // descriptor version
  d |= uint64_t(2) << 61;                        // 128-byte swizzle
  return d;
}
// Instruction descriptor: D FP32, A and B TF32, both K-major, M = 128, N = bn.
__host__ __device__ constexpr uint32_t tf32_idesc(int bn) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(bn >> 3) << 17) | (uint32_t(TC_BM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ uint32_t rn_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

template <int BN, int PASSES, int NS>
struct TcSmem {
  static constexpr int A_BYTES = TC_BM * TC_BK * 4;
  static constexpr int B_BYTES = BN * TC_BK * 4;
  static constexpr int STAGE = (A_BYTES + B_BYTES) * (PASSES == 3 ? 2 : 1);
  static constexpr int BYTES = NS * STAGE + 1024 /* alignment */ + 256 /* barriers */;
};

template <int BN, int PASSES, int NS>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tma_a, const __grid_constant__ CUtensorMap tma_b, int M, int N,
              int kblocks_per_split, int kblocks_total, float alpha, float beta, float* __restrict__ C, int64_t ldc,
              float* __restrict__ W) {
  using L = TcSmem<BN, PASSES, NS>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + NS * L::STAGE);
  // bars[0..NS): full (TMA landed), [NS..2NS): ready (rounded), [2NS..3NS): empty (MMA done), [3NS]: accumulator
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bars + 3 * NS + 1);
  volatile int* s_abort = reinterpret_cast<volatile int*>(s_tmem + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * TC_BM, n0 = blockIdx.x * BN;
  const int kb0 = blockIdx.z * kblocks_per_split;
  int nkb = kblocks_total - kb0;
  if (nkb > kblocks_per_split) nkb = kblocks_per_split;
  if (nkb < 0) nkb = 0;

  auto stage_a = [&](int s) { return smem + s * L::STAGE; };
  auto stage_b = [&](int s) { return smem + s * L::STAGE + L::A_BYTES; };
  auto lo_a = [&](int s) { return smem + s * L::STAGE + L::A_BYTES + L::B_BYTES; };
  auto lo_b = [&](int s) { return smem + s * L::STAGE + 2 * L::A_BYTES + L::B_BYTES; };
  auto bar = [&](int i) { return smem_u32(bars + i); };

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(bar(s), 1);
      mbar_init(bar(NS + s), 128);
      mbar_init(bar(2 * NS + s), 1);
    }
    mbar_init(bar(3 * NS), 1);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tma_a)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tma_b)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                 "r"(BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *s_tmem;

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      int issued = 0;
      for (int i = 0; i < nkb; ++i) {
        const int s = i % NS;
        if (i >= NS && !mbar_wait(bar(2 * NS + s), ((i / NS) - 1) & 1)) {
          *s_abort = 1;
          break;
        }
        if (*s_abort) break;
        mbar_expect_tx(bar(s), L::A_BYTES + L::B_BYTES);
        const int kx = (kb0 + i) * TC_BK;
        tma_load_2d(smem_u32(stage_a(s)), &tma_a, kx, m0, bar(s));
        tma_load_2d(smem_u32(stage_b(s)), &tma_b, kx, n0, bar(s));
        ++issued;
      }
      // copies issued but possibly not yet observed by the rounding warps:
      // wait for them to land before the CTA can exit
      for (int i = (issued > NS ? issued - NS : 0); i < issued; ++i) mbar_wait(bar(i % NS), (i / NS) & 1);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = tf32_idesc(BN);
      for (int i = 0; i < nkb; ++i) {
        const int s = i % NS;
        if (!mbar_wait(bar(NS + s), (i / NS) & 1)) {
          *s_abort = 1;
          break;
        }
        if (*s_abort) break;
        fence_after();
        const uint32_t a_hi = smem_u32(stage_a(s)), b_hi = smem_u32(stage_b(s));
        const uint32_t a_lo = smem_u32(lo_a(s)), b_lo = smem_u32(lo_b(s));
#pragma unroll
        for (int k = 0; k < TC_BK / 8; ++k) {
          // K = 8 TF32 per MMA = 32 bytes along the swizzled 128-byte row
          const uint64_t da = sw128_desc(a_hi + 32 * k), db = sw128_desc(b_hi + 32 * k);
          mma_tf32(tmem, da, db, idesc, (i > 0 || k > 0) ? 1u : 0u);
          if (PASSES == 3) {
            mma_tf32(tmem, da, sw128_desc(b_lo + 32 * k), idesc, 1u);
            mma_tf32(tmem, sw128_desc(a_lo + 32 * k), db, idesc, 1u);
          }
        }
        // the stage may be refilled once these MMAs have read it
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         bar(2 * NS + s))
                     : "memory");
      }
      // always signal the accumulator barrier: it also tells the epilogue
      // that every MMA issued above has completed
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       bar(3 * NS))
                   : "memory");
    }
  } else {
    // ---------------------------------------------------------------- rounding + epilogue
    const int t = threadIdx.x - 64;   // 0..127
    constexpr int NV = (L::A_BYTES + L::B_BYTES) / 16;
    for (int i = 0; i < nkb; ++i) {
      const int s = i % NS;
      if (!mbar_wait(bar(s), (i / NS) & 1)) {
        *s_abort = 1;
        break;
      }
      if (*s_abort) break;
      // A and B of a stage are contiguous; lo_a/lo_b mirror them
      float4* hi = reinterpret_cast<float4*>(stage_a(s));
      float4* lo = reinterpret_cast<float4*>(lo_a(s));
#pragma unroll 4
      for (int v = t; v < NV; v += 128) {
        const float4 x = hi[v];
        float4 h, l;
        h.x = __uint_as_float(rn_tf32(x.x));
        h.y = __uint_as_float(rn_tf32(x.y));
        h.z = __uint_as_float(rn_tf32(x.z));
        h.w = __uint_as_float(rn_tf32(x.w));
        hi[v] = h;
        if (PASSES == 3) {
          l.x = __uint_as_float(rn_tf32(x.x - h.x));
          l.y = __uint_as_float(rn_tf32(x.y - h.y));
          l.z = __uint_as_float(rn_tf32(x.z - h.z));
          l.w = __uint_as_float(rn_tf32(x.w - h.w));
          lo[v] = l;
        }
      }
      // make the generic-proxy stores visible to the tensor core's reads
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(bar(NS + s));
    }
    // epilogue
    const bool ok = mbar_wait(bar(3 * NS), 0);
    fence_after();
    if (!ok) *s_abort = 1;
    if (ok && !*s_abort && nkb > 0) {
      const int q = warp & 3;   // this warp's 32-lane quarter of tensor memory
      const int row = m0 + q * 32 + lane;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 16) {
        uint32_t r[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
            "[%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(tmem + (uint32_t(q * 32) << 16) + uint32_t(c0)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (row < M) {
          const int col0 = n0 + c0;
          if (W) {
            float* w = W + (int64_t(blockIdx.z) * M + row) * N;
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (col0 + j < N) w[col0 + j] = alpha * __uint_as_float(r[j]);
          } else {
            float* c = C + int64_t(row) * ldc;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              if (col0 + j < N) {
                float v = alpha * __uint_as_float(r[j]);
                if (beta != 0.f) v += beta * c[col0 + j];
                c[col0 + j] = v;
              }
            }
          }
        }
      }
    } else if (nkb == 0 && !*s_abort) {
      // empty K range: this split contributes zero
      const int q = warp & 3;
      const int row = m0 + q * 32 + lane;
      if (row < M) {
        for (int j = n0; j < n0 + BN && j < N; ++j) {
          if (W) {
            W[(int64_t(blockIdx.z) * M + row) * N + j] = 0.f;
          } else {
            C[int64_t(row) * ldc + j] = beta != 0.f ? beta * C[int64_t(row) * ldc + j] : 0.f;
          }
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
  }
}

__global__ void k_tc_reduce(int64_t M, int64_t N, int splits, const float* __restrict__ W, float beta,
                            float* __restrict__ C, int64_t ldc) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= M * N) return;
  const int64_t i = t / N, j = t % N;
  float s = 0.f;
  for (int z = 0; z < splits; ++z) s += W[int64_t(z) * M * N + t];
  if (beta != 0.f) s += beta * C[i * ldc + j];
  C[i * ldc + j] = s;
}

// dst (cols x ldd, row-major) = src^T, src rows x cols (row-major, lds);
// pads columns [rows, ldd) of dst with zeros.
__global__ void k_transpose(int64_t rows, int64_t cols, const float* __restrict__ src, int64_t lds,
                            float* __restrict__ dst, int64_t ldd) {
  __shared__ float tile[32][33];
  const int64_t r0 = int64_t(blockIdx.x) * 32, c0 = int64_t(blockIdx.y) * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int64_t r = r0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < rows && c < cols) ? src[r * lds + c] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int64_t c = c0 + i, r = r0 + threadIdx.x;
    if (c < cols && r < ldd) dst[c * ldd + r] = tile[threadIdx.x][i];
  }
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
  // initialised once, thread-safely (concurrent factorizations of a batch
  // reach their first tensor-core product at the same time)
  static const EncodeTiled fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<EncodeTiled>(p);
    (void)cudaGetLastError();
    return EncodeTiled(nullptr);
  }();
  return fn;
}

// 2-D tensor map over a row-major rows x K matrix (ld in elements), box of
// box_rows x 32 FP32, 128-byte swizzle, zero fill out of range.
CUtensorMap make_map(const float* p, int64_t rows, int64_t K, int64_t ld, int box_rows) {
  CUtensorMap map;
  const cuuint64_t dims[2] = {cuuint64_t(K), cuuint64_t(rows)};
  const cuuint64_t strides[1] = {cuuint64_t(ld) * sizeof(float)};
  const cuuint32_t box[2] = {cuuint32_t(TC_BK), cuuint32_t(box_rows)};
  const cuuint32_t estr[2] = {1, 1};
  const EncodeTiled enc = encoder();
  if (!enc) fail(FASTPI_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  const CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(p), dims, strides, box,
                               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) fail(FASTPI_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string(int(r)) + ")");
  return map;
}

int g_tc_ok[64];   // per device: 0 unknown, 1 sm_103 with the encoder, -1 not usable

bool tc_device_ok() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
  if (g_tc_ok[dev] == 0) {
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    g_tc_ok[dev] = (major == 10 && minor == 3 && encoder() != nullptr) ? 1 : -1;
  }
  return g_tc_ok[dev] > 0;
}

int num_sms_dense() {
  static int n[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 152;
  if (!n[dev]) {
    cudaDeviceGetAttribute(&n[dev], cudaDevAttrMultiProcessorCount, dev);
    if (n[dev] <= 0) n[dev] = 1;
  }
  return n[dev];
}

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

constexpr int TC_BN = 128;

template <int PASSES>
void launch_tc(cudaStream_t st, int64_t M, int64_t N, int64_t K, float alpha, const float* A, int64_t lda,
               const float* B, int64_t ldb, float beta, float* C, int64_t ldc) {
  constexpr int NS = PASSES == 3 ? 3 : 6;
  using L = TcSmem<TC_BN, PASSES, NS>;
  static bool attr_set[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (!attr_set[dev]) {
    CK(cudaFuncSetAttribute(k_gemm_tc<TC_BN, PASSES, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::BYTES));
    attr_set[dev] = true;
  }
  const CUtensorMap ma = make_map(A, M, K, lda, TC_BM);
  const CUtensorMap mb = make_map(B, N, K, ldb, TC_BN);
  const int64_t tm = (M + TC_BM - 1) / TC_BM, tn = (N + TC_BN - 1) / TC_BN;
  const int kbt = int((K + TC_BK - 1) / TC_BK);
  // split K when the output has too few tiles to fill the SMs
  int splits = 1;
  const int64_t tiles = tm * tn, target = int64_t(num_sms_dense());
  if (tiles < target && kbt >= 16) {
    int64_t s = (target + tiles - 1) / tiles;
    if (s > kbt / 8) s = kbt / 8;
    if (s > 64) s = 64;
    if (s > 1) splits = int(s);
  }
  int per = (kbt + splits - 1) / splits;
  splits = (kbt + per - 1) / per;
  DArr<float> work;
  if (splits > 1) work = DArr<float>(int64_t(splits) * M * N, st);
  const dim3 grid{unsigned(tn), unsigned(tm), unsigned(splits)};
  k_gemm_tc<TC_BN, PASSES, NS><<<grid, TC_THREADS, L::BYTES, st>>>(ma, mb, int(M), int(N), per, kbt, alpha, beta, C,
                                                                    ldc, splits > 1 ? work.get() : nullptr);
  CK_LAUNCH();
  if (splits > 1) {
    k_tc_reduce<<<unsigned((M * N + 255) / 256), 256, 0, st>>>(M, N, splits, work.get(), beta, C, ldc);
    CK_LAUNCH();
  }
}

}  // namespace

bool gemm_tf32_supported(bool ta, bool tb, int64_t M, int64_t N, int64_t K, int64_t, int64_t, int64_t ldc,
                         const void*, const void*, const void* C) {
  // operands that are not K-major or not 16-byte aligned are re-laid into
  // scratch, so only the output and the sizes constrain the tensor path
  if (M <= 0 || N <= 0 || K <= 0) return false;
  if (M >= (int64_t(1) << 31) || N >= (int64_t(1) << 31) || K >= (int64_t(1) << 31)) return false;
  if ((M + TC_BM - 1) / TC_BM > 65535) return false;
  // the K-major re-layout of a transposed A (M rows) or a non-transposed B
  // (N rows) runs 32 rows per grid row (gridDim.y <= 65535)
  if ((ta && (M + 31) / 32 > 65535) || (!tb && (N + 31) / 32 > 65535)) return false;
  (void)ldc;
  (void)C;
  return tc_device_ok();
}

void gemm_tf32(cudaStream_t st, bool ta, bool tb, int64_t M, int64_t N, int64_t K, float alpha, const float* A,
               int64_t lda, const float* B, int64_t ldb, float beta, float* C, int64_t ldc, int passes) {
  if (M <= 0 || N <= 0) return;
  if (K <= 0) {
    gemm<float>(st, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    return;
  }
  const int64_t Kp = (K + 3) / 4 * 4;
  // K-major copies where needed: op(A) must be M x K with K contiguous,
  // op(B)^T must be N x K with K contiguous
  DArr<float> at, bt;
  const float* a = A;
  int64_t la = lda;
  if (ta || (lda % 4) != 0 || !aligned16(A)) {
    at = DArr<float>(M * Kp, st);
    if (ta) {
      // A is K x M: transpose into M x Kp
      const dim3 g{unsigned((K + 31) / 32), unsigned((M + 31) / 32)};
      k_transpose<<<g, dim3{32, 8}, 0, st>>>(K, M, A, lda, at.get(), Kp);
      CK_LAUNCH();
    } else {
      copy2d<float, float>(st, M, K, A, lda, at.get(), Kp);
    }
    a = at.get();
    la = Kp;
  }
  const float* b = B;
  int64_t lb = ldb;
  if (!tb || (ldb % 4) != 0 || !aligned16(B)) {
    bt = DArr<float>(N * Kp, st);
    if (!tb) {
      // B is K x N: transpose into N x Kp
      const dim3 g{unsigned((K + 31) / 32), unsigned((N + 31) / 32)};
      k_transpose<<<g, dim3{32, 8}, 0, st>>>(K, N, B, ldb, bt.get(), Kp);
      CK_LAUNCH();
    } else {
      copy2d<float, float>(st, N, K, B, ldb, bt.get(), Kp);
    }
    b = bt.get();
    lb = Kp;
  }
  if (passes == 3)
    launch_tc<3>(st, M, N, K, alpha, a, la, b, lb, beta, C, ldc);
  else
    launch_tc<1>(st, M, N, K, alpha, a, la, b, lb, beta, C, ldc);
}

unsigned gemm_tc_status(cudaStream_t st, bool clear) {
  unsigned v = 0;
  CK(cudaMemcpyFromSymbolAsync(&v, g_tc_status, sizeof v, 0, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (clear && v) {
    const unsigned z = 0;
    CK(cudaMemcpyToSymbolAsync(g_tc_status, &z, sizeof z, 0, cudaMemcpyHostToDevice, st));
  }
  return v;
}

}  // namespace fastpi
