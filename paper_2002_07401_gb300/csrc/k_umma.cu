// k_umma.cu -- the dense lambda contraction on the 5th-generation tensor cores
// (tcgen05.mma kind::f16, BF16 operands, FP32 accumulator in tensor memory),
// fed by TMA through a multi-stage mbarrier pipeline.
//
// C[m][n] = sum_p sum_k A[m][a_p Kp + k] * B[n][b_p Kp + k]
//
// A holds up to 3 BF16 "terms" of each row side by side (hi, mid, lo of an
// FP32 value, each Kp wide, Kp a multiple of 64); B likewise.  Summing the
// pairs (a_p, b_p) with a_p + b_p <= 2 reproduces an FP32-accurate product of
// the unsplit operands; one pair (0, 0) is the plain BF16 product.
//
// One CTA computes a 128 x BN tile: warp 0 lane 0 issues the TMA loads, warp 1
// lane 0 issues the MMAs (one per 16-wide K slice), all four warps drain the
// accumulator from tensor memory (warp w owns TMEM lanes 32w..32w+31 = rows).
// Every wait is bounded by the global timer; a timeout sets *err.
#include <cuda.h>

#include <mutex>

#include "jagp_launch.h"

namespace jagp {

namespace {

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s per wait

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// wait for the phase with the given parity to complete; false after the limit
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > kWaitLimitNs) return false;
  return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major tile written by TMA with the
// 128-byte swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t desc_sw128_kmajor(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);  // start address
  d |= static_cast<uint64_t>(1) << 16;                  // leading byte offset (unused here)
  d |= static_cast<uint64_t>(1024 >> 4) << 32;          // stride byte offset
  d |= static_cast<uint64_t>(1) << 46;                  // descriptor version for tcgen05
  d |= static_cast<uint64_t>(2) << 61;                  // 128-byte swizzle
  return d;
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

struct UmmaArgs {
  int m_max;             // rows the grid covers
  const int *m_dev;      // live row count on the device, or null (= m_max)
  int n;                 // output columns
  int kp;                // K per term, multiple of 64
  int bn;                // output columns per CTA (multiple of 16, <= 256)
  int stages;
  int npairs;
  int pair_a[8], pair_b[8];
  uint32_t idesc;
  uint32_t tmem_cols;    // power of two >= max(32, bn)
  float *out;
  long long ldo;         // output row pitch (elements)
  const int *out_rows;   // destination row of row m, or null (= m)
  int *err;
};

__global__ void __launch_bounds__(128, 1) k_umma_gemm(const __grid_constant__ CUtensorMap tmA,
                                                      const __grid_constant__ CUtensorMap tmB, UmmaArgs g) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int M = g.m_dev ? *g.m_dev : g.m_max;
  const int m0 = blockIdx.y * 128;
  if (m0 >= M) return;  // whole CTA, before any barrier or tensor-memory use
  const int n0 = blockIdx.x * g.bn;
  const uint32_t a_bytes = 128u * 128u;
  const uint32_t b_bytes = static_cast<uint32_t>(g.bn) * 128u;
  const uint32_t stage_bytes = a_bytes + b_bytes;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + g.stages * stage_bytes);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * g.stages + 1);
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8u * g.stages, done = full0 + 16u * g.stages;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < g.stages; ++s) {
      mbar_init(full0 + 8u * s, 1);
      mbar_init(empty0 + 8u * s, 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(g.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int kchunks = g.kp / 64;
  const int iters = g.npairs * kchunks;
  const uint32_t tiles = smem_u32(smem);

  if (warp == 0 && lane == 0) {
    // producer: one A tile (128 x 64) and one B tile (bn x 64) per stage
    for (int it = 0; it < iters; ++it) {
      const int s = it % g.stages;
      const uint32_t use = static_cast<uint32_t>(it / g.stages);
      if (it >= g.stages && !mbar_wait(empty0 + 8u * s, (use & 1u) ^ 1u)) {
        atomicExch(g.err, 1);
        break;
      }
      const uint32_t full = full0 + 8u * s;
      mbar_expect_tx(full, stage_bytes);
      const int p = it / kchunks, c = it - p * kchunks;
      tma_load_2d(tiles + s * stage_bytes, &tmA, g.pair_a[p] * g.kp + c * 64, m0, full);
      tma_load_2d(tiles + s * stage_bytes + a_bytes, &tmB, g.pair_b[p] * g.kp + c * 64, n0, full);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: four K = 16 slices per 64-wide chunk, accumulating in TMEM
    for (int it = 0; it < iters; ++it) {
      const int s = it % g.stages;
      const uint32_t use = static_cast<uint32_t>(it / g.stages);
      if (!mbar_wait(full0 + 8u * s, use & 1u)) {
        atomicExch(g.err, 2);
        break;
      }
      tc_fence_after();
      const uint32_t a0 = tiles + s * stage_bytes, b0 = a0 + a_bytes;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        umma_bf16(tmem, desc_sw128_kmajor(a0 + kk * 32), desc_sw128_kmajor(b0 + kk * 32), g.idesc,
                  (it > 0 || kk > 0) ? 1u : 0u);
      umma_commit(empty0 + 8u * s);
    }
    umma_commit(done);  // arrives once every MMA issued above has completed
  }
  __syncwarp();

  // epilogue: tensor memory -> registers -> FP32 rows
  const bool ready = __all_sync(0xffffffffu, mbar_wait(done, 0));  // warp-uniform for tcgen05.ld
  tc_fence_after();
  if (ready) {
    const int row = m0 + warp * 32 + lane;
    const bool live = row < M;
    const long long dst = live ? (g.out_rows ? g.out_rows[row] : row) : 0;
    const uint32_t t_row = tmem + (static_cast<uint32_t>(warp * 32) << 16);
    for (int c = 0; c < g.bn; c += 16) {
      float v[16];
      tmem_ld16(t_row + static_cast<uint32_t>(c), v);
      if (live) {
        float *o = g.out + dst * g.ldo + n0 + c;
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (n0 + c + j < g.n) o[j] = v[j];
      }
    }
  } else if (lane == 0) {
    atomicExch(g.err, 3);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(g.tmem_cols) : "memory");
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// 2-D BF16 map with a 128-byte-swizzled box of 64 (inner) x box_rows
bool make_map(CUtensorMap *m, const void *base, uint64_t inner, uint64_t rows, uint32_t box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {inner * 2};
  cuuint32_t box[2] = {64, box_rows};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

int umma_pick_bn(int n) {
  if (n <= 256) return ((n + 15) / 16) * 16 < 32 ? 32 : ((n + 15) / 16) * 16;
  const int tiles = (n + 255) / 256;
  return (((n + tiles - 1) / tiles) + 15) / 16 * 16;
}

cudaError_t launch_umma_gemm(const uint16_t *A, int m_max, const int *m_dev, int a_terms, const uint16_t *B, int n,
                             int b_terms, int kp, int npairs, const int *pair_a, const int *pair_b, float *out,
                             long long ldo, const int *out_rows, int *err, cudaStream_t st) {
  if (m_max <= 0 || n <= 0) return cudaSuccess;
  if (kp <= 0 || kp % 64 != 0 || npairs < 1 || npairs > 8 || a_terms < 1 || b_terms < 1) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(A) & 15u) || (reinterpret_cast<uintptr_t>(B) & 15u)) return cudaErrorInvalidValue;
  for (int p = 0; p < npairs; ++p)
    if (pair_a[p] < 0 || pair_a[p] >= a_terms || pair_b[p] < 0 || pair_b[p] >= b_terms) return cudaErrorInvalidValue;
  UmmaArgs g{};
  g.m_max = m_max;
  g.m_dev = m_dev;
  g.n = n;
  g.kp = kp;
  g.bn = umma_pick_bn(n);
  const uint32_t stage_bytes = 128u * 128u + static_cast<uint32_t>(g.bn) * 128u;
  g.stages = static_cast<int>((200u * 1024u) / stage_bytes);
  if (g.stages > 6) g.stages = 6;
  g.npairs = npairs;
  for (int p = 0; p < npairs; ++p) {
    g.pair_a[p] = pair_a[p];
    g.pair_b[p] = pair_b[p];
  }
  g.idesc = (1u << 4)                                   // D: FP32
            | (1u << 7) | (1u << 10)                    // A, B: BF16
            | (static_cast<uint32_t>(g.bn >> 3) << 17)  // N
            | (static_cast<uint32_t>(128 >> 4) << 24);  // M
  uint32_t cols = 32;
  while (cols < static_cast<uint32_t>(g.bn)) cols <<= 1;
  g.tmem_cols = cols;
  g.out = out;
  g.ldo = ldo;
  g.out_rows = out_rows;
  g.err = err;
  CUtensorMap ta, tb;
  if (!make_map(&ta, A, static_cast<uint64_t>(a_terms) * kp, static_cast<uint64_t>(m_max), 128) ||
      !make_map(&tb, B, static_cast<uint64_t>(b_terms) * kp, static_cast<uint64_t>(n), static_cast<uint32_t>(g.bn)))
    return cudaErrorInvalidValue;
  const size_t smem = 1024 + static_cast<size_t>(g.stages) * stage_bytes + 8 * (2 * g.stages + 1) + 16;
  dim3 grid((n + g.bn - 1) / g.bn, (m_max + 127) / 128);
  k_umma_gemm<<<grid, 128, smem, st>>>(ta, tb, g);
  return cudaGetLastError();
}

cudaError_t setup_umma_attributes() {
  return cudaFuncSetAttribute(k_umma_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
}

}  // namespace jagp
