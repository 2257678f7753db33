// k_umma.cu -- the dense lambda contraction on the 5th-generation tensor cores
// (tcgen05.mma kind::f16, BF16 operands, FP32 accumulator in tensor memory),
// fed by TMA through a multi-stage mbarrier pipeline.
//
// Plain mode:  C[m][n] = sum_p sum_k A[m][a_p Kp + k] * B[n][b_p Kp + k]
// A holds up to four BF16 "terms" of each row side by side (each Kp wide, Kp a
// multiple of 64); B likewise.  All pairs accumulate into one FP32 tensor-
// memory accumulator.
//
// Fixed-point mode (row exponents ea[m], column exponents eb[n] given): the
// terms are 8-bit integer slices of rows scaled by powers of two,
//   a = 2^(ea - 7) (t0 + t1 / 256 + t2 / 256^2 + ...),  |t_i| <= 128,
// (exact in BF16), so every slice product is an integer below 2^14 and the
// tensor cores sum them exactly while partial sums stay below 2^24.  Pairs of
// equal weight d = a_p + b_p share an accumulator S_d (up to eight), and the
// epilogue forms C = 2^(ea + eb - 14) (S_0 + S_1 / 256 + S_2 / 256^2 + ...) as
// an unevaluated two-float sum: products of two-float rows far beyond FP32
// accuracy, which the lossy FP32 accumulation inside the tensor cores would
// not give.
//
// One CTA computes a 128 x BN tile: warp 0 lane 0 issues the TMA loads, warp 1
// lane 0 issues the MMAs (one per 16-wide K slice), all four warps drain the
// accumulator from tensor memory (warp w owns TMEM lanes 32w..32w+31 = rows).
// Stages hold one A and one B slice of a 64-wide K chunk, pair after pair; in
// chunk-major modes (stages_max = -1, -2, -3: K chunks of 64, 32, 16) a stage holds every slice of
// the chunk and the MMA thread issues all pairs from it.  CTAs walk kGroupM row
// tiles of one column tile before the next, so that a wave shares operand
// tiles in L2.  Every wait is bounded by the global timer; a timeout sets *err.
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "jagp_group.cuh"
#include "jagp_group.cuh"
#include "jagp_launch.h"

namespace jagp {

namespace {

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s per wait
constexpr int kGroupM = 8;                         // row tiles per group of the tile order

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
// swizzle of its row width: rows of 128, 64 or 32 bytes (K chunks of 64, 32 or
// 16 BF16 elements), 8-row groups 8 row widths apart; the PTX layout codes of
// the 128-, 64- and 32-byte swizzles are 2, 4 and 6.
__device__ __forceinline__ uint64_t desc_kmajor(uint32_t saddr, uint32_t row_bytes) {
  const uint64_t layout = row_bytes == 128 ? 2 : (row_bytes == 64 ? 4 : 6);
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);      // start address
  d |= static_cast<uint64_t>(1) << 16;                      // leading byte offset (unused here)
  d |= static_cast<uint64_t>((8u * row_bytes) >> 4) << 32;  // stride byte offset
  d |= static_cast<uint64_t>(1) << 46;                      // descriptor version for tcgen05
  d |= layout << 61;                                        // swizzle
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

// tensor maps read from global memory (the grouped launches keep them with
// their arguments there): order the generic-proxy writes that placed them
// before their use by the tensor-map proxy.  Kernel-parameter maps need nothing.
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap *a, const CUtensorMap *b) {
  if (__isGlobal(a)) asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(a) : "memory");
  if (__isGlobal(b)) asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(b) : "memory");
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
  int pair_a[kMaxPairs], pair_b[kMaxPairs], pair_group[kMaxPairs];
  int ngroups;           // accumulators (1 in plain mode)
  int slice_bits;        // fixed-point mode: bits per slice (8, or 7 for long K)
  double *out64;         // fixed-point mode: FP64 result instead of out / out_lo, or null
  int batch_rows;        // batched mode (> 0): A and B are stacked per-batch blocks of batch_rows
                         // rows; batch b's rows of A meet only batch b's rows of B
  int tiles_per_batch;   // batched mode: 128-row tiles per batch
  int b_batch_rows;      // batched mode: rows of B per batch (= batch_rows unless given)
  int chunk_major;       // 1: one stage holds every slice of one K chunk of A (na) and B (nb),
  int na, nb;            //    and the MMA thread issues all pairs from it (slices loaded once per chunk)
  int cw;                // K chunk width in elements: 64, or 32 / 16 for chunk-major stages of many slices
  const int *a_exp;      // fixed-point mode: row exponents [m_max], else null
  const int *b_exp;      // fixed-point mode: column exponents [n]
  uint32_t idesc;
  uint32_t tmem_cols;    // power of two >= max(32, bn)
  float *out;
  float *out_lo;         // fixed-point mode: low part of a two-float result, or null
  long long ldo;         // output row pitch (elements)
  const int *out_rows;   // destination row of row m, or null (= m)
  // batched mode, affine output (o_cstride != 0): the element of local row r
  // (within its batch b) and column c goes to out[b o_bstride + r o_rstride + c o_cstride]
  long long o_bstride, o_rstride, o_cstride;
  int *err;
};

struct UmmaGemm {
  static __device__ __forceinline__ void run(const CUtensorMap &tmA, const CUtensorMap &tmB, const UmmaArgs &g,
                                             const uint3 bid, const uint3 gdim) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int M = g.m_dev ? *g.m_dev : g.m_max;
    // batched mode: tile t of batch b starts at row b * batch_rows + 128 t; rows
    // past the batch's end (read from the next batch) are computed but not written
    // grouped tile order: CTAs in launch order walk kGroupM row tiles of one
    // column tile before the next column tile, so that a wave reuses both A and
    // B tiles from L2 (with large K the operands exceed L2)
    int tile_y, tile_x;
    {
      const int tiles_n = gdim.x, tiles_m = gdim.y;
      const int pid = bid.x + bid.y * tiles_n;
      const int span = kGroupM * tiles_n;
      const int first = (pid / span) * kGroupM;
      const int gsize = tiles_m - first < kGroupM ? tiles_m - first : kGroupM;
      const int r = pid - (pid / span) * span;
      tile_y = first + r % gsize;
      tile_x = r / gsize;
    }
    const int bb = g.batch_rows ? tile_y / g.tiles_per_batch : 0;
    const int bt0 = g.batch_rows ? (tile_y - bb * g.tiles_per_batch) * 128 : 0;
    const int m0 = g.batch_rows ? bb * g.batch_rows + bt0 : tile_y * 128;
    const int bbase = bb * g.b_batch_rows;  // first B row (and column exponent) of this batch
    if (m0 >= M) return;  // whole CTA, before any barrier or tensor-memory use
    const int n0 = tile_x * g.bn;
    const uint32_t row_bytes = static_cast<uint32_t>(g.cw) * 2u;  // 128, 64 or 32
    const uint32_t a_bytes = 128u * row_bytes;
    const uint32_t b_bytes = static_cast<uint32_t>(g.bn) * row_bytes;
    const int ksteps = g.cw / 16;  // MMAs (K = 16) per chunk
    const uint32_t stage_bytes =
        g.chunk_major ? static_cast<uint32_t>(g.na) * a_bytes + static_cast<uint32_t>(g.nb) * b_bytes : a_bytes + b_bytes;
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
    const int kchunks = g.kp / g.cw;
    const int iters = g.chunk_major ? kchunks : g.npairs * kchunks;
    const uint32_t tiles = smem_u32(smem);

    if (warp == 0 && lane == 0) tensormap_acquire(&tmA, &tmB);
    if (warp == 0 && lane == 0 && g.chunk_major) {
      // producer, chunk-major: every slice of A and B for one K chunk per stage
      for (int it = 0; it < iters; ++it) {
        const int s = it % g.stages;
        const uint32_t use = static_cast<uint32_t>(it / g.stages);
        if (it >= g.stages && !mbar_wait(empty0 + 8u * s, (use & 1u) ^ 1u)) {
          atomicExch(g.err, 1);
          break;
        }
        const uint32_t full = full0 + 8u * s, base = tiles + s * stage_bytes;
        mbar_expect_tx(full, stage_bytes);
        for (int a = 0; a < g.na; ++a) tma_load_2d(base + a * a_bytes, &tmA, a * g.kp + it * g.cw, m0, full);
        for (int b = 0; b < g.nb; ++b)
          tma_load_2d(base + g.na * a_bytes + b * b_bytes, &tmB, b * g.kp + it * g.cw, bbase + n0, full);
      }
    } else if (warp == 1 && lane == 0 && g.chunk_major) {
      // MMA issuer, chunk-major: all pairs of the chunk from the one stage
      uint32_t started = 0;
      for (int it = 0; it < iters; ++it) {
        const int s = it % g.stages;
        const uint32_t use = static_cast<uint32_t>(it / g.stages);
        if (!mbar_wait(full0 + 8u * s, use & 1u)) {
          atomicExch(g.err, 2);
          break;
        }
        tc_fence_after();
        const uint32_t base = tiles + s * stage_bytes;
        for (int p = 0; p < g.npairs; ++p) {
          const int grp = g.pair_group[p];
          const uint32_t a0 = base + g.pair_a[p] * a_bytes, b0 = base + g.na * a_bytes + g.pair_b[p] * b_bytes;
          const uint32_t d_tmem = tmem + static_cast<uint32_t>(grp * g.bn);
          for (int kk = 0; kk < ksteps; ++kk) {
            umma_bf16(d_tmem, desc_kmajor(a0 + kk * 32, row_bytes), desc_kmajor(b0 + kk * 32, row_bytes), g.idesc,
                      (started >> grp) & 1u);
            started |= 1u << grp;
          }
        }
        umma_commit(empty0 + 8u * s);
      }
      umma_commit(done);
    } else if (warp == 0 && lane == 0) {
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
        tma_load_2d(tiles + s * stage_bytes + a_bytes, &tmB, g.pair_b[p] * g.kp + c * 64, bbase + n0, full);
      }
    } else if (warp == 1 && lane == 0) {
      // MMA issuer: four K = 16 slices per 64-wide chunk, accumulating in TMEM
      uint32_t started = 0;  // bit g: accumulator g has received its first product
      for (int it = 0; it < iters; ++it) {
        const int s = it % g.stages;
        const uint32_t use = static_cast<uint32_t>(it / g.stages);
        if (!mbar_wait(full0 + 8u * s, use & 1u)) {
          atomicExch(g.err, 2);
          break;
        }
        tc_fence_after();
        const uint32_t a0 = tiles + s * stage_bytes, b0 = a0 + a_bytes;
        const int grp = g.pair_group[it / kchunks];
        const uint32_t d_tmem = tmem + static_cast<uint32_t>(grp * g.bn);
  #pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          umma_bf16(d_tmem, desc_kmajor(a0 + kk * 32, 128u), desc_kmajor(b0 + kk * 32, 128u), g.idesc,
                    (started >> grp) & 1u);
          started |= 1u << grp;
        }
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
      const bool live = row < M && (!g.batch_rows || bt0 + warp * 32 + lane < g.batch_rows);
      const long long dst = live ? (g.out_rows ? g.out_rows[row] : row) : 0;
      // element offset of this row's column 0 and the stride between columns
      const long long obase = g.o_cstride ? (long long)bb * g.o_bstride + (long long)(bt0 + warp * 32 + lane) * g.o_rstride
                                          : dst * g.ldo;
      const long long ocs = g.o_cstride ? g.o_cstride : 1;
      const uint32_t t_row = tmem + (static_cast<uint32_t>(warp * 32) << 16);
      const int ea = (g.a_exp && live) ? g.a_exp[row] : 0;
      for (int c = 0; c < g.bn; c += 16) {
        if (g.out64) {
          // FP64 result: v = S_0 + 2^-b (S_1 + 2^-b (S_2 + ...)) by Horner in FP64
          // from the exact integer sums, then the power-of-two scale
          double acc[16];
  #pragma unroll
          for (int j = 0; j < 16; ++j) acc[j] = 0.0;
          const double wq = ldexp(1.0, -g.slice_bits);
          for (int q = g.ngroups - 1; q >= 0; --q) {
            float u[16];
            tmem_ld16(t_row + static_cast<uint32_t>(q * g.bn + c), u);
  #pragma unroll
            for (int j = 0; j < 16; ++j) acc[j] = fma(acc[j], wq, static_cast<double>(u[j]));
          }
          if (live) {
            double *o = g.out64 + obase;
  #pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int col = n0 + c + j;
              if (col < g.n) o[col * ocs] = ldexp(acc[j], ea + g.b_exp[bbase + col] - 2 * (g.slice_bits - 1));
            }
          }
          continue;
        }
        float v[16];
        tmem_ld16(t_row + static_cast<uint32_t>(c), v);
        if (g.a_exp) {
          // v = S_0 + S_1 / 256 + S_2 / 256^2 + ... as an unevaluated sum
          // hi + lo of FP32 numbers: every S_d is an exact integer below 2^24 and
          // each addition goes through an error-free transformation (TwoSum)
          float lo[16];
  #pragma unroll
          for (int j = 0; j < 16; ++j) lo[j] = 0.0f;
          float scale = 1.0f;
          for (int q = 1; q < g.ngroups; ++q) {
            float u[16];
            tmem_ld16(t_row + static_cast<uint32_t>(q * g.bn + c), u);
            scale *= 0.00390625f;
  #pragma unroll
            for (int j = 0; j < 16; ++j) {
              const float b = __fmul_rn(u[j], scale);  // exact: power-of-two scaling
              const float s = __fadd_rn(v[j], b);
              const float z = __fsub_rn(s, v[j]);
              const float e = __fadd_rn(__fsub_rn(v[j], __fsub_rn(s, z)), __fsub_rn(b, z));
              v[j] = s;
              lo[j] = __fadd_rn(lo[j], e);
            }
          }
  #pragma unroll
          for (int j = 0; j < 16; ++j) {
            const float hi = __fadd_rn(v[j], lo[j]);
            const float l2 = __fsub_rn(lo[j], __fsub_rn(hi, v[j]));
            const int col = n0 + c + j;
            const int sh = ea + (col < g.n ? g.b_exp[bbase + col] : 0) - 14;
            v[j] = ldexpf(hi, sh);
            lo[j] = ldexpf(l2, sh);
          }
          if (live && g.out_lo) {
            float *ol = g.out_lo + obase;
  #pragma unroll
            for (int j = 0; j < 16; ++j)
              if (n0 + c + j < g.n) ol[(n0 + c + j) * ocs] = lo[j];
          }
        }
        if (live) {
          float *o = g.out + obase;
  #pragma unroll
          for (int j = 0; j < 16; ++j)
            if (n0 + c + j < g.n) o[(n0 + c + j) * ocs] = v[j];
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
};

__global__ void __launch_bounds__(128) k_umma_gemm(const __grid_constant__ CUtensorMap tmA,
                                                   const __grid_constant__ CUtensorMap tmB,
                                                   const __grid_constant__ UmmaArgs g) {
  UmmaGemm::run(tmA, tmB, g, blockIdx, gridDim);
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
// box of cw x box_rows BF16 elements, swizzled by its row width (cw = 64, 32
// or 16: 128-, 64- or 32-byte rows)
bool make_map(CUtensorMap *m, const void *base, uint64_t inner, uint64_t rows, uint32_t box_rows, uint32_t cw) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {inner * 2};
  cuuint32_t box[2] = {cw, box_rows};
  cuuint32_t es[2] = {1, 1};
  const CUtensorMapSwizzle sw =
      cw == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : (cw == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

int umma_pick_bn(int n, int max_bn) {
  if (n <= max_bn) return ((n + 15) / 16) * 16 < 32 ? 32 : ((n + 15) / 16) * 16;
  const int tiles = (n + max_bn - 1) / max_bn;
  return (((n + tiles - 1) / tiles) + 15) / 16 * 16;
}

namespace {
int g_smem_optin = 220 * 1024;  // the kernel's dynamic shared-memory limit, set once per process

uint32_t chunk_stage_bytes(int na, int nb, int bn, int cw) {
  return (static_cast<uint32_t>(na) * 128u + static_cast<uint32_t>(nb * bn)) * static_cast<uint32_t>(cw) * 2u;
}
// chunk width of the chunk-major modes: stages_max -1, -2, -3 -> 64, 32, 16
int chunk_width(int stages_max) { return stages_max == -1 ? 64 : (stages_max == -2 ? 32 : 16); }
// room for the stages: the limit less the 1 KB alignment slack and the barriers
uint32_t chunk_budget() { return static_cast<uint32_t>(g_smem_optin - 1024 - 64); }
}  // namespace

bool umma_chunk_fits(int npairs, const int *pair_a, const int *pair_b, int bn, int stages_max) {
  int na = 0, nb = 0;
  for (int p = 0; p < npairs; ++p) {
    na = pair_a[p] + 1 > na ? pair_a[p] + 1 : na;
    nb = pair_b[p] + 1 > nb ? pair_b[p] + 1 : nb;
  }
  return 2u * chunk_stage_bytes(na, nb, bn, chunk_width(stages_max)) <= chunk_budget();
}

cudaError_t launch_umma_gemm(const uint16_t *A, int m_max, const int *m_dev, int a_terms, const uint16_t *B, int n,
                             int b_terms, int kp, int npairs, const int *pair_a, const int *pair_b, float *out,
                             long long ldo, const int *out_rows, int *err, cudaStream_t st, const int *a_exp,
                             const int *b_exp, float *out_lo, int bn_max, double *out64, int slice_bits,
                             int batch_rows, int batches, int stages_max, int b_batch_rows, long long o_bstride,
                             long long o_rstride, long long o_cstride, const int *pair_group) {
  if (m_max <= 0 || n <= 0) return cudaSuccess;
  if (kp <= 0 || kp % 64 != 0 || npairs < 1 || npairs > kMaxPairs || a_terms < 1 || b_terms < 1)
    return cudaErrorInvalidValue;
  if (out64 && (!a_exp || (slice_bits != 7 && slice_bits != 8))) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(A) & 15u) || (reinterpret_cast<uintptr_t>(B) & 15u)) return cudaErrorInvalidValue;
  if ((a_exp == nullptr) != (b_exp == nullptr)) return cudaErrorInvalidValue;
  UmmaArgs g{};
  g.ngroups = 1;
  for (int p = 0; p < npairs; ++p) {
    if (pair_a[p] < 0 || pair_a[p] >= a_terms || pair_b[p] < 0 || pair_b[p] >= b_terms) return cudaErrorInvalidValue;
    g.pair_a[p] = pair_a[p];
    g.pair_b[p] = pair_b[p];
    // fixed-point mode: the accumulator of weight 256^-(a + b), or the one the
    // caller names (terms pre-scaled by powers of 256 share an accumulator)
    g.pair_group[p] = a_exp ? (pair_group ? pair_group[p] : pair_a[p] + pair_b[p]) : 0;
    if (g.pair_group[p] < 0 || g.pair_group[p] >= 8) return cudaErrorInvalidValue;
    if (g.pair_group[p] + 1 > g.ngroups) g.ngroups = g.pair_group[p] + 1;
  }
  if (g.ngroups > 8) return cudaErrorInvalidValue;
  g.slice_bits = slice_bits;
  g.out64 = out64;
  if (b_batch_rows <= 0) b_batch_rows = batch_rows;
  if (batch_rows < 0 || (batch_rows > 0 && (batches <= 0 || n > b_batch_rows))) return cudaErrorInvalidValue;
  g.batch_rows = batch_rows;
  g.b_batch_rows = b_batch_rows;
  g.tiles_per_batch = batch_rows > 0 ? (batch_rows + 127) / 128 : 0;
  g.a_exp = a_exp;
  g.b_exp = b_exp;
  g.m_max = m_max;
  g.m_dev = m_dev;
  g.n = n;
  g.kp = kp;
  // the ngroups accumulators of bn columns share the 512 tensor-memory columns;
  // bn_max (a multiple of 16, from the autotuner) may lower the limit
  int limit = g.ngroups <= 2 ? 256 : (g.ngroups <= 4 ? 128 : (g.ngroups <= 5 ? 96 : 64));
  if (bn_max > 0) {
    if (bn_max % 16) return cudaErrorInvalidValue;
    limit = bn_max < limit ? bn_max : limit;
  }
  g.bn = umma_pick_bn(n, limit);
  g.na = g.nb = 0;
  for (int p = 0; p < npairs; ++p) {
    g.na = pair_a[p] + 1 > g.na ? pair_a[p] + 1 : g.na;
    g.nb = pair_b[p] + 1 > g.nb ? pair_b[p] + 1 : g.nb;
  }
  uint32_t stage_bytes = 128u * 128u + static_cast<uint32_t>(g.bn) * 128u;
  if (stages_max < -3) return cudaErrorInvalidValue;
  // stages_max = -1, -2, -3: chunk-major, every slice of a 64-, 32- or 16-wide
  // K chunk per stage, as many stages as fit (two to four)
  g.chunk_major = stages_max < 0 ? 1 : 0;
  g.cw = g.chunk_major ? chunk_width(stages_max) : 64;
  if (g.chunk_major) {
    stage_bytes = chunk_stage_bytes(g.na, g.nb, g.bn, g.cw);
    if (2u * stage_bytes > chunk_budget()) return cudaErrorInvalidValue;
    g.stages = static_cast<int>(chunk_budget() / stage_bytes);
    if (g.stages > 4) g.stages = 4;
  } else {
    // pipeline depth: as many stages as fit in 200 KB, at most 6, or fewer
    // (stages_max, from the autotuner) so that several CTAs share an SM
    g.stages = static_cast<int>((200u * 1024u) / stage_bytes);
    if (g.stages > 6) g.stages = 6;
    if (stages_max > 0 && stages_max < g.stages) g.stages = stages_max < 2 ? 2 : stages_max;
  }
  g.npairs = npairs;
  g.idesc = (1u << 4)                                   // D: FP32
            | (1u << 7) | (1u << 10)                    // A, B: BF16
            | (static_cast<uint32_t>(g.bn >> 3) << 17)  // N
            | (static_cast<uint32_t>(128 >> 4) << 24);  // M
  uint32_t cols = 32;
  while (cols < static_cast<uint32_t>(g.bn * g.ngroups)) cols <<= 1;
  if (cols > 512) return cudaErrorInvalidValue;
  g.tmem_cols = cols;
  g.out = out;
  g.out_lo = a_exp ? out_lo : nullptr;
  g.ldo = ldo;
  g.out_rows = out_rows;
  if (o_cstride != 0 && (batch_rows <= 0 || out_rows)) return cudaErrorInvalidValue;
  g.o_bstride = o_bstride;
  g.o_rstride = o_rstride;
  g.o_cstride = o_cstride;
  g.err = err;
  CUtensorMap ta, tb;
  const uint64_t b_rows = batch_rows > 0 ? static_cast<uint64_t>(b_batch_rows) * batches : static_cast<uint64_t>(n);
  if (!make_map(&ta, A, static_cast<uint64_t>(a_terms) * kp, static_cast<uint64_t>(m_max), 128,
                static_cast<uint32_t>(g.cw)) ||
      !make_map(&tb, B, static_cast<uint64_t>(b_terms) * kp, b_rows, static_cast<uint32_t>(g.bn),
                static_cast<uint32_t>(g.cw)))
    return cudaErrorInvalidValue;
  const size_t smem = 1024 + static_cast<size_t>(g.stages) * stage_bytes + 8 * (2 * g.stages + 1) + 16;
  dim3 grid((n + g.bn - 1) / g.bn, batch_rows > 0 ? batches * g.tiles_per_batch : (m_max + 127) / 128);
  return launch_or_record<UmmaGemm, 128>(k_umma_gemm, grid, dim3(128), smem, st, ta, tb, g);
}

// ---------------------------------------------------------------------------
// Fixed-point operand packing.  Operand rows are compacted in list order: row
// m comes from table row list[m] (m < *count) or, without a list, from
// (m / nsub) * stride + m % nsub (m < nrows); rows_out[m] records it so that
// the contraction can write its result row back in place.  One warp per row.
// Each FP32 row is scaled by
// 2^-e (e = 1 + the binary exponent of its largest magnitude) and cut into
// kFixedSlices exact 8-bit integer slices t0, t1, ... (|t| <= 128), stored as
// BF16 side by side, with e in exps[m].  Every step of the cut is exact in
// FP32.  A two-float row P + P_lo is cut the same way, its remainder carried
// from slice to slice as an exact two-float sum (TwoSum), so that the slices
// take the low part's bits as well.
// ---------------------------------------------------------------------------
struct PackFixed {
  static __device__ __forceinline__ void run(const float *__restrict__ P, const float *__restrict__ P_lo,
                                             const int *__restrict__ list, const int *__restrict__ count, int nrows,
                                             int nsub, int stride, int L, int kp, __nv_bfloat16 *__restrict__ A,
                                             int *__restrict__ rows_out, int *__restrict__ exps, const uint3 bid,
                                             const uint3 gdim) {
    assume_global(P, A, rows_out, exps);
    const int rows = count ? *count : nrows;
    const int lane = threadIdx.x & 31;
    const long nw = (long)gdim.x * (blockDim.x >> 5);
    for (long m = (long)bid.x * (blockDim.x >> 5) + (threadIdx.x >> 5); m < rows; m += nw) {
      const long phys = list ? (long)list[m] : (m / nsub) * stride + (m % nsub);
      const float *src = P + phys * L;
      const float *srl = P_lo ? P_lo + phys * L : nullptr;
      float mx = 0.0f;
      for (int k = lane; k < L; k += 32) mx = fmaxf(mx, fabsf(src[k]));
  #pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      const int e = (mx > 0.0f) ? ilogbf(mx) + 1 : 0;
      if (lane == 0) {
        rows_out[m] = (int)phys;
        exps[m] = e;
      }
      __nv_bfloat16 *dst = A + m * kFixedSlices * (long)kp;
      for (int k = lane; k < kp; k += 32) {
        float x = k < L ? ldexpf(src[k], 7 - e) : 0.0f;  // |x| < 128
        // the low part, in the same scale
        float xl = (srl && k < L) ? ldexpf(srl[k], 7 - e) : 0.0f;
  #pragma unroll
        for (int t = 0; t < kFixedSlices; ++t) {
          const float q = rintf(x);
          dst[t * kp + k] = __float2bfloat16_rn(q);
          const fdw r = two_sum(__fsub_rn(x, q), xl);  // remainder + low part, exactly
          x = __fmul_rn(r.hi, 256.0f);
          xl = __fmul_rn(r.lo, 256.0f);
        }
      }
    }
}
};
__global__ void __launch_bounds__(256) k_pack_fixed(const float *__restrict__ P, const float *__restrict__ P_lo,
                                                    const int *__restrict__ list, const int *__restrict__ count,
                                                    int nrows, int nsub, int stride, int L, int kp,
                                                    __nv_bfloat16 *__restrict__ A, int *__restrict__ rows_out,
                                                    int *__restrict__ exps) {
  PackFixed::run(P, P_lo, list, count, nrows, nsub, stride, L, kp, A, rows_out, exps, blockIdx, gridDim);
}

cudaError_t launch_pack_fixed(const float *P, const float *P_lo, const int *list, const int *count, int nrows,
                               int nsub, int stride, int L, int kp, uint16_t *A, int *rows_out, int *exps,
                               int max_rows, cudaStream_t st) {
  if (max_rows <= 0) return cudaSuccess;
  long blocks = (max_rows + 7) / 8;
  if (blocks > 152 * 16) blocks = 152 * 16;
  return launch_or_record<PackFixed, 256>(k_pack_fixed, dim3((int)blocks), dim3(256), 0, st, P, P_lo, list, count,
                                          nrows, nsub > 0 ? nsub : 1, stride, L, kp,
                                          reinterpret_cast<__nv_bfloat16 *>(A), rows_out, exps);
}

// FP64 rows -> nsl exact slices of `bits` bits (|t| <= 2^(bits-1), BF16) per
// element relative to 2^e, e = 1 + the binary exponent of the row's largest
// magnitude, for the FP64-equivalent products (every step exact in FP64).
struct PackFixed64 {
  static __device__ __forceinline__ void run(const double *__restrict__ P, const int *__restrict__ list,
                                             const int *__restrict__ count, int nrows, int nsub, int stride, int L,
                                             int kp, int nsl, int bits, __nv_bfloat16 *__restrict__ A,
                                             int *__restrict__ rows_out, int *__restrict__ exps, long dst_stride,
                                             long dst_off, const uint3 bid, const uint3 gdim) {
    assume_global(P, A, rows_out, exps);
    const int rows = count ? *count : nrows;
    const int lane = threadIdx.x & 31;
    const long nw = (long)gdim.x * (blockDim.x >> 5);
    const double step = ldexp(1.0, bits);
    for (long m = (long)bid.x * (blockDim.x >> 5) + (threadIdx.x >> 5); m < rows; m += nw) {
      const long phys = list ? (long)list[m] : (m / nsub) * stride + (m % nsub);
      const double *src = P + phys * L;
      double mx = 0.0;
      for (int k = lane; k < L; k += 32) mx = fmax(mx, fabs(src[k]));
  #pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      const int e = (mx > 0.0) ? ilogb(mx) + 1 : 0;
      if (lane == 0) {
        // the row of the result: the source row, or (m / nsub) * dst_stride + dst_off + m % nsub
        rows_out[m] = dst_stride > 0 ? (int)((m / nsub) * dst_stride + dst_off + m % nsub) : (int)phys;
        exps[m] = e;
      }
      __nv_bfloat16 *dst = A + m * nsl * (long)kp;
      for (int k = lane; k < kp; k += 32) {
        double x = k < L ? ldexp(src[k], bits - 1 - e) : 0.0;  // |x| < 2^(bits-1)
        for (int t = 0; t < nsl; ++t) {
          const double q = rint(x);
          dst[t * kp + k] = __float2bfloat16_rn(static_cast<float>(q));
          x = (x - q) * step;
        }
      }
    }
}
};
__global__ void __launch_bounds__(256) k_pack_fixed64(const double *__restrict__ P, const int *__restrict__ list,
                                                      const int *__restrict__ count, int nrows, int nsub, int stride,
                                                      int L, int kp, int nsl, int bits, __nv_bfloat16 *__restrict__ A,
                                                      int *__restrict__ rows_out, int *__restrict__ exps,
                                                      long dst_stride, long dst_off) {
  PackFixed64::run(P, list, count, nrows, nsub, stride, L, kp, nsl, bits, A, rows_out, exps, dst_stride, dst_off,
                   blockIdx, gridDim);
}

cudaError_t launch_pack_fixed64(const double *P, const int *list, const int *count, int nrows, int nsub, int stride,
                                int L, int kp, int nsl, int bits, uint16_t *A, int *rows_out, int *exps,
                                int max_rows, cudaStream_t st, long dst_stride, long dst_off) {
  if (max_rows <= 0) return cudaSuccess;
  long blocks = (max_rows + 7) / 8;
  if (blocks > 152 * 16) blocks = 152 * 16;
  return launch_or_record<PackFixed64, 256>(k_pack_fixed64, dim3((int)blocks), dim3(256), 0, st, P, list, count, nrows,
                                            nsub > 0 ? nsub : 1, stride, L, kp, nsl, bits,
                                            reinterpret_cast<__nv_bfloat16 *>(A), rows_out, exps, dst_stride, dst_off);
}

// ---------------------------------------------------------------------------
// Columns of per-walker matrices as fixed-point operand rows (the operands of
// the kinetic M products, whose contraction runs over the rows of G~^{-1},
// Bt and A_up): for walker w < W and column c < C of X_w = X + w xw
// ([R][C] row-major), operand row m = w C + c holds X_w[0..R)[c] (zero from R
// to kp) relative to 2^e, e = 1 + the binary exponent of the column's largest
// magnitude, cut into nsl exact slices of `bits` bits (FP64 X: 8 or 7 bits, up
// to eight slices; two-float X + Xlo: 8 bits, the remainder carried exactly)
// as k_pack_fixed cuts a row.
// exps[m] = e; rows_out[m] = w dst_stride + dst_off + c when rows_out is given.
// One CTA per (walker, 32 columns): the column maxima first, then tiles of 64
// rows through shared memory, so that the reads (32 consecutive columns of a
// row) and the writes (64 consecutive entries of one slice of an operand row)
// are both coalesced.
// ---------------------------------------------------------------------------
template <bool kF64>
struct PackCols {
  static __device__ __forceinline__ void run(const double *__restrict__ X64, const float *__restrict__ X32,
                                             const float *__restrict__ Xlo, size_t xw, int R, int C, int kp,
                                             __nv_bfloat16 *__restrict__ A, int *__restrict__ exps,
                                             int *__restrict__ rows_out, long dst_stride, long dst_off, int nsl,
                                             int bits, const uint3 bid, const uint3 gdim) {
    assume_global(A, exps);
    if constexpr (kF64) assume_global(X64); else assume_global(X32);
    constexpr int kMaxSl = 8;
    __shared__ double t64[kF64 ? 64 : 1][33];
    __shared__ float th[kF64 ? 1 : 64][33], tl[kF64 ? 1 : 64][33];
    __shared__ float cmax[8][32];
    __shared__ int cexp[32];
    const int tid = threadIdx.x, cl = tid & 31, jr = tid >> 5;
    const int w = bid.y, c0 = bid.x * 32;
    const int c = c0 + cl;
    const size_t base = (size_t)w * xw;
    float mx = 0.0f;
    double mx64 = 0.0;
    if (c < C)
      for (int j = jr; j < R; j += 8) {
        if constexpr (kF64)
          mx64 = fmax(mx64, fabs(X64[base + (size_t)j * C + c]));
        else
          mx = fmaxf(mx, fabsf(X32[base + (size_t)j * C + c]));
      }
    if constexpr (kF64) {
      // exponents from the FP64 maxima: compare through the exponent only
      cmax[jr][cl] = 0.0f;
      __shared__ double cmax64[8][32];
      cmax64[jr][cl] = mx64;
      __syncthreads();
      if (jr == 0) {
        double m = cmax64[0][cl];
        for (int q = 1; q < 8; ++q) m = fmax(m, cmax64[q][cl]);
        const int e = m > 0.0 ? ilogb(m) + 1 : 0;
        cexp[cl] = e;
        if (c < C) {
          exps[(size_t)w * C + c] = e;
          if (rows_out) rows_out[(size_t)w * C + c] = (int)(w * dst_stride + dst_off + c);
        }
      }
    } else {
      cmax[jr][cl] = mx;
      __syncthreads();
      if (jr == 0) {
        float m = cmax[0][cl];
        for (int q = 1; q < 8; ++q) m = fmaxf(m, cmax[q][cl]);
        const int e = m > 0.0f ? ilogbf(m) + 1 : 0;
        cexp[cl] = e;
        if (c < C) {
          exps[(size_t)w * C + c] = e;
          if (rows_out) rows_out[(size_t)w * C + c] = (int)(w * dst_stride + dst_off + c);
        }
      }
    }
    __syncthreads();
    for (int j0 = 0; j0 < kp; j0 += 64) {
      // tile [64 rows][32 columns], zero past R or C
  #pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int jj = jr + 8 * q, j = j0 + jj;
        const bool in = j < R && c < C;
        if constexpr (kF64) {
          t64[jj][cl] = in ? X64[base + (size_t)j * C + c] : 0.0;
        } else {
          th[jj][cl] = in ? X32[base + (size_t)j * C + c] : 0.0f;
          tl[jj][cl] = (in && Xlo) ? Xlo[base + (size_t)j * C + c] : 0.0f;
        }
      }
      __syncthreads();
      // warp jr writes columns jr, jr + 8, jr + 16, jr + 24; lane: rows 2 lane, 2 lane + 1
  #pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        const int col = jr + 8 * cc, cg = c0 + col;
        if (cg >= C) continue;
        const int e = cexp[col];
        __nv_bfloat16 sl[2][kMaxSl];
  #pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int jj = 2 * (tid & 31) + h;
          if constexpr (kF64) {
            const double step = ldexp(1.0, bits);
            double x = ldexp(t64[jj][col], bits - 1 - e);  // |x| < 2^(bits - 1)
  #pragma unroll
            for (int t = 0; t < kMaxSl; ++t) {
              if (t >= nsl) break;
              const double q = rint(x);
              sl[h][t] = __float2bfloat16_rn(static_cast<float>(q));
              x = (x - q) * step;
            }
          } else {
            float x = ldexpf(th[jj][col], 7 - e), xl = ldexpf(tl[jj][col], 7 - e);
  #pragma unroll
            for (int t = 0; t < kMaxSl; ++t) {
              if (t >= nsl) break;
              const float q = rintf(x);
              sl[h][t] = __float2bfloat16_rn(q);
              const fdw r = two_sum(__fsub_rn(x, q), xl);
              x = __fmul_rn(r.hi, 256.0f);
              xl = __fmul_rn(r.lo, 256.0f);
            }
          }
        }
        __nv_bfloat16 *dst = A + ((size_t)w * C + cg) * nsl * (size_t)kp + j0 + 2 * (tid & 31);
  #pragma unroll
        for (int t = 0; t < kMaxSl; ++t) {
          if (t >= nsl) break;
          __nv_bfloat162 v;
          v.x = sl[0][t];
          v.y = sl[1][t];
          *reinterpret_cast<__nv_bfloat162 *>(dst + (size_t)t * kp) = v;
        }
      }
      __syncthreads();
    }
}
};
template <bool kF64>
__global__ void __launch_bounds__(256) k_pack_cols(const double *__restrict__ X64, const float *__restrict__ X32,
                                                   const float *__restrict__ Xlo, size_t xw, int R, int C, int kp,
                                                   __nv_bfloat16 *__restrict__ A, int *__restrict__ exps,
                                                   int *__restrict__ rows_out, long dst_stride, long dst_off, int nsl,
                                                   int bits) {
  PackCols<kF64>::run(X64, X32, Xlo, xw, R, C, kp, A, exps, rows_out, dst_stride, dst_off, nsl, bits, blockIdx,
                      gridDim);
}

cudaError_t launch_pack_cols(const double *X64, const float *X32, const float *Xlo, size_t xw, int R, int C, int kp,
                             int W, uint16_t *A, int *exps, int *rows_out, long dst_stride, long dst_off,
                             cudaStream_t st, int nsl, int bits) {
  if (W <= 0 || C <= 0) return cudaSuccess;
  if (kp % 64 != 0 || kp < R || (X64 == nullptr) == (X32 == nullptr)) return cudaErrorInvalidValue;
  if (nsl < 1 || nsl > 8 || (bits != 8 && (bits != 7 || !X64))) return cudaErrorInvalidValue;
  dim3 grid((C + 31) / 32, W);
  const float *nf = nullptr;
  const double *nd = nullptr;
  if (X64)
    return launch_or_record<PackCols<true>, 256>(k_pack_cols<true>, grid, dim3(256), 0, st, X64, nf, nf, xw, R, C, kp,
                                                 reinterpret_cast<__nv_bfloat16 *>(A), exps, rows_out, dst_stride,
                                                 dst_off, nsl, bits);
  return launch_or_record<PackCols<false>, 256>(k_pack_cols<false>, grid, dim3(256), 0, st, nd, X32, Xlo, xw, R, C, kp,
                                                reinterpret_cast<__nv_bfloat16 *>(A), exps, rows_out, dst_stride,
                                                dst_off, nsl, bits);
}

cudaError_t setup_umma_attributes() {
  // the largest opt-in shared memory per block (227 KB on this part), so that
  // two or more chunk-major stages of six slices fit (with K chunks of 32 or 16)
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  g_smem_optin = optin < 220 * 1024 ? 220 * 1024 : optin;
  return cudaFuncSetAttribute(k_umma_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, g_smem_optin);
}

}  // namespace jagp
