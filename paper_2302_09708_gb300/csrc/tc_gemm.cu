// Split-precision tensor-core GEMMs (tcgen05 + TMA + TMEM) for the mixed
// precision projection and rotation of Algorithm 1 (paper Sec. II B, II D).
//
// Block fixed-point split (Ozaki-style): for every operand row r (a row of the
// GEMM's M or N dimension) and every chunk q of 256 K values, the entries are
// scaled by 2^-e_rq, e_rq the binary exponent of the chunk's largest entry, and
// every entry u = x 2^-e_rq in (-1, 1) is written as four signed
// 8-bit integer digits, u = 2^-7 (d1 + 2^-8 d2 + 2^-16 d3 + 2^-24 d4) + O(2^-32),
// each exactly representable in BF16.  A product is formed from the ten digit
// products of weight >= 2^-24 relative to the leading one, in four levels
//   L0 = a1 b1,  L1 = a1 b2 + a2 b1,  L2 = a1 b3 + a2 b2 + a3 b1,
//   L3 = a1 b4 + a2 b3 + a3 b2 + a4 b1,
//   a b ~ 2^(e_a + e_b - 14) (L0 + 2^-8 L1 + 2^-16 L2 + 2^-24 L3),
// each level accumulating in its own tensor-memory accumulator.  Digit products
// are integers of magnitude <= 2^14, so over a chunk of 256 K values every level
// sum stays an integer of magnitude <= 2^24 and the tensor core adds it exactly
// (its alignment/truncation of products never drops a bit).  Every
// kChunkSteps K-steps (one exponent chunk) the exact level sums are scaled by
// 2^(e_a + e_b - 14) of that chunk and folded into a double-FP32 (hi, lo)
// running sum held in registers.  Per-chunk exponents keep the digits relative
// to local magnitudes, so the first dropped level (whose diagonal terms never
// cancel) stays ~2^-32 of the local values instead of biasing long sums.
//
// Kernel structure (one CTA per 128 x 64 output tile, 192 threads):
//   warp 0     TMA producer: one 3-D TMA load per operand per K-step brings the
//              four BF16 digit tiles (128-byte swizzle) into a 2-stage
//              shared-memory ring (full/empty mbarriers);
//   warp 1     allocates 512 TMEM columns and issues tcgen05.mma (one thread):
//              2 buffers x 4 level accumulators (64 columns each);
//   warps 2-5  epilogue: fold a finished accumulator buffer into (hi, lo), and
//              finally write hi + lo.
// Every mbarrier wait is bounded; on expiry the CTA records SPARC_ERR_TIMEOUT
// in the status word, stops issuing work, drains what it issued (bounded) and
// frees its tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "internal.cuh"

namespace sparc {

namespace {

constexpr int kBM = 128, kBN = 64, kBK = 64;
constexpr int kSlices = 4;
constexpr int kLevels = 4;
constexpr int kStages = 2;
constexpr int kChunkSteps = 4;
constexpr int kProducts = 10;
constexpr uint32_t kTileBytes = kBM * kBK * 2;                 // one A slice tile (16 KB)
constexpr uint32_t kTileBytesB = kBN * kBK * 2;                // one B slice tile (8 KB)
constexpr uint32_t kOpBytes = kSlices * kTileBytes;            // A operand, 3 slices
constexpr uint32_t kStageBytes = kOpBytes + kSlices * kTileBytesB;
constexpr uint32_t kSmemBytes = kStages * kStageBytes + 1024 + 256;
constexpr uint32_t kTmemCols = 512;
constexpr int kThreads = 192;
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait; false on timeout (and then *abort is set).  Also gives up when
// another CTA of the launch has already recorded a status.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort,
                                          const int* status) {
  if (mbar_test(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_test(bar, parity)) return true;
    if (*abort) return false;
    if (*(volatile const int*)status != 0 || clock64() - t0 > kWaitCycles) {
      *abort = 1;
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row
// groups 1024 bytes apart (tcgen05 descriptor version 1).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;            // descriptor version
  d |= (uint64_t)2 << 61;            // 128-byte swizzle
  return d;
}

// Instruction descriptor: BF16 x BF16 -> FP32, A and B K-major, M = 128, N = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                            ((uint32_t)(kBM >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

#define TMEM_REGS32(r)                                                                           \
  "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),           \
      "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),    \
      "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), \
      "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), \
      "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
#define TMEM_IN32(r)                                                                          \
  "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),     \
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),       \
      "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]),     \
      "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]),     \
      "r"(r[29]), "r"(r[30]), "r"(r[31])
#define REGLIST32                                                                             \
  "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19," \
  " %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}"

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 " REGLIST32 ", [%32];"
               : TMEM_REGS32(r)
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%32], " REGLIST32 ";" ::TMEM_IN32(r),
               "r"(taddr)
               : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// slice pairs (a-slice, b-slice) of the six products, their magnitude level
// and whether the product is the first of its level (starts the accumulator)
__constant__ int c_sa[kProducts] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3};
__constant__ int c_sb[kProducts] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0};
__constant__ int c_lv[kProducts] = {0, 1, 1, 2, 2, 2, 3, 3, 3, 3};
__constant__ int c_first[kProducts] = {1, 1, 0, 1, 0, 0, 1, 0, 0, 0};

// 2^n as a float, built from the IEEE-754 exponent field for normal results.
__device__ __forceinline__ float pow2i(int n) {
  return n >= -126 ? __int_as_float((min(n, 127) + 127) << 23) : ldexpf(1.0f, n);
}

struct TcArgs {
  int M, N;
  int64_t K;
  int64_t kchunk;   // K per split (multiple of kBK)
  int upper;        // 1: enumerate only tiles with bi <= bj (symmetric outputs)
  int tiles_m;
  double* work;     // mode 0: work[(split * 2 + out) * M * N + m + n * M]
  float* out32;     // mode 1: out32[m + n * ldo]
  int64_t ldo;
  int mode;
  const int8_t* escA;   // exponent of A row r in chunk q at [q * MP + r]
  const int8_t* escB0;  // exponent of B row c (output 0) in chunk q at [q * NP + c]
  const int8_t* escB1;  // same for output 1
  int MP, NP;           // row strides of the exponent arrays (multiples of 128)
  int* status;
};

__global__ void __launch_bounds__(kThreads, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB0,
              const __grid_constant__ CUtensorMap tB1, const TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t bars[2 * kStages + 5];
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t full0 = smem_u32(&bars[0]);
  const uint32_t empty0 = smem_u32(&bars[kStages]);
  const uint32_t accf0 = smem_u32(&bars[2 * kStages]);      // 2 barriers
  const uint32_t acce0 = smem_u32(&bars[2 * kStages + 2]);  // 2 barriers
  const uint32_t drain = smem_u32(&bars[2 * kStages + 4]);

  const int bi = blockIdx.x % a.tiles_m;
  const int bj = blockIdx.x / a.tiles_m;
  // symmetric outputs: only tiles that reach the upper triangle (i <= j)
  if (a.upper && bi * kBM > bj * kBN + kBN - 1) return;
  const int out = blockIdx.z;
  const CUtensorMap* tB = out == 0 ? &tB0 : &tB1;
  const int64_t k0 = (int64_t)blockIdx.y * a.kchunk;
  const int64_t k1 = min(a.K, k0 + a.kchunk);
  const int nk = k1 > k0 ? (int)((k1 - k0 + kBK - 1) / kBK) : 0;
  const int nchunks = (nk + kChunkSteps - 1) / kChunkSteps;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf0 + 8 * b, 1);
      mbar_init(acce0 + 8 * b, 4);
    }
    mbar_init(drain, 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_sh)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;
  volatile int* abort = &abort_sh;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int issued = 0;
      for (int it = 0; it < nk; ++it) {
        const int s = it % kStages;
        const uint32_t round = (uint32_t)(it / kStages);
        if (!mbar_wait(empty0 + 8 * s, (round & 1) ^ 1, abort, a.status)) break;
        const uint32_t sa = base + s * kStageBytes;
        mbar_expect_tx(full0 + 8 * s, kStageBytes);
        const int kx = (int)(k0 + (int64_t)it * kBK);
        tma_load_3d(sa, &tA, kx, bi * kBM, 0, full0 + 8 * s);
        tma_load_3d(sa + kOpBytes, tB, kx, bj * kBN, 0, full0 + 8 * s);
        issued = it + 1;
      }
      if (*abort) {
        // drain: the loads already issued must land before the CTA exits
        for (int it = max(0, issued - kStages); it < issued; ++it) {
          const long long t0 = clock64();
          while (!mbar_test(full0 + 8 * (it % kStages), (uint32_t)(it / kStages) & 1) &&
                 clock64() - t0 < kWaitCycles) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      for (int it = 0; it < nk; ++it) {
        const int s = it % kStages;
        const uint32_t round = (uint32_t)(it / kStages);
        const int chunk = it / kChunkSteps, in_chunk = it % kChunkSteps;
        const int buf = chunk & 1;
        const uint32_t use = (uint32_t)(chunk >> 1);
        if (in_chunk == 0) {
          if (!mbar_wait(acce0 + 8 * buf, (use & 1) ^ 1, abort, a.status)) break;
          tc_fence_after();
        }
        if (!mbar_wait(full0 + 8 * s, round & 1, abort, a.status)) break;
        tc_fence_after();
        const uint32_t sa = base + s * kStageBytes, sb = sa + kOpBytes;
#pragma unroll
        for (int p = 0; p < kProducts; ++p) {
          const uint32_t d = tmem + (uint32_t)((buf * kLevels + c_lv[p]) * kBN);
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk) {
            const uint64_t da = smem_desc(sa + c_sa[p] * kTileBytes + kk * 32);
            const uint64_t db = smem_desc(sb + c_sb[p] * kTileBytesB + kk * 32);
            tc_mma(d, da, db, !(in_chunk == 0 && kk == 0 && c_first[p]));
          }
        }
        tc_commit(empty0 + 8 * s);
        if (in_chunk == kChunkSteps - 1 || it == nk - 1) tc_commit(accf0 + 8 * buf);
      }
      // all issued MMAs complete before tensor memory is released
      tc_commit(drain);
      const long long t0 = clock64();
      while (!mbar_test(drain, 0) && clock64() - t0 < kWaitCycles) {
      }
    }
  } else {
    // ---------------- epilogue (warps 2..5) ----------------
    const int q = warp & 3;  // TMEM lane quarter of this warp
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    float hi[kBN], lo[kBN];
#pragma unroll
    for (int i = 0; i < kBN; ++i) {
      hi[i] = 0.f;
      lo[i] = 0.f;
    }
    bool ok = true;
    for (int c = 0; c < nchunks && ok; ++c) {
      const int buf = c & 1;
      const uint32_t use = (uint32_t)(c >> 1);
      if (!mbar_wait(accf0 + 8 * buf, use & 1, abort, a.status)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t t_acc = tmem + lane_off + (uint32_t)(buf * kLevels * kBN);
      // exponents of this chunk: the thread's A row and the tile's 64 B rows
      const int qg = (int)(k0 / (kBK * kChunkSteps)) + c;
      const int rowc = min(bi * kBM + q * 32 + lane, a.MP - 1);
      const int ea = (int)a.escA[(int64_t)qg * a.MP + rowc] - 14;
      const uint4* eb_src = reinterpret_cast<const uint4*>(
          (out == 0 ? a.escB0 : a.escB1) + (int64_t)qg * a.NP + bj * kBN);
#pragma unroll
      for (int cb = 0; cb < kBN / 32; ++cb) {
        // t = L1 + 2^-8 L2 + 2^-16 L3 (exact integers; FP32 keeps 24 bits of it)
        uint32_t v0[32], t[32];
        const uint4 eb0 = __ldg(eb_src + 2 * cb), eb1 = __ldg(eb_src + 2 * cb + 1);
        tmem_ld32(t_acc + cb * 32, v0);
        tmem_ld32(t_acc + 3 * kBN + cb * 32, t);
        tmem_wait_ld();
        {
          uint32_t v[32];
          tmem_ld32(t_acc + 2 * kBN + cb * 32, v);
          tmem_wait_ld();
#pragma unroll
          for (int i = 0; i < 32; ++i)
            t[i] = __float_as_uint(
                __fmaf_rn(__uint_as_float(t[i]), 0.00390625f, __uint_as_float(v[i])));
          tmem_ld32(t_acc + kBN + cb * 32, v);
          tmem_wait_ld();
#pragma unroll
          for (int i = 0; i < 32; ++i)
            t[i] = __float_as_uint(
                __fmaf_rn(__uint_as_float(t[i]), 0.00390625f, __uint_as_float(v[i])) *
                0.00390625f);
        }
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          float hh = hi[cb * 32 + i], ll = lo[cb * 32 + i];
          const uint4& ew = i < 16 ? eb0 : eb1;
          const uint32_t word = (i & 15) < 4 ? ew.x : (i & 15) < 8 ? ew.y : (i & 15) < 12 ? ew.z : ew.w;
          const int eb = (int)(int8_t)(word >> (8 * (i & 3)));
          const float sc = pow2i(ea + eb);
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const float x = __uint_as_float(u == 0 ? v0[i] : t[i]) * sc;
            const float sm = __fadd_rn(hh, x);
            const float bp = __fsub_rn(sm, hh);
            const float ap = __fsub_rn(sm, bp);
            const float err = __fadd_rn(__fsub_rn(hh, ap), __fsub_rn(x, bp));
            hh = sm;
            ll = __fadd_rn(ll, err);
          }
          hi[cb * 32 + i] = hh;
          lo[cb * 32 + i] = ll;
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acce0 + 8 * buf);
    }
    if (ok && nchunks > 0) {
      const int row = bi * kBM + q * 32 + lane;
      if (row < a.M) {
#pragma unroll
        for (int i = 0; i < kBN; ++i) {
          const int col = bj * kBN + i;
          if (col < a.N) {
            if (a.mode == 0) {
              a.work[((int64_t)blockIdx.y * 2 + out) * a.M * a.N + row + (int64_t)col * a.M] =
                  (double)hi[i] + (double)lo[i];
            } else {
              a.out32[row + (int64_t)col * a.ldo] = __fadd_rn(hi[i], lo[i]);
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
  }
  if (threadIdx.x == 0 && abort_sh) atomicCAS(a.status, 0, SPARC_ERR_TIMEOUT);
}

// ---------------------------------------------------------------------------
// Fixed-point digit slicing
// ---------------------------------------------------------------------------
// Binary exponent E with |v| < 2^E for the largest |v| (0 for an all-zero row).
__device__ __forceinline__ int row_exponent(double vmax) {
  if (!(vmax > 0.0)) return 0;
  int e;
  frexp(vmax, &e);  // vmax = m 2^e, m in [0.5, 1)
  return e;
}

// Chunk exponent stored as int8. Raising E keeps |x 2^-E| < 1, so the clamp
// only costs digits of chunks whose largest entry is below 2^-120.
__device__ __forceinline__ int8_t chunk_exponent(double vmax) {
  return (int8_t)max(-120, min(127, row_exponent(vmax)));
}

// Four signed 8-bit digits of u = x 2^-E (|u| < 1):
// u = 2^-7 (d1 + d2/2^8 + d3/2^16 + d4/2^24), each |d| <= 128.
__device__ __forceinline__ void digits(double x, int E, __nv_bfloat16 (&d)[kSlices]) {
  double u = ldexp(x, 7 - E);
#pragma unroll
  for (int k = 0; k < kSlices; ++k) {
    const double r = rint(u);
    d[k] = __double2bfloat16(r);
    u = (u - r) * 256.0;
  }
}
__device__ __forceinline__ void digitsf(float x, int E, __nv_bfloat16 (&d)[kSlices]) {
  // FP32 input: its 24-bit mantissa spans at most the first four digits, and
  // every step below is exact in FP32
  float u = ldexpf(x, 7 - E);
#pragma unroll
  for (int k = 0; k < kSlices; ++k) {
    const float r = rintf(u);
    d[k] = __float2bfloat16_rn(r);
    u = (u - r) * 256.0f;
  }
}

constexpr int kQ = kBK * kChunkSteps;  // K values per exponent chunk

// Chunk exponents of the columns of X: esc[q * NP + col] = E(max over t in chunk
// q of |X[t + col ldx]|), one warp per (column, chunk).
__global__ void k_chunk_exp_cols(const float* __restrict__ X, int64_t ldx, int64_t nd, int ncol,
                                 int nq, int NP, int8_t* __restrict__ esc) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= (int64_t)ncol * nq) return;
  const int col = (int)(w % ncol), q = (int)(w / ncol);
  const float* x = X + (int64_t)col * ldx;
  float m = 0.f;
  const int64_t t1 = min((int64_t)(q + 1) * kQ, nd);
  for (int64_t t = (int64_t)q * kQ + lane; t < t1; t += 32) m = fmaxf(m, fabsf(x[t]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) esc[(int64_t)q * NP + col] = chunk_exponent((double)m);
}

// Column exponents f_k of X (one block per column), used to balance columns.
__global__ void k_col_exponent(const float* __restrict__ X, int64_t ldx, int64_t nd,
                               int* __restrict__ esc) {
  __shared__ float sm[32];
  const float* x = X + (int64_t)blockIdx.x * ldx;
  float m = 0.f;
  for (int64_t t = threadIdx.x; t < nd; t += blockDim.x) m = fmaxf(m, fabsf(x[t]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float r = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmaxf(r, sm[w]);
    esc[blockIdx.x] = row_exponent((double)r);
  }
}

// Chunk exponents of the rows of the column-balanced X (rotation A operand):
// esc[q * MP + t] = E(max over k in chunk q of |X[t + k ldx]| 2^-f_k).
__global__ void k_chunk_exp_rows(const float* __restrict__ X, int64_t ldx, int64_t nd, int ns,
                                 const int* __restrict__ fcol, int MP, int8_t* __restrict__ esc) {
  const int q = blockIdx.y;
  const int k1 = min((q + 1) * kQ, ns);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nd;
       t += (int64_t)gridDim.x * blockDim.x) {
    float m = 0.f;
    for (int k = q * kQ; k < k1; ++k)
      m = fmaxf(m, ldexpf(fabsf(X[t + (int64_t)k * ldx]), -fcol[k]));
    esc[(int64_t)q * MP + t] = chunk_exponent((double)m);
  }
}

// Chunk exponents of the rows of the row-scaled Z (rotation B operand, row j =
// output column j): esc[q * NP + j] = E(max over k in chunk q of |Z[k + j n]| 2^f_k).
__global__ void k_chunk_exp_z(const double* __restrict__ Z, int n, const int* __restrict__ fcol,
                              int nq, int NP, int8_t* __restrict__ esc) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= (int64_t)n * nq) return;
  const int j = (int)(w % n), q = (int)(w / n);
  double m = 0.0;
  const int k1 = min((q + 1) * kQ, n);
  for (int k = q * kQ + lane; k < k1; k += 32) m = fmax(m, ldexp(fabs(Z[k + (int64_t)j * n]), fcol[k]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) esc[(int64_t)q * NP + j] = chunk_exponent(m);
}

// S[s][col][t] = digit s of X[t + col ldx] at its chunk's exponent (ld = lds)
__global__ void k_slice_cols(const float* __restrict__ X, int64_t ldx, int64_t nd, int ncol,
                             const int8_t* __restrict__ esc, int NP,
                             __nv_bfloat16* __restrict__ S, int64_t lds) {
  const int col = blockIdx.y;
  const int64_t plane = lds * ncol;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < lds;
       t += (int64_t)gridDim.x * blockDim.x) {
    __nv_bfloat16 d[kSlices];
    const int E = esc[(t / kQ) * NP + col];
    digitsf(t < nd ? X[t + col * ldx] : 0.f, E, d);
    const int64_t o = t + col * lds;
#pragma unroll
    for (int k = 0; k < kSlices; ++k) S[k * plane + o] = d[k];
  }
}

// Transposed digits of the column-balanced X: S[s][t][k] = digit s of
// X[t + k ldx] 2^-f_k at row t's exponent (ld = ldk)
__global__ void k_slice_transpose(const float* __restrict__ X, int64_t ldx, int64_t nd, int ns,
                                  const int* __restrict__ fcol, const int8_t* __restrict__ esc,
                                  int MP, __nv_bfloat16* __restrict__ S, int64_t ldk) {
  __shared__ float tile[32][33];
  const int64_t t0 = (int64_t)blockIdx.x * 32;
  const int k0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int k = k0 + r;
    const int64_t t = t0 + threadIdx.x;
    tile[r][threadIdx.x] = (k < ns && t < nd) ? ldexpf(X[t + (int64_t)k * ldx], -fcol[k]) : 0.f;
  }
  __syncthreads();
  const int64_t plane = ldk * nd;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t t = t0 + r;
    const int k = k0 + threadIdx.x;
    if (t < nd && k < ldk) {
      __nv_bfloat16 d[kSlices];
      digitsf(tile[threadIdx.x][r], esc[(int64_t)(k / kQ) * MP + t], d);
      const int64_t o = t * ldk + k;
#pragma unroll
      for (int q = 0; q < kSlices; ++q) S[q * plane + o] = d[q];
    }
  }
}

// Z digits of the row-scaled Z: S[s][j][k] = digit s of Z[k + j n] 2^f_k at
// column j's exponent, ld = ldk  (X Z = (X 2^-f) (2^f Z): the scalings cancel)
__global__ void k_slice_z(const double* __restrict__ Z, int n, const int* __restrict__ fcol,
                          const int8_t* __restrict__ esc, int NP, __nv_bfloat16* __restrict__ S,
                          int64_t ldk) {
  const int64_t plane = ldk * n;
  const int64_t tot = (int64_t)n * ldk;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / ldk), k = (int)(e % ldk);
    __nv_bfloat16 d[kSlices];
    digits(k < n ? ldexp(Z[k + (int64_t)j * n], fcol[k]) : 0.0, esc[(int64_t)(k / kQ) * NP + j], d);
#pragma unroll
    for (int q = 0; q < kSlices; ++q) S[q * plane + e] = d[q];
  }
}

// cuTensorMapEncodeTiled, resolved through the runtime so that the library does
// not link the driver library directly (it then also loads on hosts without one).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 3-D BF16 tensor map: dims (inner, rows, slices), box (64, box_rows, slices), 128-byte swizzle.
bool make_map(CUtensorMap* m, const void* base, uint64_t inner, uint64_t rows, uint64_t ld,
              uint32_t box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[3] = {inner, rows, (cuuint64_t)kSlices};
  cuuint64_t strides[2] = {ld * 2, ld * rows * 2};
  cuuint32_t box[3] = {kBK, box_rows, (cuuint32_t)kSlices};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                                      const_cast<void*>(base), dims, strides, box, estr,
                                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

cudaError_t launch_tc(const CUtensorMap& tA, const CUtensorMap& tB0, const CUtensorMap& tB1,
                      const TcArgs& a, dim3 grid, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e =
        cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  note_launch(), k_tc_gemm<<<grid, kThreads, kSmemBytes, st>>>(tA, tB0, tB1, a);
  return cudaGetLastError();
}

}  // namespace

size_t tc_esc_bytes(int64_t ld, int64_t nd, int ns_max) {
  const int64_t lds = (nd + 63) / 64 * 64;
  const int64_t nqp = (lds + kQ - 1) / kQ, NP = (ns_max + 127) / 128 * 128;
  const int64_t ldk = (ns_max + 7) / 8 * 8, nqr = (ldk + kQ - 1) / kQ;
  const int64_t MP = (nd + 127) / 128 * 128;
  const int64_t proj = 2 * nqp * NP;
  const int64_t rot = 4 * ((ns_max + 63) / 64 * 64) + nqr * (MP + NP);
  (void)ld;
  return (size_t)std::max(proj, rot) + 256;
}

size_t tc_slice_elems(int64_t ld, int64_t nd, int ns_max) {
  const int64_t ldk = (ns_max + 7) / 8 * 8;
  return (size_t)kSlices * std::max<int64_t>(ld * ns_max, nd * ldk);
}

int tc_project_nsplit(int ns) {
  const int tm = (ns + kBM - 1) / kBM, tn = (ns + kBN - 1) / kBN;
  int tiles = 0;
  for (int bj = 0; bj < tn; ++bj)
    for (int bi = 0; bi < tm; ++bi)
      if (bi * kBM <= bj * kBN + kBN - 1) ++tiles;
  tiles *= 2;  // Hs and Ms
  int s = (2 * 152 + tiles - 1) / tiles;
  return std::max(1, std::min(s, 64));
}

cudaError_t tc_project(const float* Xt, const float* Yt, int64_t ld, int64_t nd, int ns,
                       double* Hs, double* Ms, double* work, int nsplit, __nv_bfloat16* SX,
                       __nv_bfloat16* SY, int* esc, int* status, cudaStream_t st) {
  // digits of both operands, K-major (t contiguous per orbital column), each
  // orbital column at its own exponent
  const int64_t lds = (nd + 63) / 64 * 64;
  const int nq = (int)((lds + kQ - 1) / kQ);
  const int NP = (ns + 127) / 128 * 128;
  int8_t* escX = reinterpret_cast<int8_t*>(esc);
  int8_t* escY = escX + (size_t)nq * NP;
  const unsigned eg = (unsigned)(((int64_t)ns * nq * 32 + 255) / 256);
  note_launch(), k_chunk_exp_cols<<<eg, 256, 0, st>>>(Xt, ld, nd, ns, nq, NP, escX);
  note_launch(), k_chunk_exp_cols<<<eg, 256, 0, st>>>(Yt, ld, nd, ns, nq, NP, escY);
  dim3 sg((unsigned)std::min<int64_t>((lds + 255) / 256, 64), ns);
  note_launch(), k_slice_cols<<<sg, 256, 0, st>>>(Xt, ld, nd, ns, escX, NP, SX, lds);
  note_launch(), k_slice_cols<<<sg, 256, 0, st>>>(Yt, ld, nd, ns, escY, NP, SY, lds);
  CUtensorMap mXa, mXb, mYb;
  if (!make_map(&mXa, SX, (uint64_t)lds, (uint64_t)ns, (uint64_t)lds, kBM) ||
      !make_map(&mXb, SX, (uint64_t)lds, (uint64_t)ns, (uint64_t)lds, kBN) ||
      !make_map(&mYb, SY, (uint64_t)lds, (uint64_t)ns, (uint64_t)lds, kBN))
    return cudaErrorInvalidValue;
  TcArgs a{};
  a.M = ns;
  a.N = ns;
  a.K = lds;
  int64_t kc = (lds + nsplit - 1) / nsplit;
  a.kchunk = (kc + kQ - 1) / kQ * kQ;  // splits start on exponent chunks
  a.upper = 1;
  a.tiles_m = (ns + kBM - 1) / kBM;
  a.work = work;
  a.mode = 0;
  a.escA = escX;
  a.escB0 = escY;
  a.escB1 = escX;
  a.MP = NP;
  a.NP = NP;
  a.status = status;
  const int tn = (ns + kBN - 1) / kBN;
  const int nsp = (int)((lds + a.kchunk - 1) / a.kchunk);
  // out 0: Hs = X^T Y (B = Y slices), out 1: Ms = X^T X (B = X slices); tiles
  // entirely below the diagonal exit at once
  cudaError_t e = launch_tc(mXa, mYb, mXb, a, dim3(a.tiles_m * tn, nsp, 2), st);
  if (e != cudaSuccess) return e;
  // the SIMT path's deterministic split reduction (upper elements, mirrored)
  return project_reduce(work, nsp, ns, Hs, Ms, st);
}

cudaError_t tc_rotate(const float* Xt, int64_t ld, int64_t nd, int ns, const double* Z, float* Xout,
                      int64_t ldo, __nv_bfloat16* SA, __nv_bfloat16* SZ, int* esc, int* status,
                      cudaStream_t st) {
  // digits of Xt per grid point t (over its ns entries) and of Z per column j
  const int64_t ldk = (ns + 7) / 8 * 8;
  const int nq = (int)((ldk + kQ - 1) / kQ);
  const int MP = (int)((nd + 127) / 128 * 128), NP = (ns + 127) / 128 * 128;
  int* fcol = esc;  // ns entries: column exponents of Xt
  int8_t* escT = reinterpret_cast<int8_t*>(esc + ((ns + 63) / 64 * 64));
  int8_t* escZ = escT + (size_t)nq * MP;
  note_launch(), k_col_exponent<<<ns, 256, 0, st>>>(Xt, ld, nd, fcol);
  note_launch(), k_chunk_exp_rows<<<dim3((unsigned)std::min<int64_t>((nd + 255) / 256, 4096), nq),
                                    256, 0, st>>>(Xt, ld, nd, ns, fcol, MP, escT);
  note_launch(), k_chunk_exp_z<<<(unsigned)(((int64_t)ns * nq * 32 + 255) / 256), 256, 0, st>>>(
      Z, ns, fcol, nq, NP, escZ);
  dim3 tg((unsigned)((nd + 31) / 32), (unsigned)((ldk + 31) / 32));
  note_launch(), k_slice_transpose<<<tg, dim3(32, 8), 0, st>>>(Xt, ld, nd, ns, fcol, escT, MP, SA,
                                                               ldk);
  note_launch(), k_slice_z<<<(unsigned)std::min<int64_t>(((int64_t)ns * ldk + 255) / 256, 4096),
                             256, 0, st>>>(Z, ns, fcol, escZ, NP, SZ, ldk);
  CUtensorMap mA, mZ;
  if (!make_map(&mA, SA, (uint64_t)ldk, (uint64_t)nd, (uint64_t)ldk, kBM) ||
      !make_map(&mZ, SZ, (uint64_t)ldk, (uint64_t)ns, (uint64_t)ldk, kBN))
    return cudaErrorInvalidValue;
  TcArgs a{};
  a.M = (int)nd;
  a.N = ns;
  a.K = ldk;
  a.kchunk = (ldk + kQ - 1) / kQ * kQ;
  a.upper = 0;
  a.tiles_m = (int)((nd + kBM - 1) / kBM);
  a.out32 = Xout;
  a.ldo = ldo;
  a.mode = 1;
  a.escA = escT;
  a.escB0 = escZ;
  a.escB1 = escZ;
  a.MP = MP;
  a.NP = NP;
  a.status = status;
  const int tn = (ns + kBN - 1) / kBN;
  return launch_tc(mA, mZ, mZ, a, dim3(a.tiles_m * tn, 1, 1), st);
}

}  // namespace sparc
