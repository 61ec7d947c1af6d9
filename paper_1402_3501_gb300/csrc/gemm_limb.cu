// fgemm, limb form: C <- C - A B mod p on the tcgen05 tensor cores.
//
// Delayed modular reduction (Sec. 3.1) needs products summed exactly; the
// paper does it in the 53-bit mantissa of doubles.  Here the residues are
// balanced to |x| <= (p-1)/2 and split into L signed base-2^8 digits
// (x = sum_l d_l 2^{8l}), each held exactly in FP16.  One tcgen05.mma
// kind::f16 per digit pair accumulates into FP32 in tensor memory (TMEM);
// products of equal weight 2^{8w} share one accumulator (2L-1 of them).  An
// FP32 accumulator is exact while every partial sum stays within 2^24, so a
// block of at most k_flush = floor(2^24 / max weight-class product) columns of
// K is accumulated before the epilogue warps drain the accumulators:
// t = sum_w c_w 2^{8w} (int64, exact), reduced mod p by one Montgomery step
// and added to a residue kept in the epilogue's registers.  The last drain
// writes C - residue.
//
// Digits: L = 1 or 2 for p up to about 2^17 (classes recombined into one int64
// and reduced once), L = 3 or 4 up to 2^31.  For L >= 3 the tile is 128 x 64
// so that the 2L-1 class accumulators fit in the 512 TMEM columns, and since
// the recombined t may exceed 64 bits it is formed as t_lo + 2^32 t_hi
// (classes 0-3 and 4-6) and each part is reduced on its own.
//
// Structure (one CTA per 128 x TN tile of C, TN = 128, 80, 64, 64 for
// L = 1..4; warp-specialised):
//   warp 0     TMA producer: digit planes of A (128 x 64 FP16, 128B swizzle)
//              and of B^T into a shared-memory ring (6, 4, 3 or 2 stages for L = 1..4);
//   warp 1     TMEM allocation and the single MMA-issuing thread;
//   warps 2-9  epilogue: two warps per TMEM lane quadrant, TN/2 columns each,
//              the running residue in registers.
// For L <= 2 the accumulators are double-buffered: two sets of the 2L-1 class
// accumulators fit in TMEM, so the MMAs of the next K group run while the
// epilogue drains the previous one (L = 3, 4: one set, the MMAs wait).
// The digit planes of both operands are written by one packing launch into
// workspace.  Every mbarrier wait is bounded; on expiry the kernel records
// PLUQ_ERR_TIMEOUT in the error word, drains, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "common.cuh"

namespace {

constexpr int kTM = 128, kTK = 64;  // CTA tile rows, K block (one 128B swizzle row)
constexpr int kLimbBits = 8;
constexpr int kGemmThreads = 320;               // 10 warps
constexpr int kBandTiles = 8;                    // tile rows per rasterization band
constexpr int kTileBytes = kTM * kTK * 2;        // 16 KiB per digit plane tile
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

// ------------------------------------------------------------ PTX helpers --

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false (and the error word set) when the phase never completes.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (clock64() - t0 > kWaitCycles) {
      atomicExch(err, PLUQ_ERR_TIMEOUT);
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 128B swizzle, 8-row groups of
// 1024 B (stride byte offset), descriptor version 1 (tcgen05).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::f16: F32 accumulate, F16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t idesc_f16(int n) {
  return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTM >> 4) << 24);
}

__device__ __forceinline__ void umma_f16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
      "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
      "r"(v[15])
      : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&v)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
               : "r"(taddr));
}

template <int W>
__device__ __forceinline__ void tmem_ldw(uint32_t taddr, uint32_t (&v)[W]) {
  if constexpr (W == 8)
    tmem_ld8(taddr, v);
  else
    tmem_ld4(taddr, v);
}

// ------------------------------------------------------------ the kernel --

// Tile variants of the limb fgemm (chosen per shape by the autotuner):
//   0  128 x TN tile, TN = 128 (L <= 2) or 64 (L >= 3), one set of the 2L-1
//      weight-class accumulators in TMEM: the MMAs wait while the epilogue
//      drains a finished K group;
//   1  as 0 for L = 2, with the two products of the middle weight class in
//      accumulators of their own (4 x 128 TMEM columns): every accumulator
//      holds single digit products, so an exact K group is twice as long for
//      p < 2^16 and the tile is drained half as often;
//   2  two accumulator sets of a narrower tile (TN = 128 for L = 1, 80 for
//      L = 2): the MMAs of the next K group run while the epilogue drains the
//      previous one.
// The residue lives in the epilogue's registers in every variant.
template <int L, int V>
struct LimbCfg {
  static constexpr bool kSplit = V == 1 && L == 2;
  static constexpr bool kDouble = V == 2 && L <= 2;
  static constexpr int TN = L >= 3 ? 64 : (kDouble && L == 2 ? 80 : 128);  // CTA tile width
  static constexpr int kBufs = kDouble ? 2 : 1;                            // accumulator sets
  static constexpr int kAccs = kSplit ? 4 : 2 * L - 1;                     // accumulators a set
  static constexpr int kATile = kTileBytes;               // 128 x 64 FP16
  static constexpr int kBTile = TN * kTK * 2;             // TN x 64 FP16
  static constexpr int kStageBytes = L * (kATile + kBTile);
  static constexpr int kStages = (220 * 1024) / kStageBytes > 6 ? 6 : (220 * 1024) / kStageBytes;
  static constexpr int kAccCols = kAccs * TN;             // one accumulator set
  static constexpr int kEpiCols = TN / 2;                 // columns per epilogue thread
  static constexpr int kChunk = L <= 2 ? 8 : 4;           // columns per TMEM read
  static constexpr int kSmem = kStages * kStageBytes + 1024 + 256;
  static constexpr uint32_t kIdesc = idesc_f16(TN);
  // accumulator of digit product (i, j) and the exponent of its weight 2^{8 w}
  static __host__ __device__ constexpr int acc_of(int i, int j) { return kSplit ? i * 2 + j : i + j; }
  static __host__ __device__ constexpr int weight_of(int a) {
    return kSplit ? (a == 0 ? 0 : (a == 3 ? 2 : 1)) : a;
  }
  static_assert(kBufs * kAccCols <= 512, "accumulators exceed TMEM");
  static_assert(kEpiCols % kChunk == 0, "epilogue reads kChunk columns at a time");
  static_assert(kTM * (TN + 1) * 4 <= kStages * kStageBytes, "staging exceeds the ring");
};

template <int L, int V>
__global__ void __launch_bounds__(kGemmThreads, 1)
    k_fgemm_limb(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 int64_t M, int64_t N, int Mp, int Np, int num_kb, int group_kb,
                 uint32_t* __restrict__ C, int64_t ldc, FieldP F, uint64_t bias,
                 uint64_t bias_hi, int* __restrict__ err, int beta0) {
  using Cfg = LimbCfg<L, V>;
  constexpr int TN = Cfg::TN;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Cfg::kStages * Cfg::kStageBytes);
  uint64_t* full = bars;                      // [kStages]
  uint64_t* empty = bars + Cfg::kStages;      // [kStages]
  uint64_t* acc_full = bars + 2 * Cfg::kStages;   // [2]: a set holds a finished group
  uint64_t* acc_empty = acc_full + 2;             // [2]: the epilogue has read a set
  uint64_t* mma_done = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // grouped rasterization: consecutive CTAs walk down a band of kBandTiles
  // tile rows before moving right, so the CTAs resident at once share a few A
  // and B panels in L2 instead of streaming all of B once per tile row
  const int tiles_n = gridDim.x, tiles_m = gridDim.y;
  const int lin = blockIdx.y * tiles_n + blockIdx.x;
  const int band = lin / (kBandTiles * tiles_n);
  const int first_m = band * kBandTiles;
  const int band_h = min(tiles_m - first_m, kBandTiles);
  const int in_band = lin - band * kBandTiles * tiles_n;
  const int m0 = (first_m + in_band % band_h) * kTM, n0 = (in_band / band_h) * TN;
  const int num_groups = (num_kb + group_kb - 1) / group_kb;

  if (threadIdx.x == 0) {
    for (int s = 0; s < Cfg::kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 8);
    }
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------------------------------------------- TMA producer
      int issued = 0;
      for (int kb = 0; kb < num_kb; ++kb) {
        const int s = kb % Cfg::kStages;
        const uint32_t ph = (kb / Cfg::kStages) & 1;
        if (!mbar_wait(&empty[s], ph ^ 1, err)) {
          *abort_flag = 1;
          break;
        }
        if (*(volatile int*)abort_flag) break;
        mbar_expect_tx(&full[s], Cfg::kStageBytes);
        const uint32_t st = smem_u32(smem + s * Cfg::kStageBytes);
#pragma unroll
        for (int l = 0; l < L; ++l) {
          tma_load_2d(st + l * Cfg::kATile, &tmA, kb * kTK, l * Mp + m0, &full[s]);
          tma_load_2d(st + L * Cfg::kATile + l * Cfg::kBTile, &tmB, kb * kTK, l * Np + n0,
                      &full[s]);
        }
        issued = kb + 1;
      }
      // drain: every issued copy lands before the CTA may exit (a load of
      // k-block kb was only issued once k-block kb - kStages had been consumed)
      for (int kb = (issued > Cfg::kStages ? issued - Cfg::kStages : 0); kb < issued; ++kb)
        mbar_wait(&full[kb % Cfg::kStages], (kb / Cfg::kStages) & 1, err);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------------------------------------------- MMA issuer
      for (int kb = 0; kb < num_kb; ++kb) {
        const int s = kb % Cfg::kStages;
        const int g = kb / group_kb;
        const int buf = g % Cfg::kBufs;
        const bool first = (kb % group_kb) == 0;
        const bool last = (kb % group_kb) == group_kb - 1 || kb == num_kb - 1;
        if (first && g >= Cfg::kBufs) {
          // the set of group g - kBufs must have been read by the epilogue
          if (!mbar_wait(&acc_empty[buf], (g / Cfg::kBufs - 1) & 1, err)) {
            *abort_flag = 1;
            break;
          }
        }
        if (!mbar_wait(&full[s], (kb / Cfg::kStages) & 1, err)) {
          *abort_flag = 1;
          break;
        }
        tc_fence_after();
        const uint32_t st = smem_u32(smem + s * Cfg::kStageBytes);
        const uint32_t acc_base = tmem + (uint32_t)(buf * Cfg::kAccCols);
#pragma unroll
        for (int kk = 0; kk < kTK / 16; ++kk) {
          uint32_t seen = 0;  // classes already written in this k-step
#pragma unroll
          for (int i = 0; i < L; ++i) {
            const uint64_t da = smem_desc_sw128(st + i * Cfg::kATile + kk * 32);
#pragma unroll
            for (int j = 0; j < L; ++j) {
              const uint64_t db = smem_desc_sw128(st + L * Cfg::kATile + j * Cfg::kBTile + kk * 32);
              const int w = Cfg::acc_of(i, j);
              // the first product of each accumulator at the start of a group overwrites
              const uint32_t acc = (first && kk == 0 && !((seen >> w) & 1u)) ? 0u : 1u;
              seen |= 1u << w;
              umma_f16(acc_base + (uint32_t)(w * TN), da, db, Cfg::kIdesc, acc);
            }
          }
        }
        umma_commit(&empty[s]);
        if (last) umma_commit(&acc_full[buf]);
      }
      // every issued MMA completes before TMEM is released
      umma_commit(mma_done);
      mbar_wait(mma_done, 0, err);
    }
  } else {
    // -------------------------------------------------------- epilogue
    // warp e = warp - 2 reads TMEM lane quadrant e % 4 (the quadrant its warp
    // rank may access) and columns [h TN/2, (h+1) TN/2) of the tile
    const int q = warp & 3;
    const int h = (warp - 2) >> 2;
    const int row = q * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
    constexpr int EC = Cfg::kEpiCols;
    uint32_t res[EC];  // sum over drained groups of REDC(t): (sum t) R^{-1} mod p
#pragma unroll
    for (int e = 0; e < EC; ++e) res[e] = 0u;
    bool ok = true;
    for (int g = 0; g < num_groups; ++g) {
      const int buf = g % Cfg::kBufs;
      if (!mbar_wait(&acc_full[buf], (g / Cfg::kBufs) & 1, err)) {
        *abort_flag = 1;
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t set = lane_base + (uint32_t)(buf * Cfg::kAccCols + h * EC);
      constexpr int CW = Cfg::kChunk;
#pragma unroll
      for (int ch = 0; ch < EC / CW; ++ch) {
        uint32_t c[Cfg::kAccs][CW];
#pragma unroll
        for (int w = 0; w < Cfg::kAccs; ++w) tmem_ldw<CW>(set + w * TN + ch * CW, c[w]);
        tmem_wait_ld();
        if (ch == EC / CW - 1) {
          // the whole set is read: hand it back to the MMA issuer before the
          // arithmetic on the last chunk
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&acc_empty[buf]);
        }
#pragma unroll
        for (int e = 0; e < CW; ++e) {
          uint32_t v;
          if (L <= 2) {
            int64_t t = 0;
#pragma unroll
            for (int w = 0; w < Cfg::kAccs; ++w)
              t += (int64_t)__float2int_rn(__uint_as_float(c[w][e])) *
                   (1 << (kLimbBits * Cfg::weight_of(w)));
            v = F.is2 ? (uint32_t)((uint64_t)(t + (int64_t)bias) & 1u)
                      : f_redc((uint64_t)(t + (int64_t)bias), F);
          } else {
            // classes 0..3 and 4.. recombine into two int64 values t_lo and
            // t_hi with t = t_lo + 2^32 t_hi; as R = 2^32,
            // t R^{-1} = t_lo R^{-1} + t_hi = REDC(t_lo) + REDC(REDC(t_hi) R^2).
            int64_t tlo = 0, thi = 0;
#pragma unroll
            for (int w = 0; w < Cfg::kAccs; ++w) {
              const int64_t cw = (int64_t)__float2int_rn(__uint_as_float(c[w][e]));
              if (w < 4)
                tlo += cw * ((int64_t)1 << (kLimbBits * w));
              else
                thi += cw * ((int64_t)1 << (kLimbBits * (w - 4)));
            }
            const uint32_t vlo = f_redc((uint64_t)(tlo + (int64_t)bias), F);
            const uint32_t vhi = f_redc((uint64_t)(thi + (int64_t)bias_hi), F);
            v = f_add(vlo, f_redc((uint64_t)vhi * F.r2, F), F);
          }
          res[ch * CW + e] = f_add(res[ch * CW + e], v, F);
        }
      }
    }
    // the residue holds (sum t) R^{-1}; one more step with R^2 undoes it.
    // Stage the tile in the (now idle) pipeline shared memory so that C is
    // updated with row-contiguous accesses below.
    asm volatile("bar.sync 1, 256;" ::: "memory");  // every warp is past the ring
    if (ok) {
      uint32_t* stage = reinterpret_cast<uint32_t*>(smem) + row * (TN + 1) + h * EC;
#pragma unroll
      for (int e = 0; e < EC; ++e) stage[e] = F.is2 ? res[e] : f_redc((uint64_t)res[e] * F.r2, F);
    }
    // C <- C - residue (C <- -residue when beta0: the product overwrites C,
    // whose old values are never read), one warp per row, 32 consecutive
    // columns per access
    asm volatile("bar.sync 1, 256;" ::: "memory");
    if (*(volatile int*)abort_flag == 0) {
      const int ew = warp - 2;
      const uint32_t* stage = reinterpret_cast<const uint32_t*>(smem);
      for (int rr = ew; rr < kTM; rr += 8) {
        const int64_t gr = (int64_t)m0 + rr;
        if (gr >= M) break;
        uint32_t* crow = C + gr * ldc + n0;
        constexpr int NQ = (TN + 31) / 32;
        uint32_t cv[NQ];
#pragma unroll
        for (int q2 = 0; q2 < NQ; ++q2) {
          const int j = lane + 32 * q2;
          cv[q2] = (!beta0 && j < TN && n0 + j < N) ? crow[j] : 0u;
        }
#pragma unroll
        for (int q2 = 0; q2 < NQ; ++q2) {
          const int j = lane + 32 * q2;
          if (j < TN && n0 + j < N) crow[j] = f_sub(cv[q2], stage[rr * (TN + 1) + j], F);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// Signed base-2^8 digits of a balanced residue x, |x| <= p/2: the low L - 1
// digits in [-2^7, 2^7), the top digit whatever remains, each exact in FP16.
template <int L>
__device__ __forceinline__ void split_digits(int32_t x, __half (&d)[L]) {
#pragma unroll
  for (int l = 0; l < L; ++l) {
    int32_t v;
    if (l == L - 1) {
      v = x;
    } else {
      v = ((x + (1 << (kLimbBits - 1))) & ((1 << kLimbBits) - 1)) - (1 << (kLimbBits - 1));
      x = (x - v) >> kLimbBits;
    }
    d[l] = __int2half_rn(v);
  }
}

__device__ __forceinline__ int32_t balance(uint32_t a, uint32_t p) {
  return a > (p - 1) / 2 ? (int32_t)(a - p) : (int32_t)a;
}

// Digit planes of A (M x K) in K-major layout: out[l][i][k], rows padded to
// Mp and columns to Kp (a multiple of 64) with zeros.  A thread takes 8
// consecutive k of one row and writes 16 bytes per plane; `vec` marks a
// 16-byte aligned A (base and row stride), read as two 16-byte loads.
template <int L>
__device__ __forceinline__ void pack_rows(const uint32_t* __restrict__ A, int64_t lda, int64_t M,
                                          int64_t K, int64_t Mp, int64_t Kp, uint32_t p, bool vec,
                                          __half* __restrict__ out, int64_t item0,
                                          int64_t nitems_step) {
  const int64_t chunks = Kp / 8, total = Mp * chunks;
  for (int64_t it = item0; it < total; it += nitems_step) {
    const int64_t i = it / chunks, k0 = (it - i * chunks) * 8;
    uint32_t a[8];
    if (i < M && vec && k0 + 8 <= K) {
      const uint4* src = reinterpret_cast<const uint4*>(A + i * lda + k0);
      const uint4 u0 = __ldg(src), u1 = __ldg(src + 1);
      a[0] = u0.x; a[1] = u0.y; a[2] = u0.z; a[3] = u0.w;
      a[4] = u1.x; a[5] = u1.y; a[6] = u1.z; a[7] = u1.w;
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) a[q] = (i < M && k0 + q < K) ? __ldg(A + i * lda + k0 + q) : 0u;
    }
    __align__(16) __half h[L][8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      __half d[L];
      split_digits<L>(balance(a[q], p), d);
#pragma unroll
      for (int l = 0; l < L; ++l) h[l][q] = d[l];
    }
#pragma unroll
    for (int l = 0; l < L; ++l)
      *reinterpret_cast<uint4*>(out + (int64_t)l * Mp * Kp + i * Kp + k0) =
          *reinterpret_cast<const uint4*>(h[l]);
  }
}

// Digit planes of B^T: B is K x N row-major; out[l][j][k] (K-major rows of
// B^T), padded to Np x Kp.  A 64 (k) x 64 (j) tile is staged in shared memory
// as balanced residues (16-byte loads along j when B is aligned), then each
// thread writes 8 consecutive k of one j: 16 bytes per plane.
constexpr int kPackT = 64;

template <int L>
__device__ __forceinline__ void pack_cols(const uint32_t* __restrict__ B, int64_t ldb, int64_t K,
                                          int64_t N, int64_t Np, int64_t Kp, uint32_t p, bool vec,
                                          __half* __restrict__ out, int tk, int tj, int tid) {
  __shared__ int32_t tile[kPackT][kPackT + 1];
  const int64_t k0 = (int64_t)tk * kPackT, j0 = (int64_t)tj * kPackT;
  // load: 64 rows x 16 four-element groups; 256 threads, 4 groups each
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int g = tid + q * 256, kk = g >> 4, jj = (g & 15) * 4;
    const int64_t k = k0 + kk, j = j0 + jj;
    uint32_t v[4];
    if (k < K && vec && j + 4 <= N) {
      const uint4 u = __ldg(reinterpret_cast<const uint4*>(B + k * ldb + j));
      v[0] = u.x; v[1] = u.y; v[2] = u.z; v[3] = u.w;
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) v[e] = (k < K && j + e < N) ? __ldg(B + k * ldb + j + e) : 0u;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) tile[kk][jj + e] = balance(v[e], p);
  }
  __syncthreads();
  // store: 64 j x 8 chunks of 8 k; eight consecutive threads write the 128
  // contiguous bytes of one j (per plane)
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int item = tid + 256 * half, jj = item >> 3, kc = (item & 7) * 8;
    const int64_t j = j0 + jj, k = k0 + kc;
    if (j >= Np || k >= Kp) continue;
    __align__(16) __half h[L][8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      __half d[L];
      split_digits<L>(tile[kc + q][jj], d);
#pragma unroll
      for (int l = 0; l < L; ++l) h[l][q] = d[l];
    }
#pragma unroll
    for (int l = 0; l < L; ++l)
      *reinterpret_cast<uint4*>(out + (int64_t)l * Np * Kp + j * Kp + k) =
          *reinterpret_cast<const uint4*>(h[l]);
  }
}

// Both operands' digit planes in one launch: blocks [0, ga) pack A
// (grid-stride over 8-element items), blocks [ga, ga + gbk * gbj) pack one
// 64 x 64 tile of B^T each.
template <int L>
__global__ void __launch_bounds__(256)
    k_pack_both(const uint32_t* __restrict__ A, int64_t lda, int64_t M, int64_t Mp,
                const uint32_t* __restrict__ B, int64_t ldb, int64_t N, int64_t Np, int64_t K,
                int64_t Kp, uint32_t p, __half* __restrict__ outA, __half* __restrict__ outB,
                int ga, int gbk, bool veca, bool vecb) {
  const int b = blockIdx.x;
  if (b < ga) {
    pack_rows<L>(A, lda, M, K, Mp, Kp, p, veca, outA, (int64_t)b * 256 + threadIdx.x,
                 (int64_t)ga * 256);
  } else {
    const int t = b - ga;
    pack_cols<L>(B, ldb, K, N, Np, Kp, p, vecb, outB, t % gbk, t / gbk, threadIdx.x);
  }
}

template <int L>
int launch_pack(cudaStream_t s, const uint32_t* A, int64_t lda, int64_t M, int64_t Mp,
                const uint32_t* B, int64_t ldb, int64_t N, int64_t Np, int64_t K, int64_t Kp,
                uint32_t p, __half* Ap, __half* Bp) {
  // A: about 16 items (8 elements each) per thread, at most 8 CTAs per SM-ish
  const int64_t itemsA = Mp * (Kp / 8);
  const int ga = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(itemsA, 256 * 16), 4096));
  const int64_t gbk = cdiv(Kp, kPackT), gbj = cdiv(Np, kPackT);
  if (ga + gbk * gbj > INT32_MAX) return PLUQ_ERR_INVALID_ARG;
  const bool veca = ((reinterpret_cast<uintptr_t>(A) | (uintptr_t)(lda * 4)) & 15u) == 0;
  const bool vecb = ((reinterpret_cast<uintptr_t>(B) | (uintptr_t)(ldb * 4)) & 15u) == 0;
  k_pack_both<L><<<(unsigned)(ga + gbk * gbj), 256, 0, s>>>(A, lda, M, Mp, B, ldb, N, Np, K, Kp,
                                                            p, Ap, Bp, ga, (int)gbk, veca, vecb);
  PLUQ_CUDA(cudaGetLastError());
  return PLUQ_OK;
}

// ---------------------------------------------------------------------------
// Fused digit split: the same product with the digit split done by the
// producer warps inside the fgemm instead of a separate packing pass.  Four
// converter warps read raw uint32 tiles of A (128 x 64) and B (64 x TN) from
// global memory, balance each residue, split it into its L signed base-2^8
// digits and store the FP16 digit tiles straight into the shared-memory ring in
// the layout the MMA descriptors expect (K-major rows of 128 bytes, 16-byte
// chunks XOR-swizzled by the row index modulo 8, B transposed on the way), then
// publish the stage through a proxy fence and an mbarrier arrival.  Every
// element is converted once per tile that reads it (N/TN times for A, M/128
// for B), against once per call for the packing pass, so this pays where K is
// small and the packing launch and pipeline fill would dominate.
constexpr int kFusedConv = 4;                                // converter warps
constexpr int kFusedThreads = (kFusedConv + 1 + 8) * 32;     // + MMA warp + epilogue

template <int L>
struct FusedCfg {
  static constexpr int TN = L <= 2 ? 128 : 64;
  static constexpr int kAccs = 2 * L - 1;
  static constexpr int kATile = kTileBytes;               // 128 x 64 FP16
  static constexpr int kBTile = TN * kTK * 2;
  static constexpr int kStageBytes = L * (kATile + kBTile);
  static constexpr int kStages = (200 * 1024) / kStageBytes > 4 ? 4 : (200 * 1024) / kStageBytes;
  static constexpr int kSmem = kStages * kStageBytes + 1024 + 256;
  static constexpr uint32_t kIdesc = idesc_f16(TN);
  static constexpr int kEpiCols = TN / 2;
  static constexpr int kChunk = L <= 2 ? 8 : 4;
  static_assert(kAccs * TN <= 512, "accumulators exceed TMEM");
  static_assert(kTM * (TN + 1) * 4 <= kStages * kStageBytes, "staging exceeds the ring");
};

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <int L>
__device__ __forceinline__ uint4 digits_to_u4(const __half (&h)[8]) {
  return *reinterpret_cast<const uint4*>(h);
}

template <int L>
__global__ void __launch_bounds__(kFusedThreads, 1)
    k_fgemm_limb_fused(const uint32_t* __restrict__ A, int64_t lda, const uint32_t* __restrict__ B,
                       int64_t ldb, int64_t M, int64_t N, int64_t K, int num_kb, int group_kb,
                       uint32_t* __restrict__ C, int64_t ldc, FieldP F, uint64_t bias,
                       uint64_t bias_hi, int* __restrict__ err) {
  using Cfg = FusedCfg<L>;
  constexpr int TN = Cfg::TN;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Cfg::kStages * Cfg::kStageBytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + Cfg::kStages;
  uint64_t* acc_full = bars + 2 * Cfg::kStages;
  uint64_t* acc_empty = acc_full + 1;
  uint64_t* mma_done = acc_empty + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_n = gridDim.x, tiles_m = gridDim.y;
  const int lin = blockIdx.y * tiles_n + blockIdx.x;
  const int band = lin / (kBandTiles * tiles_n);
  const int first_m = band * kBandTiles;
  const int band_h = min(tiles_m - first_m, kBandTiles);
  const int in_band = lin - band * kBandTiles * tiles_n;
  const int m0 = (first_m + in_band % band_h) * kTM, n0 = (in_band / band_h) * TN;
  const int num_groups = (num_kb + group_kb - 1) / group_kb;
  constexpr int kMmaWarp = kFusedConv;

  if (threadIdx.x == 0) {
    for (int s = 0; s < Cfg::kStages; ++s) {
      mbar_init(&full[s], kFusedConv);
      mbar_init(&empty[s], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, 8);
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp < kFusedConv) {
    // ------------------------------------------------- converter warps
    const int ct = threadIdx.x;  // 0 .. 127
    const uint32_t p = F.p;
    const bool veca = ((reinterpret_cast<uintptr_t>(A) | (uintptr_t)(lda * 4)) & 15u) == 0;
    for (int kb = 0; kb < num_kb; ++kb) {
      const int s = kb % Cfg::kStages;
      const uint32_t ph = (kb / Cfg::kStages) & 1;
      bool ok = true;
      if (lane == 0) {
        ok = mbar_wait(&empty[s], ph ^ 1, err);
        if (!ok) *abort_flag = 1;
      }
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok || *(volatile int*)abort_flag) break;
      uint8_t* st = smem + s * Cfg::kStageBytes;
      const int64_t k0 = (int64_t)kb * kTK;
      // A: 128 rows x 8 chunks of 8 k; 8 consecutive threads read one row
#pragma unroll 2
      for (int it = ct; it < kTM * 8; it += kFusedConv * 32) {
        const int r = it >> 3, c = it & 7;
        const int64_t gr = m0 + r, gk = k0 + 8 * c;
        uint32_t a[8];
        if (gr < M && veca && gk + 8 <= K) {
          const uint4* src = reinterpret_cast<const uint4*>(A + gr * lda + gk);
          const uint4 u0 = __ldg(src), u1 = __ldg(src + 1);
          a[0] = u0.x; a[1] = u0.y; a[2] = u0.z; a[3] = u0.w;
          a[4] = u1.x; a[5] = u1.y; a[6] = u1.z; a[7] = u1.w;
        } else {
#pragma unroll
          for (int q = 0; q < 8; ++q) a[q] = (gr < M && gk + q < K) ? __ldg(A + gr * lda + gk + q) : 0u;
        }
        __align__(16) __half h[L][8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          __half d[L];
          split_digits<L>(balance(a[q], p), d);
#pragma unroll
          for (int l = 0; l < L; ++l) h[l][q] = d[l];
        }
        const int off = r * 128 + ((c ^ (r & 7)) << 4);
#pragma unroll
        for (int l = 0; l < L; ++l)
          *reinterpret_cast<uint4*>(st + l * Cfg::kATile + off) =
              *reinterpret_cast<const uint4*>(h[l]);
      }
      // B^T: TN rows (columns of B) x 8 chunks; 32 consecutive threads read 32
      // consecutive columns of one row of B at a time
#pragma unroll 2
      for (int it = ct; it < TN * 8; it += kFusedConv * 32) {
        const int n = it % TN, c = it / TN;
        const int64_t gn = n0 + n, gk = k0 + 8 * c;
        uint32_t b[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) b[q] = (gn < N && gk + q < K) ? __ldg(B + (gk + q) * ldb + gn) : 0u;
        __align__(16) __half h[L][8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          __half d[L];
          split_digits<L>(balance(b[q], p), d);
#pragma unroll
          for (int l = 0; l < L; ++l) h[l][q] = d[l];
        }
        const int off = n * 128 + ((c ^ (n & 7)) << 4);
#pragma unroll
        for (int l = 0; l < L; ++l)
          *reinterpret_cast<uint4*>(st + L * Cfg::kATile + l * Cfg::kBTile + off) =
              *reinterpret_cast<const uint4*>(h[l]);
      }
      // the generic-proxy stores become visible to the tensor core's reads
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&full[s]);
    }
  } else if (warp == kMmaWarp) {
    if (lane == 0) {
      // ---------------------------------------------------- MMA issuer
      for (int kb = 0; kb < num_kb; ++kb) {
        const int s = kb % Cfg::kStages;
        const int g = kb / group_kb;
        const bool first = (kb % group_kb) == 0;
        const bool last = (kb % group_kb) == group_kb - 1 || kb == num_kb - 1;
        if (first && g > 0) {
          if (!mbar_wait(acc_empty, (g - 1) & 1, err)) {
            *abort_flag = 1;
            break;
          }
        }
        if (!mbar_wait(&full[s], (kb / Cfg::kStages) & 1, err)) {
          *abort_flag = 1;
          break;
        }
        tc_fence_after();
        const uint32_t st = smem_u32(smem + s * Cfg::kStageBytes);
#pragma unroll
        for (int kk = 0; kk < kTK / 16; ++kk) {
          uint32_t seen = 0;
#pragma unroll
          for (int i = 0; i < L; ++i) {
            const uint64_t da = smem_desc_sw128(st + i * Cfg::kATile + kk * 32);
#pragma unroll
            for (int j = 0; j < L; ++j) {
              const uint64_t db = smem_desc_sw128(st + L * Cfg::kATile + j * Cfg::kBTile + kk * 32);
              const int w = i + j;
              const uint32_t acc = (first && kk == 0 && !((seen >> w) & 1u)) ? 0u : 1u;
              seen |= 1u << w;
              umma_f16(tmem + (uint32_t)(w * TN), da, db, Cfg::kIdesc, acc);
            }
          }
        }
        umma_commit(&empty[s]);
        if (last) umma_commit(acc_full);
      }
      umma_commit(mma_done);
      mbar_wait(mma_done, 0, err);
    }
  } else {
    // -------------------------------------------------------- epilogue
    const int e = warp - kMmaWarp - 1;  // 0 .. 7
    const int q = warp & 3;             // the TMEM lane quadrant this warp may access
    const int h = e >> 2;
    const int row = q * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
    constexpr int EC = Cfg::kEpiCols;
    constexpr int CW = Cfg::kChunk;
    uint32_t res[EC];
#pragma unroll
    for (int i = 0; i < EC; ++i) res[i] = 0u;
    bool ok = true;
    for (int g = 0; g < num_groups; ++g) {
      if (!mbar_wait(acc_full, g & 1, err)) {
        *abort_flag = 1;
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t set = lane_base + (uint32_t)(h * EC);
#pragma unroll
      for (int ch = 0; ch < EC / CW; ++ch) {
        uint32_t c[Cfg::kAccs][CW];
#pragma unroll
        for (int w = 0; w < Cfg::kAccs; ++w) tmem_ldw<CW>(set + w * TN + ch * CW, c[w]);
        tmem_wait_ld();
        if (ch == EC / CW - 1) {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(acc_empty);
        }
#pragma unroll
        for (int i = 0; i < CW; ++i) {
          uint32_t v;
          if (L <= 2) {
            int64_t t = 0;
#pragma unroll
            for (int w = 0; w < Cfg::kAccs; ++w)
              t += (int64_t)__float2int_rn(__uint_as_float(c[w][i])) * (1 << (kLimbBits * w));
            v = F.is2 ? (uint32_t)((uint64_t)(t + (int64_t)bias) & 1u)
                      : f_redc((uint64_t)(t + (int64_t)bias), F);
          } else {
            int64_t tlo = 0, thi = 0;
#pragma unroll
            for (int w = 0; w < Cfg::kAccs; ++w) {
              const int64_t cw = (int64_t)__float2int_rn(__uint_as_float(c[w][i]));
              if (w < 4)
                tlo += cw * ((int64_t)1 << (kLimbBits * w));
              else
                thi += cw * ((int64_t)1 << (kLimbBits * (w - 4)));
            }
            const uint32_t vlo = f_redc((uint64_t)(tlo + (int64_t)bias), F);
            const uint32_t vhi = f_redc((uint64_t)(thi + (int64_t)bias_hi), F);
            v = f_add(vlo, f_redc((uint64_t)vhi * F.r2, F), F);
          }
          res[ch * CW + i] = f_add(res[ch * CW + i], v, F);
        }
      }
    }
    asm volatile("bar.sync 1, 256;" ::: "memory");
    if (ok) {
      uint32_t* stage = reinterpret_cast<uint32_t*>(smem) + row * (TN + 1) + h * EC;
#pragma unroll
      for (int i = 0; i < EC; ++i) stage[i] = F.is2 ? res[i] : f_redc((uint64_t)res[i] * F.r2, F);
    }
    asm volatile("bar.sync 1, 256;" ::: "memory");
    if (*(volatile int*)abort_flag == 0) {
      const uint32_t* stage = reinterpret_cast<const uint32_t*>(smem);
      for (int rr = e; rr < kTM; rr += 8) {
        const int64_t gr = (int64_t)m0 + rr;
        if (gr >= M) break;
        uint32_t* crow = C + gr * ldc + n0;
        constexpr int NQ = (TN + 31) / 32;
        uint32_t cv[NQ];
#pragma unroll
        for (int q2 = 0; q2 < NQ; ++q2) {
          const int j = lane + 32 * q2;
          cv[q2] = (j < TN && n0 + j < N) ? crow[j] : 0u;
        }
#pragma unroll
        for (int q2 = 0; q2 < NQ; ++q2) {
          const int j = lane + 32 * q2;
          if (j < TN && n0 + j < N) crow[j] = f_sub(cv[q2], stage[rr * (TN + 1) + j], F);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// ------------------------------------------------------------ host side --

struct LimbPlan {
  int L = 0;
  int group_kb = 0;  // K blocks of 64 per exact accumulation group
  uint64_t bias = 0;     // multiple of p making the (low) recombined drain value >= 0
  uint64_t bias_hi = 0;  // same for the high part (L >= 3)
  // L = 2 with the middle class split (tile variant 1): its group and bias
  int group_kb_split = 0;
  uint64_t bias_split = 0;
};

// Largest |digit| of each of the L digits over all balanced residues.
void digit_bounds(uint32_t p, int L, int64_t* bound) {
  const int64_t h = p / 2;  // balanced residues lie in [-(p/2), p/2] (p = 2: {-1, 0})
  for (int l = 0; l < L; ++l) bound[l] = 0;
  if (L >= 3) {
    // low digits take every value of [-2^7, 2^7); the top digit of x is
    // floor((x + c) / 2^{8(L-1)}) with c = 2^7 (1 + 2^8 + ... + 2^{8(L-2)}),
    // monotone in x, so its extremes sit at x = +-h
    for (int l = 0; l < L - 1; ++l) bound[l] = (int64_t)1 << (kLimbBits - 1);
    const int64_t base = (int64_t)1 << (kLimbBits * (L - 1));
    const int64_t c = ((int64_t)1 << (kLimbBits - 1)) * ((base - 1) / ((1 << kLimbBits) - 1));
    auto fdiv = [](int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); };
    const int64_t top_hi = fdiv(h + c, base), top_lo = fdiv(-h + c, base);
    bound[L - 1] = std::max(top_hi < 0 ? -top_hi : top_hi, top_lo < 0 ? -top_lo : top_lo);
    return;
  }
  auto digits = [&](int64_t x) {
    for (int l = 0; l < L; ++l) {
      int64_t d;
      if (l == L - 1) {
        d = x;
      } else {
        d = ((x + (1 << (kLimbBits - 1))) & ((1 << kLimbBits) - 1)) - (1 << (kLimbBits - 1));
        x = (x - d) >> kLimbBits;
      }
      const int64_t a = d < 0 ? -d : d;
      if (a > bound[l]) bound[l] = a;
    }
  };
  // low digits never exceed 2^(s-1); the top digit is monotone in x, so its
  // extremes sit at x = +-h (checked with a window for the rounding carry)
  const int64_t span = L == 1 ? 0 : (int64_t)1 << (kLimbBits * (L - 1));
  for (int64_t x = h - span; x <= h; ++x)
    if (x >= -h) digits(x);
  for (int64_t x = -h; x <= -h + span; ++x)
    if (x <= h) digits(x);
}

LimbPlan plan_for(uint32_t p) {
  LimbPlan pl;
  const long double lim = (long double)p * 4294967296.0L;  // REDC input bound p R
  for (int L = 1; L <= 4; ++L) {
    int64_t b[4] = {0, 0, 0, 0};
    digit_bounds(p, L, b);
    // weight-class bounds: class w collects digit pairs (i, w - i)
    int64_t cls[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int i = 0; i < L; ++i)
      for (int j = 0; j < L; ++j) cls[i + j] += b[i] * b[j];
    int64_t worst = 1;
    for (int w = 0; w < 2 * L - 1; ++w) worst = cls[w] > worst ? cls[w] : worst;
    const int64_t kmax = ((int64_t)1 << 24) / worst;
    const int64_t gkb = kmax / kTK;
    const int64_t need = L == 1 ? 4 : 1;  // L = 1 only when it needs few drains
    if (gkb < need) continue;
    const int64_t kflush = gkb * kTK;
    // largest |t| per drain: t = sum_w kflush cls[w] 2^{8w} (L <= 2); for
    // L >= 3 the same sum split at w = 4 into t_lo and t_hi
    long double tmax = 0, tmax_hi = 0;
    for (int w = 0; w < 2 * L - 1; ++w) {
      if (L >= 3 && w >= 4)
        tmax_hi += (long double)kflush * cls[w] * powl(2.0L, 8 * (w - 4));
      else
        tmax += (long double)kflush * cls[w] * powl(2.0L, 8 * w);
    }
    if (p != 2 && (2 * tmax + p >= lim || 2 * tmax_hi + p >= lim)) continue;
    pl.L = L;
    pl.group_kb = (int)(gkb > 1 << 20 ? 1 << 20 : gkb);
    const uint64_t tm = (uint64_t)tmax + 1, tmh = (uint64_t)tmax_hi + 1;
    pl.bias = p == 2 ? 0 : (tm + p - 1) / p * p;
    pl.bias_hi = p == 2 ? 0 : (tmh + p - 1) / p * p;
    pl.group_kb_split = pl.group_kb;
    pl.bias_split = pl.bias;
    if (L == 2) {
      // each accumulator holds one digit product: bound b_i b_j instead of the
      // class sum; the drained t has the same form, so only its size changes
      int64_t worst1 = 1;
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) worst1 = std::max(worst1, b[i] * b[j]);
      const int64_t g1 = std::min<int64_t>((((int64_t)1 << 24) / worst1) / kTK, 1 << 20);
      long double t1 = 0;
      for (int w = 0; w < 3; ++w) t1 += (long double)(g1 * kTK) * cls[w] * powl(2.0L, 8 * w);
      if (g1 >= 1 && (p == 2 || 2 * t1 + p < lim)) {
        pl.group_kb_split = (int)g1;
        const uint64_t t1m = (uint64_t)t1 + 1;
        pl.bias_split = p == 2 ? 0 : (t1m + p - 1) / p * p;
      }
    }
    return pl;
  }
  return pl;
}

using EncodeTiled = PFN_cuTensorMapEncodeTiled_v12000;

EncodeTiled lookup_encode() {
  void* ptr = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                       &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    return reinterpret_cast<EncodeTiled>(ptr);
  return nullptr;
}

EncodeTiled get_encode() {
  static const EncodeTiled fn = lookup_encode();  // thread-safe one-time lookup
  return fn;
}

int make_map(CUtensorMap* map, const __half* base, int64_t rows, int64_t kp, int box_rows) {
  EncodeTiled enc = get_encode();
  if (!enc) return PLUQ_ERR_CUDA;
  cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kp * 2};
  cuuint32_t box[2] = {(cuuint32_t)kTK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, (void*)base, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? PLUQ_OK : PLUQ_ERR_CUDA;
}

template <int L, int V>
int run_limb(pluq_ctx* c, const LimbPlan& pl, int64_t M, int64_t N, int64_t K, const uint32_t* A,
             int64_t lda, const uint32_t* B, int64_t ldb, uint32_t* C, int64_t ldc) {
  using Cfg = LimbCfg<L, V>;
  static const cudaError_t attr = cudaFuncSetAttribute(
      k_fgemm_limb<L, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::kSmem);
  PLUQ_CUDA(attr);
  constexpr int TN = Cfg::TN;
  const int64_t Mp = cdiv(M, kTM) * kTM, Np = cdiv(N, TN) * TN, Kp = cdiv(K, kTK) * kTK;
  if (L * Mp > INT32_MAX || L * Np > INT32_MAX || Kp > INT32_MAX) return PLUQ_ERR_INVALID_ARG;
  const size_t abytes = sizeof(__half) * L * Mp * Kp, bbytes = sizeof(__half) * L * Np * Kp;
  PLUQ_TRY(c->pack.ensure(abytes + bbytes + 1024));
  __half* Ap = c->pack.as<__half>();
  __half* Bp = reinterpret_cast<__half*>(reinterpret_cast<char*>(Ap) + ((abytes + 1023) / 1024) * 1024);
  {
    ProfScope ps(c, PC_PACK, 0, 4.0 * (M * K + K * N) + (double)abytes + (double)bbytes, 1);
    PLUQ_TRY(launch_pack<L>(c->stream, A, lda, M, Mp, B, ldb, N, Np, K, Kp, c->F.p, Ap, Bp));
  }
  CUtensorMap ma, mb;
  PLUQ_TRY(make_map(&ma, Ap, L * Mp, Kp, kTM));
  PLUQ_TRY(make_map(&mb, Bp, L * Np, Kp, TN));
  const dim3 grid((unsigned)(Np / TN), (unsigned)(Mp / kTM));
  if (grid.y > 65535) return PLUQ_ERR_INVALID_ARG;
  int* err = c->small.as<int>() + 16;
  ProfScope ps(c, PC_FGEMM, 2.0 * M * N * K,
               (double)abytes + (double)bbytes + 8.0 * M * N, 1,
               2.0 * Mp * Np * Kp * L * L);
  k_fgemm_limb<L, V><<<grid, kGemmThreads, Cfg::kSmem, c->stream>>>(
      ma, mb, M, N, (int)Mp, (int)Np, (int)(Kp / kTK),
      Cfg::kSplit ? pl.group_kb_split : pl.group_kb, C, ldc, c->F,
      Cfg::kSplit ? pl.bias_split : pl.bias, pl.bias_hi, err, c->fgemm_beta0 ? 1 : 0);
  PLUQ_CUDA(cudaGetLastError());
  return PLUQ_OK;
}

template <int L>
int run_limb_fused(pluq_ctx* c, const LimbPlan& pl, int64_t M, int64_t N, int64_t K,
                   const uint32_t* A, int64_t lda, const uint32_t* B, int64_t ldb, uint32_t* C,
                   int64_t ldc) {
  using Cfg = FusedCfg<L>;
  static const cudaError_t attr = cudaFuncSetAttribute(
      k_fgemm_limb_fused<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::kSmem);
  PLUQ_CUDA(attr);
  constexpr int TN = Cfg::TN;
  const int64_t Mt = cdiv(M, kTM), Nt = cdiv(N, TN), Kp = cdiv(K, kTK) * kTK;
  if (Mt > 65535 || Nt > INT32_MAX || Kp > INT32_MAX) return PLUQ_ERR_INVALID_ARG;
  const dim3 grid((unsigned)Nt, (unsigned)Mt);
  int* err = c->small.as<int>() + 16;
  ProfScope ps(c, PC_FGEMM, 2.0 * M * N * K, 4.0 * (M * K + K * N) + 8.0 * M * N, 1,
               2.0 * Mt * kTM * Nt * TN * Kp * L * L);
  k_fgemm_limb_fused<L><<<grid, kFusedThreads, Cfg::kSmem, c->stream>>>(
      A, lda, B, ldb, M, N, K, (int)(Kp / kTK), pl.group_kb, C, ldc, c->F, pl.bias, pl.bias_hi,
      err);
  PLUQ_CUDA(cudaGetLastError());
  return PLUQ_OK;
}

}  // namespace

int limb_form_supported(uint32_t p) { return plan_for(p).L > 0; }

int fgemm_sub_limb(pluq_ctx* c, int64_t M, int64_t N, int64_t K, const uint32_t* A, int64_t lda,
                   const uint32_t* B, int64_t ldb, uint32_t* C, int64_t ldc) {
  if (M <= 0 || N <= 0 || K <= 0) return PLUQ_OK;
  // the plan depends on p only; cached in the context (L, groups, biases)
  if (c->limb_plan_p != c->F.p) {
    const LimbPlan pl = plan_for(c->F.p);
    c->limb_plan[0] = (uint64_t)pl.L;
    c->limb_plan[1] = (uint64_t)pl.group_kb;
    c->limb_plan[2] = pl.bias;
    c->limb_plan[3] = pl.bias_hi;
    c->limb_plan[4] = (uint64_t)pl.group_kb_split;
    c->limb_plan[5] = pl.bias_split;
    c->limb_plan_p = c->F.p;
  }
  LimbPlan cached;
  cached.L = (int)c->limb_plan[0];
  cached.group_kb = (int)c->limb_plan[1];
  cached.bias = c->limb_plan[2];
  cached.bias_hi = c->limb_plan[3];
  cached.group_kb_split = (int)c->limb_plan[4];
  cached.bias_split = c->limb_plan[5];
  // a short inner dimension: the producer warps split the digits themselves
  // (no packing launch, one pass over the operands per tile)
  if (K <= c->fused_kmax && !c->fgemm_beta0) {
    if (cached.L == 1) return run_limb_fused<1>(c, cached, M, N, K, A, lda, B, ldb, C, ldc);
    if (cached.L == 2) return run_limb_fused<2>(c, cached, M, N, K, A, lda, B, ldb, C, ldc);
    if (cached.L == 3) return run_limb_fused<3>(c, cached, M, N, K, A, lda, B, ldb, C, ldc);
    if (cached.L == 4) return run_limb_fused<4>(c, cached, M, N, K, A, lda, B, ldb, C, ldc);
  }
  const int v = c->limb_variant;
  if (cached.L == 1)
    return v == 2 ? run_limb<1, 2>(c, cached, M, N, K, A, lda, B, ldb, C, ldc)
                  : run_limb<1, 0>(c, cached, M, N, K, A, lda, B, ldb, C, ldc);
  if (cached.L == 2) {
    if (v == 1) return run_limb<2, 1>(c, cached, M, N, K, A, lda, B, ldb, C, ldc);
    if (v == 2) return run_limb<2, 2>(c, cached, M, N, K, A, lda, B, ldb, C, ldc);
    return run_limb<2, 0>(c, cached, M, N, K, A, lda, B, ldb, C, ldc);
  }
  if (cached.L == 3) return run_limb<3, 0>(c, cached, M, N, K, A, lda, B, ldb, C, ldc);
  if (cached.L == 4) return run_limb<4, 0>(c, cached, M, N, K, A, lda, B, ldb, C, ldc);
  return PLUQ_ERR_UNSUPPORTED_FORM;
}

// ---------------------------------------------------------------------------
// fgemm_modp_noalloc: the limb fgemm without any device allocation.
//
// Some callers cannot call cudaMalloc: code running while another component
// owns the device memory through its own pool, latency-critical paths that
// must not hit the implicit device synchronisation of an allocation, or
// embedded hosts with a fixed memory budget.  This entry point serves them:
// the digit planes that fgemm_modp keeps in context workspace live instead in
// a file-scope __device__ array of kNoAllocScratchBytes (32 MiB) that every
// GPU loading the library holds until the process exits.
//
// The host refers to that array only through its device address, obtained
// once per device with cudaGetSymbolAddress while that device is current;
// the first call on a device performs this set-up, so make it before any
// stream capture.  Every call reuses the same array (the previous contents
// remain; the packing pass rewrites every byte the kernel reads and the
// error word is cleared on the call's stream), so calls that overlap on the
// GPU - concurrent streams, or several host threads - race on it.  The call
// reads the kernel's error word back (into a host variable on its own stack,
// no allocation) and so returns once the product is complete.
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
__device__ int g_noalloc_err;

struct NoAllocDevice {
  bool ready = false;
  unsigned char* scratch = nullptr;
  int* err = nullptr;
};
constexpr int kNoAllocMaxDevices = 64;
NoAllocDevice g_noalloc_dev[kNoAllocMaxDevices];
std::mutex g_noalloc_mutex;

int noalloc_setup(int dev, NoAllocDevice** out) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) return PLUQ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  NoAllocDevice& d = g_noalloc_dev[dev];
  if (!d.ready) {
    void* s = nullptr;
    void* e = nullptr;
    if (cudaGetSymbolAddress(&s, g_noalloc_scratch) != cudaSuccess ||
        cudaGetSymbolAddress(&e, g_noalloc_err) != cudaSuccess) {
      cudaGetLastError();
      return PLUQ_ERR_CUDA;
    }
    PLUQ_CUDA(cudaFuncSetAttribute(k_fgemm_limb<1, 0>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   LimbCfg<1, 0>::kSmem));
    PLUQ_CUDA(cudaFuncSetAttribute(k_fgemm_limb<2, 0>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   LimbCfg<2, 0>::kSmem));
    PLUQ_CUDA(cudaFuncSetAttribute(k_fgemm_limb<3, 0>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   LimbCfg<3, 0>::kSmem));
    PLUQ_CUDA(cudaFuncSetAttribute(k_fgemm_limb<4, 0>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   LimbCfg<4, 0>::kSmem));
    d.scratch = static_cast<unsigned char*>(s);
    d.err = static_cast<int*>(e);
    d.ready = true;
  }
  *out = &d;
  return PLUQ_OK;
}

template <int L>
int noalloc_run(const NoAllocDevice& d, const LimbPlan& pl, const FieldP& F, int64_t M, int64_t N,
                int64_t K, const uint32_t* A, int64_t lda, const uint32_t* B, int64_t ldb,
                uint32_t* C, int64_t ldc, cudaStream_t s) {
  using Cfg = LimbCfg<L, 0>;
  constexpr int TN = Cfg::TN;
  // each dimension alone is checked against the array before any product of
  // them is formed, so the byte counts below cannot wrap
  const int64_t cap = (int64_t)(kNoAllocScratchBytes / sizeof(__half));
  if (M > cap || N > cap || K > cap) return PLUQ_ERR_TOO_LARGE;
  const int64_t Mp = cdiv(M, kTM) * kTM, Np = cdiv(N, TN) * TN, Kp = cdiv(K, kTK) * kTK;
  if (L * Mp > cap || L * Np > cap || Kp > cap) return PLUQ_ERR_TOO_LARGE;
  if ((L * Mp + L * Np) > cap / Kp) return PLUQ_ERR_TOO_LARGE;
  const size_t abytes = sizeof(__half) * L * Mp * Kp, bbytes = sizeof(__half) * L * Np * Kp;
  const size_t aoff = ((abytes + 1023) / 1024) * 1024;
  if (aoff + bbytes > kNoAllocScratchBytes) return PLUQ_ERR_TOO_LARGE;
  if (Mp / kTM > 65535) return PLUQ_ERR_TOO_LARGE;
  __half* Ap = reinterpret_cast<__half*>(d.scratch);
  __half* Bp = reinterpret_cast<__half*>(d.scratch + aoff);
  PLUQ_CUDA(cudaMemsetAsync(d.err, 0, sizeof(int), s));
  PLUQ_TRY(launch_pack<L>(s, A, lda, M, Mp, B, ldb, N, Np, K, Kp, F.p, Ap, Bp));
  CUtensorMap ma, mb;
  PLUQ_TRY(make_map(&ma, Ap, L * Mp, Kp, kTM));
  PLUQ_TRY(make_map(&mb, Bp, L * Np, Kp, TN));
  const dim3 grid((unsigned)(Np / TN), (unsigned)(Mp / kTM));
  k_fgemm_limb<L, 0><<<grid, kGemmThreads, Cfg::kSmem, s>>>(ma, mb, M, N, (int)Mp, (int)Np,
                                                         (int)(Kp / kTK), pl.group_kb, C, ldc, F,
                                                         pl.bias, pl.bias_hi, d.err, 0);
  PLUQ_CUDA(cudaGetLastError());
  // the kernel's error word (a bounded wait that ran out leaves C as it was)
  // comes back to the host: the call returns once the product is done
  int err = 0;
  PLUQ_CUDA(cudaMemcpyAsync(&err, d.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  PLUQ_CUDA(cudaStreamSynchronize(s));
  return err != 0 ? err : PLUQ_OK;
}

}  // namespace

extern "C" int fgemm_modp_noalloc(uint32_t p, int64_t M, int64_t N, int64_t K, const uint32_t* A,
                                  int64_t lda, const uint32_t* B, int64_t ldb, uint32_t* C,
                                  int64_t ldc, void* stream) {
  if (M < 0 || N < 0 || K < 0) return PLUQ_ERR_INVALID_ARG;
  if (M == 0 || N == 0 || K == 0) return PLUQ_OK;
  if (!A || !B || !C || lda < K || ldb < N || ldc < N) return PLUQ_ERR_INVALID_ARG;
  PLUQ_TRY(check_prime_range(p));
  const LimbPlan pl = plan_for(p);
  if (pl.L == 0) return PLUQ_ERR_UNSUPPORTED_FORM;
  int dev = 0;
  PLUQ_CUDA(cudaGetDevice(&dev));
  NoAllocDevice* d = nullptr;
  PLUQ_TRY(noalloc_setup(dev, &d));
  const FieldP F = make_field(p);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (pl.L == 1) return noalloc_run<1>(*d, pl, F, M, N, K, A, lda, B, ldb, C, ldc, s);
  if (pl.L == 2) return noalloc_run<2>(*d, pl, F, M, N, K, A, lda, B, ldb, C, ldc, s);
  if (pl.L == 3) return noalloc_run<3>(*d, pl, F, M, N, K, A, lda, B, ldb, C, ldc, s);
  return noalloc_run<4>(*d, pl, F, M, N, K, A, lda, B, ldb, C, ldc, s);
}
