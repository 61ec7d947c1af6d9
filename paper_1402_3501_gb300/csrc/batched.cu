// Batched PLUQ: many independent matrices (each at most kBatchMax x kBatchMax)
// factored by one persistent launch.
//
// CTAs take matrices from an atomic work counter in an order the host sorts by
// decreasing work (m n min(m, n)), so the longest factorizations start first.
// One CTA factors one matrix with the rank-profile-revealing pivoting of
// Sec. 4.1: the next pivot is the row-major first non-zero of the Schur
// complement, so the rows are taken in order and each row, once reduced by all
// earlier pivots, is either zero or gives a pivot at its first non-zero column.
//
// The elimination is the tiled iterative scheme of Sec. 4.1 with one column
// tile, its row slabs cut by pivot count rather than by row count, so that every
// update of the rows below carries many pivots.  A slab collects pivots in a
// shared-memory buffer of kSlab rows (16, 24 or 32: the template parameter that
// trades pivots an update against CTAs an SM) -- pivot rows at the top,
// candidate rows below -- in rounds:
//   1. the next rows of the matrix fill the free buffer rows (the pivot columns
//      of earlier slabs zeroed);
//   2. they are reduced by the slab's pivots so far: multipliers by forward
//      substitution on the pivot columns, then rows -= L U with the products of
//      every entry summed in 64 bits and reduced once (delayed reduction,
//      Sec. 3.1);
//   3. they are eliminated among themselves in row order (pivot search, rank-1
//      updates of the rows below the pivot row, a warp a row);
//   4. the rows that gave no pivot are final and go back to the matrix; the new
//      pivot rows move up.
// The slab closes once fewer than kSlab / 4 buffer rows are free (or the matrix
// ends): its pivot rows go back to the matrix and the rows below are reduced by
// its pivots at once.  For p < 2^16 on the tensor cores (trailing_mma, with
// W = U_JJ^{-1} U formed once a slab, so the multipliers come out of the same
// products); otherwise L from a forward substitution per row, then C <- C - L U
// in 64 x 64 tiles of 4 x 4 register micro-tiles on the CUDA cores.  One factor
// of every product is kept in Montgomery form (x R mod p, R = 2^32), so the
// reduction of a sum of products is one REDC.  L multipliers overwrite the
// pivot column entries.  For p < 2^16 the buffer holds 16-bit residues.
//
// The final P^T A Q^T layout is written in place: the multipliers of the
// non-pivot rows are first copied to the CTA's scratch, the pivot rows are then
// moved up eight at a time through shared memory (a pivot row never moves down),
// and the non-pivot rows are written from the scratch.  Entries >= p mark the
// matrix with PLUQ_ERR_ENTRY_OUT_OF_RANGE and leave it untouched.
#include <algorithm>
#include <climits>
#include <numeric>
#include <type_traits>
#include <vector>

#include "common.cuh"

namespace {

constexpr int kBatchThreads = 256;
constexpr int kBatchWarps = kBatchThreads / 32;
constexpr int kBatchMax = 1024;
constexpr int kRowBlock = 128;  // rows below the slab whose multipliers are formed together
constexpr int kTile = 64;       // C tile of the update below the slab, 4 x 4 per thread
constexpr int kLd = 256;        // buffer rows hold a multiple of this many columns ...
constexpr int kPadS = 4;        // ... plus this many words, so that rows 2t and 2t + 1 (t < 4)
                                // of a column fall in distinct banks
constexpr int kLdL = kRowBlock + 4;  // row stride of the multipliers of a row block, likewise
constexpr int kLdE = 36;             // row stride of U_JJ^{-1}, likewise
constexpr int kLoadBatch = 8;   // global loads a lane keeps in flight
constexpr int kRowUnroll = 8;   // 32-column chunks of a row a warp updates together

struct BatchDesc {
  uint32_t* A;
  int32_t* P;
  int32_t* Q;
  int64_t lda;
  int32_t m, n;
};

// Field arithmetic specialised by the size of p:
//   0: p = 2 (bits);
//   1: p < 2^27 (32 products of residues sum to less than p 2^32: one REDC);
//   2: otherwise (a REDC per product);
//   3: p < 2^16: as 1, and the update of the rows below runs on the tensor
//      cores (residues split into two 8-bit digits, exact in FP16; see
//      trailing_mma).
__host__ __device__ constexpr bool one_redc(int mode) { return mode == 1 || mode == 3; }
template <int kMode>
struct BField {
  __device__ __forceinline__ static uint32_t mulm(uint32_t cm, uint32_t w, const FieldP& F) {
    if (kMode == 0) return cm & w;
    return f_redc((uint64_t)cm * w, F);
  }
  __device__ __forceinline__ static uint32_t to_mont(uint32_t v, const FieldP& F) {
    if (kMode == 0) return v & 1u;
    return f_redc((uint64_t)v * F.r2, F);
  }
  __device__ __forceinline__ static uint32_t from_mont(uint32_t v, const FieldP& F) {
    if (kMode == 0) return v;
    return f_redc((uint64_t)v, F);
  }
};

// REDC(t) for t < 2^32: t + m p vanishes mod 2^32 (m = -t p^{-1} mod 2^32), so
// (t + m p) / 2^32 is the high word of m p plus the carry out of the low
// words, which is 1 exactly when t != 0; the result is at most p.
__device__ __forceinline__ uint32_t f_redc32(uint32_t t, const FieldP& F) {
  const uint32_t u = __umulhi(t * F.pneg_inv, F.p) + (t != 0u ? 1u : 0u);
  return u >= F.p ? u - F.p : u;
}

// sum of Montgomery a times plain b over a dot product, as a plain residue
template <int kMode>
struct Dot {
  uint64_t acc = 0;
  uint32_t red = 0;
  __device__ __forceinline__ void add(uint32_t am, uint32_t b, const FieldP& F) {
    if (kMode == 0) {
      red ^= am & b;
    } else if (one_redc(kMode)) {
      acc += (uint64_t)am * b;
    } else {
      red = f_add(red, f_redc((uint64_t)am * b, F), F);
    }
  }
  __device__ __forceinline__ uint32_t value(const FieldP& F) const {
    if (kMode == 0) return red & 1u;
    if (one_redc(kMode)) return f_redc(acc, F);
    return red;
  }
  __device__ __forceinline__ void merge(const Dot& o, const FieldP& F) {
    if (kMode == 0) red ^= o.red;
    else if (one_redc(kMode)) acc += o.acc;
    else red = f_add(red, o.red, F);
  }
};

// sum_{q < k} a[q lda] b[q ldb] (a Montgomery, b plain) as a plain residue, in
// four independent partial sums (k <= 32: the merged sum stays below p 2^32
// in mode 1)
template <int kMode, typename TB>
__device__ __forceinline__ uint32_t dot_prefix(const uint32_t* a, int lda, const TB* b,
                                               size_t ldb, int k, const FieldP& F) {
  Dot<kMode> s0, s1, s2, s3;
  int q = 0;
  for (; q + 4 <= k; q += 4) {
    s0.add(a[q * lda], b[q * ldb], F);
    s1.add(a[(q + 1) * lda], b[(q + 1) * ldb], F);
    s2.add(a[(q + 2) * lda], b[(q + 2) * ldb], F);
    s3.add(a[(q + 3) * lda], b[(q + 3) * ldb], F);
  }
  for (; q < k; ++q) s0.add(a[q * lda], b[q * ldb], F);
  s0.merge(s1, F);
  s2.merge(s3, F);
  s0.merge(s2, F);
  return s0.value(F);
}

__device__ __forceinline__ int bt_block_or(int v, int* red) {
  v = __any_sync(0xffffffffu, v != 0) ? 1 : 0;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  int out = 0;
  for (int w = 0; w < kBatchWarps; ++w) out |= red[w];
  return out;
}

// out[base + k] = k-th index i < cnt with !flag[i] (ascending), block-wide.
__device__ void bt_compact(const int32_t* flag, int cnt, int32_t* out, int base, int* red) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int per = (cnt + kBatchThreads - 1) / kBatchThreads;
  const int i0 = tid * per, i1 = min(cnt, i0 + per);
  int mine = 0;
  for (int i = i0; i < i1; ++i) mine += flag[i] ? 0 : 1;
  int incl = mine;
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  __syncthreads();
  if (lane == 31) red[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int v = lane < kBatchWarps ? red[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    if (lane < kBatchWarps) red[lane] = v;
  }
  __syncthreads();
  int pos = base + incl - mine + (warp > 0 ? red[warp - 1] : 0);
  for (int i = i0; i < i1; ++i)
    if (!flag[i]) out[pos++] = i;
  __syncthreads();
}

// n words of row src (global) into dst (shared), zero where drop(j), zero
// from n to ld; kLoadBatch loads of a lane in flight.  One warp.
template <typename T, typename Drop>
__device__ __forceinline__ void bt_load_row(T* dst, const uint32_t* src, int n, int ld, Drop drop) {
  const int lane = threadIdx.x & 31;
  for (int jb0 = 0; jb0 < ld; jb0 += 32 * kLoadBatch) {
    uint32_t v[kLoadBatch];
#pragma unroll
    for (int q = 0; q < kLoadBatch; ++q) {
      const int j = jb0 + 32 * q + lane;
      v[q] = (j < n && !drop(j)) ? src[j] : 0u;
    }
#pragma unroll
    for (int q = 0; q < kLoadBatch; ++q) {
      const int j = jb0 + 32 * q + lane;
      if (j < ld) dst[j] = (T)v[q];
    }
  }
}

// Two 8-bit digits (v0 >> shift, v1 >> shift, low bytes) as an FP16 pair, exact:
// 0x6400 | d is 1024 + d in FP16, and 1024 is subtracted.
__device__ __forceinline__ uint32_t digit_pair(uint32_t v0, uint32_t v1, int shift) {
  const uint32_t w = ((v0 >> shift) & 0xFFu) | (((v1 >> shift) & 0xFFu) << 16) | 0x64006400u;
  uint32_t out;
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(out) : "r"(w), "r"(0x64006400u));
  return out;
}

__device__ __forceinline__ uint32_t hadd2(uint32_t a, uint32_t b) {
  uint32_t out;
  asm("add.rn.f16x2 %0, %1, %2;" : "=r"(out) : "r"(a), "r"(b));
  return out;
}

// c += a b on a 16 x 8 x 16 tile (legacy warp-level tensor-core product; FP16
// in, FP32 accumulate)
__device__ __forceinline__ void mma16816(float* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// an FP32 holding an integer in [0, 2^23), as that integer
__device__ __forceinline__ uint32_t f2u_exact(float x) {
  return __float_as_uint(x + 8388608.0f) & 0x7FFFFFu;
}

// Buffer storage: 16-bit residues for p < 2^16 (mode 3), else 32-bit.
template <int kMode>
using SlabT = std::conditional_t<kMode == 3, uint16_t, uint32_t>;

// CTAs an SM the register budget is set for.
__host__ __device__ constexpr int slab_min_blocks(int slab, bool narrow) {
  return (slab >= 32 && !narrow) ? 2 : 3;
}

// Shared memory of one CTA, in bytes, for buffer rows of ldN columns of TS.
template <int kSlab, typename TS>
__host__ __device__ constexpr size_t slab_smem_bytes_for(int ldN) {
  return sizeof(TS) * ((size_t)kSlab * (ldN + kPadS)  // S: pivot rows, then candidate rows
                       + (size_t)kSlab * kLdE)        // Uinv: U_JJ^{-1} of the tensor-core update
         + 4 * ((size_t)kSlab * kLdL                  // LT: multipliers (or entries) of a row block
                + (size_t)kSlab * kSlab               // Ls: multipliers of the buffer rows (plain)
                + 6 * kSlab                           // spr, spc, invm, first, srow, pslot
                + (size_t)ldN                         // ispiv
                + (size_t)kBatchMax                   // prow, pcol (16-bit)
                + kBatchWarps + 8);                   // red, misc
}


// A block of nr <= kRowBlock rows below a slab, for p < 2^16, on the tensor
// cores: with X the rows' entries at the slab's P <= 32 pivot columns (plain,
// pivot-major in XT), W = U_JJ^{-1} U (P x n, Montgomery form, in S) and
// U_JJ^{-1} (P x P, Montgomery form, Uinv),
//   C <- C - X W    at the other columns,
//   L  = X U_JJ^{-1} at the pivot columns (the multipliers),
// i.e. C <- C - L U.  Every residue is split into two 8-bit digits,
// x = x1 2^8 + x0, exact in FP16; per 16-deep step three products are
// accumulated in FP32: X0 W0, X1 W1 and (X0 + X1)(W0 + W1) (digit sums <= 510),
// each a sum of at most 32 products below 2^18, so below 2^23 and exact.  The
// middle term is K - X0W0 - X1W1 and the dot product
// x = X1W1 2^16 + mid 2^8 + X0W0 < 32 p^2 is reduced by one REDC (W carries R).
// Warp w takes rows 16w..16w+15 of the block (its A fragments stay in
// registers) and sweeps the columns 16 at a time, then the P columns of
// U_JJ^{-1}.
template <int kMode, typename TS>
__device__ __forceinline__ void trailing_mma(uint32_t* C, int64_t ldc, int nr, int n, int P,
                                             const int32_t* spc, const uint32_t* XT, const TS* S,
                                             int ldS, const TS* Uinv, const int32_t* ispiv, int r,
                                             const FieldP& F) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int m0 = warp * 16;
  if (m0 >= nr) return;
  // A fragments: a[q] holds rows m0 + g (+8 for odd q), depth 2t, 2t + 1 (+8 for q >= 2)
  uint32_t alo[2][4], ahi[2][4];
#pragma unroll
  for (int ks = 0; ks < 2; ++ks)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int row = m0 + g + ((q & 1) ? 8 : 0);
      const int k0 = 16 * ks + 2 * t + ((q & 2) ? 8 : 0);
      const uint32_t v0 = k0 < P ? XT[k0 * kLdL + row] : 0u;
      const uint32_t v1 = k0 + 1 < P ? XT[(k0 + 1) * kLdL + row] : 0u;
      alo[ks][q] = digit_pair(v0, v1, 0);
      ahi[ks][q] = digit_pair(v0, v1, 8);
    }
  const bool two = P > 16;
  const int ntiles = (n + 15) / 16, etiles = (P + 15) / 16;
  for (int tile = 0; tile < ntiles + etiles; ++tile) {
    const bool ext = tile >= ntiles;
    const int c0 = ext ? 16 * (tile - ntiles) : 16 * tile;
    // C entries of this lane: rows m0 + g (+8), columns c0 + 8 nt + 2t (+1)
    uint32_t cv[2][4];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int row = m0 + g + (i >= 2 ? 8 : 0), col = c0 + 8 * nt + 2 * t + (i & 1);
        cv[nt][i] = (!ext && row < nr && col < n) ? C[(int64_t)row * ldc + col] : 0u;
      }
    float acc[2][3][4];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[nt][d][i] = 0.0f;
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      if (ks == 1 && !two) break;
      uint32_t asum[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) asum[q] = hadd2(alo[ks][q], ahi[ks][q]);
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        const int col = c0 + 8 * nt + g;
        const int k0 = 16 * ks + 2 * t;
        uint32_t u[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          const int k = k0 + (h & 1) + ((h & 2) ? 8 : 0);
          u[h] = k < P ? (ext ? (col < P ? Uinv[k * kLdE + col] : 0u) : S[(size_t)k * ldS + col])
                       : 0u;
        }
        const uint32_t bl0 = digit_pair(u[0], u[1], 0), bl1 = digit_pair(u[2], u[3], 0);
        const uint32_t bh0 = digit_pair(u[0], u[1], 8), bh1 = digit_pair(u[2], u[3], 8);
        mma16816(acc[nt][0], alo[ks], bl0, bl1);
        mma16816(acc[nt][1], ahi[ks], bh0, bh1);
        mma16816(acc[nt][2], asum, hadd2(bl0, bh0), hadd2(bl1, bh1));
      }
    }
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int row = m0 + g + (i >= 2 ? 8 : 0), col = c0 + 8 * nt + 2 * t + (i & 1);
        if (row >= nr || col >= (ext ? P : n)) continue;
        const uint32_t ll = f2u_exact(acc[nt][0][i]), hh = f2u_exact(acc[nt][1][i]);
        const uint32_t mid = f2u_exact(acc[nt][2][i]) - ll - hh;
        const uint32_t red = f_redc(((uint64_t)hh << 16) + (uint64_t)((mid << 8) + ll), F);
        if (ext) {
          C[(int64_t)row * ldc + spc[col]] = red;  // the multiplier of pivot col
        } else if (ispiv[col] <= r) {            // not one of the slab's pivot columns
          C[(int64_t)row * ldc + col] = f_sub(cv[nt][i], red, F);
        }
      }
  }
}

template <int kMode, int kSlab>
__global__ void __launch_bounds__(kBatchThreads, slab_min_blocks(kSlab, kMode == 3))
    k_batched_pluq(const BatchDesc* __restrict__ descs, const int32_t* __restrict__ order,
                   int batch, int* __restrict__ counter, FieldP F,
                   const uint32_t* __restrict__ inv_table, uint32_t* __restrict__ scratch,
                   size_t scratch_per_cta, int ldN, int64_t* __restrict__ ranks,
                   int32_t* __restrict__ status) {
  using BF = BField<kMode>;
  constexpr int kMinFree = kSlab / 4;  // a slab closes when fewer buffer rows are free
  constexpr int kRG = kSlab <= 16 ? 4 : 8;   // row groups of 4 in the refill update
  constexpr int kCL = kBatchThreads / kRG;   // column lanes: the update's tile is 4 kCL wide
  using TS = SlabT<kMode>;
  extern __shared__ __align__(16) uint32_t smem[];
  const int ldS = ldN + kPadS;  // row stride of the buffer
  TS* S = reinterpret_cast<TS*>(smem);
  uint32_t* LT = reinterpret_cast<uint32_t*>(S + (size_t)kSlab * ldS);
  TS* Uinv = reinterpret_cast<TS*>(LT + kSlab * kLdL);
  uint32_t* Ls = reinterpret_cast<uint32_t*>(Uinv + kSlab * kLdE);
  int32_t* spr = reinterpret_cast<int32_t*>(Ls + kSlab * kSlab);  // slab pivot -> matrix row
  int32_t* spc = spr + kSlab;                                      // slab pivot -> column
  uint32_t* invm = reinterpret_cast<uint32_t*>(spc + kSlab);       // inverse pivot (Montgomery)
  int32_t* first = reinterpret_cast<int32_t*>(invm + kSlab);       // buffer row -> first non-zero
  int32_t* srow = first + kSlab;                                   // buffer row -> matrix row
  int32_t* pslot = srow + kSlab;                                   // a round's pivots' buffer rows
  int32_t* ispiv = pslot + kSlab;  // 0: not a pivot column; else 1 + its pivot index
  int16_t* prow = reinterpret_cast<int16_t*>(ispiv + ldN);  // pivot -> row (< kBatchMax)
  int16_t* pcol = prow + kBatchMax;                          // pivot -> column
  int* red = reinterpret_cast<int*>(pcol + kBatchMax);
  int* s_idx = red + kBatchWarps;
  // the final layout's index arrays reuse the multiplier space
  int32_t* isprow = reinterpret_cast<int32_t*>(S);   // kSlab * ldS >= kBatchMax words
  int32_t* rowpos = reinterpret_cast<int32_t*>(LT);  // kSlab * kLdL >= 2 kBatchMax words
  int32_t* colpos = rowpos + kBatchMax;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t* SC = scratch + (size_t)blockIdx.x * scratch_per_cta;

  while (true) {
    if (tid == 0) *s_idx = atomicAdd(counter, 1);
    __syncthreads();
    const int idx = *s_idx;
    __syncthreads();
    if (idx >= batch) break;
    const int b = order[idx];
    const BatchDesc d = descs[b];
    const int m = d.m, n = d.n;
    uint32_t* A = d.A;
    const int64_t lda = d.lda;
    if (m == 0 || n == 0) {
      for (int t = tid; t < m; t += kBatchThreads) d.P[t] = t;
      for (int u = tid; u < n; u += kBatchThreads) d.Q[u] = u;
      if (tid == 0) {
        ranks[b] = 0;
        status[b] = PLUQ_OK;
      }
      continue;
    }
    // entries must be residues
    int bad = 0;
    for (int l = warp; l < m; l += kBatchWarps) {
      const uint32_t* row = A + (int64_t)l * lda;
      for (int jb0 = 0; jb0 < n; jb0 += 32 * kLoadBatch) {
        uint32_t v[kLoadBatch];
#pragma unroll
        for (int q = 0; q < kLoadBatch; ++q) {
          const int j = jb0 + 32 * q + lane;
          v[q] = j < n ? row[j] : 0u;
        }
#pragma unroll
        for (int q = 0; q < kLoadBatch; ++q) bad |= v[q] >= F.p;
      }
    }
    if (bt_block_or(bad, red)) {
      if (tid == 0) {
        ranks[b] = -1;
        status[b] = PLUQ_ERR_ENTRY_OUT_OF_RANGE;
      }
      continue;
    }
    for (int j = tid; j < ldN; j += kBatchThreads) ispiv[j] = 0;
    __syncthreads();
    int r = 0, next = 0;
    while (next < m) {
      int P = 0;  // pivots of this slab so far, in buffer rows 0..P-1
      while (true) {
        const int c = min(kSlab - P, m - next);  // rows taken in this round
        // 1. rows next.. into buffer rows P..P+c-1, earlier slabs' pivot columns zeroed
        for (int i = warp; i < c; i += kBatchWarps) {
          const int s = P + i;
          bt_load_row(S + (size_t)s * ldS, A + (int64_t)(next + i) * lda, n, ldN, [&](int j) {
            const int f = ispiv[j];
            return f != 0 && f <= r;
          });
          if (lane < kSlab) Ls[s * kSlab + lane] = 0u;
          if (lane == 0) srow[s] = next + i;
        }
        __syncthreads();
        if (P > 0) {
          // 2. their multipliers for the slab's pivots (forward substitution on the
          // pivot columns, a thread a row) ...
          if (tid < c) {
            const TS* st = S + (size_t)(P + tid) * ldS;
            for (int k = 0; k < P; ++k) {
              const int jk = spc[k];
              const uint32_t sk = dot_prefix<kMode>(LT + tid, kLdL, S + jk, ldS, k, F);
              const uint32_t l = BF::mulm(invm[k], f_sub(st[jk], sk, F), F);
              Ls[(P + tid) * kSlab + k] = l;
              LT[k * kLdL + tid] = BF::to_mont(l, F);
            }
          } else if (tid < kSlab) {
            for (int k = 0; k < P; ++k) LT[k * kLdL + tid] = 0u;
          }
          __syncthreads();
          // ... then rows -= L U over every column: thread t takes rows
          // 4 (t / kCL) .. + 3 and columns c0 + t % kCL + kCL jj
          const int rt = (tid / kCL) * 4, cl = tid % kCL;
          for (int c0 = 0; c0 < n; c0 += 4 * kCL) {
            Dot<kMode> acc[4][4];
#pragma unroll 2
            for (int k = 0; k < P; ++k) {
              const uint4 a4 = *reinterpret_cast<const uint4*>(LT + k * kLdL + rt);
              const uint32_t a[4] = {a4.x, a4.y, a4.z, a4.w};
              uint32_t bv[4];
#pragma unroll
              for (int jj = 0; jj < 4; ++jj) bv[jj] = S[(size_t)k * ldS + c0 + cl + kCL * jj];
#pragma unroll
              for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) acc[i][jj].add(a[i], bv[jj], F);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
              for (int jj = 0; jj < 4; ++jj) {
                const int row = rt + i, col = c0 + cl + kCL * jj;
                if (row < c && col < n) {
                  TS* e = S + (size_t)(P + row) * ldS + col;
                  *e = (TS)f_sub(*e, acc[i][jj].value(F), F);
                }
              }
          }
          __syncthreads();
        }
        // first non-zero of each new row
        for (int i = warp; i < c; i += kBatchWarps) {
          const TS* st = S + (size_t)(P + i) * ldS;
          int fz = INT_MAX;
          for (int jb = 0; jb < n; jb += 32) {
            const unsigned nz = __ballot_sync(0xffffffffu, jb + lane < n && st[jb + lane] != 0u);
            if (nz) {
              fz = jb + __ffs(nz) - 1;
              break;
            }
          }
          if (lane == 0) first[P + i] = fz;
        }
        __syncthreads();
        // 3. the new rows among themselves, in row order: for each pivot, every
        // warp looks up the inverse and updates its own rows below the pivot row
        // (kRowUnroll chunks of 32 columns at a time), tracking their first
        // non-zero; one barrier a pivot
        int np = 0;
        for (int s = P; s < P + c; ++s) {
          const int js = first[s];
          if (js == INT_MAX) continue;  // a zero row: no pivot
          const int k = P + np;
          const TS* pr = S + (size_t)s * ldS;
          const uint32_t im = BF::to_mont(f_inv(pr[js], F, inv_table), F);
          for (int u = s + 1 + warp; u < P + c; u += kBatchWarps) {
            TS* ur = S + (size_t)u * ldS;
            const uint32_t w = ur[js];
            if (w == 0u) continue;  // unchanged; its first non-zero is not js
            const uint32_t l = BF::mulm(im, w, F);
            const uint32_t lm = BF::to_mont(l, F);
            int fz = INT_MAX;  // this lane's first non-zero column, then the row's
            if constexpr (kMode == 3) {
              // 16-bit residues two at a time (32-bit shared accesses); the
              // products are below 2^32, so a 32-bit Montgomery reduction
              const uint32_t* pr2 = reinterpret_cast<const uint32_t*>(pr);
              uint32_t* ur2 = reinterpret_cast<uint32_t*>(ur);
              const int n2 = (n + 1) >> 1;  // an odd n pairs with the zero column n
              for (int jb0 = 0; jb0 < n2; jb0 += 32 * kRowUnroll) {
                uint32_t nv[kRowUnroll];
#pragma unroll
                for (int q = 0; q < kRowUnroll; ++q) {
                  const int j2 = jb0 + 32 * q + lane;
                  nv[q] = 0u;
                  if (j2 < n2) {
                    const uint32_t a = ur2[j2], b = pr2[j2];
                    const uint32_t lo = f_sub(a & 0xFFFFu, f_redc32(lm * (b & 0xFFFFu), F), F);
                    const uint32_t hi = f_sub(a >> 16, f_redc32(lm * (b >> 16), F), F);
                    nv[q] = lo | (hi << 16);
                  }
                }
#pragma unroll
                for (int q = 0; q < kRowUnroll; ++q) {
                  const int j2 = jb0 + 32 * q + lane;
                  if (j2 < n2) ur2[j2] = nv[q];
                  if (nv[q] != 0u && fz == INT_MAX) fz = 2 * j2 + ((nv[q] & 0xFFFFu) ? 0 : 1);
                }
              }
            } else {
              for (int jb0 = 0; jb0 < n; jb0 += 32 * kRowUnroll) {
                uint32_t nv[kRowUnroll];
#pragma unroll
                for (int q = 0; q < kRowUnroll; ++q) {
                  const int j = jb0 + 32 * q + lane;
                  nv[q] = j < n ? f_sub(ur[j], BF::mulm(lm, pr[j], F), F) : 0u;
                }
#pragma unroll
                for (int q = 0; q < kRowUnroll; ++q) {
                  const int j = jb0 + 32 * q + lane;
                  if (j < n) ur[j] = (TS)nv[q];
                  if (nv[q] != 0u && fz == INT_MAX) fz = j;
                }
              }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) fz = min(fz, __shfl_xor_sync(0xffffffffu, fz, o));
            if (lane == 0) {
              Ls[u * kSlab + k] = l;
              first[u] = fz;
            }
          }
          if (tid == 0) {
            spr[k] = srow[s];
            spc[k] = js;
            invm[k] = im;
            pslot[np] = s;
            ispiv[js] = r + k + 1;
          }
          ++np;
          __syncthreads();
        }
        // 4. rows without a pivot are final: back to the matrix (the multipliers
        // of this slab at its pivot columns, zero elsewhere; earlier slabs'
        // pivot columns keep their multipliers)
        for (int s = P + warp; s < P + c; s += kBatchWarps) {
          if (first[s] != INT_MAX) continue;
          uint32_t* row = A + (int64_t)srow[s] * lda;
          for (int j = lane; j < n; j += 32) {
            const int f = ispiv[j];
            if (f != 0 && f <= r) continue;
            row[j] = f > r ? Ls[s * kSlab + (f - r - 1)] : 0u;
          }
        }
        __syncthreads();
        // the round's pivot rows move up to buffer rows P..P+np-1 (pslot[i] >=
        // P + i, increasing: each column moved in increasing i)
        for (int j = tid; j < ldN; j += kBatchThreads)
          for (int i = 0; i < np; ++i)
            if (pslot[i] != P + i) S[(size_t)(P + i) * ldS + j] = S[(size_t)pslot[i] * ldS + j];
        if (tid < kSlab)
          for (int i = 0; i < np; ++i)
            if (pslot[i] != P + i) Ls[(P + i) * kSlab + tid] = Ls[pslot[i] * kSlab + tid];
        __syncthreads();
        P += np;
        next += c;
        if (P > kSlab - kMinFree || next >= m) break;
      }
      // the slab's pivot rows back to the matrix: multipliers at the columns of
      // the slab's earlier pivots, the reduced row elsewhere
      for (int k = warp; k < P; k += kBatchWarps) {
        uint32_t* row = A + (int64_t)spr[k] * lda;
        const TS* st = S + (size_t)k * ldS;
        for (int j = lane; j < n; j += 32) {
          const int f = ispiv[j];
          if (f != 0 && f <= r) continue;
          const int kk = f - r - 1;
          row[j] = (f > r && kk < k) ? Ls[k * kSlab + kk] : st[j];
        }
      }
      for (int k = tid; k < P; k += kBatchThreads) {
        prow[r + k] = (int16_t)spr[k];
        pcol[r + k] = (int16_t)spc[k];
      }
      __syncthreads();
      // the rows below reduced by the slab's P pivots
      if (P > 0 && next < m) {
        if constexpr (kMode == 3) {
          // U_JJ (plain), then W = U_JJ^{-1} U in place and U_JJ^{-1}, both in
          // Montgomery form, by back substitution down each column:
          // w_k = (u_k - sum_{q>k} U_k[j_q] w_q) / U_k[j_k]
          uint32_t* Ujj = LT;  // [k][q], stride kSlab + 1; then X of a row block
          for (int e = tid; e < P * P; e += kBatchThreads) {
            const int k = e / P, q = e - k * P;
            Ujj[k * (kSlab + 1) + q] = S[(size_t)k * ldS + spc[q]];
          }
          __syncthreads();
          for (int col = tid; col < n + P; col += kBatchThreads) {
            const bool ext = col >= n;
            const int e = col - n;
            TS* w = ext ? Uinv + e : S + col;
            const size_t ldw = ext ? (size_t)kLdE : (size_t)ldS;
            for (int k = P - 1; k >= 0; --k) {
              const uint32_t u = ext ? (k == e ? 1u : 0u) : w[(size_t)k * ldw];
              Dot<kMode> d;
              for (int q = k + 1; q < P; ++q) d.add(Ujj[k * (kSlab + 1) + q], w[(size_t)q * ldw], F);
              w[(size_t)k * ldw] = (TS)BF::to_mont(BF::mulm(invm[k], f_sub(u, d.value(F), F), F), F);
            }
          }
          __syncthreads();
          uint32_t* XT = LT;  // [k][row], stride kLdL
          for (int rb = next; rb < m; rb += kRowBlock) {
            const int nr = min(kRowBlock, m - rb);
            if (tid < nr) {
              const uint32_t* ar = A + (int64_t)(rb + tid) * lda;
              for (int k0 = 0; k0 < P; k0 += kLoadBatch) {
                uint32_t x[kLoadBatch];
#pragma unroll
                for (int q = 0; q < kLoadBatch; ++q) x[q] = k0 + q < P ? ar[spc[k0 + q]] : 0u;
#pragma unroll
                for (int q = 0; q < kLoadBatch; ++q)
                  if (k0 + q < P) XT[(k0 + q) * kLdL + tid] = x[q];
              }
            } else if (tid < kRowBlock) {
              for (int k = 0; k < P; ++k) XT[k * kLdL + tid] = 0u;
            }
            __syncthreads();
            trailing_mma<kMode>(A + (int64_t)rb * lda, lda, nr, n, P, spc, XT, S, ldS, Uinv,
                                ispiv, r, F);
            __syncthreads();
          }
        } else {
          for (int rb = next; rb < m; rb += kRowBlock) {
            const int nr = min(kRowBlock, m - rb);
            if (tid < kRowBlock) {
              if (tid < nr) {
                // the row's entries at the pivot columns, then L by forward substitution
                const uint32_t* ar = A + (int64_t)(rb + tid) * lda;
                for (int k0 = 0; k0 < P; k0 += kLoadBatch) {
                  uint32_t x[kLoadBatch];
  #pragma unroll
                  for (int q = 0; q < kLoadBatch; ++q) x[q] = k0 + q < P ? ar[spc[k0 + q]] : 0u;
  #pragma unroll
                  for (int q = 0; q < kLoadBatch; ++q)
                    if (k0 + q < P) LT[(k0 + q) * kLdL + tid] = x[q];
                }
                for (int k = 0; k < P; ++k) {
                  const int jk = spc[k];
                  const uint32_t sk = dot_prefix<kMode>(LT + tid, kLdL, S + jk, ldS, k, F);
                  const uint32_t l = BF::mulm(invm[k], f_sub(LT[k * kLdL + tid], sk, F), F);
                  LT[k * kLdL + tid] = BF::to_mont(l, F);
                }
              } else {
                for (int k = 0; k < P; ++k) LT[k * kLdL + tid] = 0u;
              }
            }
            __syncthreads();
            // C <- C - L U; the slab's pivot columns take L
            {
              const int tx = tid & 15, ty = tid >> 4;
              for (int sub = 0; sub < nr; sub += kTile) {
                const int rl = sub + ty * 4;  // first of this thread's rows within the block
                for (int c0 = 0; c0 < n; c0 += kTile) {
                  uint32_t cv[4][4];
    #pragma unroll
                  for (int i = 0; i < 4; ++i)
    #pragma unroll
                    for (int jj = 0; jj < 4; ++jj) {
                      const int row = rl + i, col = c0 + tx + 16 * jj;
                      cv[i][jj] = (row < nr && col < n) ? A[(int64_t)(rb + row) * lda + col] : 0u;
                    }
                  Dot<kMode> acc[4][4];
    #pragma unroll 2
                  for (int k = 0; k < P; ++k) {
                    const uint4 a4 = *reinterpret_cast<const uint4*>(LT + k * kLdL + rl);
                    const uint32_t a[4] = {a4.x, a4.y, a4.z, a4.w};
                    uint32_t bv[4];
    #pragma unroll
                    for (int jj = 0; jj < 4; ++jj) bv[jj] = S[(size_t)k * ldS + c0 + tx + 16 * jj];
    #pragma unroll
                    for (int i = 0; i < 4; ++i)
    #pragma unroll
                      for (int jj = 0; jj < 4; ++jj) acc[i][jj].add(a[i], bv[jj], F);
                  }
    #pragma unroll
                  for (int i = 0; i < 4; ++i)
    #pragma unroll
                    for (int jj = 0; jj < 4; ++jj) {
                      const int row = rl + i, col = c0 + tx + 16 * jj;
                      if (row < nr && col < n) {
                        const int f = ispiv[col];
                        const uint32_t v = f > r ? BF::from_mont(LT[(f - r - 1) * kLdL + row], F)
                                                 : f_sub(cv[i][jj], acc[i][jj].value(F), F);
                        A[(int64_t)(rb + row) * lda + col] = v;
                      }
                    }
                }
              }
            }
            __syncthreads();
          }
        }
      }
      r += P;
    }
    // P = [pivot rows, others ascending], Q likewise
    for (int i = tid; i < m; i += kBatchThreads) isprow[i] = 0;
    for (int j = tid; j < n; j += kBatchThreads) ispiv[j] = 0;
    __syncthreads();
    for (int k = tid; k < r; k += kBatchThreads) {
      isprow[prow[k]] = 1;
      ispiv[pcol[k]] = 1;
      rowpos[k] = prow[k];
      colpos[k] = pcol[k];
    }
    __syncthreads();
    bt_compact(isprow, m, rowpos, r, red);
    bt_compact(ispiv, n, colpos, r, red);
    // the non-pivot rows' multipliers (at the pivot columns, in pivot order) to scratch
    for (int t = r + warp; t < m; t += kBatchWarps) {
      const uint32_t* src = A + (int64_t)rowpos[t] * lda;
      uint32_t* dst = SC + (size_t)(t - r) * r;
      for (int u = lane; u < r; u += 32) dst[u] = src[colpos[u]];
    }
    __syncthreads();
    // pivot rows up, eight at a time through shared memory: row t comes from
    // rowpos[t] >= t, and rows below t0 + 8 are not read again
    for (int t0 = 0; t0 < r; t0 += kBatchWarps) {
      const int t = t0 + warp;
      TS* w = S + (size_t)warp * ldS;
      if (t < r) bt_load_row(w, A + (int64_t)rowpos[t] * lda, n, ldN, [](int) { return false; });
      __syncthreads();
      if (t < r) {
        uint32_t* dst = A + (int64_t)t * lda;
        for (int u = lane; u < n; u += 32) dst[u] = w[colpos[u]];
      }
      __syncthreads();
    }
    // non-pivot rows: their multipliers, then zeros
    for (int t = r + warp; t < m; t += kBatchWarps) {
      const uint32_t* src = SC + (size_t)(t - r) * r;
      uint32_t* dst = A + (int64_t)t * lda;
      for (int u = lane; u < n; u += 32) dst[u] = u < r ? src[u] : 0u;
    }
    for (int t = tid; t < m; t += kBatchThreads) d.P[t] = rowpos[t];
    for (int u = tid; u < n; u += kBatchThreads) d.Q[u] = colpos[u];
    if (tid == 0) {
      ranks[b] = r;
      status[b] = PLUQ_OK;
    }
    __syncthreads();
  }
}

__global__ void k_batch_reset(int* counter) { *counter = 0; }

int slab_ld(int max_n) { return (int)cdiv(std::max(max_n, 1), kLd) * kLd; }

template <int kMode, int kSlab>
size_t slab_smem_bytes(int max_n) {
  return slab_smem_bytes_for<kSlab, SlabT<kMode>>(slab_ld(max_n));
}

template <int kMode, int kSlab>
int batched_occupancy(int max_n) {
  if (cudaFuncSetAttribute(k_batched_pluq<kMode, kSlab>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) != cudaSuccess)
    return 0;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batched_pluq<kMode, kSlab>,
                                                    kBatchThreads,
                                                    slab_smem_bytes<kMode, kSlab>(max_n)) != cudaSuccess)
    return 0;
  return occ;
}

int batched_mode(const FieldP& F) {
  return F.is2 ? 0 : F.p < (1u << 16) ? 3 : F.p < (1u << 27) ? 1 : 2;
}

// Buffer height: the option's, else 32 for p < 2^16 (16-bit buffer: three CTAs
// an SM at 512 columns), 16 otherwise.
int batched_slab(const pluq_ctx* c, int max_n) {
  (void)max_n;
  if (c->batch_slab) return c->batch_slab;
  return batched_mode(c->F) == 3 ? 32 : 16;
}

template <int kMode>
int occupancy_for(int slab, int max_n) {
  switch (slab) {
    case 16: return batched_occupancy<kMode, 16>(max_n);
    case 24: return batched_occupancy<kMode, 24>(max_n);
    default: return batched_occupancy<kMode, 32>(max_n);
  }
}

template <int kMode, int kSlab>
void launch_slab(pluq_ctx* c, int G, const BatchDesc* d, const int32_t* order, int count,
                 int* counter, uint32_t* sc, size_t per, int max_n, int64_t* ranks,
                 int32_t* status) {
  k_batched_pluq<kMode, kSlab><<<G, kBatchThreads, slab_smem_bytes<kMode, kSlab>(max_n),
                                 c->stream>>>(
      d, order, count, counter, c->F, inv_table_ptr(c), sc, per, slab_ld(max_n), ranks, status);
}

template <int kMode>
void launch_mode(pluq_ctx* c, int slab, int G, const BatchDesc* d, const int32_t* order,
                 int count, int* counter, uint32_t* sc, size_t per, int max_n, int64_t* ranks,
                 int32_t* status) {
  switch (slab) {
    case 16:
      launch_slab<kMode, 16>(c, G, d, order, count, counter, sc, per, max_n, ranks, status);
      break;
    case 24:
      launch_slab<kMode, 24>(c, G, d, order, count, counter, sc, per, max_n, ranks, status);
      break;
    default:
      launch_slab<kMode, 32>(c, G, d, order, count, counter, sc, per, max_n, ranks, status);
      break;
  }
}

}  // namespace

int batched_max_dim() { return kBatchMax; }

// CTAs of the persistent launch for matrices of at most max_n columns.
int batched_grid(pluq_ctx* c, int max_n) {
  const int slab = batched_slab(c, max_n);
  int occ = 0;
  switch (batched_mode(c->F)) {
    case 0: occ = occupancy_for<0>(slab, max_n); break;
    case 1: occ = occupancy_for<1>(slab, max_n); break;
    case 2: occ = occupancy_for<2>(slab, max_n); break;
    default: occ = occupancy_for<3>(slab, max_n); break;
  }
  return occ > 0 ? occ * c->sm_count : 0;
}

// Persistent launch over `count` matrices already described on the device.
int launch_batched(pluq_ctx* c, const void* descs, const int32_t* order, int count,
                   int64_t* ranks, int32_t* status, int max_elems, int max_n) {
  int* counter = c->small.as<int>() + 24;
  const int G = batched_grid(c, max_n);
  if (G <= 0) return PLUQ_ERR_CUDA;
  const size_t per = (size_t)std::max(max_elems, 1);
  PLUQ_TRY(c->batch_scratch.ensure(sizeof(uint32_t) * per * G));
  {
    ProfScope pr(c, PC_INDEX);
    k_batch_reset<<<1, 1, 0, c->stream>>>(counter);
  }
  ProfScope ps(c, PC_BASE);
  const auto* d = static_cast<const BatchDesc*>(descs);
  const int slab = batched_slab(c, max_n);
  uint32_t* sc = c->batch_scratch.as<uint32_t>();
  switch (batched_mode(c->F)) {
    case 0:
      launch_mode<0>(c, slab, G, d, order, count, counter, sc, per, max_n, ranks, status);
      break;
    case 1:
      launch_mode<1>(c, slab, G, d, order, count, counter, sc, per, max_n, ranks, status);
      break;
    case 2:
      launch_mode<2>(c, slab, G, d, order, count, counter, sc, per, max_n, ranks, status);
      break;
    default:
      launch_mode<3>(c, slab, G, d, order, count, counter, sc, per, max_n, ranks, status);
      break;
  }
  PLUQ_CUDA(cudaGetLastError());
  return PLUQ_OK;
}

size_t batched_desc_size() { return sizeof(BatchDesc); }

void batched_fill_desc(void* out, int i, uint32_t* A, int32_t* P, int32_t* Q, int64_t lda, int m,
                       int n) {
  static_cast<BatchDesc*>(out)[i] = BatchDesc{A, P, Q, lda, m, n};
}
