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
// shared-memory buffer of kSlab rows (pivot rows at the top, candidate rows
// below), in rounds:
//   1. the next rows of the matrix fill the free buffer rows (the pivot columns
//      of earlier slabs zeroed);
//   2. they are reduced by the slab's pivots so far: multipliers by forward
//      substitution on the pivot columns, then rows -= L U with the products of
//      every entry summed in 64 bits and reduced once (delayed reduction,
//      Sec. 3.1);
//   3. they are eliminated among themselves in row order (pivot search, rank-1
//      updates spread over all warps as (row, 32-column) items);
//   4. the rows that gave no pivot are final and go back to the matrix; the new
//      pivot rows move up.
// The slab closes once fewer than kMinFree buffer rows are free (or the matrix
// ends): its pivot rows go back to the matrix and the rows below are reduced by
// its pivots at once, L from a forward substitution per row, then C <- C - L U
// in 64 x 64 tiles of 4 x 4 register micro-tiles.  Multipliers are kept in
// Montgomery form (x R mod p, R = 2^32) as left operands, so the reduction of
// a sum of products (L R) * U is one REDC.  L multipliers overwrite the pivot
// column entries.
//
// The final P^T A Q^T layout is written in place: the multipliers of the
// non-pivot rows are first copied to the CTA's scratch, the pivot rows are then
// moved up eight at a time through shared memory (a pivot row never moves down),
// and the non-pivot rows are written from the scratch.  Entries >= p mark the
// matrix with PLUQ_ERR_ENTRY_OUT_OF_RANGE and leave it untouched.
#include <algorithm>
#include <climits>
#include <numeric>
#include <vector>

#include "common.cuh"

namespace {

constexpr int kBatchThreads = 256;
constexpr int kBatchWarps = kBatchThreads / 32;
constexpr int kBatchMax = 1024;
constexpr int kSlab = 32;       // rows of the shared-memory buffer; most pivots of a slab
constexpr int kMinFree = 8;     // a slab closes when fewer buffer rows than this are free
constexpr int kRowBlock = 128;  // rows below the slab whose multipliers are formed together
constexpr int kTile = 64;       // C tile of the update below the slab, 4 x 4 per thread
constexpr int kLd = 128;        // buffer rows are padded to a multiple of this many words
constexpr int kLoadBatch = 8;   // global loads a lane keeps in flight
constexpr int kItemUnroll = 4;  // (row, chunk) items a warp updates together

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
//   2: otherwise (a REDC per product).
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

// sum of Montgomery a times plain b over a dot product, as a plain residue
template <int kMode>
struct Dot {
  uint64_t acc = 0;
  uint32_t red = 0;
  __device__ __forceinline__ void add(uint32_t am, uint32_t b, const FieldP& F) {
    if (kMode == 0) {
      red ^= am & b;
    } else if (kMode == 1) {
      acc += (uint64_t)am * b;
    } else {
      red = f_add(red, f_redc((uint64_t)am * b, F), F);
    }
  }
  __device__ __forceinline__ uint32_t value(const FieldP& F) const {
    if (kMode == 0) return red & 1u;
    if (kMode == 1) return f_redc(acc, F);
    return red;
  }
};

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
template <typename Drop>
__device__ __forceinline__ void bt_load_row(uint32_t* dst, const uint32_t* src, int n, int ld,
                                            Drop drop) {
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
      if (j < ld) dst[j] = v[q];
    }
  }
}

// Shared memory of one CTA, in 32-bit words, for buffer rows of ldS words.
__host__ __device__ constexpr size_t slab_smem_words(int ldS) {
  return (size_t)kSlab * ldS              // S: pivot rows, then candidate rows (plain)
         + (size_t)kSlab * kRowBlock      // LT: multipliers of a row block, pivot-major (Montgomery)
         + (size_t)kSlab * kSlab          // Ls: multipliers of the buffer rows (plain)
         + 8 * kSlab                      // spr, spc, invm, first, srow, lrow, lmrow, pslot
         + (size_t)ldS                    // ispiv
         + 2 * (size_t)kBatchMax          // prow, pcol
         + kBatchWarps + 8;               // red, misc
}

template <int kMode>
__global__ void __launch_bounds__(kBatchThreads)
    k_batched_pluq(const BatchDesc* __restrict__ descs, const int32_t* __restrict__ order,
                   int batch, int* __restrict__ counter, FieldP F,
                   const uint32_t* __restrict__ inv_table, uint32_t* __restrict__ scratch,
                   size_t scratch_per_cta, int ldS, int64_t* __restrict__ ranks,
                   int32_t* __restrict__ status) {
  using BF = BField<kMode>;
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t* S = smem;
  uint32_t* LT = S + (size_t)kSlab * ldS;
  uint32_t* Ls = LT + kSlab * kRowBlock;
  int32_t* spr = reinterpret_cast<int32_t*>(Ls + kSlab * kSlab);  // slab pivot -> matrix row
  int32_t* spc = spr + kSlab;                                      // slab pivot -> column
  uint32_t* invm = reinterpret_cast<uint32_t*>(spc + kSlab);       // inverse pivot (Montgomery)
  int32_t* first = reinterpret_cast<int32_t*>(invm + kSlab);       // buffer row -> first non-zero
  int32_t* srow = first + kSlab;                                   // buffer row -> matrix row
  uint32_t* lrow = reinterpret_cast<uint32_t*>(srow + kSlab);      // multipliers of one step
  uint32_t* lmrow = lrow + kSlab;
  int32_t* pslot = reinterpret_cast<int32_t*>(lmrow + kSlab);      // a round's pivots' buffer rows
  int32_t* ispiv = pslot + kSlab;  // 0: not a pivot column; else 1 + its pivot index
  int32_t* prow = ispiv + ldS;
  int32_t* pcol = prow + kBatchMax;
  int* red = pcol + kBatchMax;
  int* s_idx = red + kBatchWarps;
  // the final layout's index arrays reuse the multiplier space
  int32_t* isprow = reinterpret_cast<int32_t*>(Ls);  // kSlab * kSlab = kBatchMax words
  int32_t* rowpos = reinterpret_cast<int32_t*>(LT);  // kSlab * kRowBlock >= 2 kBatchMax words
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
    for (int j = tid; j < ldS; j += kBatchThreads) ispiv[j] = 0;
    __syncthreads();
    int r = 0, next = 0;
    while (next < m) {
      int P = 0;  // pivots of this slab so far, in buffer rows 0..P-1
      while (true) {
        const int c = min(kSlab - P, m - next);  // rows taken in this round
        // 1. rows next.. into buffer rows P..P+c-1, earlier slabs' pivot columns zeroed
        for (int i = warp; i < c; i += kBatchWarps) {
          const int s = P + i;
          bt_load_row(S + (size_t)s * ldS, A + (int64_t)(next + i) * lda, n, ldS, [&](int j) {
            const int f = ispiv[j];
            return f != 0 && f <= r;
          });
          Ls[s * kSlab + lane] = 0u;
          if (lane == 0) srow[s] = next + i;
        }
        __syncthreads();
        if (P > 0) {
          // 2. their multipliers for the slab's pivots (forward substitution on the
          // pivot columns, a thread a row) ...
          if (tid < c) {
            const uint32_t* st = S + (size_t)(P + tid) * ldS;
            for (int k = 0; k < P; ++k) {
              const int jk = spc[k];
              Dot<kMode> s;
              for (int q = 0; q < k; ++q) s.add(LT[q * kRowBlock + tid], S[(size_t)q * ldS + jk], F);
              const uint32_t l = BF::mulm(invm[k], f_sub(st[jk], s.value(F), F), F);
              Ls[(P + tid) * kSlab + k] = l;
              LT[k * kRowBlock + tid] = BF::to_mont(l, F);
            }
          } else if (tid < kSlab) {
            for (int k = 0; k < P; ++k) LT[k * kRowBlock + tid] = 0u;
          }
          __syncthreads();
          // ... then rows -= L U over every column: warp w takes rows 4w..4w+3,
          // lane l columns c0 + l + 32 jj
          const int rt = warp * 4;
          for (int c0 = 0; c0 < n; c0 += 128) {
            Dot<kMode> acc[4][4];
#pragma unroll 2
            for (int k = 0; k < P; ++k) {
              const uint4 a4 = *reinterpret_cast<const uint4*>(LT + k * kRowBlock + rt);
              const uint32_t a[4] = {a4.x, a4.y, a4.z, a4.w};
              uint32_t bv[4];
#pragma unroll
              for (int jj = 0; jj < 4; ++jj) bv[jj] = S[(size_t)k * ldS + c0 + lane + 32 * jj];
#pragma unroll
              for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) acc[i][jj].add(a[i], bv[jj], F);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
              for (int jj = 0; jj < 4; ++jj) {
                const int row = rt + i, col = c0 + lane + 32 * jj;
                if (row < c && col < n) {
                  uint32_t* e = S + (size_t)(P + row) * ldS + col;
                  *e = f_sub(*e, acc[i][jj].value(F), F);
                }
              }
          }
          __syncthreads();
        }
        // first non-zero of each new row
        for (int i = warp; i < c; i += kBatchWarps) {
          const uint32_t* st = S + (size_t)(P + i) * ldS;
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
        // 3. the new rows among themselves, in row order
        int np = 0;
        const int nch = (n + 31) >> 5;
        for (int s = P; s < P + c; ++s) {
          const int js = first[s];
          if (js == INT_MAX) continue;  // a zero row: no pivot
          const int k = P + np;
          const uint32_t* pr = S + (size_t)s * ldS;
          const int ub = s + 1, ue = P + c;
          if (warp == 0) {
            const uint32_t im = BF::to_mont(f_inv(pr[js], F, inv_table), F);
            const int u = ub + lane;
            if (u < ue) {
              const uint32_t w = S[(size_t)u * ldS + js];
              const uint32_t l = w != 0u ? BF::mulm(im, w, F) : 0u;
              lrow[u] = l;
              lmrow[u] = BF::to_mont(l, F);
              Ls[u * kSlab + k] = l;
              if (w != 0u) first[u] = INT_MAX;
            }
            if (lane == 0) {
              spr[k] = srow[s];
              spc[k] = js;
              invm[k] = im;
              pslot[np] = s;
              ispiv[js] = r + k + 1;
            }
          }
          ++np;
          __syncthreads();
          // rank-1 update of the rows below it, as (row, 32-column chunk) items
          const int items = (ue - ub) * nch;
          for (int it0 = warp * kItemUnroll; it0 < items; it0 += kBatchWarps * kItemUnroll) {
            uint32_t nv[kItemUnroll];
            int iu[kItemUnroll], jb[kItemUnroll];
            bool act[kItemUnroll];
#pragma unroll
            for (int q = 0; q < kItemUnroll; ++q) {
              const int it = it0 + q;
              const int du = it / nch;
              iu[q] = ub + du;
              jb[q] = (it - du * nch) * 32;
              const uint32_t lm = it < items ? lmrow[iu[q]] : 0u;
              act[q] = lm != 0u;
              const int j = jb[q] + lane;
              nv[q] = (act[q] && j < n)
                          ? f_sub(S[(size_t)iu[q] * ldS + j], BF::mulm(lm, pr[j], F), F)
                          : 0u;
            }
#pragma unroll
            for (int q = 0; q < kItemUnroll; ++q) {
              if (!act[q]) continue;  // warp-uniform
              const int j = jb[q] + lane;
              if (j < n) S[(size_t)iu[q] * ldS + j] = nv[q];
              const unsigned nz = __ballot_sync(0xffffffffu, nv[q] != 0u);
              if (nz && lane == 0) atomicMin(first + iu[q], jb[q] + __ffs(nz) - 1);
            }
          }
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
        for (int j = tid; j < ldS; j += kBatchThreads)
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
        const uint32_t* st = S + (size_t)k * ldS;
        for (int j = lane; j < n; j += 32) {
          const int f = ispiv[j];
          if (f != 0 && f <= r) continue;
          const int kk = f - r - 1;
          row[j] = (f > r && kk < k) ? Ls[k * kSlab + kk] : st[j];
        }
      }
      for (int k = tid; k < P; k += kBatchThreads) {
        prow[r + k] = spr[k];
        pcol[r + k] = spc[k];
      }
      __syncthreads();
      // the rows below reduced by the slab's P pivots
      if (P > 0 && next < m) {
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
                  if (k0 + q < P) LT[(k0 + q) * kRowBlock + tid] = x[q];
              }
              for (int k = 0; k < P; ++k) {
                const int jk = spc[k];
                Dot<kMode> s;
                for (int q = 0; q < k; ++q) s.add(LT[q * kRowBlock + tid], S[(size_t)q * ldS + jk], F);
                const uint32_t l =
                    BF::mulm(invm[k], f_sub(LT[k * kRowBlock + tid], s.value(F), F), F);
                LT[k * kRowBlock + tid] = BF::to_mont(l, F);
              }
            } else {
              for (int k = 0; k < P; ++k) LT[k * kRowBlock + tid] = 0u;
            }
          }
          __syncthreads();
          // C <- C - L U; the slab's pivot columns take L
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
                const uint4 a4 = *reinterpret_cast<const uint4*>(LT + k * kRowBlock + rl);
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
                    const uint32_t v = f > r ? BF::from_mont(LT[(f - r - 1) * kRowBlock + row], F)
                                             : f_sub(cv[i][jj], acc[i][jj].value(F), F);
                    A[(int64_t)(rb + row) * lda + col] = v;
                  }
                }
            }
          }
          __syncthreads();
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
      uint32_t* w = S + (size_t)warp * ldS;
      if (t < r) bt_load_row(w, A + (int64_t)rowpos[t] * lda, n, ldS, [](int) { return false; });
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

size_t slab_smem_bytes(int max_n) { return sizeof(uint32_t) * slab_smem_words(slab_ld(max_n)); }

template <int kMode>
int batched_occupancy(size_t smem) {
  if (cudaFuncSetAttribute(k_batched_pluq<kMode>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           227 * 1024) != cudaSuccess)
    return 0;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batched_pluq<kMode>, kBatchThreads,
                                                    smem) != cudaSuccess)
    return 0;
  return occ;
}

int batched_mode(const FieldP& F) { return F.is2 ? 0 : (F.p < (1u << 27) ? 1 : 2); }

}  // namespace

int batched_max_dim() { return kBatchMax; }

// CTAs of the persistent launch for matrices of at most max_n columns.
int batched_grid(pluq_ctx* c, int max_n) {
  const size_t smem = slab_smem_bytes(max_n);
  int occ = 0;
  switch (batched_mode(c->F)) {
    case 0: occ = batched_occupancy<0>(smem); break;
    case 1: occ = batched_occupancy<1>(smem); break;
    default: occ = batched_occupancy<2>(smem); break;
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
  const int ldS = slab_ld(max_n);
  const size_t smem = slab_smem_bytes(max_n);
  uint32_t* sc = c->batch_scratch.as<uint32_t>();
  const uint32_t* tab = inv_table_ptr(c);
  switch (batched_mode(c->F)) {
    case 0:
      k_batched_pluq<0><<<G, kBatchThreads, smem, c->stream>>>(d, order, count, counter, c->F, tab,
                                                               sc, per, ldS, ranks, status);
      break;
    case 1:
      k_batched_pluq<1><<<G, kBatchThreads, smem, c->stream>>>(d, order, count, counter, c->F, tab,
                                                               sc, per, ldS, ranks, status);
      break;
    default:
      k_batched_pluq<2><<<G, kBatchThreads, smem, c->stream>>>(d, order, count, counter, c->F, tab,
                                                               sc, per, ldS, ranks, status);
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
