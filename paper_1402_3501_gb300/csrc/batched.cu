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
// The elimination is blocked by row slabs of kSlab rows, the tiled iterative
// scheme of Sec. 4.1 with one column tile:
//   1. the slab (reduced by every earlier slab) is loaded into shared memory
//      with the earlier pivot columns zeroed, and eliminated row by row there
//      (pivot search, rank-1 updates of the slab rows below the pivot row);
//   2. the slab goes back to the matrix: multipliers at its pivot columns,
//      reduced rows elsewhere; earlier pivot columns keep the multipliers the
//      earlier slabs wrote;
//   3. the rows below are reduced by the slab's nb pivots at once: their
//      multipliers L = X U_JJ^{-1} (X: their entries at the slab's pivot
//      columns, U_JJ: the pivot rows at those columns, upper triangular in
//      pivot order) by a forward substitution per row, then C <- C - L U in
//      64 x 64 tiles of 4 x 4 register micro-tiles, the nb products of every
//      output summed in 64 bits and reduced once (delayed reduction, Sec. 3.1).
// The pivot rows are kept in Montgomery form (x R mod p, R = 2^32) for step 3,
// so the reduction of a sum of products L * (U R) is one REDC.  L multipliers
// overwrite the pivot column entries; the final P^T A Q^T layout is gathered
// through the CTA's scratch and copied back.  Entries >= p mark the matrix with
// PLUQ_ERR_ENTRY_OUT_OF_RANGE and leave it untouched.
#include <algorithm>
#include <climits>
#include <numeric>
#include <vector>

#include "common.cuh"

namespace {

constexpr int kBatchThreads = 256;
constexpr int kBatchWarps = kBatchThreads / 32;
constexpr int kBatchMax = 1024;
constexpr int kSlab = 32;  // rows eliminated in shared memory together
constexpr int kRowBlock = 128;  // rows below the slab whose multipliers are formed together
constexpr int kTile = 64;       // C tile of the update, 4 x 4 per thread

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
};

// sum of plain a times Montgomery b over a dot product, as a plain residue
template <int kMode>
struct Dot {
  uint64_t acc = 0;
  uint32_t red = 0;
  __device__ __forceinline__ void add(uint32_t a, uint32_t bm, const FieldP& F) {
    if (kMode == 0) {
      red ^= a & bm;
    } else if (kMode == 1) {
      acc += (uint64_t)a * bm;
    } else {
      red = f_add(red, f_redc((uint64_t)a * bm, F), F);
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

// Shared memory of one CTA, in 32-bit words, for rows of ldS words.
__host__ __device__ constexpr size_t slab_smem_words(int ldS) {
  return (size_t)kSlab * ldS              // S: the slab, then the pivot rows (Montgomery)
         + (size_t)kSlab * kRowBlock      // LT: multipliers of a row block, pivot-major
         + (size_t)kSlab * kSlab          // Ls: multipliers inside the slab
         + (size_t)kSlab * (kSlab + 1)    // Ujj: pivot rows at the pivot columns (Montgomery)
         + kSlab                          // invm: inverse pivots (Montgomery)
         + 3 * kSlab                      // first, spr, spc
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
  uint32_t* Ujj = Ls + kSlab * kSlab;
  uint32_t* invm = Ujj + kSlab * (kSlab + 1);
  int32_t* first = reinterpret_cast<int32_t*>(invm + kSlab);
  int32_t* spr = first + kSlab;
  int32_t* spc = spr + kSlab;
  int32_t* ispiv = spc + kSlab;  // 0: not a pivot column; else 1 + its pivot index
  int32_t* prow = ispiv + ldS;
  int32_t* pcol = prow + kBatchMax;
  int* red = pcol + kBatchMax;
  int* s_idx = red + kBatchWarps;
  // the final gather's index arrays reuse the slab and multiplier space
  int32_t* isprow = reinterpret_cast<int32_t*>(S);
  int32_t* rowpos = isprow + kBatchMax;
  int32_t* colpos = rowpos + kBatchMax;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tx = tid & 15, ty = tid >> 4;
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
    for (int l = warp; l < m; l += kBatchWarps)
      for (int j = lane; j < n; j += 32) bad |= A[(int64_t)l * lda + j] >= F.p;
    if (bt_block_or(bad, red)) {
      if (tid == 0) {
        ranks[b] = -1;
        status[b] = PLUQ_ERR_ENTRY_OUT_OF_RANGE;
      }
      continue;
    }
    for (int j = tid; j < ldS; j += kBatchThreads) ispiv[j] = 0;
    __syncthreads();
    int r = 0;
    for (int i0 = 0; i0 < m; i0 += kSlab) {
      const int bh = min(kSlab, m - i0);
      // 1. the slab, earlier pivot columns and columns >= n zeroed; first non-zeros
      for (int t = warp; t < kSlab; t += kBatchWarps) {
        const uint32_t* row = A + (int64_t)(i0 + t) * lda;
        uint32_t* st = S + (size_t)t * ldS;
        int fz = INT_MAX;
        for (int jb = 0; jb < ldS; jb += 32) {
          const int j = jb + lane;
          const uint32_t v = (t < bh && j < n && ispiv[j] == 0) ? row[j] : 0u;
          st[j] = v;
          const unsigned nz = __ballot_sync(0xffffffffu, v != 0u);
          if (nz && fz == INT_MAX) fz = jb + __ffs(nz) - 1;
        }
        if (lane == 0) first[t] = fz;
        Ls[t * kSlab + lane] = 0u;
      }
      __syncthreads();
      int nb = 0;
      for (int t = 0; t < bh; ++t) {
        const int js = first[t];
        if (js == INT_MAX) continue;  // row t of the slab is zero: no pivot
        const uint32_t* pr = S + (size_t)t * ldS;
        const uint32_t inv = f_inv(pr[js], F, inv_table);
        const uint32_t im = BF::to_mont(inv, F);
        for (int u = t + 1 + warp; u < bh; u += kBatchWarps) {
          uint32_t* ur = S + (size_t)u * ldS;
          const uint32_t w = ur[js];
          if (w == 0u) continue;  // unchanged; its first non-zero is not js
          const uint32_t l = BF::mulm(im, w, F);
          const uint32_t lm = BF::to_mont(l, F);
          int fz = INT_MAX;
          for (int jb = 0; jb < n; jb += 32) {
            const int j = jb + lane;
            uint32_t nv = 0u;
            if (j < n) {
              nv = f_sub(ur[j], BF::mulm(lm, pr[j], F), F);
              ur[j] = nv;
            }
            const unsigned nz = __ballot_sync(0xffffffffu, nv != 0u);
            if (nz && fz == INT_MAX) fz = jb + __ffs(nz) - 1;
          }
          if (lane == 0) {
            Ls[u * kSlab + nb] = l;
            first[u] = fz;
          }
        }
        if (tid == 0) {
          spr[nb] = t;
          spc[nb] = js;
          invm[nb] = im;
        }
        ++nb;
        __syncthreads();
      }
      for (int k = tid; k < nb; k += kBatchThreads) {
        prow[r + k] = i0 + spr[k];
        pcol[r + k] = spc[k];
        ispiv[spc[k]] = r + k + 1;
      }
      __syncthreads();
      // 2. back to the matrix
      for (int t = warp; t < bh; t += kBatchWarps) {
        uint32_t* row = A + (int64_t)(i0 + t) * lda;
        const uint32_t* st = S + (size_t)t * ldS;
        for (int j = lane; j < n; j += 32) {
          const int f = ispiv[j];
          if (f != 0 && f <= r) continue;  // an earlier pivot column: its multiplier stays
          uint32_t v = st[j];
          if (f > r && spr[f - r - 1] < t) v = Ls[t * kSlab + (f - r - 1)];
          row[j] = v;
        }
      }
      __syncthreads();
      if (nb > 0 && i0 + bh < m) {
        // 3. pivot rows to rows 0..nb-1 of S in Montgomery form (spr[k] >= k, so
        // each column is moved in place in increasing k)
        for (int j = tid; j < ldS; j += kBatchThreads)
          for (int k = 0; k < nb; ++k)
            S[(size_t)k * ldS + j] = BF::to_mont(S[(size_t)spr[k] * ldS + j], F);
        __syncthreads();
        for (int e = tid; e < nb * nb; e += kBatchThreads) {
          const int q = e / nb, k = e - q * nb;
          Ujj[q * (kSlab + 1) + k] = S[(size_t)q * ldS + spc[k]];
        }
        __syncthreads();
        for (int rb = i0 + bh; rb < m; rb += kRowBlock) {
          const int nr = min(kRowBlock, m - rb);
          if (tid < kRowBlock) {
            // multipliers of row rb + tid: L_k = (x_k - sum_{q<k} L_q U_q[j_k]) / U_k[j_k]
            if (tid < nr) {
              const uint32_t* ar = A + (int64_t)(rb + tid) * lda;
              for (int k = 0; k < nb; ++k) {
                const uint32_t x = ar[spc[k]];
                Dot<kMode> s;
                for (int q = 0; q < k; ++q) s.add(LT[q * kRowBlock + tid], Ujj[q * (kSlab + 1) + k], F);
                LT[k * kRowBlock + tid] = BF::mulm(invm[k], f_sub(x, s.value(F), F), F);
              }
            } else {
              for (int k = 0; k < nb; ++k) LT[k * kRowBlock + tid] = 0u;
            }
          }
          __syncthreads();
          // C <- C - L U; the slab's pivot columns take L
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
              for (int k = 0; k < nb; ++k) {
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
                    const uint32_t v = f > r ? LT[(f - r - 1) * kRowBlock + row]
                                             : f_sub(cv[i][jj], acc[i][jj].value(F), F);
                    A[(int64_t)(rb + row) * lda + col] = v;
                  }
                }
            }
          }
          __syncthreads();
        }
      }
      r += nb;
    }
    // P = [pivot rows, others ascending], Q likewise; gather through scratch
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
    for (int t = warp; t < m; t += kBatchWarps) {
      const uint32_t* src = A + (int64_t)rowpos[t] * lda;
      uint32_t* dst = SC + (size_t)t * n;
      for (int u = lane; u < n; u += 32) dst[u] = (t >= r && u >= r) ? 0u : src[colpos[u]];
    }
    __syncthreads();
    for (int t = warp; t < m; t += kBatchWarps) {
      const uint32_t* src = SC + (size_t)t * n;
      uint32_t* dst = A + (int64_t)t * lda;
      for (int u = lane; u < n; u += 32) dst[u] = src[u];
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

int slab_ld(int max_n) { return std::max(kTile, (int)cdiv(std::max(max_n, 1), kTile) * kTile); }

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
