// Batched PLUQ: many independent matrices (each at most kBatchMax x kBatchMax)
// factored by one persistent launch.
//
// CTAs take matrices from an atomic work counter in an order the host sorts by
// decreasing work (m n min(m, n)), so the longest factorizations start first.
// One CTA factors one matrix with the rank-profile-revealing elimination of
// Sec. 4.1: the next pivot is the row-major first non-zero of the Schur
// complement.  The matrix stays in global memory (it is L2-resident while its
// CTA works on it); each row's first non-zero column outside the pivot columns
// is kept in shared memory and refreshed as the row is eliminated, so rows
// that become zero cost nothing further.  L multipliers overwrite the pivot
// column entries; the final P^T A Q^T layout is gathered through the CTA's
// scratch and copied back.  Entries >= p mark the matrix with
// PLUQ_ERR_ENTRY_OUT_OF_RANGE and leave it untouched.
#include <algorithm>
#include <climits>
#include <numeric>
#include <vector>

#include "common.cuh"

namespace {

constexpr int kBatchThreads = 512;
constexpr int kBatchWarps = kBatchThreads / 32;
constexpr int kBatchMax = 1024;
constexpr int kUnroll = 8;          // row loads in flight per lane
constexpr int kBatchCtasPerSm = 2;  // co-resident CTAs hide L2 latency

struct BatchDesc {
  uint32_t* A;
  int32_t* P;
  int32_t* Q;
  int64_t lda;
  int32_t m, n;
};

__device__ __forceinline__ int bt_block_min(int v, int* red) {
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  int out = INT_MAX;
  for (int w = 0; w < kBatchWarps; ++w) out = min(out, red[w]);
  return out;
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

template <bool kIs2>
__device__ __forceinline__ uint32_t bt_mulm(uint32_t cm, uint32_t w, const FieldP& F) {
  if (kIs2) return cm & w;
  return f_redc((uint64_t)cm * w, F);
}

template <bool kIs2>
__global__ void __launch_bounds__(kBatchThreads, kBatchCtasPerSm)
    k_batched_pluq(const BatchDesc* __restrict__ descs, const int32_t* __restrict__ order,
                   int batch, int* __restrict__ counter, FieldP F,
                   const uint32_t* __restrict__ inv_table, uint32_t* __restrict__ scratch,
                   size_t scratch_per_cta, int64_t* __restrict__ ranks,
                   int32_t* __restrict__ status) {
  __shared__ int32_t first[kBatchMax];   // first non-zero column per row (INT_MAX: none)
  __shared__ uint32_t piv[kBatchMax];    // current pivot row, pivot columns zeroed
  __shared__ int32_t ispiv[kBatchMax];
  __shared__ int32_t isprow[kBatchMax];
  __shared__ int32_t rowpos[kBatchMax];
  __shared__ int32_t colpos[kBatchMax];
  __shared__ int32_t prow[kBatchMax];
  __shared__ int32_t pcol[kBatchMax];
  __shared__ int red[kBatchWarps];
  __shared__ int s_idx;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t* S = scratch + (size_t)blockIdx.x * scratch_per_cta;

  while (true) {
    if (tid == 0) s_idx = atomicAdd(counter, 1);
    __syncthreads();
    const int idx = s_idx;
    __syncthreads();
    if (idx >= batch) break;
    const int b = order[idx];
    const BatchDesc d = descs[b];
    const int m = d.m, n = d.n, mn = min(m, n);
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
    for (int j = tid; j < n; j += kBatchThreads) ispiv[j] = 0;
    for (int l = warp; l < m; l += kBatchWarps) {
      const uint32_t* row = A + (int64_t)l * lda;
      int fz = INT_MAX;
      for (int jb = 0; jb < n; jb += 32) {
        const int j = jb + lane;
        const unsigned bb = __ballot_sync(0xffffffffu, j < n && row[j] != 0u);
        if (bb) {
          fz = jb + __ffs(bb) - 1;
          break;
        }
      }
      if (lane == 0) first[l] = fz;
    }
    __syncthreads();
    int r = 0, cursor = 0;
    while (r < mn) {
      int cand = INT_MAX;
      for (int l = cursor + tid; l < m; l += kBatchThreads)
        if (first[l] != INT_MAX) {
          cand = l;
          break;
        }
      const int istar = bt_block_min(cand, red);
      if (istar == INT_MAX) break;
      const int j0 = first[istar];
      const uint32_t* prow_g = A + (int64_t)istar * lda;
      for (int j = tid; j < n; j += kBatchThreads) piv[j] = ispiv[j] ? 0u : prow_g[j];
      __syncthreads();
      const uint32_t inv = f_inv(piv[j0], F, inv_table);
      const uint32_t inv_m = f_to_mont(inv, F);
      if (tid == 0) {
        prow[r] = istar;
        pcol[r] = j0;
        ispiv[j0] = 1;
        first[istar] = INT_MAX;
      }
      // eliminate the rows below the pivot row
      for (int l = istar + 1 + warp; l < m; l += kBatchWarps) {
        uint32_t* row = A + (int64_t)l * lda;
        const uint32_t wl = row[j0];
        __syncwarp();
        if (wl == 0u) continue;  // unchanged; its first non-zero is not j0
        const uint32_t cmul = bt_mulm<kIs2>(inv_m, wl, F);
        const uint32_t cm = f_to_mont(cmul, F);
        int fz = INT_MAX;
        // eight loads in flight per lane before the dependent updates
        for (int jb0 = 0; jb0 < n; jb0 += 32 * kUnroll) {
          uint32_t v[kUnroll];
#pragma unroll
          for (int q = 0; q < kUnroll; ++q) {
            const int j = jb0 + 32 * q + lane;
            v[q] = j < n ? row[j] : 0u;
          }
#pragma unroll
          for (int q = 0; q < kUnroll; ++q) {
            const int j = jb0 + 32 * q + lane;
            bool nz = false;
            if (j < n) {
              const uint32_t nv = f_sub(v[q], bt_mulm<kIs2>(cm, piv[j], F), F);
              row[j] = nv;
              nz = nv != 0u && j != j0 && !ispiv[j];
            }
            const unsigned bb = __ballot_sync(0xffffffffu, nz);
            if (bb && fz == INT_MAX) fz = jb0 + 32 * q + __ffs(bb) - 1;
          }
        }
        __syncwarp();
        if (lane == 0) {
          row[j0] = cmul;
          first[l] = fz;
        }
      }
      __syncthreads();
      cursor = istar + 1;
      ++r;
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
      uint32_t* dst = S + (size_t)t * n;
      for (int u = lane; u < n; u += 32) dst[u] = (t >= r && u >= r) ? 0u : src[colpos[u]];
    }
    __syncthreads();
    for (int t = warp; t < m; t += kBatchWarps) {
      const uint32_t* src = S + (size_t)t * n;
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

}  // namespace

int batched_max_dim() { return kBatchMax; }

// Persistent launch over `count` matrices already described on the device.
int launch_batched(pluq_ctx* c, const void* descs, const int32_t* order, int count,
                   int64_t* ranks, int32_t* status, int max_elems) {
  int* counter = c->small.as<int>() + 24;
  const int G = c->sm_count * kBatchCtasPerSm;
  const size_t per = (size_t)std::max(max_elems, 1);
  PLUQ_TRY(c->batch_scratch.ensure(sizeof(uint32_t) * per * G));
  {
    ProfScope pr(c, PC_INDEX);
    k_batch_reset<<<1, 1, 0, c->stream>>>(counter);
  }
  ProfScope ps(c, PC_BASE);
  const auto* d = static_cast<const BatchDesc*>(descs);
  if (c->F.is2)
    k_batched_pluq<true><<<G, kBatchThreads, 0, c->stream>>>(
        d, order, count, counter, c->F, inv_table_ptr(c), c->batch_scratch.as<uint32_t>(), per, ranks,
        status);
  else
    k_batched_pluq<false><<<G, kBatchThreads, 0, c->stream>>>(
        d, order, count, counter, c->F, inv_table_ptr(c), c->batch_scratch.as<uint32_t>(), per, ranks,
        status);
  PLUQ_CUDA(cudaGetLastError());
  return PLUQ_OK;
}

size_t batched_desc_size() { return sizeof(BatchDesc); }

void batched_fill_desc(void* out, int i, uint32_t* A, int32_t* P, int32_t* Q, int64_t lda, int m,
                       int n) {
  static_cast<BatchDesc*>(out)[i] = BatchDesc{A, P, Q, lda, m, n};
}

int batched_ctas_per_sm() { return kBatchCtasPerSm; }
