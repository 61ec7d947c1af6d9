// Base case of the tile-recursive PLUQ: rank-profile-revealing elimination of
// one tile (at most kBM x kBN) held in shared memory by one CTA.
//
// The pivot of each step is the row-major first non-zero of the remaining
// (Schur-complement) tile, the search order of Sec. 4.1 that reveals the row
// rank profile; combined with the recursion's block order it reveals both
// profiles.  Rows that reduce to zero are skipped in one parallel scan instead
// of one step each, so a step costs O(1) barriers per pivot: warps own rows,
// each warp reports its first row with a non-zero entry on a non-pivot
// column, and the minimum over warps is the next pivot row.
//
// Output, in place: the tile becomes the compressed L\U of T' = P^T T Q^T with
//   P = [pivot rows in pivot order, other rows ascending]
//   Q = [pivot columns in pivot order, other columns ascending]
// (the other rows/columns must stay ascending so that the caller's recursive
// calls see them in their original order), the trailing block zero.  perm_r,
// perm_c receive P, Q as local index vectors and rank_out the rank.
#include <climits>

#include "common.cuh"

namespace {

constexpr int kBaseThreads = 512;
constexpr int kBaseWarps = kBaseThreads / 32;
constexpr int kBM = 128;
constexpr int kBN = 128;
constexpr int kSlots = kBN / 32;
constexpr size_t kBaseSmem =
    sizeof(uint32_t) * kBM * kBN + sizeof(int32_t) * (3 * kBM + 3 * kBN + 2 * kBaseWarps);

__global__ void __launch_bounds__(kBaseThreads)
    k_base_pluq(uint32_t* __restrict__ A, int64_t lda, int m, int n, FieldP F,
                const uint32_t* __restrict__ inv_table, int32_t* __restrict__ perm_r,
                int32_t* __restrict__ perm_c, int32_t* __restrict__ rank_out) {
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t* T = smem;                                   // [kBM][kBN]
  int32_t* prow = reinterpret_cast<int32_t*>(T + kBM * kBN);  // [kBM]
  int32_t* rowpos = prow + kBM;                         // [kBM]
  int32_t* isprow = rowpos + kBM;                       // [kBM]
  int32_t* pcol = isprow + kBM;                         // [kBN]
  int32_t* colpos = pcol + kBN;                         // [kBN]
  int32_t* ispcol = colpos + kBN;                       // [kBN]
  int32_t* cand = ispcol + kBN;                         // [2][kBaseWarps]

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned full = 0xffffffffu;

  for (int i = warp; i < m; i += kBaseWarps) {
    const uint32_t* src = A + (int64_t)i * lda;
    for (int j = lane; j < kBN; j += 32) T[i * kBN + j] = (j < n) ? src[j] : 0u;
  }
  for (int i = tid; i < kBM; i += kBaseThreads) isprow[i] = 0;
  for (int j = tid; j < kBN; j += kBaseThreads) ispcol[j] = 0;
  __syncthreads();

  // first candidate row of each warp: first owned row with a non-zero
  {
    int first = INT_MAX;
    for (int l = warp; l < m; l += kBaseWarps) {
      bool nz = false;
#pragma unroll
      for (int s = 0; s < kSlots; ++s) nz |= T[l * kBN + lane + 32 * s] != 0u;
      if (__any_sync(full, nz)) {
        first = l;
        break;
      }
    }
    if (lane == 0) cand[warp] = first;
  }
  __syncthreads();

  uint32_t mypiv = 0;  // bit s: column lane + 32 s is a pivot column
  int r = 0, buf = 0;
  while (true) {
    int istar = INT_MAX;
#pragma unroll
    for (int w = 0; w < kBaseWarps; ++w) istar = min(istar, cand[buf * kBaseWarps + w]);
    if (istar == INT_MAX) break;
    const uint32_t* Ti = T + istar * kBN;
    // pivot column: first non-zero of row istar outside the pivot columns
    int j0 = -1;
#pragma unroll
    for (int s = 0; s < kSlots; ++s) {
      const bool nz = !((mypiv >> s) & 1u) && Ti[lane + 32 * s] != 0u;
      const unsigned b = __ballot_sync(full, nz);
      if (b && j0 < 0) j0 = 32 * s + __ffs(b) - 1;
    }
    if (j0 < 0) break;  // unreachable: the candidate row has a non-zero off the pivots
    const uint32_t inv = f_inv(Ti[j0], F, inv_table);
    const uint32_t inv_m = f_to_mont(inv, F);
    uint32_t pv[kSlots];
#pragma unroll
    for (int s = 0; s < kSlots; ++s) pv[s] = Ti[lane + 32 * s];
    const int jslot = j0 >> 5, jlane = j0 & 31;
    if (lane == jlane) mypiv |= 1u << jslot;
    if (tid == 0) {
      prow[r] = istar;
      pcol[r] = j0;
    }
    int first = INT_MAX;
    for (int l = warp; l < m; l += kBaseWarps) {
      if (l <= istar) continue;
      uint32_t* Tl = T + l * kBN;
      const uint32_t wl = Tl[j0];
      __syncwarp();
      bool nz = false;
      if (wl != 0u) {
        const uint32_t cmul = f_mul_mont(inv_m, wl, F);  // multiplier L[l, r]
        const uint32_t cm = f_to_mont(cmul, F);
#pragma unroll
        for (int s = 0; s < kSlots; ++s) {
          const int j = lane + 32 * s;
          if (j == j0) {
            Tl[j] = cmul;
          } else if (!((mypiv >> s) & 1u)) {
            const uint32_t nv = f_sub(Tl[j], f_mul_mont(cm, pv[s], F), F);
            Tl[j] = nv;
            nz |= nv != 0u;
          }
        }
      } else {
#pragma unroll
        for (int s = 0; s < kSlots; ++s)
          nz |= !((mypiv >> s) & 1u) && Tl[lane + 32 * s] != 0u;
      }
      if (first == INT_MAX && __any_sync(full, nz)) first = l;
    }
    if (lane == 0) cand[(buf ^ 1) * kBaseWarps + warp] = first;
    __syncthreads();
    buf ^= 1;
    ++r;
  }

  // P = [pivot rows, other rows ascending], Q likewise
  for (int k = tid; k < r; k += kBaseThreads) {
    isprow[prow[k]] = 1;
    ispcol[pcol[k]] = 1;
    rowpos[k] = prow[k];
    colpos[k] = pcol[k];
  }
  __syncthreads();
  if (warp < 2) {
    const int cnt = warp == 0 ? m : n;
    const int32_t* flag = warp == 0 ? isprow : ispcol;
    int32_t* pos = warp == 0 ? rowpos : colpos;
    int base = r;
    for (int c0 = 0; c0 < cnt; c0 += 32) {
      const int i = c0 + lane;
      const bool np = i < cnt && !flag[i];
      const unsigned b = __ballot_sync(full, np);
      if (np) pos[base + __popc(b & ((1u << lane) - 1u))] = i;
      base += __popc(b);
    }
  }
  __syncthreads();
  if (r > 0) {
    for (int t = warp; t < m; t += kBaseWarps) {
      uint32_t* dst = A + (int64_t)t * lda;
      const uint32_t* src = T + rowpos[t] * kBN;
      for (int u = lane; u < n; u += 32) dst[u] = (t >= r && u >= r) ? 0u : src[colpos[u]];
    }
  }
  for (int t = tid; t < m; t += kBaseThreads) perm_r[t] = rowpos[t];
  for (int u = tid; u < n; u += kBaseThreads) perm_c[u] = colpos[u];
  if (tid == 0) rank_out[0] = r;
}

__global__ void k_inv_table(uint32_t* table, uint32_t p) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= p) return;
  table[a] = a == 0 ? 0u : f_inv_euclid((uint32_t)a, p);
}

}  // namespace

int launch_base_pluq(pluq_ctx* c, uint32_t* A, int64_t lda, int m, int n, int32_t* perm_r,
                     int32_t* perm_c, int32_t* rank_out) {
  // set once, thread-safely (function-local static initialisation)
  static const cudaError_t attr =
      cudaFuncSetAttribute(k_base_pluq, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBaseSmem);
  PLUQ_CUDA(attr);
  if (m > kBM || n > kBN || m <= 0 || n <= 0) return PLUQ_ERR_INVALID_ARG;
  ProfScope ps(c, PC_BASE, 0, 8.0 * m * n);
  k_base_pluq<<<1, kBaseThreads, kBaseSmem, c->stream>>>(A, lda, m, n, c->F, inv_table_ptr(c),
                                                        perm_r, perm_c, rank_out);
  PLUQ_CUDA(cudaGetLastError());
  return PLUQ_OK;
}

// Inverse table for p below 2^22 (16 MiB): one load replaces a Euclid chain.
constexpr uint32_t kInvTableMaxP = 1u << 22;

int ensure_inv_table(pluq_ctx* c) {
  const uint32_t p = c->F.p;
  if (p >= kInvTableMaxP || p == 2) return PLUQ_OK;
  if (c->inv_table_p == p) return PLUQ_OK;
  PLUQ_TRY(c->inv_table.ensure(sizeof(uint32_t) * p));
  ProfScope ps(c, PC_OTHER, 0, 4.0 * p);
  k_inv_table<<<(unsigned)cdiv(p, 256), 256, 0, c->stream>>>(c->inv_table.as<uint32_t>(), p);
  PLUQ_CUDA(cudaGetLastError());
  c->inv_table_p = p;
  return PLUQ_OK;
}

const uint32_t* inv_table_ptr(pluq_ctx* c) {
  return (c->inv_table_p == c->F.p && c->inv_table.ptr) ? c->inv_table.as<uint32_t>() : nullptr;
}
