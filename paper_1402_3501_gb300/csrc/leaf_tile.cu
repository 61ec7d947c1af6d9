// One-CTA leaf for primes below 2^16: rank-profile-revealing elimination of a
// block of up to 256 x 256 residues held as 16-bit words in the shared memory
// of one CTA (128 KiB), the base case of the tile recursion (Sec. 4.1) for
// small fields.
//
// Pivot search as in the other leaves: the next pivot is the row-major first
// non-zero of the remaining Schur complement (the search of Sec. 4.1 that
// reveals the row rank profile).  Warp w owns rows w, w + 32, ...; after each
// step every warp reports its first owned row (below the pivot) with a
// non-zero outside the pivot columns, and the minimum over the 32 reports is
// the next pivot row, so rows that reduce to zero cost nothing more and one
// block barrier is taken per pivot.  A row is updated in chunks of eight
// columns (one 16-byte shared-memory word); a warp spreads the (row, chunk)
// pairs of its rows below the pivot over its lanes, taking only the chunks
// from the first one that still holds a non-pivot column, so the work of a
// step follows the live part of the Schur complement.
//
// Products c x mod p (c, x < 2^16, so c x < 2^32) are reduced by Barrett's
// method with mu = floor(2^32 / p): q = floor(c x mu / 2^32) undershoots the
// quotient by at most 2, so r = c x - q p needs at most two corrections.
//
// Output as the other leaves: the block becomes the compressed L\U of
// P^T X Q^T with P = [pivot rows, other rows ascending], Q likewise, and
// perm_r / perm_c / rank_out receive the local index vectors and the rank.
#include <algorithm>
#include <climits>

#include "common.cuh"

namespace {

constexpr int kTileMax = 256;
constexpr int kTileThreads = 1024;
constexpr int kTileWarps = kTileThreads / 32;
constexpr int kTileRowsPerWarp = kTileMax / kTileWarps;  // 8
constexpr size_t kTileSmem = sizeof(uint16_t) * kTileMax * kTileMax +
                             sizeof(int32_t) * (4 * kTileMax + 2 * kTileWarps);

struct Barrett16 {
  uint32_t p, mu;  // mu = floor(2^32 / p)
  __device__ __forceinline__ uint32_t mul(uint32_t a, uint32_t b) const {
    const uint32_t x = a * b;  // < 2^32
    const uint32_t q = __umulhi(x, mu);
    uint32_t r = x - q * p;
    r = r >= p ? r - p : r;
    return r >= p ? r - p : r;
  }
  __device__ __forceinline__ uint32_t sub(uint32_t a, uint32_t b) const {
    return a >= b ? a - b : a + p - b;
  }
};

__device__ __forceinline__ void unpack8(const uint4 v, uint32_t (&x)[8]) {
  x[0] = v.x & 0xFFFFu; x[1] = v.x >> 16;
  x[2] = v.y & 0xFFFFu; x[3] = v.y >> 16;
  x[4] = v.z & 0xFFFFu; x[5] = v.z >> 16;
  x[6] = v.w & 0xFFFFu; x[7] = v.w >> 16;
}

__device__ __forceinline__ uint4 pack8(const uint32_t (&x)[8]) {
  return make_uint4(x[0] | (x[1] << 16), x[2] | (x[3] << 16), x[4] | (x[5] << 16),
                    x[6] | (x[7] << 16));
}

__global__ void __launch_bounds__(kTileThreads, 1)
    k_leaf_tile16(uint32_t* __restrict__ X, int64_t ldx, int m, int n, uint32_t p, uint32_t mu,
                  const uint32_t* __restrict__ inv_table, int32_t* __restrict__ perm_r,
                  int32_t* __restrict__ perm_c, int32_t* __restrict__ rank_out) {
  extern __shared__ __align__(16) uint8_t tile_smem[];
  uint16_t* T = reinterpret_cast<uint16_t*>(tile_smem);  // [256][256]
  int32_t* prow = reinterpret_cast<int32_t*>(T + kTileMax * kTileMax);  // [256]
  int32_t* pcol = prow + kTileMax;                                      // [256]
  int32_t* rowpos = pcol + kTileMax;                                    // [256]
  int32_t* colpos = rowpos + kTileMax;                                  // [256]
  int32_t* cand = colpos + kTileMax;                                    // [2][32]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned full = 0xffffffffu;
  const Barrett16 B{p, mu};
  const int c0 = lane * 8;  // this lane's eight columns

  // load the block (zero padded to 256 columns): rows by warps, 8 columns a lane
  for (int i = warp; i < kTileMax; i += kTileWarps) {
    uint32_t x[8];
    const uint32_t* src = X + (int64_t)i * ldx;
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = (i < m && c0 + q < n) ? __ldg(src + c0 + q) : 0u;
    *reinterpret_cast<uint4*>(T + i * kTileMax + c0) = pack8(x);
  }
  __syncthreads();
  // each warp's first owned row with a non-zero
  {
    int first = INT_MAX;
    for (int k = 0; k < kTileRowsPerWarp; ++k) {
      const int l = warp + k * kTileWarps;
      if (l >= m) break;
      const uint4 v = *reinterpret_cast<const uint4*>(T + l * kTileMax + c0);
      if (__any_sync(full, (v.x | v.y | v.z | v.w) != 0u)) {
        first = l;
        break;
      }
    }
    if (lane == 0) cand[warp] = first;
  }
  __syncthreads();

  // lane c holds the pivot-column mask of chunk c (columns [8c, 8c + 8));
  // chunks past the last column count as fully eliminated
  const int nchunk = (n + 7) / 8;
  uint32_t pivmask = lane < nchunk ? 0u : 0xFFu;
  int r = 0, buf = 0;
  while (true) {
    // elected row: the smallest report
    int istar = cand[buf * kTileWarps + lane];
    for (int o = 16; o > 0; o >>= 1) istar = min(istar, __shfl_xor_sync(full, istar, o));
    if (istar == INT_MAX) break;
    const uint16_t* Ti = T + istar * kTileMax;
    uint32_t pv[8];
    unpack8(*reinterpret_cast<const uint4*>(Ti + c0), pv);
    // pivot column: first non-zero of the row outside the pivot columns
    int local = 8;
#pragma unroll
    for (int q = 7; q >= 0; --q)
      if (pv[q] != 0u && !((pivmask >> q) & 1u)) local = q;
    const unsigned bal = __ballot_sync(full, local < 8);
    const int src = __ffs(bal) - 1;
    const int jl = __shfl_sync(full, local, src);  // the pivot's slot in chunk src
    const int j0 = 8 * src + jl;
    uint32_t mine = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (q == jl) mine = pv[q];
    const uint32_t piv = __shfl_sync(full, mine, src);
    const uint32_t inv =
        p == 2 ? 1u : (inv_table ? __ldg(inv_table + piv) : f_inv_euclid(piv, p));
    // live chunks [lo, nchunk): before lo every column was a pivot column
    // before this step (chunk src, whose last live column may be the new pivot,
    // still receives the multipliers)
    const unsigned live = __ballot_sync(full, pivmask != 0xFFu);
    const int lo = live ? __ffs(live) - 1 : nchunk;
    const int nlive = nchunk - lo;
    if (lane == src) pivmask |= 1u << jl;
    if (tid == 0) {
      prow[r] = istar;
      pcol[r] = j0;
    }
    // this warp's rows below the pivot row: l_k = warp + 32 (kb + k), k < nr;
    // lane k computes row k's multiplier (its L entry)
    const int kb = istar < warp ? 0 : (istar - warp) / kTileWarps + 1;
    const int nr = max(0, min(kTileRowsPerWarp, (m - warp + kTileWarps - 1) / kTileWarps) - kb);
    uint32_t cm_mine = 0;
    if (lane < nr) cm_mine = B.mul(T[(warp + kTileWarps * (kb + lane)) * kTileMax + j0], inv);
    __syncwarp();  // every multiplier is read before chunk src is rewritten
    // (row, chunk) items of this warp over the live chunks only
    uint32_t rownz = 0;  // bit k: row k keeps a non-zero outside the pivot columns
    const int items = nr * nlive;
    for (int t0 = 0; t0 < items; t0 += 32) {
      const int t = t0 + lane;
      const int k = t < items ? t / nlive : 0;
      const int ch = t < items ? lo + (t - k * nlive) : 0;
      const uint32_t cm = __shfl_sync(full, cm_mine, k);
      const uint32_t mask = __shfl_sync(full, pivmask, ch);
      if (t < items) {
        uint16_t* Tl = T + (warp + kTileWarps * (kb + k)) * kTileMax + 8 * ch;
        uint32_t x[8];
        unpack8(*reinterpret_cast<const uint4*>(Tl), x);
        bool nz = false;
        if (cm != 0u) {
          uint32_t y[8];
          unpack8(*reinterpret_cast<const uint4*>(Ti + 8 * ch), y);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            if ((mask >> q) & 1u) continue;  // L entries and the new pivot column
            x[q] = B.sub(x[q], B.mul(cm, y[q]));
            nz |= x[q] != 0u;
          }
          if (ch == src) {
#pragma unroll
            for (int q = 0; q < 8; ++q)
              if (q == jl) x[q] = cm;
          }
          *reinterpret_cast<uint4*>(Tl) = pack8(x);
        } else {
#pragma unroll
          for (int q = 0; q < 8; ++q) nz |= !((mask >> q) & 1u) && x[q] != 0u;
        }
        if (nz) rownz |= 1u << k;
      }
    }
    rownz = __reduce_or_sync(full, rownz);
    const int first = rownz ? warp + kTileWarps * (kb + __ffs(rownz) - 1) : INT_MAX;
    if (lane == 0) cand[(buf ^ 1) * kTileWarps + warp] = first;
    __syncthreads();
    buf ^= 1;
    ++r;
  }

  // P = [pivot rows in pivot order, other rows ascending], Q likewise
  __shared__ uint32_t rbits[kTileMax / 32], cbits[kTileMax / 32];
  if (tid < kTileMax / 32) {
    rbits[tid] = 0u;
    cbits[tid] = 0u;
  }
  __syncthreads();
  for (int k = tid; k < r; k += kTileThreads) {
    atomicOr(&rbits[prow[k] >> 5], 1u << (prow[k] & 31));
    atomicOr(&cbits[pcol[k] >> 5], 1u << (pcol[k] & 31));
    rowpos[k] = prow[k];
    colpos[k] = pcol[k];
  }
  __syncthreads();
  if (warp < 2) {
    const int cnt = warp == 0 ? m : n;
    const uint32_t* bits = warp == 0 ? rbits : cbits;
    int32_t* pos = warp == 0 ? rowpos : colpos;
    int base = r;
    for (int s0 = 0; s0 < cnt; s0 += 32) {
      const int i = s0 + lane;
      const bool np = i < cnt && !((bits[i >> 5] >> (i & 31)) & 1u);
      const unsigned b = __ballot_sync(full, np);
      if (np) pos[base + __popc(b & ((1u << lane) - 1u))] = i;
      base += __popc(b);
    }
  }
  __syncthreads();
  for (int t = warp; t < m; t += kTileWarps) {
    uint32_t* dst = X + (int64_t)t * ldx;
    const uint16_t* srow = T + rowpos[t] * kTileMax;
    for (int u = lane; u < n; u += 32) dst[u] = (t >= r && u >= r) ? 0u : srow[colpos[u]];
  }
  for (int t = tid; t < m; t += kTileThreads) perm_r[t] = rowpos[t];
  for (int u = tid; u < n; u += kTileThreads) perm_c[u] = colpos[u];
  if (tid == 0) rank_out[0] = r;
}

}  // namespace

// Whether the one-CTA 16-bit leaf takes an m x n block: p < 2^16 and both
// sides within 256 (and within the context's leaf cut-off).
int tile_leaf_fits(pluq_ctx* c, int64_t m, int64_t n) {
  return c->F.p < (1u << 16) && m > 0 && n > 0 && m <= kTileMax && n <= kTileMax &&
         m <= std::max(c->leaf_dim, 1) && n <= std::max(c->leaf_dim, 1);
}

int launch_leaf_tile(pluq_ctx* c, uint32_t* X, int64_t ldx, int m, int n, int32_t* perm_r,
                     int32_t* perm_c, int32_t* rank_out) {
  static const cudaError_t attr = cudaFuncSetAttribute(
      k_leaf_tile16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmem);
  PLUQ_CUDA(attr);
  if (!tile_leaf_fits(c, m, n)) return PLUQ_ERR_INVALID_ARG;
  const uint32_t p = c->F.p;
  const uint32_t mu = (uint32_t)((((uint64_t)1) << 32) / p);
  ProfScope ps(c, PC_BASE, 0, 8.0 * m * n);
  k_leaf_tile16<<<1, kTileThreads, kTileSmem, c->stream>>>(X, ldx, m, n, p, mu, inv_table_ptr(c),
                                                          perm_r, perm_c, rank_out);
  PLUQ_CUDA(cudaGetLastError());
  return PLUQ_OK;
}
