// Leaves of the tile-recursive PLUQ on one thread-block cluster.
//
// The elimination is the one of the cooperative barrier leaf: each step takes
// the row-major first non-zero of the remaining Schur complement as the pivot
// (the pivot search of Sec. 4.1), so the result is the same rank-profile-
// revealing L\U.  Here the block is held by the G <= 16 CTAs of a single
// cluster (row l in CTA l mod G, in shared memory), and a step synchronises
// with one hardware cluster barrier instead of a grid barrier in global
// memory: every CTA leaves its candidate (its first row with a live column,
// that column and the inverse of the entry there) in its own shared memory;
// after the barrier every CTA reads the G candidates, then copies the elected
// row right of its pivot column from the winner's shared memory into its own
// (distributed shared memory), with no L2 round trip on the way.
//
// Storage per residue: 16 bits for p < 2^16, a 16-bit and an 8-bit plane for
// p < 2^24, else 32 bits, so that a 1024 x 1024 block fits the shared memory
// of 16 SMs for p < 2^24 (n <= 1024: thread tid of 1024 copies column tid of
// the elected row).  The row updates run over work items of 4 active rows by
// 64 columns, one warp each, with Shoup's precomputed-quotient products; the
// first live column of an updated row is found afterwards, inside the first
// 64-column chunk the update left non-zero (a per-row chunk mask).
//
// There is no wait on a memory word: the cluster barrier is a hardware barrier
// and every CTA passes it the same number of times (the loop ends on the
// elected row, which all CTAs read alike).  Output as the other leaves: the
// block becomes the compressed L\U of P^T X Q^T, P = [pivot rows, other rows
// ascending] and Q likewise, with perm_r / perm_c / rank_out as local index
// vectors.
#include <cooperative_groups.h>

#include <algorithm>
#include <climits>
#include <mutex>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int kClThreads = 1024;
constexpr int kClWarps = kClThreads / 32;
constexpr int kClCols = 1;                     // columns per thread
constexpr int kClMaxDim = kClThreads * kClCols;  // rows and columns, at most
constexpr int kClMaxRows = 128;                // owned rows per CTA, at most
constexpr int kClMaxCtas = 16;
constexpr int kClGroup = 4;                  // rows per elimination work item
constexpr int kClChunk = 64;                 // columns per elimination work item
constexpr uint32_t kPivFlag = 0x80000000u;   // pivot column in the elected-row copy

// The CTA's dynamic shared memory (the regions of ClLayout).
extern __shared__ __align__(16) unsigned char cl_smem[];

// Residue storage of the owned rows: 0: uint32; 1: uint16 (p < 2^16);
// 2: uint16 low plane and uint8 high plane (p < 2^24).  Indexed from the
// shared array itself (byte offsets of the planes), so that every access is
// a shared-memory access; peer() gives generic pointers into the same rows of
// another CTA of the cluster.
template <int kStore>
struct ClRows {
  uint32_t lo_off = 0, hi_off = 0;  // byte offsets of the planes in cl_smem
  int ns = 0;                       // row stride (elements)

  __device__ __forceinline__ uint32_t ld(int lr, int j) const {
    const int i = lr * ns + j;
    if (kStore == 0) return reinterpret_cast<const uint32_t*>(cl_smem + lo_off)[i];
    const uint32_t l = reinterpret_cast<const uint16_t*>(cl_smem + lo_off)[i];
    if (kStore == 1) return l;
    return l | ((uint32_t)(cl_smem + hi_off)[i] << 16);
  }
  __device__ __forceinline__ void st(int lr, int j, uint32_t v) const {
    const int i = lr * ns + j;
    if (kStore == 0) {
      reinterpret_cast<uint32_t*>(cl_smem + lo_off)[i] = v;
      return;
    }
    reinterpret_cast<uint16_t*>(cl_smem + lo_off)[i] = (uint16_t)v;
    if (kStore == 2) (cl_smem + hi_off)[i] = (uint8_t)(v >> 16);
  }

  struct Peer {
    const void* lo;
    const uint8_t* hi;
    int ns;
    __device__ __forceinline__ uint32_t ld(int lr, int j) const {
      const int i = lr * ns + j;
      if (kStore == 0) return static_cast<const uint32_t*>(lo)[i];
      const uint32_t l = static_cast<const uint16_t*>(lo)[i];
      if (kStore == 1) return l;
      return l | ((uint32_t)hi[i] << 16);
    }
  };
  // the same rows in the shared memory of CTA `rank` of the cluster
  __device__ __forceinline__ Peer peer(const cg::cluster_group& cl, unsigned rank) const {
    Peer o;
    o.ns = ns;
    o.lo = cl.map_shared_rank(static_cast<void*>(cl_smem + lo_off), rank);
    o.hi = kStore == 2 ? static_cast<const uint8_t*>(
                             cl.map_shared_rank(static_cast<void*>(cl_smem + hi_off), rank))
                       : nullptr;
    return o;
  }
};

// Byte offsets of the dynamic shared memory regions.
struct ClLayout {
  size_t lo, hi, pivrow, colpos, prow, pcol, fcol, posk, total;
};

__host__ __device__ inline size_t cl_align(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline ClLayout cl_layout(int m, int n, int G, int store) {
  const int rown = (m + G - 1) / G;
  const int ns = (n + 15) & ~15;
  const int mn = m < n ? m : n;
  ClLayout L;
  size_t o = 0;
  L.lo = o;
  o = cl_align(o + (size_t)rown * ns * (store == 0 ? 4 : 2));
  L.hi = o;
  if (store == 2) o = cl_align(o + (size_t)rown * ns);
  L.pivrow = o;
  o = cl_align(o + sizeof(uint32_t) * n);
  L.colpos = o;
  o = cl_align(o + sizeof(int32_t) * n);
  L.prow = o;
  o = cl_align(o + sizeof(int32_t) * mn);
  L.pcol = o;
  o = cl_align(o + sizeof(int32_t) * mn);
  L.fcol = o;
  o = cl_align(o + sizeof(int32_t) * rown);
  L.posk = o;
  o = cl_align(o + sizeof(int32_t) * rown);
  L.total = o;
  return L;
}

// Products by a fixed multiplier c < p with Shoup's precomputed quotient
// (V. Shoup, NTL's MulModPrecon): c' = floor(c 2^32 / p); for any 32-bit x,
// q = floor(x c' / 2^32) is floor(x c / p) or one less, so x c - q p lies in
// [0, 2p) and is exact in 32-bit wrap-around arithmetic (p < 2^31).
// c' from pinv64 = floor((2^64 - 1) / p), which is within one of 2^64 / p:
// the estimate floor(c 2^32 pinv64 / 2^64) is c' or c' - 1, fixed by one
// comparison.
__device__ __forceinline__ uint32_t shoup_pre(uint32_t c, uint32_t p, uint64_t pinv64) {
  const uint64_t x = (uint64_t)c << 32;
  uint64_t e = __umul64hi(x, pinv64);
  if (x - e * p >= p) ++e;
  return (uint32_t)e;
}

__device__ __forceinline__ uint32_t shoup_mul(uint32_t x, uint32_t c, uint32_t cpre, uint32_t p) {
  const uint32_t t = x * c - __umulhi(x, cpre) * p;  // [0, 2p)
  return min(t, t - p);
}

// a - b mod p for a, b < p
__device__ __forceinline__ uint32_t sub_mod(uint32_t a, uint32_t b, uint32_t p) {
  const uint32_t d = a - b;
  return min(d, d + p);
}

// pivots among the first i rows (columns): mask bits below i plus the prefix
// count of the whole words before
__device__ __forceinline__ int count_below(const unsigned* mask, const int* pre, int i) {
  return pre[i >> 5] + __popc(mask[i >> 5] & ((1u << (i & 31)) - 1u));
}

template <int kStore>
__global__ void __launch_bounds__(kClThreads, 1)
    k_leaf_cluster(uint32_t* __restrict__ X, int64_t ldx, int m, int n, FieldP F,
                   uint64_t pinv64, const uint32_t* __restrict__ inv_table, int32_t* __restrict__ perm_r,
                   int32_t* __restrict__ perm_c, int32_t* __restrict__ rank_out) {
  __shared__ int4 s_cand[2];  // (global row, column, inverse of the entry, owned index) by parity
  __shared__ int4 s_win;      // the elected candidate
  // active rows of a step: (owned row | bit 16 when its first live column
  // must be found again, multiplier c, Shoup's c', unused)
  __shared__ int4 s_act[kClMaxRows];
  __shared__ int s_nact;
  __shared__ unsigned s_nz[kClMaxRows];  // per active row: chunks left with a live non-zero
  __shared__ unsigned s_pmask[32];       // pivot columns
  __shared__ unsigned s_rmask[32];
  __shared__ int s_rpre[33], s_cpre[33];

  const cg::cluster_group cl = cg::this_cluster();
  const int G = (int)cl.num_blocks();
  const int g = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int mn = min(m, n);
  const ClLayout Lo = cl_layout(m, n, G, kStore);
  ClRows<kStore> W;
  W.ns = (n + 15) & ~15;
  W.lo_off = (uint32_t)Lo.lo;
  W.hi_off = (uint32_t)Lo.hi;
  uint32_t* pivrow = reinterpret_cast<uint32_t*>(cl_smem + Lo.pivrow);
  int32_t* colpos = reinterpret_cast<int32_t*>(cl_smem + Lo.colpos);
  int32_t* prow = reinterpret_cast<int32_t*>(cl_smem + Lo.prow);
  int32_t* pcol = reinterpret_cast<int32_t*>(cl_smem + Lo.pcol);
  int32_t* fcol = reinterpret_cast<int32_t*>(cl_smem + Lo.fcol);
  int32_t* posk = reinterpret_cast<int32_t*>(cl_smem + Lo.posk);
  const int owned = m > g ? (m - 1 - g) / G + 1 : 0;  // rows l = lr G + g < m

  // owned rows into shared memory, eight loads in flight per lane
  for (int lr = warp; lr < owned; lr += kClWarps) {
    const uint32_t* src = X + (int64_t)(lr * G + g) * ldx;
    for (int j0 = lane; j0 < n; j0 += 32 * 8) {
      uint32_t v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = j0 + 32 * q < n ? __ldcg(src + j0 + 32 * q) : 0u;
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (j0 + 32 * q < n) W.st(lr, j0 + 32 * q, v[q]);
    }
  }
  for (int i = tid; i < 32; i += kClThreads) s_rmask[i] = s_pmask[i] = 0u;
  __syncthreads();
  // fcol[lr]: first non-zero column of owned row lr outside the pivot columns
  // (INT_MAX: none left, or the row became a pivot row)
  for (int lr = warp; lr < owned; lr += kClWarps) {
    int jl = INT_MAX;
    for (int j = lane; j < n; j += 32)
      if (W.ld(lr, j) != 0u) {
        jl = j;
        break;
      }
    jl = __reduce_min_sync(0xffffffffu, jl);
    if (lane == 0) {
      fcol[lr] = jl;
      posk[lr] = -1;
    }
  }
  bool mypiv[kClCols];
#pragma unroll
  for (int c = 0; c < kClCols; ++c) mypiv[c] = false;
  // every CTA of the cluster has loaded its rows (X is overwritten at the
  // end) and runs before any distributed shared memory access
  cl.sync();

  int r = 0;
  for (int k = 0;; ++k) {
    const int par = k & 1;
    // this CTA's candidate: its first owned row with a live column
    if (warp == 0) {
      int first = INT_MAX;
      for (int b0 = 0; b0 < owned; b0 += 32) {
        const int lr = b0 + lane;
        const unsigned hit = __ballot_sync(0xffffffffu, lr < owned && fcol[lr] != INT_MAX);
        if (hit) {
          first = b0 + __ffs(hit) - 1;
          break;
        }
      }
      if (lane == 0) {
        int4 cd = make_int4(INT_MAX, 0, 0, 0);
        if (first != INT_MAX) {
          const int j = fcol[first];
          cd = make_int4(first * G + g, j, (int)f_inv(W.ld(first, j), F, inv_table), first);
        }
        s_cand[par] = cd;
        s_nact = 0;
      }
    }
    // one cluster barrier a step; the candidate slots are double-buffered by
    // step parity, so slot par is rewritten two barriers after it was read
    cl.sync();
    if (warp == 0) {
      int4 cd = make_int4(INT_MAX, 0, 0, 0);
      if (lane < G) cd = *cl.map_shared_rank(&s_cand[par], (unsigned)lane);
      const int best = __reduce_min_sync(0xffffffffu, cd.x);
      if (lane == 0 && best == INT_MAX) s_win = cd;
      if (best != INT_MAX && cd.x == best) s_win = cd;  // rows are distinct: one lane
    }
    __syncthreads();
    const int4 w = s_win;
    if (w.x == INT_MAX || r >= mn) break;
    const int istar = w.x, j0 = w.y, lrw = w.w;
    const int wr = istar % G;
    // rows to eliminate: owned rows below the pivot row with a non-zero in its
    // column (one thread a row), with their multipliers; rows whose first
    // live column lies left of the pivot column keep it (bit 16 clear).  The
    // list order does not matter: one slot per warp from a shared counter.
    if (tid < ((owned + 31) & ~31)) {
      const uint32_t pinv = (uint32_t)w.z;
      const int lr = tid;
      bool act = false;
      int4 e = make_int4(0, 0, 0, 0);
      if (lr < owned && lr * G + g > istar) {
        const uint32_t wl = W.ld(lr, j0);
        if (wl != 0u) {
          act = true;
          const uint32_t cmul = shoup_mul(wl, pinv, shoup_pre(pinv, F.p, pinv64), F.p);
          e = make_int4(lr | (fcol[lr] < j0 ? 0 : 0x10000), (int)cmul,
                        (int)shoup_pre(cmul, F.p, pinv64), 0);
        }
      }
      const unsigned mask = __ballot_sync(0xffffffffu, act);
      int base = 0;
      if (lane == 0 && mask) base = atomicAdd(&s_nact, __popc(mask));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (act) {
        const int pos = base + __popc(mask & ((1u << lane) - 1u));
        s_act[pos] = e;
        s_nz[pos] = 0u;
      }
    }
    // the elected row right of its pivot column, read once from CTA wr into
    // this CTA's shared memory; the pivot columns (which hold L entries) are
    // kPivFlag: the update subtracts zero there and does not count them live
    {
      const typename ClRows<kStore>::Peer P = W.peer(cl, (unsigned)wr);
#pragma unroll
      for (int c = 0; c < kClCols; ++c) {
        const int j = tid + c * kClThreads;
        if (j > j0 && j < n) pivrow[j] = mypiv[c] ? kPivFlag : P.ld(lrw, j);
      }
    }
    __syncthreads();
    // W[l, :] -= c_l piv[:] right of the pivot column, the multiplier into it.
    // Work items of up to kClGroup active rows x kClChunk columns, one warp
    // each: a lane reads each elected-row entry once for the rows of its item.
    const int na = s_nact;
    for (int a = tid; a < na; a += kClThreads) W.st(s_act[a].x & 0xffff, j0, (uint32_t)s_act[a].y);
    // the pivot row and column leave (read again after the next barrier)
    if (tid == 0) {
      if (wr == g) {
        fcol[lrw] = INT_MAX;
        posk[lrw] = r;
      }
      prow[r] = istar;
      pcol[r] = j0;
      s_pmask[j0 >> 5] |= 1u << (j0 & 31);
    }
#pragma unroll
    for (int c = 0; c < kClCols; ++c)
      if (tid + c * kClThreads == j0) mypiv[c] = true;
    {
      const int ngrp = (na + kClGroup - 1) / kClGroup;
      const int nch = (n - j0 - 1 + kClChunk - 1) / kClChunk;
      for (int it = warp; it < ngrp * nch; it += kClWarps) {
        const int gi = it / nch, ch = it - gi * nch;
        const int a0 = gi * kClGroup;
        const int nr = min(kClGroup, na - a0);
        int lrs[kClGroup];
        uint32_t cs[kClGroup], cps[kClGroup], nz[kClGroup];
        bool redo[kClGroup];
#pragma unroll
        for (int q = 0; q < kClGroup; ++q) {
          const int4 e = q < nr ? s_act[a0 + q] : make_int4(0, 0, 0, 0);
          lrs[q] = e.x & 0xffff;
          redo[q] = (e.x & 0x10000) != 0;
          cs[q] = (uint32_t)e.y;
          cps[q] = (uint32_t)e.z;
          nz[q] = 0u;
        }
        const int jb = j0 + 1 + ch * kClChunk + lane;
#pragma unroll
        for (int u = 0; u < kClChunk / 32; ++u) {
          const int j = jb + 32 * u;
          if (j < n) {
            const uint32_t pw = pivrow[j];
            const uint32_t pvj = pw & ~kPivFlag;
            const uint32_t keep = (pw & kPivFlag) ? 0u : ~0u;
            uint32_t v[kClGroup];
#pragma unroll
            for (int q = 0; q < kClGroup; ++q)
              if (q < nr) v[q] = W.ld(lrs[q], j);
#pragma unroll
            for (int q = 0; q < kClGroup; ++q) {
              if (q < nr) {
                const uint32_t d = sub_mod(v[q], shoup_mul(pvj, cs[q], cps[q], F.p), F.p);
                W.st(lrs[q], j, d);
                nz[q] |= d & keep;
              }
            }
          }
        }
        // chunks where a row that needs its first live column has one
#pragma unroll
        for (int q = 0; q < kClGroup; ++q)
          if (q < nr && redo[q] && __any_sync(0xffffffffu, nz[q] != 0u) && lane == 0)
            atomicOr(&s_nz[a0 + q], 1u << ch);
      }
    }
    __syncthreads();
    // first live column of the rows whose first live column was the pivot
    // column, one warp a row: inside the first chunk the elimination found a
    // live non-zero in (none: the row is zero right of the pivot column, and
    // was zero left of it); pivot columns hold L entries and do not count
    for (int a = warp; a < na; a += kClWarps) {
      const int ae = s_act[a].x;
      if (!(ae & 0x10000)) continue;
      const int lr = ae & 0xffff;
      const unsigned chunks = s_nz[a];
      int f = INT_MAX;
      if (chunks) {
        const int jc = j0 + 1 + (__ffs(chunks) - 1) * kClChunk;
        for (int j1 = jc; j1 < jc + kClChunk && j1 < n; j1 += 32) {
          const int j = j1 + lane;
          const bool live =
              j < n && !((s_pmask[j >> 5] >> (j & 31)) & 1u) && W.ld(lr, j) != 0u;
          const unsigned b = __ballot_sync(0xffffffffu, live);
          if (b) {
            f = j1 + __ffs(b) - 1;
            break;
          }
        }
      }
      if (lane == 0) fcol[lr] = f;
    }
    ++r;
    __syncthreads();
  }

  // P = [pivot rows, other rows ascending], Q likewise, from bit masks of the
  // pivot rows and columns and prefix counts of their words
  for (int t = tid; t < r; t += kClThreads) atomicOr(&s_rmask[prow[t] >> 5], 1u << (prow[t] & 31));
  __syncthreads();
  if (warp == 0) {
    int rv = __popc(s_rmask[lane]), cv = __popc(s_pmask[lane]);
    for (int o = 1; o < 32; o <<= 1) {
      const int ru = __shfl_up_sync(0xffffffffu, rv, o);
      const int cu = __shfl_up_sync(0xffffffffu, cv, o);
      if (lane >= o) {
        rv += ru;
        cv += cu;
      }
    }
    s_rpre[lane + 1] = rv;
    s_cpre[lane + 1] = cv;
    if (lane == 0) s_rpre[0] = s_cpre[0] = 0;
  }
  __syncthreads();
  for (int u = tid; u < n; u += kClThreads) {
    if (u < r) colpos[u] = pcol[u];
    if (!((s_pmask[u >> 5] >> (u & 31)) & 1u)) colpos[r + u - count_below(s_pmask, s_cpre, u)] = u;
  }
  __syncthreads();
  for (int lr = warp; lr < owned; lr += kClWarps) {
    const int l = lr * G + g;
    const int t = posk[lr] >= 0 ? posk[lr] : r + l - count_below(s_rmask, s_rpre, l);
    uint32_t* dst = X + (int64_t)t * ldx;
    for (int u = lane; u < n; u += 32) dst[u] = (t >= r && u >= r) ? 0u : W.ld(lr, colpos[u]);
  }
  if (g == 0) {
    for (int t = tid; t < r; t += kClThreads) perm_r[t] = prow[t];
    for (int l = tid; l < m; l += kClThreads)
      if (!((s_rmask[l >> 5] >> (l & 31)) & 1u)) perm_r[r + l - count_below(s_rmask, s_rpre, l)] = l;
    for (int u = tid; u < n; u += kClThreads) perm_c[u] = colpos[u];
    if (tid == 0) rank_out[0] = r;
  }
  // no CTA leaves while another may still read its shared memory
  cl.sync();
}

template <int kStore>
const void* cl_kernel() {
  return reinterpret_cast<const void*>(&k_leaf_cluster<kStore>);
}

int cl_store(const pluq_ctx* c) {
  if (c->F.p < (1u << 16)) return 1;
  if (c->F.p < (1u << 24)) return 2;
  return 0;
}

// Per device: the cluster size the leaf uses (16 where a cluster of 16 CTAs
// with this shared memory can be resident, else 8; 0: no cluster launch) and
// the dynamic shared memory a CTA may take.
struct ClCaps {
  int ctas = -1;
  size_t smem = 0;
};

const ClCaps& cl_caps(int device) {
  static std::mutex mu;
  static ClCaps caps[64];
  std::lock_guard<std::mutex> lock(mu);
  ClCaps& cc = caps[device & 63];
  if (cc.ctas >= 0) return cc;
  cc.ctas = 0;
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) !=
      cudaSuccess) {
    cudaGetLastError();
    return cc;
  }
  size_t stat = 0;
  const void* ks[3] = {cl_kernel<0>(), cl_kernel<1>(), cl_kernel<2>()};
  for (const void* k : ks) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) {
      cudaGetLastError();
      return cc;
    }
    stat = std::max(stat, fa.sharedSizeBytes);
  }
  if ((size_t)optin <= stat + 1024) return cc;
  const size_t dyn = (size_t)optin - stat;
  for (const void* k : ks) {
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
            cudaSuccess) {
      cudaGetLastError();
      return cc;
    }
  }
  for (int G : {kClMaxCtas, 8}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = dyn;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = G;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, ks[2], &cfg) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (nclusters >= 1) {
      cc.ctas = G;
      cc.smem = dyn;
      break;
    }
  }
  return cc;
}

}  // namespace

// Whether an m x n leaf fits the shared memory of one cluster.
int cluster_leaf_fits(pluq_ctx* c, int64_t m, int64_t n) {
  if (m <= 0 || n <= 0 || m > c->leaf_dim || n > c->leaf_dim) return 0;
  if (m > kClMaxDim || n > kClMaxDim) return 0;
  const ClCaps& cc = cl_caps(c->device);
  if (cc.ctas <= 0) return 0;
  const int G = (int)std::min<int64_t>(cc.ctas, m);
  if ((m + G - 1) / G > kClMaxRows) return 0;
  return cl_layout((int)m, (int)n, G, cl_store(c)).total <= cc.smem;
}

int launch_leaf_cluster(pluq_ctx* c, uint32_t* X, int64_t ldx, int m, int n, int32_t* perm_r,
                        int32_t* perm_c, int32_t* rank_out) {
  if (!cluster_leaf_fits(c, m, n)) return PLUQ_ERR_INVALID_ARG;
  const ClCaps& cc = cl_caps(c->device);
  const int G = std::min(cc.ctas, m);
  const int store = cl_store(c);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(kClThreads);
  cfg.dynamicSmemBytes = cl_layout(m, n, G, store).total;
  cfg.stream = c->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = G;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const uint32_t* tab = inv_table_ptr(c);
  const FieldP F = c->F;
  const uint64_t pinv64 = ~0ull / F.p;  // floor((2^64 - 1) / p)
  ProfScope ps(c, PC_BASE, 0, 8.0 * m * n);
  if (store == 0)
    PLUQ_CUDA(cudaLaunchKernelEx(&cfg, k_leaf_cluster<0>, X, ldx, m, n, F, pinv64, tab, perm_r,
                                 perm_c, rank_out));
  else if (store == 1)
    PLUQ_CUDA(cudaLaunchKernelEx(&cfg, k_leaf_cluster<1>, X, ldx, m, n, F, pinv64, tab, perm_r,
                                 perm_c, rank_out));
  else
    PLUQ_CUDA(cudaLaunchKernelEx(&cfg, k_leaf_cluster<2>, X, ldx, m, n, F, pinv64, tab, perm_r,
                                 perm_c, rank_out));
  return PLUQ_OK;
}
