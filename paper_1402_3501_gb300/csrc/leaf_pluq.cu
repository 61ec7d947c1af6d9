// Large leaves of the tile-recursive PLUQ: rank-profile-revealing elimination
// of a block of up to kLeafMax x kLeafMax residues by one cooperative grid.
//
// The block is distributed over the shared memory of G CTAs (row l lives in
// CTA l mod G), so it is read from HBM once and written once.  Each step picks
// the row-major first non-zero of the remaining Schur complement (the pivot
// search of Sec. 4.1): every CTA proposes its first row with a non-zero
// outside the pivot columns, publishing the row itself, and an atomicMin over
// the row indices elects the pivot row; after one grid barrier every CTA
// reads the elected row, finds its first non-zero column, and eliminates its
// own rows below it.  Rows that reduce to zero are never visited again, so a
// step costs one grid barrier per pivot, whatever the number of zero rows:
// the cost follows the rank, which is what rank-deficient blocks need.
//
// Output as the one-CTA base case: the block becomes the compressed L\U of
// P^T X Q^T with P = [pivot rows, other rows ascending] and Q likewise,
// perm_r / perm_c / rank_out as local index vectors.  The grid barrier spins
// with a time limit; on expiry the kernel records PLUQ_ERR_TIMEOUT, raises an
// abort flag seen by every CTA and returns without writing the block.
#include <climits>

#include "common.cuh"

namespace {

constexpr int kLeafThreads = 512;
constexpr int kLeafWarps = kLeafThreads / 32;
constexpr long long kBarrierCycles = 4000000000LL;  // ~2 s

struct LeafSync {
  unsigned count;
  unsigned gen;
  int best[3];
  int abort;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_volatile_i(const int* p) {
  return *reinterpret_cast<const volatile int*>(p);
}

// Grid-wide barrier for a cooperative launch; false once any CTA aborted.
__device__ bool grid_barrier(LeafSync* s, unsigned G, unsigned& gen, int* err) {
  __shared__ int aborted;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned arrived = atomicAdd(&s->count, 1u);
    if (arrived == G - 1) {
      s->count = 0;
      __threadfence();
      atomicAdd(&s->gen, 1u);
    } else {
      const long long t0 = clock64();
      while (ld_acquire(&s->gen) == gen) {
        if (ld_volatile_i(&s->abort)) break;
        if (clock64() - t0 > kBarrierCycles) {
          atomicExch(err, PLUQ_ERR_TIMEOUT);
          atomicExch(&s->abort, 1);
          break;
        }
      }
    }
    ++gen;
    __threadfence();
    aborted = ld_volatile_i(&s->abort);
  }
  __syncthreads();
  return aborted == 0;
}

// Block-wide: out[base + rank] = i for every i < count with !flag[i], in
// ascending order (flags in shared memory).
__device__ void compact_unflagged(const int32_t* flag, int count, int32_t* out, int base,
                                  int32_t* scratch /* kLeafWarps + 1 ints */) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int per = (count + kLeafThreads - 1) / kLeafThreads;
  const int i0 = tid * per, i1 = min(count, i0 + per);
  int mine = 0;
  for (int i = i0; i < i1; ++i) mine += flag[i] ? 0 : 1;
  int incl = mine;
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) scratch[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int v = lane < kLeafWarps ? scratch[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    if (lane < kLeafWarps) scratch[lane] = v;
  }
  __syncthreads();
  int pos = base + incl - mine + (warp > 0 ? scratch[warp - 1] : 0);
  for (int i = i0; i < i1; ++i)
    if (!flag[i]) out[pos++] = i;
  __syncthreads();
}

__global__ void __launch_bounds__(kLeafThreads, 1)
    k_leaf_pluq(uint32_t* __restrict__ X, int64_t ldx, int m, int n, FieldP F,
                const uint32_t* __restrict__ inv_table, int32_t* __restrict__ perm_r,
                int32_t* __restrict__ perm_c, int32_t* __restrict__ rank_out, LeafSync* sync,
                uint32_t* __restrict__ candbuf, int* __restrict__ err) {
  extern __shared__ __align__(16) uint32_t sm[];
  const unsigned G = gridDim.x;
  const int cta = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rown = (m + G - 1) / G;  // owned-row capacity
  const int mn = min(m, n);
  uint32_t* W = sm;                                             // [rown][n]
  uint32_t* piv = W + (size_t)rown * n;                         // [n] elected row
  int32_t* ispiv = reinterpret_cast<int32_t*>(piv + n);         // [n]
  int32_t* prow = ispiv + n;                                    // [mn]
  int32_t* pcol = prow + mn;                                    // [mn]
  int32_t* rowflag = pcol + mn;                                 // [rown]
  int32_t* red = rowflag + rown;                                // [64]
  int32_t* rowpos = red + 64;                                   // [m]
  int32_t* rowinv = rowpos + m;                                 // [m]
  int32_t* isprow = rowinv + m;                                 // [m]
  int32_t* colpos = isprow + m;                                 // [n]

  // owned rows into shared memory
  int owned = 0;
  for (int lr = 0; lr < rown; ++lr)
    if ((int64_t)lr * G + cta < m) owned = lr + 1;
  for (int lr = warp; lr < owned; lr += kLeafWarps) {
    const uint32_t* src = X + ((int64_t)lr * G + cta) * ldx;
    for (int j = lane; j < n; j += 32) W[(size_t)lr * n + j] = src[j];
  }
  for (int j = tid; j < n; j += kLeafThreads) ispiv[j] = 0;
  __syncthreads();

  unsigned gen = 0;
  // first candidate: first owned row with a non-zero
  for (int lr = warp; lr < owned; lr += kLeafWarps) {
    bool nz = false;
    for (int j = lane; j < n; j += 32) nz |= W[(size_t)lr * n + j] != 0u;
    nz = __any_sync(0xffffffffu, nz);
    if (lane == 0) rowflag[lr] = nz ? 1 : 0;
  }
  __syncthreads();
  {
    int first = -1;
    for (int lr = 0; lr < owned; ++lr)
      if (rowflag[lr]) {
        first = lr;
        break;
      }
    if (first >= 0) {
      uint32_t* dst = candbuf + (size_t)cta * n;
      for (int j = tid; j < n; j += kLeafThreads) dst[j] = W[(size_t)first * n + j];
      if (tid == 0) atomicMin(&sync->best[0], first * (int)G + cta);
    }
  }
  bool ok = grid_barrier(sync, G, gen, err);

  int r = 0;
  for (int k = 0; ok; ++k) {
    const int istar = ld_volatile_i(&sync->best[k % 3]);
    if (cta == 0 && tid == 0) sync->best[(k + 2) % 3] = INT_MAX;
    if (istar == INT_MAX || r >= mn) break;
    const int winner = istar % (int)G;
    const uint32_t* crow = candbuf + ((size_t)(k & 1) * G + winner) * n;
    // L2 loads: the buffer is rewritten every other step by other SMs
    for (int j = tid; j < n; j += kLeafThreads) piv[j] = __ldcg(crow + j);
    __syncthreads();
    // pivot column: first non-zero of the elected row outside the pivots
    int jl = INT_MAX;
    for (int j = tid; j < n; j += kLeafThreads)
      if (!ispiv[j] && piv[j] != 0u) {
        jl = j;
        break;
      }
    for (int o = 16; o > 0; o >>= 1) jl = min(jl, __shfl_xor_sync(0xffffffffu, jl, o));
    if (lane == 0) red[warp] = jl;
    __syncthreads();
    int j0 = INT_MAX;
    for (int w = 0; w < kLeafWarps; ++w) j0 = min(j0, red[w]);
    if (j0 == INT_MAX) {  // unreachable: the elected row has a non-zero off the pivots
      if (tid == 0) atomicExch(err, PLUQ_ERR_INVALID_ARG);
      break;
    }
    const uint32_t inv = f_inv(piv[j0], F, inv_table);
    const uint32_t inv_m = f_to_mont(inv, F);
    __syncthreads();
    if (tid == 0) {
      prow[r] = istar;
      pcol[r] = j0;
      ispiv[j0] = 1;
    }
    __syncthreads();
    // eliminate owned rows below the pivot row
    for (int lr = warp; lr < owned; lr += kLeafWarps) {
      const int l = lr * (int)G + cta;
      uint32_t* Wl = W + (size_t)lr * n;
      bool nz = false;
      if (l > istar) {
        const uint32_t wl = Wl[j0];
        __syncwarp();
        if (wl != 0u) {
          const uint32_t cmul = f_mul_mont(inv_m, wl, F);
          const uint32_t cm = f_to_mont(cmul, F);
          for (int j = lane; j < n; j += 32) {
            if (j == j0) {
              Wl[j] = cmul;
            } else if (!ispiv[j]) {
              const uint32_t nv = f_sub(Wl[j], f_mul_mont(cm, piv[j], F), F);
              Wl[j] = nv;
              nz |= nv != 0u;
            }
          }
        } else {
          for (int j = lane; j < n; j += 32) nz |= !ispiv[j] && Wl[j] != 0u;
        }
      }
      nz = __any_sync(0xffffffffu, nz);
      if (lane == 0) rowflag[lr] = nz ? 1 : 0;
    }
    __syncthreads();
    int first = -1;
    for (int lr = 0; lr < owned; ++lr)
      if (rowflag[lr]) {
        first = lr;
        break;
      }
    if (first >= 0) {
      uint32_t* dst = candbuf + ((size_t)((k + 1) & 1) * G + cta) * n;
      for (int j = tid; j < n; j += kLeafThreads) dst[j] = W[(size_t)first * n + j];
      if (tid == 0) atomicMin(&sync->best[(k + 1) % 3], first * (int)G + cta);
    }
    ++r;
    ok = grid_barrier(sync, G, gen, err);
  }
  if (!ok || ld_volatile_i(err) != 0) return;

  // P = [pivot rows, other rows ascending], Q likewise; every CTA builds both
  for (int i = tid; i < m; i += kLeafThreads) isprow[i] = 0;
  __syncthreads();
  for (int k = tid; k < r; k += kLeafThreads) {
    isprow[prow[k]] = 1;
    rowpos[k] = prow[k];
    colpos[k] = pcol[k];
  }
  __syncthreads();
  compact_unflagged(isprow, m, rowpos, r, red);
  compact_unflagged(ispiv, n, colpos, r, red);
  for (int t = tid; t < m; t += kLeafThreads) rowinv[rowpos[t]] = t;
  __syncthreads();
  for (int lr = warp; lr < owned; lr += kLeafWarps) {
    const int s = lr * (int)G + cta;
    const int t = rowinv[s];
    uint32_t* dst = X + (int64_t)t * ldx;
    const uint32_t* src = W + (size_t)lr * n;
    for (int u = lane; u < n; u += 32) dst[u] = (t >= r && u >= r) ? 0u : src[colpos[u]];
  }
  if (cta == 0) {
    for (int t = tid; t < m; t += kLeafThreads) perm_r[t] = rowpos[t];
    for (int u = tid; u < n; u += kLeafThreads) perm_c[u] = colpos[u];
    if (tid == 0) rank_out[0] = r;
  }
}

__global__ void k_leaf_init(LeafSync* s) {
  s->count = 0u;
  s->gen = 0u;
  s->best[0] = s->best[1] = s->best[2] = INT_MAX;
  s->abort = 0;
}

size_t leaf_smem(int m, int n, int G) {
  const int rown = (m + G - 1) / G;
  const int mn = m < n ? m : n;
  return sizeof(uint32_t) * ((size_t)rown * n + n + n + 2 * mn + rown + 64 + 3 * m + n);
}

}  // namespace

// Largest block a leaf launch accepts (rows and columns).
int leaf_max_dim() { return 2048; }

// Whether a leaf of m x n fits the shared memory of the cooperative grid.
int leaf_fits(pluq_ctx* c, int64_t m, int64_t n) {
  if (m <= 0 || n <= 0 || m > c->leaf_dim || n > c->leaf_dim) return 0;
  return leaf_smem((int)m, (int)n, c->sm_count) <= 220 * 1024;
}

int launch_leaf_pluq(pluq_ctx* c, uint32_t* X, int64_t ldx, int m, int n, int32_t* perm_r,
                     int32_t* perm_c, int32_t* rank_out) {
  static int max_smem_set = 0;
  // grid: at most one CTA per SM, at least ~8 owned rows per CTA
  int G = (m + 7) / 8;
  if (G > c->sm_count) G = c->sm_count;
  if (G < 1) G = 1;
  size_t smem = leaf_smem(m, n, G);
  while (smem > 220 * 1024 && G < c->sm_count) {
    ++G;
    smem = leaf_smem(m, n, G);
  }
  if (smem > 220 * 1024) return PLUQ_ERR_INVALID_ARG;
  if (max_smem_set < (int)smem) {
    PLUQ_CUDA(cudaFuncSetAttribute(k_leaf_pluq, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   220 * 1024));
    max_smem_set = 220 * 1024;
  }
  // grid sync words and two candidate-row buffers of G rows each
  const size_t need = 256 + sizeof(uint32_t) * 2 * (size_t)G * n;
  PLUQ_TRY(c->leaf.ensure(need));
  LeafSync* sync = c->leaf.as<LeafSync>();
  uint32_t* candbuf = reinterpret_cast<uint32_t*>(c->leaf.as<char>() + 256);
  {
    ProfScope pi(c, PC_INDEX);
    k_leaf_init<<<1, 1, 0, c->stream>>>(sync);
  }
  int* err = c->small.as<int>() + 16;
  const uint32_t* tab = inv_table_ptr(c);
  FieldP F = c->F;
  void* args[] = {&X, &ldx, &m, &n, &F, &tab, &perm_r, &perm_c, &rank_out, &sync, &candbuf, &err};
  ProfScope ps(c, PC_BASE, 0, 8.0 * m * n);
  PLUQ_CUDA(cudaLaunchCooperativeKernel((const void*)k_leaf_pluq, dim3(G), dim3(kLeafThreads), args,
                                        smem, c->stream));
  return PLUQ_OK;
}
