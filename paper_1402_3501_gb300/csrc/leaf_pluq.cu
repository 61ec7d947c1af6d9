// Large leaves of the tile-recursive PLUQ: rank-profile-revealing elimination
// of a block of up to kLeafMax x kLeafMax residues by one cooperative grid.
//
// The block is distributed over the shared memory of G CTAs (row l lives in
// CTA l mod G), so it is read from HBM once and written once.  Each step picks
// the row-major first non-zero of the remaining Schur complement (the pivot
// search of Sec. 4.1): every CTA proposes its first row with a non-zero
// outside the pivot columns (tracked per row during elimination), publishing
// the row with that column and the inverse of its entry there; after one grid
// barrier every CTA elects the smallest proposed row index, reads that row and
// eliminates its own rows below it.  Rows that reduce to zero are never visited again, so a
// step costs one grid barrier per pivot, whatever the number of zero rows:
// the cost follows the rank, which is what rank-deficient blocks need.
//
// Output as the one-CTA base case: the block becomes the compressed L\U of
// P^T X Q^T with P = [pivot rows, other rows ascending] and Q likewise,
// perm_r / perm_c / rank_out as local index vectors.  The grid barrier spins
// with a time limit; on expiry the kernel records PLUQ_ERR_TIMEOUT, raises an
// abort flag seen by every CTA and returns without writing the block.
#include <algorithm>
#include <climits>

#include "common.cuh"

namespace {

constexpr int kLeafThreads = 512;
constexpr int kLeafWarps = kLeafThreads / 32;

// Grid barrier words and the candidate election of the barrier leaf.  Each
// CTA writes its candidate (global row index, INT_MAX for none) to its own
// slot cand[step & 1][cta] before arriving; after the barrier every CTA
// reduces the G slots itself (one round of parallel loads) instead of all
// CTAs contending for one atomicMin word.  Two slot arrays by step parity: a
// CTA rewrites cand[s & 1] at the end of step s + 1, after every CTA passed
// the barrier of step s + 1 and so finished reading step s's slots.
constexpr int kLeafMaxCtas = 256;
struct LeafSync {
  unsigned count;  // grid-barrier arrivals; bit 31: abort
  int pad0;
  long long wait_cycles;  // bound of every wait, in SM clock cycles
  int pad[28];
  int cand[2][kLeafMaxCtas];
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
// Grid-wide barrier: one monotonic arrival counter.  Each CTA adds 1 with a
// release atomic (publishing the CTA's writes, ordered before it by the block
// barrier) and polls with acquire loads until the counter reaches G times the
// number of barriers passed; no reset, no generation word, no separate fence.
// Bit 31 of the counter is the abort flag (a timed-out CTA sets it), seen by
// the same polls.  false once any CTA aborted.
constexpr unsigned kAbortBit = 0x80000000u;

__device__ __forceinline__ unsigned atom_add_release(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

__device__ bool grid_barrier(LeafSync* s, unsigned G, unsigned& target, int* err) {
  __shared__ int aborted;
  __syncthreads();
  if (threadIdx.x == 0) {
    target += G;
    unsigned v = atom_add_release(&s->count, 1u) + 1u;
    const long long t0 = clock64();
    const long long limit = s->wait_cycles;
    while ((v & ~kAbortBit) < target && !(v & kAbortBit)) {
      if (clock64() - t0 > limit) {
        atomicExch(err, PLUQ_ERR_TIMEOUT);
        atomicOr(&s->count, kAbortBit);
        v = kAbortBit;
        break;
      }
      v = ld_acquire(&s->count);
    }
    aborted = (v & kAbortBit) != 0;
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

constexpr int kLeafMaxRows = 128;  // owned rows per CTA of a barrier leaf

// Words per candidate slot: the row, its live column and the Montgomery
// inverse of its entry there, padded to 16 bytes.
__host__ __device__ inline int leaf_slot(int n) { return (n + 2 + 3) & ~3; }

__global__ void __launch_bounds__(kLeafThreads, 1)
    k_leaf_pluq(uint32_t* __restrict__ X, int64_t ldx, int m, int n, FieldP F,
                const uint32_t* __restrict__ inv_table, int32_t* __restrict__ perm_r,
                int32_t* __restrict__ perm_c, int32_t* __restrict__ rank_out, LeafSync* sync,
                uint32_t* __restrict__ candbuf, int* __restrict__ err) {
  extern __shared__ __align__(16) uint32_t sm[];
  __shared__ uint32_t s_hdr[2];  // elected pivot column and Montgomery inverse
  __shared__ int s_act[kLeafMaxRows], s_newf[kLeafMaxRows], s_nact;
  __shared__ uint32_t s_cm[kLeafMaxRows], s_cmul[kLeafMaxRows];
  const unsigned G = gridDim.x;
  const int cta = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rown = (m + G - 1) / G;  // owned-row capacity
  const int mn = min(m, n);
  const int slot = leaf_slot(n);
  uint32_t* W = sm;                                             // [rown][n]
  uint32_t* piv = W + (size_t)rown * n;                         // [n] elected row
  int32_t* ispiv = reinterpret_cast<int32_t*>(piv + n);         // [n]
  int32_t* prow = ispiv + n;                                    // [mn]
  int32_t* pcol = prow + mn;                                    // [mn]
  int32_t* fcol = pcol + mn;                                    // [rown] first live column
  int32_t* red = fcol + rown;                                   // [64]
  int32_t* rowpos = red + 64;                                   // [m]
  int32_t* rowinv = rowpos + m;                                 // [m]
  int32_t* isprow = rowinv + m;                                 // [m]
  int32_t* colpos = isprow + m;                                 // [n]

  // owned rows into shared memory
  int owned = 0;
  for (int lr = 0; lr < rown; ++lr)
    if ((int64_t)lr * G + cta < m) owned = lr + 1;
  copy_rows_g2s(W, X + (int64_t)cta * ldx, ldx * (int64_t)G, owned, n, warp, lane, kLeafWarps);
  for (int j = tid; j < n; j += kLeafThreads) ispiv[j] = 0;
  __syncthreads();
  // fcol[lr]: first non-zero column of owned row lr outside the pivot columns
  // (INT_MAX: none left, or the row became a pivot row), refreshed by the
  // warp that eliminates the row
  for (int lr = warp; lr < owned; lr += kLeafWarps) {
    const uint32_t* Wl = W + (size_t)lr * n;
    int jl = INT_MAX;
    for (int j = lane; j < n; j += 32)
      if (Wl[j] != 0u) {
        jl = j;
        break;
      }
    jl = __reduce_min_sync(0xffffffffu, jl);
    if (lane == 0) fcol[lr] = jl;
  }
  __syncthreads();

  // this CTA's candidate for the next step: its first owned row with a live
  // column, published with that column and the inverse of its entry there
  auto publish = [&](int buf) {
    int first = INT_MAX;
    for (int b0 = 0; b0 < owned; b0 += 32) {
      const int lr = b0 + lane;
      const unsigned hit = __ballot_sync(0xffffffffu, lr < owned && fcol[lr] != INT_MAX);
      if (hit) {
        first = b0 + __ffs(hit) - 1;
        break;
      }
    }
    if (first != INT_MAX) {
      uint32_t* dst = candbuf + ((size_t)buf * G + cta) * slot;
      const uint32_t* src = W + (size_t)first * n;
      for (int j = tid; j < n; j += kLeafThreads) dst[j] = src[j];
      if (tid == 0) {
        const int j0 = fcol[first];
        dst[n] = (uint32_t)j0;
        dst[n + 1] = f_to_mont(f_inv(src[j0], F, inv_table), F);
      }
    }
    if (tid == 0) sync->cand[buf][cta] = first == INT_MAX ? INT_MAX : first * (int)G + cta;
  };
  // elected row of step k: smallest candidate over the G slots (all threads)
  auto elect = [&](int buf) {
    int v = tid < (int)G ? __ldcg(&sync->cand[buf][tid]) : INT_MAX;
    v = __reduce_min_sync(0xffffffffu, v);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    int best = INT_MAX;
    for (int w = 0; w < kLeafWarps; ++w) best = min(best, red[w]);
    return best;
  };

  unsigned target = 0;  // grid-barrier arrivals expected so far
  publish(0);
  bool ok = grid_barrier(sync, G, target, err);

  int r = 0;
  for (int k = 0; ok; ++k) {
    const int istar = elect(k & 1);
    if (istar == INT_MAX || r >= mn) break;
    const int winner = istar % (int)G;
    const uint32_t* crow = candbuf + ((size_t)(k & 1) * G + winner) * slot;
    // L2 loads: the buffer is rewritten every other step by other SMs
    for (int j = tid; j < n; j += kLeafThreads) piv[j] = __ldcg(crow + j);
    if (tid < 2) s_hdr[tid] = __ldcg(crow + n + tid);
    __syncthreads();
    const int j0 = (int)s_hdr[0];
    const uint32_t inv_m = s_hdr[1];
    // rows to eliminate: owned rows below the pivot row with a non-zero in its
    // column (the others keep their first live column); the pivot row leaves
    // the race.  Listed with their multipliers by warp 0.
    if (warp == 0) {
      int cnt = 0;
      for (int b0 = 0; b0 < owned; b0 += 32) {
        const int lr = b0 + lane;
        bool act = false;
        uint32_t cmul = 0, cm = 0;
        if (lr < owned) {
          const int l = lr * (int)G + cta;
          if (l == istar) {
            fcol[lr] = INT_MAX;
          } else if (l > istar) {  // rows above are zero or pivot rows
            const uint32_t wl = W[(size_t)lr * n + j0];
            if (wl != 0u) {
              act = true;
              cmul = f_mul_mont(inv_m, wl, F);
              cm = f_to_mont(cmul, F);
            }
          }
        }
        const unsigned mask = __ballot_sync(0xffffffffu, act);
        if (act) {
          const int pos = cnt + __popc(mask & ((1u << lane) - 1u));
          s_act[pos] = lr;
          s_cm[pos] = cm;
          s_cmul[pos] = cmul;
          s_newf[pos] = INT_MAX;
        }
        cnt += __popc(mask);
      }
      if (lane == 0) s_nact = cnt;
    }
    __syncthreads();
    // W[l, :] -= c_l piv[:], all threads over (row, column): a thread keeps
    // the same columns for every row, its first live column per row reduced
    // over the warp and then over the CTA
    const int na = s_nact;
    for (int a = 0; a < na; ++a) {
      uint32_t* Wl = W + (size_t)s_act[a] * n;
      const uint32_t cm = s_cm[a];
      int jl = INT_MAX;
      for (int j = tid; j < n; j += kLeafThreads) {
        if (j == j0) {
          Wl[j] = s_cmul[a];
        } else if (!ispiv[j]) {
          const uint32_t nv = f_sub(Wl[j], f_mul_mont(cm, piv[j], F), F);
          Wl[j] = nv;
          if (nv != 0u && jl == INT_MAX) jl = j;
        }
      }
      jl = __reduce_min_sync(0xffffffffu, jl);
      if (lane == 0 && jl != INT_MAX) atomicMin(&s_newf[a], jl);
    }
    __syncthreads();
    if (tid < na) fcol[s_act[tid]] = s_newf[tid];
    if (tid == 0) {
      prow[r] = istar;
      pcol[r] = j0;
      ispiv[j0] = 1;
    }
    __syncthreads();
    publish((k + 1) & 1);
    ++r;
    ok = grid_barrier(sync, G, target, err);
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

__global__ void k_leaf_init(LeafSync* s, long long wait_cycles) {
  if (threadIdx.x == 0) {
    s->count = 0u;
    s->wait_cycles = wait_cycles;
  }
  for (int i = threadIdx.x; i < kLeafMaxCtas; i += blockDim.x) s->cand[0][i] = s->cand[1][i] = INT_MAX;
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
  if ((m + c->sm_count - 1) / c->sm_count > kLeafMaxRows) return 0;
  return leaf_smem((int)m, (int)n, c->sm_count) <= 220 * 1024;
}

int launch_leaf_pluq(pluq_ctx* c, uint32_t* X, int64_t ldx, int m, int n, int32_t* perm_r,
                     int32_t* perm_c, int32_t* rank_out) {
  static const cudaError_t attr =
      cudaFuncSetAttribute(k_leaf_pluq, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  PLUQ_CUDA(attr);
  // grid: at most one CTA per SM, at least ~8 owned rows per CTA
  int G = (m + 7) / 8;
  if (G > c->sm_count) G = c->sm_count;
  if (G < 1) G = 1;
  size_t smem = leaf_smem(m, n, G);
  while (smem > 220 * 1024 && G < c->sm_count) {
    ++G;
    smem = leaf_smem(m, n, G);
  }
  if (smem > 220 * 1024 || (m + G - 1) / G > kLeafMaxRows) return PLUQ_ERR_INVALID_ARG;
  // barrier words, election slots and two candidate-row buffers of G rows each
  if (G > kLeafMaxCtas || G > kLeafThreads) return PLUQ_ERR_INVALID_ARG;
  const size_t head = (sizeof(LeafSync) + 255) / 256 * 256;
  const size_t need = head + sizeof(uint32_t) * 2 * (size_t)G * leaf_slot(n);
  PLUQ_TRY(c->leaf.ensure(need));
  LeafSync* sync = c->leaf.as<LeafSync>();
  uint32_t* candbuf = reinterpret_cast<uint32_t*>(c->leaf.as<char>() + head);
  {
    ProfScope pi(c, PC_INDEX);
    k_leaf_init<<<1, 256, 0, c->stream>>>(sync, c->wait_cycles);
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

// ---------------------------------------------------------------------------
// Wavefront leaf: the same rank-profile elimination with rows distributed in
// consecutive blocks (CTA c owns rows [c R, c R + R)).  Pivots are searched
// row by row in row order (Sec. 4.1), so CTA c's pivots are all found after
// those of CTAs < c.  A CTA first applies, in pivot order and as they are
// published, the pivot rows of all earlier CTAs to its own rows (several at a
// time, one reduction per element and batch); once every earlier CTA is done
// it factors its own rows, publishing each pivot row (pivot-column entries
// zeroed) with its column and inverse, then hands over with one release
// store.  A single 64-bit word, (CTAs done << 32) | pivots published, is the
// only synchronisation: one hand-off per CTA instead of one grid barrier per
// pivot.  Waits are bounded; on expiry PLUQ_ERR_TIMEOUT is recorded, an abort
// flag stops every CTA and the block is not written.
namespace {

struct ChainSync {
  unsigned long long word;
  int abort;
  int pad0;
  long long wait_cycles;  // bound of every wait, in SM clock cycles
  int pad[58];
};

struct PivInfo {
  int row;
  int col;
  uint32_t inv_m;
  int pad;
};

constexpr int kChainBatch = 8;     // pivot rows applied per pass
constexpr int kChainMaxRows = 64;  // rows per CTA, at most

__device__ __forceinline__ unsigned long long chain_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void chain_release(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

template <bool kIs2>
__device__ __forceinline__ uint32_t ch_mulm(uint32_t cm, uint32_t w, const FieldP& F) {
  if (kIs2) return cm & w;
  return f_redc((uint64_t)cm * w, F);
}

// Block-wide minimum of v (all threads get it); red holds kLeafWarps ints.
__device__ __forceinline__ int block_min(int v, int* red) {
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  int out = INT_MAX;
  for (int w = 0; w < kLeafWarps; ++w) out = min(out, red[w]);
  return out;
}

template <bool kIs2>
__global__ void __launch_bounds__(kLeafThreads, 1)
    k_leaf_chain(uint32_t* __restrict__ X, int64_t ldx, int m, int n, int R, FieldP F,
                 const uint32_t* __restrict__ inv_table, int32_t* __restrict__ perm_r,
                 int32_t* __restrict__ perm_c, int32_t* __restrict__ rank_out, ChainSync* sync,
                 uint32_t* __restrict__ pub, PivInfo* __restrict__ pinfo, int* __restrict__ err) {
  extern __shared__ __align__(16) uint32_t sm[];
  __shared__ unsigned long long s_word;
  __shared__ int s_red[kLeafWarps];
  __shared__ int s_col[kChainBatch];
  __shared__ uint32_t s_inv[kChainBatch];
  __shared__ uint32_t s_cm[kChainBatch * 32];  // multipliers per (batch pivot, row < 32)
  __shared__ uint32_t s_mul[kChainMaxRows], s_mulm[kChainMaxRows];  // phase-2 multipliers
  const int G = gridDim.x, cta = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int mn = min(m, n);
  const int r0 = cta * R;
  const int own = max(0, min(R, m - r0));
  const int ubuf = max(kChainBatch * n, 3 * m + n);  // U, reused by the output phase
  uint32_t* W = sm;                                                 // [R][n]
  uint32_t* U = W + (size_t)R * n;                                  // [kChainBatch][n]
  int32_t* ispiv = reinterpret_cast<int32_t*>(U + ubuf);           // [n]
  int32_t* rowpos = reinterpret_cast<int32_t*>(U);                  // [m]   (output phase)
  int32_t* rowinv = rowpos + m;                                     // [m]
  int32_t* isprow = rowinv + m;                                     // [m]
  int32_t* colpos = isprow + m;                                     // [n]

  copy_rows_g2s(W, X + (int64_t)r0 * ldx, ldx, own, n, warp, lane, kLeafWarps);
  for (int j = tid; j < n; j += kLeafThreads) ispiv[j] = 0;
  __syncthreads();

  // wait until `cond(word)`; false on abort / timeout
  auto wait_word = [&](int need_done, int need_piv) -> bool {
    if (tid == 0) {
      unsigned long long w = chain_acquire(&sync->word);
      const long long t0 = clock64();
      const long long limit = sync->wait_cycles;
      bool ok = true;
      // the abort flag is an error path: checked every 32nd poll only, so a
      // poll is one L2 round trip
      for (unsigned it = 1; (int)(w >> 32) < need_done && (int)(w & 0xffffffffu) < need_piv;
           ++it) {
        if ((it & 31u) == 0 && (ld_volatile_i(&sync->abort) || clock64() - t0 > limit)) {
          if (!ld_volatile_i(&sync->abort)) atomicExch(err, PLUQ_ERR_TIMEOUT);
          atomicExch(&sync->abort, 1);
          ok = false;
          break;
        }
        w = chain_acquire(&sync->word);
      }
      s_word = ok ? w : ~0ull;
    }
    __syncthreads();
    return s_word != ~0ull;
  };

  // phase 1: apply the pivots of earlier CTAs as they are published
  int applied = 0;
  bool ok = true;
  while (true) {
    if (!wait_word(cta, applied + 1)) {
      ok = false;
      break;
    }
    const unsigned long long w = s_word;
    const int npub = (int)(w & 0xffffffffu);
    const int done = (int)(w >> 32);
    while (applied < npub) {
      const int K = min(kChainBatch, npub - applied);
      // pivot rows (pivot-column entries already zero) and their columns
      copy_g2s(U, pub + (size_t)applied * n, K * n, tid, kLeafThreads);
      if (tid < K) {
        const int4 pi = __ldcg(reinterpret_cast<const int4*>(pinfo + applied + tid));
        s_col[tid] = pi.y;
        s_inv[tid] = (uint32_t)pi.z;
      }
      __syncthreads();
      // multipliers of each own row by forward substitution on the K pivot
      // columns (one thread per row)
      for (int lr0 = 0; lr0 < own; lr0 += 32) {
        if (tid < 32 && lr0 + tid < own) {
          const uint32_t* Wl = W + (size_t)(lr0 + tid) * n;
          uint32_t cmv[kChainBatch];
          for (int kk = 0; kk < K; ++kk) {
            uint32_t v = Wl[s_col[kk]];
            for (int q = 0; q < kk; ++q)
              v = f_sub(v, ch_mulm<kIs2>(cmv[q], U[(size_t)q * n + s_col[kk]], F), F);
            const uint32_t cmul = ch_mulm<kIs2>(s_inv[kk], v, F);
            cmv[kk] = f_to_mont(cmul, F);
            s_cm[kk * 32 + tid] = cmv[kk];
          }
        }
        __syncthreads();
        // W[l][j] -= sum_k c_k U_k[j]  (one Montgomery reduction per element)
        const int rows = min(32, own - lr0);
        for (int idx = tid; idx < rows * n; idx += kLeafThreads) {
          const int rr = idx / n, j = idx - rr * n;
          uint32_t* wp = W + (size_t)(lr0 + rr) * n + j;
          uint32_t sub;
          if (kIs2) {
            uint32_t s2 = 0;
            for (int kk = 0; kk < K; ++kk) s2 ^= s_cm[kk * 32 + rr] & U[(size_t)kk * n + j];
            sub = s2;
          } else if (K * (uint64_t)F.p < (1ull << 32)) {
            uint64_t acc = 0;
            for (int kk = 0; kk < K; ++kk) acc += (uint64_t)s_cm[kk * 32 + rr] * U[(size_t)kk * n + j];
            sub = f_redc(acc, F);
          } else {
            sub = 0;
            for (int kk = 0; kk < K; ++kk)
              sub = f_add(sub, f_redc((uint64_t)s_cm[kk * 32 + rr] * U[(size_t)kk * n + j], F), F);
          }
          *wp = f_sub(*wp, sub, F);
        }
        __syncthreads();
        // store the multipliers (plain form) at the pivot columns
        for (int idx = tid; idx < rows * K; idx += kLeafThreads) {
          const int rr = idx / K, kk = idx - rr * K;
          const uint32_t cm = s_cm[kk * 32 + rr];
          W[(size_t)(lr0 + rr) * n + s_col[kk]] = kIs2 ? cm : f_redc((uint64_t)cm, F);
        }
        __syncthreads();
      }
      for (int kk = tid; kk < K; kk += kLeafThreads) ispiv[s_col[kk]] = 1;
      __syncthreads();
      applied += K;
    }
    if (done >= cta) break;
  }

  // phase 2: factor the own rows in order (every earlier pivot is applied)
  int np = applied;
  if (ok) {
    for (int lr = 0; lr < own && np < mn; ++lr) {
      uint32_t* Wl = W + (size_t)lr * n;
      int jl = INT_MAX;
      for (int j = tid; j < n; j += kLeafThreads)
        if (!ispiv[j] && Wl[j] != 0u) {
          jl = j;
          break;
        }
      const int j0 = block_min(jl, s_red);
      if (j0 == INT_MAX) continue;  // the row reduced to zero
      const uint32_t inv = f_inv(Wl[j0], F, inv_table);
      const uint32_t inv_m = f_to_mont(inv, F);
      // publish the pivot row with its pivot-column entries zeroed; the
      // multipliers of the own rows below it
      uint32_t* dst = pub + (size_t)np * n;
      for (int j = tid; j < n; j += kLeafThreads) {
        const uint32_t v = ispiv[j] ? 0u : Wl[j];
        U[j] = v;
        dst[j] = v;
      }
      const int below = own - lr - 1;
      if (tid < below) {
        const uint32_t wl = W[(size_t)(lr + 1 + tid) * n + j0];
        const uint32_t cmul = ch_mulm<kIs2>(inv_m, wl, F);
        s_mul[tid] = cmul;
        s_mulm[tid] = f_to_mont(cmul, F);
      }
      if (tid == 0) pinfo[np] = PivInfo{r0 + lr, j0, inv_m, 0};
      __syncthreads();
      if (tid == 0) {
        ispiv[j0] = 1;
        // the release store publishes the row written by the whole CTA
        // (ordered before it by the block barrier)
        chain_release(&sync->word, ((unsigned long long)cta << 32) | (unsigned)(np + 1));
      }
      // eliminate the own rows below it: all threads over (row, column), the
      // pivot column receiving the multiplier (an L entry)
      for (int b = 0; b < below; ++b) {
        const uint32_t cm = s_mulm[b];
        if (cm == 0u) continue;
        uint32_t* W2 = W + (size_t)(lr + 1 + b) * n;
        for (int j = tid; j < n; j += kLeafThreads)
          W2[j] = j == j0 ? s_mul[b] : f_sub(W2[j], ch_mulm<kIs2>(cm, U[j], F), F);
      }
      __syncthreads();
      ++np;
    }
    if (tid == 0)
      chain_release(&sync->word, ((unsigned long long)(cta + 1) << 32) | (unsigned)np);
  }

  // phase 3: once every CTA is done, write the own rows in the (P, Q) frame
  if (!ok || !wait_word(G, INT_MAX)) return;
  const int r = (int)(s_word & 0xffffffffu);
  for (int i = tid; i < m; i += kLeafThreads) isprow[i] = 0;
  for (int j = tid; j < n; j += kLeafThreads) ispiv[j] = 0;
  __syncthreads();
  for (int k = tid; k < r; k += kLeafThreads) {
    const int4 pi = __ldcg(reinterpret_cast<const int4*>(pinfo + k));
    isprow[pi.x] = 1;
    ispiv[pi.y] = 1;
    rowpos[k] = pi.x;
    colpos[k] = pi.y;
  }
  __syncthreads();
  compact_unflagged(isprow, m, rowpos, r, s_red);
  compact_unflagged(ispiv, n, colpos, r, s_red);
  for (int t = tid; t < m; t += kLeafThreads) rowinv[rowpos[t]] = t;
  __syncthreads();
  for (int lr = warp; lr < own; lr += kLeafWarps) {
    const int t = rowinv[r0 + lr];
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

__global__ void k_chain_init(ChainSync* s, long long wait_cycles) {
  s->word = 0ull;
  s->abort = 0;
  s->wait_cycles = wait_cycles;
}

size_t chain_smem(int m, int n, int R) {
  const size_t ubuf = std::max<size_t>((size_t)kChainBatch * n, 3 * (size_t)m + n);
  return sizeof(uint32_t) * ((size_t)R * n + ubuf + n);
}

}  // namespace

// Rows per CTA of a wavefront leaf: `chain_rows` within what shared memory
// allows (default: the fewest that cover m with one CTA per SM, i.e. the
// most CTAs, which measured fastest), at least that many; 0 when m does not
// fit.
int chain_rows(pluq_ctx* c, int m, int n) {
  int rmax = kChainMaxRows;
  while (rmax > 0 && chain_smem(m, n, rmax) > 220 * 1024) --rmax;
  const int rmin = (m + c->sm_count - 1) / c->sm_count;
  if (rmax < 1 || rmin > rmax) return 0;
  int R = c->chain_rows > 0 ? c->chain_rows : rmin;
  if (R > rmax) R = rmax;
  if (R < rmin) R = rmin;
  if (R > m) R = m;
  return R < 1 ? 1 : R;
}

int launch_leaf_chain(pluq_ctx* c, uint32_t* X, int64_t ldx, int m, int n, int32_t* perm_r,
                      int32_t* perm_c, int32_t* rank_out) {
  static const cudaError_t attr0 = cudaFuncSetAttribute(
      k_leaf_chain<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  static const cudaError_t attr1 = cudaFuncSetAttribute(
      k_leaf_chain<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  PLUQ_CUDA(attr0);
  PLUQ_CUDA(attr1);
  int R = chain_rows(c, m, n);
  if (R < 1) return PLUQ_ERR_INVALID_ARG;
  const int G = (m + R - 1) / R;
  const size_t smem = chain_smem(m, n, R);
  if (smem > 220 * 1024) return PLUQ_ERR_INVALID_ARG;
  const int mn = m < n ? m : n;
  const size_t head = sizeof(ChainSync);
  const size_t need = head + sizeof(PivInfo) * mn + sizeof(uint32_t) * (size_t)mn * n + 256;
  PLUQ_TRY(c->leaf.ensure(need));
  ChainSync* sync = c->leaf.as<ChainSync>();
  PivInfo* pinfo = reinterpret_cast<PivInfo*>(c->leaf.as<char>() + head);
  uint32_t* pub = reinterpret_cast<uint32_t*>(c->leaf.as<char>() + head + sizeof(PivInfo) * mn);
  {
    ProfScope pi(c, PC_INDEX);
    k_chain_init<<<1, 1, 0, c->stream>>>(sync, c->wait_cycles);
  }
  int* err = c->small.as<int>() + 16;
  const uint32_t* tab = inv_table_ptr(c);
  FieldP F = c->F;
  void* args[] = {&X, &ldx, &m, &n, &R, &F, &tab, &perm_r, &perm_c, &rank_out, &sync, &pub,
                  &pinfo, &err};
  ProfScope ps(c, PC_BASE, 0, 8.0 * m * n);
  const void* fn = F.is2 ? (const void*)k_leaf_chain<true> : (const void*)k_leaf_chain<false>;
  PLUQ_CUDA(cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kLeafThreads), args, smem, c->stream));
  return PLUQ_OK;
}

int chain_fits(pluq_ctx* c, int64_t m, int64_t n) {
  if (m <= 0 || n <= 0 || m > c->leaf_dim || n > c->leaf_dim) return 0;
  return chain_rows(c, (int)m, (int)n) > 0;
}
