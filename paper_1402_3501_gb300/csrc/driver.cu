// Host driver of the tile-recursive PLUQ (Sec. 4.1, "Tiled recursive
// elimination"), the C ABI, and the output kernels (rank profiles, rank
// profile matrix, reduced echelon form).
//
// Recursion, for a block A = [A1 A2; A3 A4] (A1 of size m1 x n1), in place:
//   A1 = P1 [L1; M1] [U1 V1] Q1                      (recursive, rank r1)
//   [B1; B2] = P1^T A2,  [C1 C2] = A3 Q1^T           (row / column gathers)
//   D = L1^{-1} B1,  E = C1 U1^{-1}                   (ftrsm)
//   F = B2 - M1 D,  H = A4 - E D,  G = C2 - E V1      (fgemm, F and H as one)
//   F = P2 [L2; M2] [U2 V2] Q2,  G = P3 [L3; M3] [U3 V3] Q3   (recursive; independent)
//   H <- P3^T H Q2^T = [H1 H2; H3 H4]
//   [I; K] = [H1; H3] U2^{-1}                         (ftrsm)
//   [H2; H4] -= [I; K] V2                             (fgemm)
//   O = L3^{-1} H2,  R = H4 - M3 O                    (ftrsm, fgemm)
//   R = P4 [L4; M4] [U4 V4] Q4                        (recursive, rank r4)
// followed by the block-cyclic shifts that bring the four pivot blocks to the
// front: rows [A1p F2p | F_rest | G3p R4p] -> [A1p F2p G3p R4p | F_rest ...],
// columns [A1p | G3p G_rest | F2p R4p] -> [A1p F2p G3p R4p | G_rest ...].
// The L entries of the G-pivot rows on the F-pivot columns are I (not
// L3^{-1} I): G-pivot row = I [0 U2 V2] + L3 [U3 0 O] on the column blocks.
// Each recursive call returns local index vectors for its rows and columns;
// the caller applies them to the parts of its block outside the child and
// composes them into its own.  The pivots of the four calls together are the
// rank profile matrix because every call keeps its non-pivot rows and
// columns in their original relative order.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <thread>
#include <vector>

#include "common.cuh"

namespace {

bool is_prime_u32(uint32_t n) {
  if (n < 2) return false;
  for (uint32_t d : {2u, 3u, 5u, 7u, 11u, 13u}) {
    if (n % d == 0) return n == d;
  }
  // deterministic Miller-Rabin for n < 3,215,031,751 with bases 2, 3, 5, 7
  uint64_t d = n - 1;
  int s = 0;
  while ((d & 1) == 0) {
    d >>= 1;
    ++s;
  }
  for (uint64_t a : {2ull, 3ull, 5ull, 7ull}) {
    uint64_t x = 1, b = a % n, e = d;
    while (e) {
      if (e & 1) x = x * b % n;
      b = b * b % n;
      e >>= 1;
    }
    if (x == 1 || x == n - 1) continue;
    bool comp = true;
    for (int i = 1; i < s; ++i) {
      x = x * x % n;
      if (x == n - 1) {
        comp = false;
        break;
      }
    }
    if (comp) return false;
  }
  return true;
}

int check_p(uint32_t p) {
  if (p < 2 || p >= 0x80000000u) return PLUQ_ERR_P_OUT_OF_RANGE;
  if (!is_prime_u32(p)) return PLUQ_ERR_P_NOT_PRIME;
  return PLUQ_OK;
}

int resolve_form(uint32_t p, int form) {
  if (form == PLUQ_FORM_AUTO) {
    if (limb_form_supported(p)) return PLUQ_FORM_LIMB_F16;
    if (fp64_form_supported(p)) return PLUQ_FORM_FP64;
    return -1;
  }
  if (form == PLUQ_FORM_FP64) return fp64_form_supported(p) ? form : -1;
  if (form == PLUQ_FORM_LIMB_F16) return limb_form_supported(p) ? form : -1;
  return -2;
}

__global__ void k_check_range(const uint32_t* __restrict__ A, int64_t lda, int64_t m, int64_t n,
                              uint32_t p, int* __restrict__ flag) {
  for (int64_t t = blockIdx.y; t < m; t += gridDim.y) {
    const uint32_t* row = A + t * lda;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x)
      if (row[u] >= p) *flag = 1;
  }
}

__global__ void k_copy_mat(uint32_t* __restrict__ dst, int64_t ldd, const uint32_t* __restrict__ src,
                           int64_t lds, int64_t m, int64_t n) {
  for (int64_t t = blockIdx.y; t < m; t += gridDim.y) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x)
      dst[t * ldd + u] = src[t * lds + u];
  }
}

// Sorted set of the first r entries of a permutation of [0, cnt): a bitmap in
// shared memory, then an ordered compaction (one CTA).
// out[0..r) = the first r entries of perm (distinct, < cnt) in increasing
// order, by a bitmap in shared memory and a block prefix count.
__device__ void sorted_profile(const int32_t* __restrict__ perm, int64_t r, int64_t cnt,
                               int32_t* __restrict__ out, uint32_t* bits) {
  __shared__ int32_t warp_tot[32];
  const int64_t words = (cnt + 31) / 32;
  for (int64_t w = threadIdx.x; w < words; w += blockDim.x) bits[w] = 0u;
  __syncthreads();
  for (int64_t k = threadIdx.x; k < r; k += blockDim.x) {
    const int32_t v = perm[k];
    atomicOr(&bits[v >> 5], 1u << (v & 31));
  }
  __syncthreads();
  // each thread owns a contiguous range of words
  const int64_t per = (words + blockDim.x - 1) / blockDim.x;
  const int64_t w0 = threadIdx.x * per, w1 = min(words, w0 + per);
  int32_t mine = 0;
  for (int64_t w = w0; w < w1; ++w) mine += __popc(bits[w]);
  // block exclusive scan of `mine`
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t incl = mine;
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x / 32;
    int32_t v = lane < nw ? warp_tot[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    if (lane < nw) warp_tot[lane] = v;  // inclusive warp totals
  }
  __syncthreads();
  int32_t pos = incl - mine + (warp > 0 ? warp_tot[warp - 1] : 0);
  for (int64_t w = w0; w < w1; ++w) {
    uint32_t b = bits[w];
    while (b) {
      const int bit = __ffs(b) - 1;
      out[pos++] = (int32_t)(w * 32 + bit);
      b &= b - 1;
    }
  }
}

__global__ void k_profile(const int32_t* __restrict__ perm, int64_t r, int64_t cnt,
                          int32_t* __restrict__ out) {
  extern __shared__ uint32_t bits[];
  sorted_profile(perm, r, cnt, out, bits);
}

// Row and column rank profiles of a batch: block (b, 0) sorts matrix b's
// pivot rows, block (b, 1) its pivot columns.
struct ProfileDesc {
  const int32_t* P;
  const int32_t* Q;
  int32_t* rrp;
  int32_t* crp;
  int64_t m, n, r;
};

__global__ void k_profiles_batched(const ProfileDesc* __restrict__ d) {
  extern __shared__ uint32_t bits[];
  const ProfileDesc e = d[blockIdx.x];
  if (e.r <= 0) return;
  if (blockIdx.y == 0) {
    if (e.rrp) sorted_profile(e.P, e.r, e.m, e.rrp, bits);
  } else {
    if (e.crp) sorted_profile(e.Q, e.r, e.n, e.crp, bits);
  }
}

__global__ void k_rpm_col_of_row(const int32_t* __restrict__ P, const int32_t* __restrict__ Q,
                                 int64_t r, int64_t m, int32_t* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < m) out[t] = -1;
}
__global__ void k_rpm_fill(const int32_t* __restrict__ P, const int32_t* __restrict__ Q, int64_t r,
                           int32_t* __restrict__ out) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < r) out[P[k]] = Q[k];
}

__global__ void k_invert_perm(const int32_t* __restrict__ Q, int64_t n, int32_t* __restrict__ qinv) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u < n) qinv[Q[u]] = (int32_t)u;
}

// RREF row t = pivot ord[t] (ord[t] = qinv[crp[t]]) of X = [I | U1^{-1} U2]
// in the Q frame, scattered back to the original column order: entry (t, col)
// goes to R[t * rs + col * cs] (rs = ldr, cs = 1 for the row form; rs = 1,
// cs = ldc for its transpose, the column echelon form of the transposed input).
__global__ void k_rref_scatter(const uint32_t* __restrict__ W, int64_t ldw, int64_t r, int64_t n,
                               const int32_t* __restrict__ qinv, const int32_t* __restrict__ crp,
                               uint32_t* __restrict__ R, int64_t rs, int64_t cs) {
  for (int64_t t = blockIdx.y; t < r; t += gridDim.y) {
    const int32_t k = qinv[crp[t]];
    for (int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; col < n;
         col += (int64_t)gridDim.x * blockDim.x) {
      const int32_t j = qinv[col];
      R[t * rs + col * cs] = j < r ? (j == k ? 1u : 0u) : W[(int64_t)k * ldw + j];
    }
  }
}

// dst (cols x rows, ldd) = src (rows x cols, lds)^T through 32 x 32 tiles.
__global__ void k_transpose(uint32_t* __restrict__ dst, int64_t ldd,
                            const uint32_t* __restrict__ src, int64_t lds, int64_t rows,
                            int64_t cols) {
  __shared__ uint32_t tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t r = r0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < rows && c < cols) ? src[r * lds + c] : 0u;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t c = c0 + i, r = r0 + threadIdx.x;
    if (c < cols && r < rows) dst[c * ldd + r] = tile[threadIdx.x][i];
  }
}

__global__ void k_store_rank(int64_t* dst, int64_t r) { *dst = r; }

__global__ void k_merge_err(int* dst, const int* src) {
  if (*src != 0 && *dst == 0) *dst = *src;
}

// flags[0] = (perm_r[i] == i for all i < m), flags[1] = (perm_c[j] == j for all
// j < n): a leaf whose pivots fell on the diagonal leaves the blocks beside it
// unpermuted, and the recursion skips those permutation launches.
__global__ void k_perm_identity(const int32_t* __restrict__ perm_r, int m,
                                const int32_t* __restrict__ perm_c, int n, int32_t* flags) {
  int bad_r = 0, bad_c = 0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) bad_r |= perm_r[i] != i;
  for (int j = threadIdx.x; j < n; j += blockDim.x) bad_c |= perm_c[j] != j;
  bad_r = __syncthreads_or(bad_r);
  bad_c = __syncthreads_or(bad_c);
  if (threadIdx.x == 0) {
    flags[0] = !bad_r;
    flags[1] = !bad_c;
  }
}

dim3 grid2(int64_t rows, int64_t cols) {
  int64_t gx = cdiv(cols, 256);
  if (gx > 32) gx = 32;
  int64_t gy = rows < 65535 ? rows : 65535;
  if (gy < 1) gy = 1;
  if (gx < 1) gx = 1;
  return dim3((unsigned)gx, (unsigned)gy, 1);
}

// ------------------------------------------------ concurrent F and G --
//
// The recursive calls on F and G read and write disjoint blocks of A and
// disjoint ranges of the index vectors, and neither needs the other's result
// (Sec. 2.3: F and G are factored independently before H is updated), so
// they run on two child contexts at once: one host thread each, one stream
// each, their own workspace, half the parent's SMs for cooperative leaves.
constexpr int64_t kForkMinElems = 1024;

void destroy_lane(pluq_ctx* l) {
  if (!l) return;
  destroy_lane(l->lane[0]);
  destroy_lane(l->lane[1]);
  destroy_lane(l->lane[2]);
  for (cudaEvent_t e : l->la_ev)
    if (e) cudaEventDestroy(e);
  l->perm_r = DevBuf{};  // views of the parent's buffers
  l->perm_c = DevBuf{};
  l->inv_table = DevBuf{};
  l->scratch.release();
  l->pack.release();
  l->tmp_i.release();
  l->tri_inv.release();
  l->small.release();
  l->leaf.release();
  l->work.release();
  l->wino.release();
  for (cudaEvent_t e : l->prof.pool) cudaEventDestroy(e);
  if (l->fork_ev) cudaEventDestroy(l->fork_ev);
  for (cudaEvent_t e : l->side_ev)
    if (e) cudaEventDestroy(e);
  if (l->host_small) cudaFreeHost(l->host_small);
  if (l->own_stream) cudaStreamDestroy(l->own_stream);
  delete l;
}

// Child context i of c, configured for a branch of m x n.
int get_lane(pluq_ctx* c, int i, int64_t m, int64_t n, pluq_ctx** out) {
  pluq_ctx*& l = c->lane[i];
  if (!l) {
    pluq_ctx* nl = new pluq_ctx();
    nl->device = c->device;
    nl->parent = c;
    nl->ws = c->ws;
    bind_workspace(nl);
    nl->lane_depth = c->lane_depth + 1;
    if (cudaStreamCreateWithFlags(&nl->own_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMallocHost(&nl->host_small, 256) != cudaSuccess) {
      cudaGetLastError();
      destroy_lane(nl);
      return PLUQ_ERR_CUDA;
    }
    l = nl;
  }
  l->stream = l->own_stream;
  l->sm_count = std::max(1, c->sm_count / 2);
  l->wait_cycles = c->wait_cycles;
  l->wino_min = c->wino_min;
  l->F = c->F;
  l->form = c->form;
  l->bm = c->bm;
  l->bn = c->bn;
  l->trsm_block = c->trsm_block;
  l->strip_max = c->strip_max;
  l->leaf_dim = c->leaf_dim;
  l->leaf_kind = c->leaf_kind;
  l->leaf_density = c->leaf_density;
  l->chain_rows = c->chain_rows;
  l->fork_depth = c->fork_depth;
  l->thin_gemm = c->thin_gemm;
  l->decomposition = c->decomposition;
  l->slab_rows = c->slab_rows;
  l->depth_slots = c->depth_slots;
  l->mmax = c->mmax;
  l->nmax = c->nmax;
  l->limb_plan_p = c->limb_plan_p;
  for (int k = 0; k < 6; ++k) l->limb_plan[k] = c->limb_plan[k];
  l->limb_variant = c->limb_variant;
  l->lookahead = c->lookahead;
  l->fused_kmax = c->fused_kmax;
  l->perm_r = c->perm_r;
  l->perm_c = c->perm_c;
  l->inv_table = c->inv_table;
  l->inv_table_p = c->inv_table_p;
  l->prof.on = false;
  for (int k = 0; k < PC_COUNT; ++k) l->launches[k] = 0;
  l->n_base = l->n_nodes = l->n_gemm = 0;
  // workspace for everything inside an m x n block, sized once (a growing
  // allocation would synchronise the device under the other branch)
  const int64_t mn = std::max<int64_t>(1, std::min(m, n));
  PLUQ_TRY(l->small.ensure(256));
  PLUQ_TRY(l->scratch.ensure(sizeof(uint32_t) * std::max<int64_t>(m * n, 1)));
  PLUQ_TRY(l->tmp_i.ensure(sizeof(int32_t) * std::max(c->mmax, c->nmax)));
  PLUQ_TRY(l->tri_inv.ensure(sizeof(uint32_t) * cdiv(mn, std::max(1, c->trsm_block)) * 64 * 64));
  if (c->form == PLUQ_FORM_LIMB_F16) {
    const int64_t kp = cdiv(mn + 64, 64) * 64;
    const int64_t rows = cdiv(m, 128) * 128 + cdiv(n, 128) * 128;
    PLUQ_TRY(l->pack.ensure(sizeof(uint16_t) * 4 * rows * kp + 4096));
  }
  const int64_t ld = std::min<int64_t>(std::max(c->leaf_dim, 1), std::max(m, n));
  PLUQ_TRY(l->leaf.ensure(4096 + 16 * ld + 4 * ld * ld + 8 * (int64_t)c->sm_count * (ld + 4)));
  PLUQ_CUDA(cudaMemsetAsync(l->small.ptr, 0, 256, l->stream));
  *out = l;
  return PLUQ_OK;
}

void merge_lane_stats(pluq_ctx* c, const pluq_ctx* l) {
  for (int k = 0; k < PC_COUNT; ++k) c->launches[k] += l->launches[k];
  c->n_base += l->n_base;
  c->n_nodes += l->n_nodes;
  c->n_gemm += l->n_gemm;
}

// Whether a recursive call's local row / column index vectors are the identity.
struct Ident {
  bool r = true, c = true;
};

// Which parts of a block's factorization must end in their compressed
// positions: L (unit lower, with M), U (upper, with V), both, or neither (only
// the index vectors and the rank).  A full PLUQ keeps both everywhere.  The
// reduced echelon form needs U only and the rank profiles neither, at the top;
// a child keeps what its parent still reads after it returns (all of A1; U2,
// V2 of F; L3, M3 of G) plus the parent's own needs for its block.
enum Keep { KEEP_NONE = 0, KEEP_L = 1, KEEP_U = 2, KEEP_LU = 3 };

struct Recursion {
  pluq_ctx* c;
  uint32_t* A;
  int64_t lda;
  int32_t* rank_slot;  // device int32
  int32_t* PR(int d) { return c->perm_r.as<int32_t>() + (int64_t)d * c->mmax; }
  int spare() const { return c->depth_slots - 1; }
  int32_t* PC(int d) { return c->perm_c.as<int32_t>() + (int64_t)d * c->nmax; }
  uint32_t* X(int64_t R0, int64_t C0, int64_t i, int64_t j) {
    return A + (R0 + i) * lda + (C0 + j);
  }

  int64_t split(int64_t x) { return x / 2; }

  // Runs the recursive calls on F and G at once on the two child contexts
  // (this thread takes G); returns after both streams have finished.
  int fork_fg(int64_t R0, int64_t C0, int64_t m1, int64_t n1, int64_t m2, int64_t n2, int64_t r1,
              int d, int64_t* r2, int64_t* r3, Ident* id2, Ident* id3, int keep) {
    pluq_ctx* lf = nullptr;
    pluq_ctx* lg = nullptr;
    // F's lane also runs f_post: D and H (r1 + m2 rows) by F's columns
    PLUQ_TRY(get_lane(c, 0, std::max(m1 - r1, m2 + r1), n2, &lf));
    PLUQ_TRY(get_lane(c, 1, m2, n1 - r1, &lg));
    if (!c->fork_ev) PLUQ_CUDA(cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming));
    PLUQ_CUDA(cudaEventRecord(c->fork_ev, c->stream));
    PLUQ_CUDA(cudaStreamWaitEvent(lf->stream, c->fork_ev, 0));
    PLUQ_CUDA(cudaStreamWaitEvent(lg->stream, c->fork_ev, 0));
    auto finish = [](pluq_ctx* l, int st) {
      // the branch's last kernels and its device error word
      if (cudaMemcpyAsync(l->host_small, l->small.ptr, 32 * sizeof(int32_t),
                          cudaMemcpyDeviceToHost, l->stream) != cudaSuccess ||
          cudaStreamSynchronize(l->stream) != cudaSuccess) {
        cudaGetLastError();
        return st != PLUQ_OK ? st : PLUQ_ERR_CUDA;
      }
      if (st != PLUQ_OK) return st;
      return l->host_small[16] != 0 ? l->host_small[16] : PLUQ_OK;
    };
    int st_f = PLUQ_OK, st_g = PLUQ_OK;
    std::thread tf([&] {
      if (cudaSetDevice(lf->device) != cudaSuccess) {
        st_f = PLUQ_ERR_CUDA;
        return;
      }
      Recursion rf{lf, A, lda, lf->small.as<int32_t>() + 8};
      int st = rf.node(R0 + r1, C0 + n1, m1 - r1, n2, d + 1, r2, id2, keep | KEEP_U);
      if (st == PLUQ_OK) st = rf.f_post(R0, C0, m1, n1, m2, n2, r1, *r2, d, *id2, keep);
      st_f = finish(lf, st);
    });
    Recursion rg{lg, A, lda, lg->small.as<int32_t>() + 8};
    st_g = finish(lg, rg.node(R0 + m1, C0 + r1, m2, n1 - r1, d + 1, r3, id3, keep | KEEP_L));
    tf.join();
    merge_lane_stats(c, lf);
    merge_lane_stats(c, lg);
    c->leaf_density = lg->leaf_density;
    return st_f != PLUQ_OK ? st_f : st_g;
  }

  // What follows F and needs nothing of G: F's permutations of the blocks
  // beside it (M1; D and H by its columns) and the first H steps,
  // [I; K] = H[:, :r2] U2^{-1} and H[:, r2:] -= [I; K] V2.  Both act on H
  // row by row, so they commute with G's later row permutation of H and run
  // in F's branch while G is still being factored.
  int f_post(int64_t R0, int64_t C0, int64_t m1, int64_t n1, int64_t m2, int64_t n2, int64_t r1,
             int64_t r2, int d, Ident id2, int keep) {
    int32_t* pr = PR(d) + R0;
    int32_t* pc = PC(d) + C0;
    int32_t* cr = PR(d + 1);
    int32_t* cc = PC(d + 1);
    PLUQ_TRY(compose_pair(pr + r1, cr + R0 + r1, m1 - r1, pc + n1, cc + C0 + n1, n2, id2));
    // M1 (L) by F's row permutation: storage only
    if (!id2.r && (keep & KEEP_L))
      PLUQ_TRY(permute_rows(c, X(R0, C0, r1, 0), lda, m1 - r1, r1, cr + R0 + r1));
    // D (rows 0..r1; U, storage only) and H (rows m1..m) by F's column permutation
    if (!id2.c) {
      if (keep & KEEP_U)
        PLUQ_TRY(permute_cols2(c, X(R0, C0, 0, n1), lda, 0, r1, m1, m2, n2, cc + C0 + n1));
      else
        PLUQ_TRY(permute_cols2(c, X(R0, C0, 0, n1), lda, m1, m2, 0, 0, n2, cc + C0 + n1));
    }
    if (r2 > 0) {
      PLUQ_TRY(trsm_right_upper(c, X(R0, C0, r1, n1), lda, r2, X(R0, C0, m1, n1), lda, m2));
      PLUQ_TRY(fgemm_sub(c, m2, n2 - r2, r2, X(R0, C0, m1, n1), lda, X(R0, C0, r1, n1 + r2), lda,
                         X(R0, C0, m1, n1 + r2), lda));
    }
    return PLUQ_OK;
  }

  // The updates after A1 on two streams (see node); returns once this
  // context's stream waits for the other's work (no host synchronisation).
  // With h1 > 0 (F and G empty: r1 = m1 = n1), H's update is split at R's
  // first quarter: H11 (h1 x w1) on this stream, the rest on the look-ahead
  // child context's stream, whose completion *la_done then records; R's
  // recursion starts on H11 at once and waits for la_done only after its own
  // A1 (see node).
  int side_stream_update(int64_t R0, int64_t C0, int64_t m1, int64_t n1, int64_t m2, int64_t n2,
                         int64_t r1, int d = 0, int64_t h1 = 0, int64_t w1 = 0,
                         cudaEvent_t* la_done = nullptr) {
    const int64_t m = m1 + m2;
    pluq_ctx* lg = nullptr;
    PLUQ_TRY(get_lane(c, 1, m2, n1, &lg));
    for (cudaEvent_t* e : {&c->fork_ev, &c->side_ev[0], &c->side_ev[1]})
      if (!*e) PLUQ_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    PLUQ_CUDA(cudaEventRecord(c->fork_ev, c->stream));
    PLUQ_CUDA(cudaStreamWaitEvent(lg->stream, c->fork_ev, 0));
    // G's stream: E, then G -= E V1
    const int64_t diag0 = R0 == C0 ? R0 : -1;
    PLUQ_TRY(trsm_right_upper(lg, X(R0, C0, 0, 0), lda, r1, X(R0, C0, m1, 0), lda, m2, diag0));
    PLUQ_CUDA(cudaEventRecord(c->side_ev[0], lg->stream));
    PLUQ_TRY(fgemm_sub(lg, m2, n1 - r1, r1, X(R0, C0, m1, 0), lda, X(R0, C0, 0, r1), lda,
                       X(R0, C0, m1, r1), lda));
    PLUQ_CUDA(cudaEventRecord(c->side_ev[1], lg->stream));
    // this stream: D, then [F; H] -= [M1; E] D once E is ready
    PLUQ_TRY(trsm_left_lower_unit(c, X(R0, C0, 0, 0), lda, r1, X(R0, C0, 0, n1), lda, n2, diag0));
    PLUQ_CUDA(cudaStreamWaitEvent(c->stream, c->side_ev[0], 0));
    if (h1 > 0) {
      pluq_ctx* la = nullptr;
      PLUQ_TRY(get_lane(c, 2, m2, n2, &la));
      if ((int)c->la_ev.size() < 2 * (d + 1)) c->la_ev.resize(2 * (d + 1), nullptr);
      for (int k = 0; k < 2; ++k)
        if (!c->la_ev[2 * d + k])
          PLUQ_CUDA(cudaEventCreateWithFlags(&c->la_ev[2 * d + k], cudaEventDisableTiming));
      PLUQ_CUDA(cudaEventRecord(c->la_ev[2 * d], c->stream));  // D and E ready
      PLUQ_CUDA(cudaStreamWaitEvent(la->stream, c->la_ev[2 * d], 0));
      PLUQ_TRY(fgemm_sub(c, h1, w1, r1, X(R0, C0, m1, 0), lda, X(R0, C0, 0, n1), lda,
                         X(R0, C0, m1, n1), lda));
      PLUQ_TRY(fgemm_sub(la, h1, n2 - w1, r1, X(R0, C0, m1, 0), lda, X(R0, C0, 0, n1 + w1), lda,
                         X(R0, C0, m1, n1 + w1), lda));
      PLUQ_TRY(fgemm_sub(la, m2 - h1, n2, r1, X(R0, C0, m1 + h1, 0), lda, X(R0, C0, 0, n1), lda,
                         X(R0, C0, m1 + h1, n1), lda));
      // its device error word joins this context's before the hand-over
      k_merge_err<<<1, 1, 0, la->stream>>>(c->small.as<int>() + 16, la->small.as<int>() + 16);
      PLUQ_CUDA(cudaGetLastError());
      PLUQ_CUDA(cudaEventRecord(c->la_ev[2 * d + 1], la->stream));
      *la_done = c->la_ev[2 * d + 1];
      merge_lane_stats(c, la);
      for (int k = 0; k < PC_COUNT; ++k) la->launches[k] = 0;
      la->n_base = la->n_nodes = la->n_gemm = 0;
    } else {
      PLUQ_TRY(fgemm_sub(c, m - r1, n2, r1, X(R0, C0, r1, 0), lda, X(R0, C0, 0, n1), lda,
                         X(R0, C0, r1, n1), lda));
    }
    PLUQ_CUDA(cudaStreamWaitEvent(c->stream, c->side_ev[1], 0));
    // the other stream's device error word joins this context's
    k_merge_err<<<1, 1, 0, c->stream>>>(c->small.as<int>() + 16, lg->small.as<int>() + 16);
    PLUQ_CUDA(cudaGetLastError());
    merge_lane_stats(c, lg);
    for (int k = 0; k < PC_COUNT; ++k) lg->launches[k] = 0;
    lg->n_base = lg->n_nodes = lg->n_gemm = 0;
    return PLUQ_OK;
  }

  // Composition with a child's local index vectors; a child whose vectors are
  // the identity changes nothing, so its launch is skipped.
  int compose_pair(int32_t* base_r, const int32_t* perm_r, int64_t count_r, int32_t* base_c,
                   const int32_t* perm_c, int64_t count_c, Ident id) {
    if (id.r && id.c) return PLUQ_OK;
    if (id.r) return launch_compose(c, base_c, perm_c, count_c);
    if (id.c) return launch_compose(c, base_r, perm_r, count_r);
    return launch_compose_pair(c, base_r, perm_r, count_r, base_c, perm_c, count_c);
  }

  // Factors the m x n block at (R0, C0); *r_out receives its rank and *id
  // whether its local row / column index vectors are the identity (then the
  // caller's permutations of the blocks beside it are no-ops and skipped).
  // pending: an event the blocks beside A1 (A2, A3, A4) wait for before this
  // node touches them (the look-ahead update of the parent's H), or null.
  int node(int64_t R0, int64_t C0, int64_t m, int64_t n, int d, int64_t* r_out, Ident* id,
           int keep = KEEP_LU, cudaEvent_t pending = nullptr) {
    int32_t* pr = PR(d) + R0;
    int32_t* pc = PC(d) + C0;
    *r_out = 0;
    *id = Ident{};
    if (m == 0 || n == 0) {
      PLUQ_TRY(launch_iota_pair(c, pr, m, pc, n));
      return PLUQ_OK;
    }
    // wavefront leaves win on dense blocks, cluster (else barrier) leaves on
    // rank-deficient ones; kind 2 guesses from the rank density of the
    // previous leaf
    const bool dense = c->leaf_density > 0.5;
    const bool tile = c->leaf_dim > 0 && (c->leaf_kind == 4 || (c->leaf_kind == 2 && dense)) &&
                      tile_leaf_fits(c, m, n);
    const bool want_chain = c->leaf_kind == 1 || ((c->leaf_kind == 2 || c->leaf_kind == 4) && dense);
    const bool chain = !tile && c->leaf_dim > 0 && want_chain && chain_fits(c, m, n);
    const bool cluster = !tile && !chain && c->leaf_dim > 0 &&
                         (c->leaf_kind == 3 || c->leaf_kind == 2 || c->leaf_kind == 4) &&
                         cluster_leaf_fits(c, m, n);
    const bool leaf = !tile && !chain && !cluster && c->leaf_dim > 0 && leaf_fits(c, m, n);
    if (tile || chain || cluster || leaf || (m <= c->bm && n <= c->bn)) {
      c->n_base++;
      if (tile)
        PLUQ_TRY(launch_leaf_tile(c, X(R0, C0, 0, 0), lda, (int)m, (int)n, pr, pc, rank_slot));
      else if (chain)
        PLUQ_TRY(launch_leaf_chain(c, X(R0, C0, 0, 0), lda, (int)m, (int)n, pr, pc, rank_slot));
      else if (cluster)
        PLUQ_TRY(launch_leaf_cluster(c, X(R0, C0, 0, 0), lda, (int)m, (int)n, pr, pc, rank_slot));
      else if (leaf)
        PLUQ_TRY(launch_leaf_pluq(c, X(R0, C0, 0, 0), lda, (int)m, (int)n, pr, pc, rank_slot));
      else
        PLUQ_TRY(launch_base_pluq(c, X(R0, C0, 0, 0), lda, (int)m, (int)n, pr, pc, rank_slot));
      // whether the leaf's index vectors are the identity (ints 12, 13)
      {
        ProfScope ps(c, PC_INDEX, 0, 4.0 * (m + n));
        k_perm_identity<<<1, 1024, 0, c->stream>>>(pr, (int)m, pc, (int)n,
                                                    c->small.as<int32_t>() + 12);
        PLUQ_CUDA(cudaGetLastError());
      }
      // rank (int 8 of the scalar block) and the device error word (int 16)
      PLUQ_CUDA(cudaMemcpyAsync(c->host_small, c->small.ptr, 32 * sizeof(int32_t),
                                cudaMemcpyDeviceToHost, c->stream));
      PLUQ_CUDA(cudaStreamSynchronize(c->stream));
      if (c->host_small[16] != 0) return c->host_small[16];
      *r_out = c->host_small[8];
      id->r = c->host_small[12] != 0;
      id->c = c->host_small[13] != 0;
      if (tile || chain || cluster || leaf)
        c->leaf_density = (double)*r_out / (double)std::min(m, n);
      const int64_t b = c->dinv_b;
      if (b > 0 && c->dinv_ok && m == b && n == b && *r_out == b && R0 == C0 && R0 % b == 0 &&
          R0 / b < (int64_t)c->dinv_valid.size()) {
        if (!c->prof.on && c->lane_depth < c->fork_depth) {
          // the two triangles at once: U's on the G child context's stream
          pluq_ctx* lg = nullptr;
          PLUQ_TRY(get_lane(c, 1, b, b, &lg));
          for (cudaEvent_t* e : {&c->fork_ev, &c->side_ev[0]})
            if (!*e) PLUQ_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
          PLUQ_CUDA(cudaEventRecord(c->fork_ev, c->stream));
          PLUQ_CUDA(cudaStreamWaitEvent(lg->stream, c->fork_ev, 0));
          PLUQ_TRY(cache_leaf_inverse(lg, c, true, X(R0, C0, 0, 0), lda, R0 / b));
          k_merge_err<<<1, 1, 0, lg->stream>>>(c->small.as<int>() + 16, lg->small.as<int>() + 16);
          PLUQ_CUDA(cudaGetLastError());
          PLUQ_CUDA(cudaEventRecord(c->side_ev[0], lg->stream));
          PLUQ_TRY(cache_leaf_inverse(c, c, false, X(R0, C0, 0, 0), lda, R0 / b));
          PLUQ_CUDA(cudaStreamWaitEvent(c->stream, c->side_ev[0], 0));
          merge_lane_stats(c, lg);
          for (int k = 0; k < PC_COUNT; ++k) lg->launches[k] = 0;
          lg->n_base = lg->n_nodes = lg->n_gemm = 0;
        } else {
          PLUQ_TRY(cache_leaf_inverses(c, X(R0, C0, 0, 0), lda, R0 / b));
        }
        c->dinv_valid[R0 / b] = 1;
      }
      return PLUQ_OK;
    }
    if (d + 2 >= c->depth_slots) return PLUQ_ERR_INVALID_ARG;  // the last slot is scratch
    c->n_nodes++;
    int64_t lim_m = c->leaf_dim > 0 ? c->leaf_dim : c->bm;
    int64_t lim_n = c->leaf_dim > 0 ? c->leaf_dim : c->bn;
    if (m <= lim_m && n <= lim_n) {
      // within the cut-off but no leaf kernel takes the block (its shared
      // memory needs more SMs than this context has): split it all the same
      lim_m = std::max<int64_t>(1, m / 2);
      lim_n = std::max<int64_t>(1, n / 2);
    }
    int64_t m1 = m > lim_m ? split(m) : m;
    int64_t n1 = n > lim_n ? split(n) : n;
    if (c->decomposition == 1 && (m > lim_m || n > lim_n)) {
      // tiled iterative (Sec. 4.1): a slab of the first rows across all
      // columns (A2, A4 empty: then G, the rows below, is the next step), and
      // within a slab a tile of the first columns (A3, A4 empty: F, the
      // columns right of it, is next)
      const int64_t b = c->slab_rows > 0 ? c->slab_rows : lim_m;
      if (m > b) {
        m1 = b;
        n1 = n;
      } else if (n > lim_n) {
        m1 = m;
        n1 = lim_n;
      } else {
        m1 = lim_m;
        n1 = n;
      }
    }
    const int64_t m2 = m - m1, n2 = n - n1;
    cudaEvent_t la_pending = nullptr;  // this node's look-ahead update of R's A2, A3, A4
    int32_t* cr = PR(d + 1);
    int32_t* cc = PC(d + 1);
    PLUQ_TRY(launch_iota_pair(c, pr, m, pc, n));

    // A1
    int64_t r1 = 0;
    Ident id1, id2, id3, id4;
    PLUQ_TRY(node(R0, C0, m1, n1, d + 1, &r1, &id1, KEEP_LU));
    // the parent's look-ahead update of this block's A2, A3, A4
    if (pending) PLUQ_CUDA(cudaStreamWaitEvent(c->stream, pending, 0));
    if (r1 < m1 || r1 < n1) {
      // F or G is non-empty: blocks move by shifts, the diagonal blocks of later
      // triangles are no longer the cached leaves
      for (pluq_ctx* o = c; o; o = o->parent) o->dinv_ok = false;
    }
    PLUQ_TRY(compose_pair(pr, cr + R0, m1, pc, cc + C0, n1, id1));
    if (!id1.r) PLUQ_TRY(permute_rows(c, X(R0, C0, 0, n1), lda, m1, n2, cr + R0));
    if (!id1.c) PLUQ_TRY(permute_cols(c, X(R0, C0, m1, 0), lda, m2, n1, cc + C0));
    if (r1 > 0) {
      // D = L1^{-1} B1 and E = C1 U1^{-1} are independent, and so is G's
      // update (it needs E only): E and G -= E V1 go to the G child context's
      // stream while this one solves D, then [F; H] -= [M1; E] D waits for E
      const bool side = c->lane_depth < c->fork_depth && !c->prof.on && m2 > 0 &&
                        (int64_t)r1 * (m2 + n2) >= kForkMinElems * 64;
      // look-ahead: A1 of full rank (F and G empty) and an R that splits
      const bool la = side && c->lookahead && c->decomposition == 0 && r1 == m1 && r1 == n1 &&
                      m2 > lim_m && n2 > lim_n;
      if (la) {
        PLUQ_TRY(side_stream_update(R0, C0, m1, n1, m2, n2, r1, d, split(m2), split(n2),
                                    &la_pending));
      } else if (side) {
        PLUQ_TRY(side_stream_update(R0, C0, m1, n1, m2, n2, r1));
      } else {
        const int64_t diag0 = R0 == C0 ? R0 : -1;
        PLUQ_TRY(trsm_left_lower_unit(c, X(R0, C0, 0, 0), lda, r1, X(R0, C0, 0, n1), lda, n2,
                                      diag0));
        PLUQ_TRY(trsm_right_upper(c, X(R0, C0, 0, 0), lda, r1, X(R0, C0, m1, 0), lda, m2, diag0));
        PLUQ_TRY(fgemm_sub(c, m - r1, n2, r1, X(R0, C0, r1, 0), lda, X(R0, C0, 0, n1), lda,
                           X(R0, C0, r1, n1), lda));
        PLUQ_TRY(fgemm_sub(c, m2, n1 - r1, r1, X(R0, C0, m1, 0), lda, X(R0, C0, 0, r1), lda,
                           X(R0, C0, m1, r1), lda));
      }
    }

    // F (rows r1..m1 of the top half, right columns) and G (bottom rows,
    // columns r1..n1 of the left half): independent, concurrent when both
    // are large; then the permutations each induces on the other blocks
    int64_t r2 = 0, r3 = 0;
    // (worth a thread when each block holds at least a quarter leaf)
    const int64_t fork_min = std::max<int64_t>(kForkMinElems, lim_m * lim_n / 4);
    const bool fork = c->lane_depth < c->fork_depth && !c->prof.on &&
                      (m1 - r1) * n2 >= fork_min && m2 * (n1 - r1) >= fork_min;
    if (fork) {
      // F's branch also runs f_post (see there)
      PLUQ_TRY(fork_fg(R0, C0, m1, n1, m2, n2, r1, d, &r2, &r3, &id2, &id3, keep));
    } else {
      PLUQ_TRY(node(R0 + r1, C0 + n1, m1 - r1, n2, d + 1, &r2, &id2, keep | KEEP_U));
      PLUQ_TRY(f_post(R0, C0, m1, n1, m2, n2, r1, r2, d, id2, keep));
      PLUQ_TRY(node(R0 + m1, C0 + r1, m2, n1 - r1, d + 1, &r3, &id3, keep | KEEP_L));
    }
    PLUQ_TRY(compose_pair(pr + m1, cr + R0 + m1, m2, pc + r1, cc + C0 + r1, n1 - r1, id3));
    // E (columns 0..r1; L, storage only) and H (columns n1..n) by G's row permutation
    if (!id3.r) {
      if (keep & KEEP_L)
        PLUQ_TRY(permute_rows2(c, X(R0, C0, m1, 0), lda, m2, 0, r1, n1, n2, cr + R0 + m1));
      else
        PLUQ_TRY(permute_rows2(c, X(R0, C0, m1, 0), lda, m2, n1, n2, 0, 0, cr + R0 + m1));
    }
    // V1 (U, storage only) by G's column permutation
    if (!id3.c && (keep & KEEP_U))
      PLUQ_TRY(permute_cols(c, X(R0, C0, 0, r1), lda, r1, n1 - r1, cc + C0 + r1));

    // H = [H1 H2; H3 H4] at rows m1.., columns n1.. ([I; K] and H2 are done
    // in f_post): O = L3^{-1} H[:r3, r2:], R -= M3 O
    if (r3 > 0) {
      PLUQ_TRY(trsm_left_lower_unit(c, X(R0, C0, m1, r1), lda, r3, X(R0, C0, m1, n1 + r2), lda,
                                    n2 - r2));
      PLUQ_TRY(fgemm_sub(c, m2 - r3, n2 - r2, r3, X(R0, C0, m1 + r3, r1), lda,
                         X(R0, C0, m1, n1 + r2), lda, X(R0, C0, m1 + r3, n1 + r2), lda));
    }

    // R
    int64_t r4 = 0;
    PLUQ_TRY(node(R0 + m1 + r3, C0 + n1 + r2, m2 - r3, n2 - r2, d + 1, &r4, &id4, keep,
                  la_pending));
    PLUQ_TRY(compose_pair(pr + m1 + r3, cr + R0 + m1 + r3, m2 - r3, pc + n1 + r2,
                          cc + C0 + n1 + r2, n2 - r2, id4));
    // E2, M3 (columns 0..r1+r3) and K (columns n1..n1+r2) by R's row
    // permutation: all L, storage only
    if (!id4.r && (keep & KEEP_L))
      PLUQ_TRY(permute_rows2(c, X(R0, C0, m1 + r3, 0), lda, m2 - r3, 0, r1 + r3, n1, r2,
                             cr + R0 + m1 + r3));
    // D2, V2 (rows 0..r1+r2) and O (rows m1..m1+r3) by R's column permutation:
    // all U, storage only
    if (!id4.c && (keep & KEEP_U))
      PLUQ_TRY(permute_cols2(c, X(R0, C0, 0, n1 + r2), lda, 0, r1 + r2, m1, r3, n2 - r2,
                             cc + C0 + n1 + r2));
    id->r = id1.r && id2.r && id3.r && id4.r;
    id->c = id1.c && id2.c && id3.c && id4.c;

    // block-cyclic shifts
    int32_t* tmp = PR(spare()) + R0;  // spare row slot (this block's range)
    {
      const int64_t a = r1 + r2, fr = m1 - r1 - r2, gr = r3 + r4;
      if (fr > 0 && gr > 0) {
        id->r = false;
        const int64_t st[2] = {fr, 0}, ln[2] = {gr, fr};
        PLUQ_TRY(launch_segperm(c, tmp, st, ln, 2));
        // (a block whose factors nobody reads needs only its index vectors)
        if (keep != KEEP_NONE) PLUQ_TRY(permute_rows(c, X(R0, C0, a, 0), lda, fr + gr, n, tmp));
        PLUQ_TRY(launch_compose(c, pr + a, tmp, fr + gr));
      }
    }
    {
      // columns from r1: [G3p (r3) | G_rest (n1-r1-r3) | F2p (r2) | R4p (r4)]
      const int64_t gn = n1 - r1 - r3;
      const bool ident = (r2 == 0 || (r3 == 0 && gn == 0)) && (r4 == 0 || gn == 0);
      if (!ident) {
        id->c = false;
        int32_t* tmpc = PC(spare()) + C0;
        const int64_t st[4] = {r3 + gn, 0, r3 + gn + r2, r3};
        const int64_t ln[4] = {r2, r3, r4, gn};
        const int64_t len = r3 + gn + r2 + r4;
        PLUQ_TRY(launch_segperm(c, tmpc, st, ln, 4));
        if (keep != KEEP_NONE) PLUQ_TRY(permute_cols(c, X(R0, C0, 0, r1), lda, m, len, tmpc));
        PLUQ_TRY(launch_compose(c, pc + r1, tmpc, len));
      }
    }
    *r_out = r1 + r2 + r3 + r4;
    return PLUQ_OK;
  }
};

int prepare(pluq_ctx* c, uint32_t p, int64_t m, int64_t n, int form, void* stream) {
  PLUQ_TRY(check_p(p));
  const int f = resolve_form(p, form);
  if (f == -2) return PLUQ_ERR_INVALID_ARG;
  if (f < 0) return PLUQ_ERR_UNSUPPORTED_FORM;
  PLUQ_CUDA(cudaSetDevice(c->device));
  c->stream = (cudaStream_t)stream;
  c->F = make_field(p);
  c->form = f;
  c->n_base = c->n_nodes = c->n_gemm = 0;
  c->leaf_density = 1.0;
  (void)m;
  (void)n;
  return PLUQ_OK;
}

// Factor A in place; leaves P = PR(0), Q = PC(0) in the workspace.
// Applies the autotuned schedule of (p, m, n, form), if any, for one call and
// restores the caller's options afterwards.
struct TunedScope {
  pluq_ctx* c;
  int leaf_dim, leaf_kind, fork_depth, limb_variant;
  TunedScope(pluq_ctx* ctx, int64_t m, int64_t n)
      : c(ctx), leaf_dim(ctx->leaf_dim), leaf_kind(ctx->leaf_kind), fork_depth(ctx->fork_depth),
        limb_variant(ctx->limb_variant) {
    if (c->tuning || !c->use_tuned) return;
    for (const pluq_ctx::Tuned& t : c->tuned)
      if (t.p == c->F.p && t.m == m && t.n == n && t.form == c->form) {
        c->leaf_dim = t.leaf_dim;
        c->leaf_kind = t.leaf_kind;
        c->fork_depth = t.fork_depth;
        c->limb_variant = t.limb_variant;
        break;
      }
  }
  ~TunedScope() {
    c->leaf_dim = leaf_dim;
    c->leaf_kind = leaf_kind;
    c->fork_depth = fork_depth;
    c->limb_variant = limb_variant;
  }
};

int factor(pluq_ctx* c, int64_t m, int64_t n, uint32_t* A, int64_t lda, int64_t* r_out,
           int keep = KEEP_LU) {
  TunedScope tuned(c, m, n);
  c->mmax = std::max<int64_t>(m, 1);
  c->nmax = std::max<int64_t>(n, 1);
  // index-vector slots: one a recursion level.  Tiled iteration nests one
  // level a slab and a tile (plus halvings of blocks no leaf takes)
  const int64_t lim = std::max(1, c->leaf_dim > 0 ? c->leaf_dim : std::min(c->bm, c->bn));
  const int64_t slab = c->slab_rows > 0 ? c->slab_rows : lim;
  c->depth_slots = c->decomposition == 1
                       ? (int)std::max<int64_t>(kMaxDepth, cdiv(m, slab) + cdiv(n, lim) +
                                                               cdiv(slab, lim) + 72)
                       : kMaxDepth;
  PLUQ_TRY(c->perm_r.ensure(sizeof(int32_t) * c->depth_slots * c->mmax));
  PLUQ_TRY(c->perm_c.ensure(sizeof(int32_t) * c->depth_slots * c->nmax));
  PLUQ_TRY(c->scratch.ensure(sizeof(uint32_t) * std::max<int64_t>(m * n, 1)));
  PLUQ_TRY(c->tmp_i.ensure(sizeof(int32_t) * std::max(c->mmax, c->nmax)));
  PLUQ_TRY(c->small.ensure(256));
  PLUQ_TRY(ensure_inv_table(c));
  if (c->form == PLUQ_FORM_LIMB_F16) {
    // digit planes of the largest fgemm operands (K <= min(m, n) / 2 + 64; a
    // tiled-iterative slab can give K up to its row count)
    const int64_t kmax = c->decomposition == 1 ? std::min(std::min(m, n), slab) : 0;
    const int64_t kp = cdiv(std::max(std::min(m, n) / 2, kmax) + 64, 64) * 64;
    const int64_t rows = cdiv(m, 128) * 128 + cdiv(n, 128) * 128;
    PLUQ_TRY(c->pack.ensure(sizeof(uint16_t) * 2 * rows * kp + 4096));
  }
  int* flag = c->small.as<int>();
  PLUQ_CUDA(cudaMemsetAsync(flag, 0, 256, c->stream));
  if (m > 0 && n > 0) {
    ProfScope ps(c, PC_OTHER, 0, 4.0 * m * n);
    k_check_range<<<grid2(m, n), 256, 0, c->stream>>>(A, lda, m, n, c->F.p, flag);
    PLUQ_CUDA(cudaGetLastError());
    PLUQ_CUDA(cudaMemcpyAsync(c->host_small, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PLUQ_CUDA(cudaStreamSynchronize(c->stream));
    if (c->host_small[0] != 0) return PLUQ_ERR_ENTRY_OUT_OF_RANGE;
  }
  // inverses of the full-rank diagonal leaves, for the solves of every ancestor
  c->dinv_b = 0;
  c->dinv_ok = false;
  c->dinv_valid.clear();
  if (c->dinv_enable && c->decomposition == 0 && c->leaf_dim > 0 && c->lane_depth == 0 &&
      std::min(m, n) >= 2 * (int64_t)c->leaf_dim) {
    const int64_t b = c->leaf_dim, slots = std::min(m, n) / b;
    if (c->dinv.ensure(sizeof(uint32_t) * slots * 2 * b * b) == PLUQ_OK) {
      c->dinv_b = b;
      c->dinv_ok = true;
      c->dinv_valid.assign(slots, 0);
    }
  }
  Recursion rec{c, A, lda, c->small.as<int32_t>() + 8};
  Ident id;
  PLUQ_TRY(rec.node(0, 0, m, n, 0, r_out, &id, keep));
  PLUQ_CUDA(cudaMemcpyAsync(c->host_small, c->small.ptr, 32 * sizeof(int32_t),
                            cudaMemcpyDeviceToHost, c->stream));
  PLUQ_CUDA(cudaStreamSynchronize(c->stream));
  if (c->host_small[16] != 0) return c->host_small[16];
  c->host_small[8] = (int32_t)*r_out;
  return PLUQ_OK;
}

int write_outputs(pluq_ctx* c, int64_t m, int64_t n, int64_t r, int32_t* P, int32_t* Q,
                  int64_t* rank_dev, int32_t* rrp, int32_t* crp) {
  const int32_t* PR = c->perm_r.as<int32_t>();
  const int32_t* PC = c->perm_c.as<int32_t>();
  if (P && m > 0)
    PLUQ_CUDA(cudaMemcpyAsync(P, PR, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice, c->stream));
  if (Q && n > 0)
    PLUQ_CUDA(cudaMemcpyAsync(Q, PC, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, c->stream));
  if (rank_dev) {
    ProfScope ps(c, PC_OTHER);
    k_store_rank<<<1, 1, 0, c->stream>>>(rank_dev, r);
    PLUQ_CUDA(cudaGetLastError());
  }
  if (rrp && r > 0) {
    ProfScope ps(c, PC_OTHER, 0, 4.0 * r);
    k_profile<<<1, 1024, sizeof(uint32_t) * cdiv(m, 32), c->stream>>>(PR, r, m, rrp);
    PLUQ_CUDA(cudaGetLastError());
  }
  if (crp && r > 0) {
    ProfScope ps(c, PC_OTHER, 0, 4.0 * r);
    k_profile<<<1, 1024, sizeof(uint32_t) * cdiv(n, 32), c->stream>>>(PC, r, n, crp);
    PLUQ_CUDA(cudaGetLastError());
  }
  return PLUQ_OK;
}

int copy_to_work(pluq_ctx* c, int64_t m, int64_t n, const uint32_t* A, int64_t lda) {
  PLUQ_TRY(c->work.ensure(sizeof(uint32_t) * std::max<int64_t>(m * n, 1)));
  if (m > 0 && n > 0) {
    ProfScope ps(c, PC_OTHER, 0, 8.0 * m * n);
    k_copy_mat<<<grid2(m, n), 256, 0, c->stream>>>(c->work.as<uint32_t>(), n, A, lda, m, n);
    PLUQ_CUDA(cudaGetLastError());
  }
  return PLUQ_OK;
}

}  // namespace

ProfScope::ProfScope(pluq_ctx* ctx, int cls, double flops, double bytes, int nlaunch,
                     double tflops)
    : c(ctx) {
  c->launches[cls] += nlaunch;
  if (!c->prof.on) return;
  Profiler& P = c->prof;
  while (P.used + 2 > P.pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    P.pool.push_back(e);
  }
  ProfRec r{cls, (int)P.used, (int)P.used + 1, flops, bytes, tflops};
  P.used += 2;
  cudaEventRecord(P.pool[r.a], c->stream);
  P.recs.push_back(r);
  idx = (int)P.recs.size() - 1;
}

ProfScope::~ProfScope() {
  if (idx >= 0) cudaEventRecord(c->prof.pool[c->prof.recs[idx].b], c->stream);
}

int check_prime_range(uint32_t p) { return check_p(p); }

int fgemm_sub(pluq_ctx* c, int64_t M, int64_t N, int64_t K, const uint32_t* A, int64_t lda,
              const uint32_t* B, int64_t ldb, uint32_t* C, int64_t ldc) {
  if (M <= 0 || N <= 0 || K <= 0) return PLUQ_OK;
  if (wino_applies(c, M, N, K)) return fgemm_sub_wino(c, M, N, K, A, lda, B, ldb, C, ldc, 0);
  return fgemm_sub_classical(c, M, N, K, A, lda, B, ldb, C, ldc);
}

int fgemm_sub_classical(pluq_ctx* c, int64_t M, int64_t N, int64_t K, const uint32_t* A,
                        int64_t lda, const uint32_t* B, int64_t ldb, uint32_t* C, int64_t ldc) {
  if (M <= 0 || N <= 0 || K <= 0) return PLUQ_OK;
  c->n_gemm++;
  if (c->form == PLUQ_FORM_LIMB_F16) {
    // a thin inner dimension does not pay for packing and a tensor pipeline
    if (c->thin_gemm && thin_fgemm_ok(c, M, N, K))
      return fgemm_sub_thin(c, M, N, K, A, lda, B, ldb, C, ldc);
    return fgemm_sub_limb(c, M, N, K, A, lda, B, ldb, C, ldc);
  }
  return fgemm_sub_fp64(c, M, N, K, A, lda, B, ldb, C, ldc);
}

extern "C" {

int pluq_create(pluq_ctx** ctx, int device) {
  if (!ctx) return PLUQ_ERR_INVALID_ARG;
  *ctx = nullptr;
  pluq_ctx* c = new pluq_ctx();
  c->device = device;
  bind_workspace(c);
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return PLUQ_ERR_CUDA;
  }
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  if (cudaMallocHost(&c->host_small, 256) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return PLUQ_ERR_CUDA;
  }
  *ctx = c;
  return PLUQ_OK;
}

int pluq_destroy(pluq_ctx* c) {
  if (!c) return PLUQ_OK;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  destroy_lane(c->lane[0]);
  destroy_lane(c->lane[1]);
  destroy_lane(c->lane[2]);
  for (cudaEvent_t e : c->la_ev)
    if (e) cudaEventDestroy(e);
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  for (cudaEvent_t e : c->side_ev)
    if (e) cudaEventDestroy(e);
  c->scratch.release();
  c->pack.release();
  c->perm_r.release();
  c->perm_c.release();
  c->tmp_i.release();
  for (cudaEvent_t e : c->prof.pool) cudaEventDestroy(e);
  c->small.release();
  c->inv_table.release();
  c->leaf.release();
  c->tune_src.release();
  c->tune_dst.release();
  c->tri_inv.release();
  c->batch_dev.release();
  c->batch_scratch.release();
  c->batch_pq.release();
  if (c->batch_graph) cudaGraphExecDestroy(c->batch_graph);
  if (c->batch_host) cudaFreeHost(c->batch_host);
  c->work.release();
  c->wino.release();
  c->dinv.release();
  if (c->host_small) cudaFreeHost(c->host_small);
  delete c;
  return PLUQ_OK;
}

int pluq_modp(pluq_ctx* c, uint32_t p, int64_t m, int64_t n, uint32_t* A, int64_t lda, int32_t* P,
              int32_t* Q, int64_t* rank_dev, int32_t* rrp, int32_t* crp, int form, void* stream) {
  if (!c || m < 0 || n < 0 || (m > 0 && !P) || (n > 0 && !Q)) return PLUQ_ERR_INVALID_ARG;
  if (m > 0 && n > 0 && (!A || lda < n)) return PLUQ_ERR_INVALID_ARG;
  if (m >= 0x7fffffff || n >= 0x7fffffff) return PLUQ_ERR_INVALID_ARG;
  PLUQ_TRY(prepare(c, p, m, n, form, stream));
  int64_t r = 0;
  PLUQ_TRY(factor(c, m, n, A, lda, &r));
  return write_outputs(c, m, n, r, P, Q, rank_dev, rrp, crp);
}

int rank_profile_modp(pluq_ctx* c, uint32_t p, int64_t m, int64_t n, const uint32_t* A, int64_t lda,
                      int64_t* rank_dev, int32_t* rrp, int32_t* crp, int32_t* rpm_col_of_row,
                      int form, void* stream) {
  if (!c || m < 0 || n < 0) return PLUQ_ERR_INVALID_ARG;
  if (m > 0 && n > 0 && (!A || lda < n)) return PLUQ_ERR_INVALID_ARG;
  PLUQ_TRY(prepare(c, p, m, n, form, stream));
  PLUQ_TRY(copy_to_work(c, m, n, A, lda));
  int64_t r = 0;
  // only the pivots are read: no L or U block needs its final position
  PLUQ_TRY(factor(c, m, n, c->work.as<uint32_t>(), std::max<int64_t>(n, 1), &r, KEEP_NONE));
  PLUQ_TRY(write_outputs(c, m, n, r, nullptr, nullptr, rank_dev, rrp, crp));
  if (rpm_col_of_row && m > 0) {
    const int32_t* PR = c->perm_r.as<int32_t>();
    const int32_t* PC = c->perm_c.as<int32_t>();
    ProfScope ps(c, PC_OTHER, 0, 4.0 * m, r > 0 ? 2 : 1);
    k_rpm_col_of_row<<<(unsigned)cdiv(m, 256), 256, 0, c->stream>>>(PR, PC, r, m, rpm_col_of_row);
    if (r > 0) k_rpm_fill<<<(unsigned)cdiv(r, 256), 256, 0, c->stream>>>(PR, PC, r, rpm_col_of_row);
    PLUQ_CUDA(cudaGetLastError());
  }
  return PLUQ_OK;
}

// RREF of the m x n matrix W (workspace, ld ldw, factored in place) written
// with strides (rs, cs); rank to rank_dev, pivot columns to crp (may be NULL).
static int echelon_core(pluq_ctx* c, int64_t m, int64_t n, uint32_t* W, int64_t ldw, uint32_t* R,
                        int64_t rs, int64_t cs, int64_t* rank_dev, int32_t* crp,
                        int64_t* r_host = nullptr) {
  int64_t r = 0;
  // the echelon form reads U (in the Q frame) and the pivots, never L
  PLUQ_TRY(factor(c, m, n, W, ldw, &r, KEEP_U));
  if (r_host) *r_host = r;
  PLUQ_TRY(write_outputs(c, m, n, r, nullptr, nullptr, rank_dev, nullptr, nullptr));
  if (r == 0) return PLUQ_OK;
  // X = U1^{-1} [U1 U2] in the Q frame: only U2 needs solving.
  PLUQ_TRY(trsm_left_upper(c, W, ldw, r, W + r, ldw, n - r));
  PLUQ_TRY(c->tmp_i.ensure(sizeof(int32_t) * (n + r + 64)));
  int32_t* ints = c->tmp_i.as<int32_t>();
  int32_t* qinv = ints;
  int32_t* crp_buf = crp ? crp : ints + n;
  const int32_t* PC = c->perm_c.as<int32_t>();
  ProfScope ps(c, PC_OTHER, 0, 8.0 * n + 4.0 * r * n, 3);
  k_invert_perm<<<(unsigned)cdiv(n, 256), 256, 0, c->stream>>>(PC, n, qinv);
  k_profile<<<1, 1024, sizeof(uint32_t) * cdiv(n, 32), c->stream>>>(PC, r, n, crp_buf);
  k_rref_scatter<<<grid2(r, n), 256, 0, c->stream>>>(W, ldw, r, n, qinv, crp_buf, R, rs, cs);
  PLUQ_CUDA(cudaGetLastError());
  return PLUQ_OK;
}

int echelon_modp(pluq_ctx* c, uint32_t p, int64_t m, int64_t n, const uint32_t* A, int64_t lda,
                 uint32_t* R, int64_t ldr, int64_t* rank_dev, int32_t* crp, int form, void* stream) {
  if (!c || m < 0 || n < 0) return PLUQ_ERR_INVALID_ARG;
  if (m > 0 && n > 0 && (!A || !R || lda < n || ldr < n)) return PLUQ_ERR_INVALID_ARG;
  PLUQ_TRY(prepare(c, p, m, n, form, stream));
  PLUQ_TRY(copy_to_work(c, m, n, A, lda));
  return echelon_core(c, m, n, c->work.as<uint32_t>(), std::max<int64_t>(n, 1), R, ldr, 1,
                      rank_dev, crp);
}

int echelon_modp_batched(pluq_ctx* c, uint32_t p, int32_t batch, const int64_t* m,
                         const int64_t* n, const uint32_t* const* A, const int64_t* lda,
                         uint32_t* const* R, const int64_t* ldr, int32_t* const* crp,
                         int64_t* ranks, int32_t* status, int form, void* stream) {
  if (!c || batch < 0 || (batch > 0 && (!m || !n || !A || !lda || !R || !ldr || !ranks)))
    return PLUQ_ERR_INVALID_ARG;
  // one matrix after the other on the stream: each needs its own triangular
  // solve X2 = U1^{-1} U2 of its own rank, so the one-CTA-per-matrix kernel of
  // the batched factorization does not carry over
  int first_bad = PLUQ_OK;
  for (int32_t b = 0; b < batch; ++b) {
    int64_t r = 0;
    int st = PLUQ_OK;
    const bool argok = m[b] >= 0 && n[b] >= 0 &&
                       (m[b] == 0 || n[b] == 0 ||
                        (A[b] && R[b] && lda[b] >= n[b] && ldr[b] >= n[b]));
    if (!argok) {
      st = PLUQ_ERR_INVALID_ARG;
    } else {
      st = prepare(c, p, m[b], n[b], form, stream);
      if (st == PLUQ_OK && m[b] > 0 && n[b] > 0) {
        st = copy_to_work(c, m[b], n[b], A[b], lda[b]);
        if (st == PLUQ_OK)
          st = echelon_core(c, m[b], n[b], c->work.as<uint32_t>(), n[b], R[b], ldr[b], 1,
                            nullptr, crp ? crp[b] : nullptr, &r);
      }
    }
    ranks[b] = st == PLUQ_OK ? r : -1;
    if (status) status[b] = st;
    if (st != PLUQ_OK && first_bad == PLUQ_OK) first_bad = st;
    if (st != PLUQ_OK && st != PLUQ_ERR_INVALID_ARG && st != PLUQ_ERR_ENTRY_OUT_OF_RANGE) {
      // not a fault of this matrix (prime, form, workspace, device): stop here
      for (int32_t e = b + 1; e < batch; ++e) {
        ranks[e] = -1;
        if (status) status[e] = st;
      }
      return st;
    }
  }
  return first_bad;
}

int column_echelon_modp(pluq_ctx* c, uint32_t p, int64_t m, int64_t n, const uint32_t* A,
                        int64_t lda, uint32_t* C, int64_t ldc, int64_t* rank_dev, int32_t* rrp,
                        int form, void* stream) {
  if (!c || m < 0 || n < 0) return PLUQ_ERR_INVALID_ARG;
  if (m > 0 && n > 0 && (!A || !C || lda < n || ldc < std::min(m, n))) return PLUQ_ERR_INVALID_ARG;
  // the RREF of A^T (n x m), transposed back: E = RREF(A^T)^T, m x r
  PLUQ_TRY(prepare(c, p, n, m, form, stream));
  PLUQ_TRY(c->work.ensure(sizeof(uint32_t) * std::max<int64_t>(m * n, 1)));
  uint32_t* W = c->work.as<uint32_t>();
  const int64_t ldw = std::max<int64_t>(m, 1);
  if (m > 0 && n > 0) {
    ProfScope ps(c, PC_OTHER, 0, 8.0 * m * n);
    k_transpose<<<dim3((unsigned)cdiv(n, 32), (unsigned)cdiv(m, 32)), dim3(32, 8), 0,
                  c->stream>>>(W, ldw, A, lda, m, n);
    PLUQ_CUDA(cudaGetLastError());
  }
  return echelon_core(c, n, m, W, ldw, C, 1, ldc, rank_dev, rrp);
}

int fgemm_modp(pluq_ctx* c, uint32_t p, int64_t M, int64_t N, int64_t K, const uint32_t* A,
               int64_t lda, const uint32_t* B, int64_t ldb, uint32_t* C, int64_t ldc, int form,
               void* stream) {
  if (!c || M < 0 || N < 0 || K < 0) return PLUQ_ERR_INVALID_ARG;
  if (M > 0 && N > 0 && K > 0 && (!A || !B || !C || lda < K || ldb < N || ldc < N))
    return PLUQ_ERR_INVALID_ARG;
  PLUQ_TRY(prepare(c, p, M, N, form, stream));
  PLUQ_TRY(c->small.ensure(256));
  PLUQ_CUDA(cudaMemsetAsync(c->small.ptr, 0, 256, c->stream));
  PLUQ_TRY(fgemm_sub(c, M, N, K, A, lda, B, ldb, C, ldc));
  // the kernels' device error word (int 16): a bounded wait that ran out
  PLUQ_CUDA(cudaMemcpyAsync(c->host_small + 16, c->small.as<int>() + 16, sizeof(int32_t),
                            cudaMemcpyDeviceToHost, c->stream));
  PLUQ_CUDA(cudaStreamSynchronize(c->stream));
  return c->host_small[16] != 0 ? c->host_small[16] : PLUQ_OK;
}

int pluq_modp_batched(pluq_ctx* c, uint32_t p, int32_t batch, const int64_t* m, const int64_t* n,
                      uint32_t* const* A, const int64_t* lda, int32_t* const* P, int32_t* const* Q,
                      int64_t* ranks, int32_t* status, int form, void* stream) {
  if (!c || batch < 0 || (batch > 0 && (!m || !n || !A || !lda || !P || !Q || !ranks)))
    return PLUQ_ERR_INVALID_ARG;
  if (batch == 0) return PLUQ_OK;
  PLUQ_TRY(prepare(c, p, 1, 1, form, stream));
  PLUQ_TRY(c->small.ensure(256));
  PLUQ_TRY(ensure_inv_table(c));
  // matrices within the persistent kernel's limits; the others go one by one
  const int64_t lim = batched_max_dim();
  std::vector<int> small, big;
  int first_bad = PLUQ_OK;
  for (int32_t b = 0; b < batch; ++b) {
    const bool argok = m[b] >= 0 && n[b] >= 0 &&
                       (m[b] == 0 || n[b] == 0 || (A[b] && lda[b] >= n[b])) &&
                       (m[b] == 0 || P[b]) && (n[b] == 0 || Q[b]);
    if (!argok) {
      ranks[b] = -1;
      if (status) status[b] = PLUQ_ERR_INVALID_ARG;
      if (first_bad == PLUQ_OK) first_bad = PLUQ_ERR_INVALID_ARG;
      continue;
    }
    (m[b] <= lim && n[b] <= lim ? small : big).push_back(b);
  }
  if (!small.empty()) {
    const int cnt = (int)small.size();
    // longest factorizations first
    std::vector<int32_t> order(cnt);
    for (int i = 0; i < cnt; ++i) order[i] = i;
    auto work = [&](int i) {
      const double mm = (double)m[small[i]], nn = (double)n[small[i]];
      return mm * nn * std::min(mm, nn);
    };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work(x) > work(y); });
    const size_t dsz = batched_desc_size();
    const size_t off_order = ((dsz * cnt + 255) / 256) * 256;
    const size_t off_rank = off_order + ((sizeof(int32_t) * cnt + 255) / 256) * 256;
    const size_t off_stat = off_rank + sizeof(int64_t) * cnt;
    const size_t total = off_stat + sizeof(int32_t) * cnt + 256;
    if (c->batch_host_bytes < total) {
      if (c->batch_graph) {
        cudaGraphExecDestroy(c->batch_graph);
        c->batch_graph = nullptr;
      }
      if (c->batch_host) cudaFreeHost(c->batch_host);
      c->batch_host = nullptr;
      c->batch_host_bytes = 0;
      if (cudaMallocHost(&c->batch_host, total) != cudaSuccess) {
        cudaGetLastError();
        return PLUQ_ERR_NO_WORKSPACE;
      }
      c->batch_host_bytes = total;
    }
    const void* old_dev = c->batch_dev.ptr;
    PLUQ_TRY(c->batch_dev.ensure(total));
    char* hb = static_cast<char*>(c->batch_host);
    char* db = c->batch_dev.as<char>();
    int max_elems = 1, max_n = 1;
    for (int i = 0; i < cnt; ++i) {
      const int b = small[i];
      batched_fill_desc(hb, i, A[b], P[b], Q[b], lda[b], (int)m[b], (int)n[b]);
      max_elems = std::max<int64_t>(max_elems, m[b] * n[b]);
      max_n = std::max<int64_t>(max_n, n[b]);
    }
    std::memcpy(hb + off_order, order.data(), sizeof(int32_t) * cnt);
    // one graph per (count, workspace): H2D descriptors, persistent kernel,
    // D2H ranks and status
    if (c->batch_graph && (c->batch_graph_count != cnt || c->batch_graph_key != db ||
                           old_dev != c->batch_dev.ptr || c->batch_graph_elems < max_elems ||
                           c->batch_graph_maxn != max_n || c->batch_graph_slab != c->batch_slab ||
                           c->batch_graph_p != c->F.p ||
                           c->batch_graph_tab != (const void*)inv_table_ptr(c))) {
      cudaGraphExecDestroy(c->batch_graph);
      c->batch_graph = nullptr;
    }
    if (!c->batch_graph) {
      // the gather scratch is sized (and captured) for this batch's largest matrix
      const int grid = batched_grid(c, max_n);
      if (grid <= 0) return PLUQ_ERR_CUDA;
      PLUQ_TRY(c->batch_scratch.ensure(sizeof(uint32_t) * (size_t)max_elems * grid));
      cudaStream_t cs;
      PLUQ_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      cudaStream_t saved = c->stream;
      c->stream = cs;
      int st = PLUQ_OK;
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        st = PLUQ_ERR_CUDA;
      } else {
        if (cudaMemcpyAsync(db, hb, off_rank, cudaMemcpyHostToDevice, cs) != cudaSuccess)
          st = PLUQ_ERR_CUDA;
        if (st == PLUQ_OK)
          st = launch_batched(c, db, reinterpret_cast<const int32_t*>(db + off_order), cnt,
                              reinterpret_cast<int64_t*>(db + off_rank),
                              reinterpret_cast<int32_t*>(db + off_stat), max_elems, max_n);
        if (st == PLUQ_OK &&
            cudaMemcpyAsync(hb + off_rank, db + off_rank, off_stat - off_rank + sizeof(int32_t) * cnt,
                            cudaMemcpyDeviceToHost, cs) != cudaSuccess)
          st = PLUQ_ERR_CUDA;
        if (cudaStreamEndCapture(cs, &g) != cudaSuccess) st = PLUQ_ERR_CUDA;
      }
      c->stream = saved;
      if (st == PLUQ_OK && cudaGraphInstantiate(&c->batch_graph, g, 0) != cudaSuccess)
        st = PLUQ_ERR_CUDA;
      if (g) cudaGraphDestroy(g);
      cudaStreamDestroy(cs);
      cudaGetLastError();
      if (st != PLUQ_OK) {
        c->batch_graph = nullptr;
        return st;
      }
      c->batch_graph_count = cnt;
      c->batch_graph_key = db;
      c->batch_graph_elems = max_elems;
      c->batch_graph_maxn = max_n;
      c->batch_graph_slab = c->batch_slab;
      c->batch_graph_p = c->F.p;
      c->batch_graph_tab = inv_table_ptr(c);
    }
    c->launches[PC_BASE] += 1;
    c->launches[PC_INDEX] += 1;
    PLUQ_CUDA(cudaGraphLaunch(c->batch_graph, c->stream));
    PLUQ_CUDA(cudaStreamSynchronize(c->stream));
    const int64_t* hr = reinterpret_cast<const int64_t*>(hb + off_rank);
    const int32_t* hs = reinterpret_cast<const int32_t*>(hb + off_stat);
    for (int i = 0; i < cnt; ++i) {
      const int b = small[i];
      ranks[b] = hr[i];
      if (status) status[b] = hs[i];
      if (hs[i] != PLUQ_OK && first_bad == PLUQ_OK) first_bad = hs[i];
    }
  }
  for (int b : big) {
    const int st = pluq_modp(c, p, m[b], n[b], A[b], lda[b], P[b], Q[b], nullptr, nullptr, nullptr,
                             form, stream);
    ranks[b] = st == PLUQ_OK ? (int64_t)c->host_small[8] : -1;
    if (status) status[b] = st;
    if (st != PLUQ_OK && first_bad == PLUQ_OK) first_bad = st;
  }
  return first_bad;
}

int rank_profile_modp_batched(pluq_ctx* c, uint32_t p, int32_t batch, const int64_t* m,
                              const int64_t* n, uint32_t* const* A, const int64_t* lda,
                              int32_t* const* rrp, int32_t* const* crp, int64_t* ranks,
                              int32_t* status, int form, void* stream) {
  if (!c || batch < 0 || (batch > 0 && (!m || !n || !A || !lda || !ranks)))
    return PLUQ_ERR_INVALID_ARG;
  if (batch == 0) return PLUQ_OK;
  // pivot index vectors of every matrix in one workspace
  std::vector<int64_t> offp(batch), offq(batch);
  int64_t total = 0, maxdim = 1;
  for (int32_t b = 0; b < batch; ++b) {
    const int64_t mb = std::max<int64_t>(m[b], 0), nb = std::max<int64_t>(n[b], 0);
    offp[b] = total;
    total += mb;
    offq[b] = total;
    total += nb;
    maxdim = std::max(maxdim, std::max(mb, nb));
  }
  PLUQ_TRY(c->batch_pq.ensure(sizeof(int32_t) * std::max<int64_t>(total, 1) +
                              sizeof(ProfileDesc) * batch + 256));
  int32_t* base = c->batch_pq.as<int32_t>();
  std::vector<int32_t*> Pp(batch), Qp(batch);
  for (int32_t b = 0; b < batch; ++b) {
    Pp[b] = base + offp[b];
    Qp[b] = base + offq[b];
  }
  const int st = pluq_modp_batched(c, p, batch, m, n, A, lda, Pp.data(), Qp.data(), ranks, status,
                                   form, stream);
  if (st != PLUQ_OK && st != PLUQ_ERR_INVALID_ARG && st != PLUQ_ERR_ENTRY_OUT_OF_RANGE) return st;
  // profiles of the matrices that factored (ranks < 0 mark the others)
  std::vector<ProfileDesc> d(batch);
  for (int32_t b = 0; b < batch; ++b)
    d[b] = ProfileDesc{Pp[b], Qp[b], rrp ? rrp[b] : nullptr, crp ? crp[b] : nullptr,
                       std::max<int64_t>(m[b], 0), std::max<int64_t>(n[b], 0),
                       ranks[b] > 0 ? ranks[b] : 0};
  ProfileDesc* dd = reinterpret_cast<ProfileDesc*>(
      reinterpret_cast<char*>(base) + ((sizeof(int32_t) * std::max<int64_t>(total, 1) + 255) / 256) * 256);
  PLUQ_CUDA(cudaMemcpyAsync(dd, d.data(), sizeof(ProfileDesc) * batch, cudaMemcpyHostToDevice,
                            c->stream));
  const size_t smem = sizeof(uint32_t) * cdiv(maxdim, 32);
  if (smem > 48 * 1024) return PLUQ_ERR_INVALID_ARG;
  {
    ProfScope ps(c, PC_OTHER, 0, 8.0 * total);
    k_profiles_batched<<<dim3((unsigned)batch, 2), 256, smem, c->stream>>>(dd);
    PLUQ_CUDA(cudaGetLastError());
  }
  // the descriptors are host vectors: wait for the copy before they go away
  PLUQ_CUDA(cudaStreamSynchronize(c->stream));
  return st;
}

int pluq_last_rank(pluq_ctx* c, int64_t* rank) {
  if (!c || !rank) return PLUQ_ERR_INVALID_ARG;
  *rank = c->host_small[8];
  return PLUQ_OK;
}

int pluq_sync_status(pluq_ctx* c) {
  if (!c) return PLUQ_ERR_INVALID_ARG;
  if (cudaSetDevice(c->device) != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess ||
      cudaGetLastError() != cudaSuccess)
    return PLUQ_ERR_CUDA;
  if (!c->small.ptr) return PLUQ_OK;
  int32_t word = 0;
  if (cudaMemcpy(&word, c->small.as<int32_t>() + 16, sizeof(word), cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return PLUQ_ERR_CUDA;
  return word != 0 ? word : PLUQ_OK;
}

int pluq_set_tuning(pluq_ctx* c, int bm, int bn, int trsm_block) {
  if (!c) return PLUQ_ERR_INVALID_ARG;
  if (bm < 0 || bm > 128 || bn < 0 || bn > 128 || trsm_block < 0 || trsm_block > 64)
    return PLUQ_ERR_INVALID_ARG;
  if (bm) c->bm = bm;
  if (bn) c->bn = bn;
  if (trsm_block) c->trsm_block = trsm_block;
  return PLUQ_OK;
}

int pluq_set_option(pluq_ctx* c, int option, int value) {
  if (!c) return PLUQ_ERR_INVALID_ARG;
  switch (option) {
    case PLUQ_OPT_LEAF_DIM:
      if (value < 0 || value > leaf_max_dim()) return PLUQ_ERR_INVALID_ARG;
      c->leaf_dim = value;
      return PLUQ_OK;
    case PLUQ_OPT_LEAF_KIND:
      if (value < 0 || value > 4) return PLUQ_ERR_INVALID_ARG;
      c->leaf_kind = value;
      return PLUQ_OK;
    case PLUQ_OPT_TILE_M:
      if (value < 1 || value > 128) return PLUQ_ERR_INVALID_ARG;
      c->bm = value;
      return PLUQ_OK;
    case PLUQ_OPT_TILE_N:
      if (value < 1 || value > 128) return PLUQ_ERR_INVALID_ARG;
      c->bn = value;
      return PLUQ_OK;
    case PLUQ_OPT_CHAIN_ROWS:
      if (value < 0 || value > 64) return PLUQ_ERR_INVALID_ARG;
      c->chain_rows = value;
      return PLUQ_OK;
    case PLUQ_OPT_THIN_GEMM:
      if (value < 0 || value > 1) return PLUQ_ERR_INVALID_ARG;
      c->thin_gemm = value;
      return PLUQ_OK;
    case PLUQ_OPT_DECOMPOSITION:
      if (value < 0 || value > 1) return PLUQ_ERR_INVALID_ARG;
      c->decomposition = value;
      return PLUQ_OK;
    case PLUQ_OPT_SLAB_ROWS:
      if (value < 0) return PLUQ_ERR_INVALID_ARG;
      c->slab_rows = value;
      return PLUQ_OK;
    case PLUQ_OPT_USE_TUNED:
      if (value < 0 || value > 1) return PLUQ_ERR_INVALID_ARG;
      c->use_tuned = value;
      return PLUQ_OK;
    case PLUQ_OPT_FORK_DEPTH:
      if (value < 0 || value > 4) return PLUQ_ERR_INVALID_ARG;
      c->fork_depth = value;
      return PLUQ_OK;
    case PLUQ_OPT_TRSM_BLOCK:
      if (value < 1 || value > 64) return PLUQ_ERR_INVALID_ARG;
      c->trsm_block = value;
      return PLUQ_OK;
    case PLUQ_OPT_WAIT_LIMIT_US:
      if (value < 0 || value > 60000000) return PLUQ_ERR_INVALID_ARG;
      c->wait_cycles = (long long)value * 2000;
      return PLUQ_OK;
    case PLUQ_OPT_DIAG_INVERSES:
      if (value < 0 || value > 1) return PLUQ_ERR_INVALID_ARG;
      c->dinv_enable = value;
      return PLUQ_OK;
    case PLUQ_OPT_FUSED_KMAX:
      if (value < 0) return PLUQ_ERR_INVALID_ARG;
      c->fused_kmax = value;
      return PLUQ_OK;
    case PLUQ_OPT_TRSM_STRIP:
      if (value != 0 && value != 256 && value != 512) return PLUQ_ERR_INVALID_ARG;
      c->strip_max = value;
      return PLUQ_OK;
    case PLUQ_OPT_FGEMM_TILE:
      if (value < 0 || value > 2) return PLUQ_ERR_INVALID_ARG;
      c->limb_variant = value;
      return PLUQ_OK;
    case PLUQ_OPT_WINOGRAD_MIN:
      if (value < 0) return PLUQ_ERR_INVALID_ARG;
      c->wino_min = value;
      return PLUQ_OK;
    case PLUQ_OPT_LOOKAHEAD:
      if (value < 0 || value > 1) return PLUQ_ERR_INVALID_ARG;
      c->lookahead = value;
      return PLUQ_OK;
    case PLUQ_OPT_BATCH_SLAB:
      if (value != 0 && value != 16 && value != 24 && value != 32) return PLUQ_ERR_INVALID_ARG;
      c->batch_slab = value;
      return PLUQ_OK;
    case PLUQ_OPT_WORKSPACE_MB:
      if (value < 0) return PLUQ_ERR_INVALID_ARG;
      c->ws->limit = (size_t)value << 20;
      return PLUQ_OK;
    default:
      return PLUQ_ERR_INVALID_ARG;
  }
}

int pluq_set_leaf(pluq_ctx* c, int leaf_dim) {
  if (!c || leaf_dim < 0 || leaf_dim > leaf_max_dim()) return PLUQ_ERR_INVALID_ARG;
  c->leaf_dim = leaf_dim;
  return PLUQ_OK;
}

int pluq_autotune(pluq_ctx* c, uint32_t p, int64_t m, int64_t n, const uint32_t* A, int64_t lda,
                  int form, void* stream, double budget_ms, int32_t* chosen, double* best_ms) {
  if (!c || m <= 0 || n <= 0 || !A || lda < n) return PLUQ_ERR_INVALID_ARG;
  if (m >= 0x7fffffff || n >= 0x7fffffff) return PLUQ_ERR_INVALID_ARG;
  PLUQ_TRY(prepare(c, p, m, n, form, stream));
  const size_t bytes = sizeof(uint32_t) * (size_t)m * n;
  PLUQ_TRY(c->tune_src.ensure(bytes));
  PLUQ_TRY(c->tune_dst.ensure(bytes));
  uint32_t* src = c->tune_src.as<uint32_t>();
  uint32_t* dst = c->tune_dst.as<uint32_t>();
  {
    ProfScope ps(c, PC_OTHER, 0, 8.0 * m * n);
    k_copy_mat<<<grid2(m, n), 256, 0, c->stream>>>(src, n, A, lda, m, n);
    PLUQ_CUDA(cudaGetLastError());
  }
  if (budget_ms <= 0) budget_ms = 10000.0;
  const int save_leaf = c->leaf_dim, save_kind = c->leaf_kind, save_fork = c->fork_depth;
  const int save_variant = c->limb_variant;
  c->tuning = true;
  // one warm run, then the best of two timed runs of a schedule (ms), or a status
  auto trial = [&](int leaf, int kind, int fork, int variant, double* ms) -> int {
    c->leaf_dim = leaf;
    c->leaf_kind = kind;
    c->fork_depth = fork;
    c->limb_variant = variant;
    double best = 1e30;
    for (int it = 0; it < 3; ++it) {
      PLUQ_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, c->stream));
      PLUQ_CUDA(cudaStreamSynchronize(c->stream));
      const auto t0 = std::chrono::steady_clock::now();
      int64_t r = 0;
      const int st = factor(c, m, n, dst, n, &r);
      if (st != PLUQ_OK) return st;
      const double t = std::chrono::duration<double, std::milli>(
                           std::chrono::steady_clock::now() - t0).count();
      if (it > 0) best = std::min(best, t);
    }
    *ms = best;
    return PLUQ_OK;
  };
  const auto start = std::chrono::steady_clock::now();
  auto spent = [&] {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - start)
        .count();
  };
  // leaf cut-offs that differ for this shape (one at or above the larger side)
  std::vector<int> leaves;
  for (int l : {1024, 512, 2048}) {
    const int64_t big = std::max(m, n);
    bool dup = false;
    for (int e : leaves) dup |= (e >= big && l >= big);
    if (!dup) leaves.push_back(l);
  }
  int b_leaf = 1024, b_kind = 2, b_fork = 2, b_var = save_variant;
  double b_ms = 1e30;
  int st = PLUQ_OK;
  // one-CTA 16-bit tiles of 256 for small primes (dense blocks take them under
  // the per-leaf choice, rank-deficient ones the cluster leaf)
  if (c->F.p < (1u << 16)) leaves.push_back(256);
  // stage 1: cut-off and leaf kind (the default schedule first); stage 2: fork depth
  for (int l : leaves) {
    for (int k : {2, 0, 1, 3, 4}) {
      if (k == 4 && l != 256) continue;
      if (l == 256 && (k == 0 || k == 1)) continue;
      if (b_ms < 1e30 && spent() > budget_ms) break;
      double ms = 0;
      st = trial(l, k, 2, b_var, &ms);
      if (st != PLUQ_OK) break;
      if (ms < b_ms) {
        b_ms = ms;
        b_leaf = l;
        b_kind = k;
      }
    }
    if (st != PLUQ_OK) break;
  }
  for (int f : {0, 1, 3}) {
    if (st != PLUQ_OK || spent() > budget_ms) break;
    double ms = 0;
    st = trial(b_leaf, b_kind, f, b_var, &ms);
    if (st == PLUQ_OK && ms < b_ms) {
      b_ms = ms;
      b_fork = f;
    }
  }
  // stage 3: the limb fgemm's tile variant (only the two-digit and one-digit
  // plans have alternatives)
  if (c->form == PLUQ_FORM_LIMB_F16 && c->F.p < (1u << 18)) {
    for (int v : {0, 1, 2}) {
      if (v == b_var || st != PLUQ_OK || spent() > budget_ms) continue;
      double ms = 0;
      st = trial(b_leaf, b_kind, b_fork, v, &ms);
      if (st == PLUQ_OK && ms < b_ms) {
        b_ms = ms;
        b_var = v;
      }
    }
  }
  c->tuning = false;
  c->leaf_dim = save_leaf;
  c->leaf_kind = save_kind;
  c->fork_depth = save_fork;
  c->limb_variant = save_variant;
  if (st != PLUQ_OK) return st;
  pluq_ctx::Tuned t{c->F.p, m, n, c->form, b_leaf, b_kind, b_fork, b_var, b_ms};
  bool replaced = false;
  for (pluq_ctx::Tuned& e : c->tuned)
    if (e.p == t.p && e.m == m && e.n == n && e.form == t.form) {
      e = t;
      replaced = true;
    }
  if (!replaced) c->tuned.push_back(t);
  if (chosen) {
    chosen[0] = b_leaf;
    chosen[1] = b_kind;
    chosen[2] = b_fork;
    chosen[3] = b_var;
  }
  if (best_ms) *best_ms = b_ms;
  return PLUQ_OK;
}

int pluq_last_stats(pluq_ctx* c, int64_t* n_base, int64_t* n_nodes, int64_t* n_gemm) {
  if (!c) return PLUQ_ERR_INVALID_ARG;
  if (n_base) *n_base = c->n_base;
  if (n_nodes) *n_nodes = c->n_nodes;
  if (n_gemm) *n_gemm = c->n_gemm;
  return PLUQ_OK;
}

int pluq_profile_enable(pluq_ctx* c, int enable) {
  if (!c) return PLUQ_ERR_INVALID_ARG;
  c->prof.on = enable != 0;
  c->prof.used = 0;
  c->prof.recs.clear();
  for (int k = 0; k < PC_COUNT; ++k) c->launches[k] = 0;
  return PLUQ_OK;
}

int pluq_profile_read(pluq_ctx* c, int cls, int64_t* launches, double* ms, double* flops,
                      double* bytes, double* tensor_flops) {
  if (!c || cls < 0 || cls >= PC_COUNT) return PLUQ_ERR_INVALID_ARG;
  PLUQ_CUDA(cudaSetDevice(c->device));
  int64_t nl = c->launches[cls];
  double t = 0, f = 0, b = 0, tf = 0;
  for (const ProfRec& r : c->prof.recs) {
    if (r.cls != cls) continue;
    float e = 0;
    PLUQ_CUDA(cudaEventSynchronize(c->prof.pool[r.b]));
    PLUQ_CUDA(cudaEventElapsedTime(&e, c->prof.pool[r.a], c->prof.pool[r.b]));
    t += e;
    f += r.flops;
    b += r.bytes;
    tf += r.tflops;
  }
  if (launches) *launches = nl;
  if (ms) *ms = t;
  if (flops) *flops = f;
  if (bytes) *bytes = b;
  if (tensor_flops) *tensor_flops = tf;
  return PLUQ_OK;
}

const char* pluq_status_string(int s) {
  switch (s) {
    case PLUQ_OK: return "ok";
    case PLUQ_ERR_INVALID_ARG: return "invalid argument";
    case PLUQ_ERR_P_NOT_PRIME: return "p is not prime";
    case PLUQ_ERR_P_OUT_OF_RANGE: return "p out of range [2, 2^31)";
    case PLUQ_ERR_ENTRY_OUT_OF_RANGE: return "matrix entry >= p";
    case PLUQ_ERR_UNSUPPORTED_FORM: return "fgemm form unsupported for this p";
    case PLUQ_ERR_NO_WORKSPACE: return "device workspace allocation failed";
    case PLUQ_ERR_CUDA: return "CUDA error";
    case PLUQ_ERR_TIMEOUT: return "device wait timed out";
    case PLUQ_ERR_TOO_LARGE: return "problem exceeds the fixed scratch array";
    default: return "unknown status";
  }
}

}  // extern "C"
