// Shared declarations of the GF(p) PLUQ library: status codes, the context,
// and the internal entry points each translation unit provides.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <vector>

#include "pluqmodp.h"
#include "field.cuh"

#define PLUQ_CUDA(call)                                   \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return PLUQ_ERR_CUDA;          \
  } while (0)

#define PLUQ_TRY(call)               \
  do {                               \
    int s_ = (call);                 \
    if (s_ != PLUQ_OK) return s_;    \
  } while (0)

static inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Global-to-shared copies for latency-bound kernels: each thread keeps kIlp
// independent L2 loads in flight before storing, instead of one dependent
// load per loop trip.  L2-only loads (ld.global.cg) also read data that other
// SMs wrote earlier in the same kernel.
template <int kIlp = 8>
__device__ __forceinline__ void copy_g2s(uint32_t* __restrict__ dst,
                                         const uint32_t* __restrict__ src, int count, int tid,
                                         int nthreads) {
  int i = tid;
  for (; i + (kIlp - 1) * nthreads < count; i += kIlp * nthreads) {
    uint32_t v[kIlp];
#pragma unroll
    for (int q = 0; q < kIlp; ++q) v[q] = __ldcg(src + i + q * nthreads);
#pragma unroll
    for (int q = 0; q < kIlp; ++q) dst[i + q * nthreads] = v[q];
  }
  for (; i < count; i += nthreads) dst[i] = __ldcg(src + i);
}

// rows x n block (row stride lds) into dense shared rows, one warp per row.
template <int kIlp = 16>
__device__ __forceinline__ void copy_rows_g2s(uint32_t* __restrict__ dst,
                                              const uint32_t* __restrict__ src, int64_t lds,
                                              int rows, int n, int warp, int lane, int nwarps) {
  for (int lr = warp; lr < rows; lr += nwarps) {
    const uint32_t* s = src + (int64_t)lr * lds;
    uint32_t* d = dst + (size_t)lr * n;
    for (int j0 = lane; j0 < n; j0 += 32 * kIlp) {
      uint32_t v[kIlp];
#pragma unroll
      for (int q = 0; q < kIlp; ++q) {
        const int j = j0 + 32 * q;
        v[q] = j < n ? __ldcg(s + j) : 0u;
      }
#pragma unroll
      for (int q = 0; q < kIlp; ++q) {
        const int j = j0 + 32 * q;
        if (j < n) d[j] = v[q];
      }
    }
  }
}

// Device workspace held by a context and its child contexts, against an
// optional cap (0: none).
struct WsAccount {
  std::atomic<size_t> used{0};  // child contexts grow buffers from their own threads
  size_t limit = 0;
};

// A growable device allocation owned by the context.
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  WsAccount* acct = nullptr;  // the context's workspace account (may be null)
  int ensure(size_t need) {
    if (need <= bytes) return PLUQ_OK;
    size_t want = need + need / 8 + 256;
    if (acct && acct->limit && acct->used - bytes + want > acct->limit) {
      // try the exact size before giving up
      want = need;
      if (acct->used - bytes + want > acct->limit) return PLUQ_ERR_NO_WORKSPACE;
    }
    release();
    if (cudaMalloc(&ptr, want) != cudaSuccess) {
      cudaGetLastError();
      ptr = nullptr;
      return PLUQ_ERR_NO_WORKSPACE;
    }
    bytes = want;
    if (acct) acct->used += want;
    return PLUQ_OK;
  }
  void release() {
    if (ptr) cudaFree(ptr);
    if (acct && ptr) acct->used -= bytes;
    ptr = nullptr;
    bytes = 0;
  }
  template <class T>
  T* as() const { return reinterpret_cast<T*>(ptr); }
};

// Index-vector slots of the tile-recursive driver (each level halves at least
// one dimension, and dimensions are < 2^31); the tiled-iterative schedule,
// whose depth grows with the number of slabs and tiles, sizes its own.
constexpr int kMaxDepth = 72;

// Kernel classes for the per-class CUDA-event timers.
enum ProfClass {
  PC_BASE = 0,  // base-case PLUQ tile
  PC_FGEMM,     // fgemm tensor kernel (limb tcgen05 or FP64 DMMA)
  PC_PACK,      // digit-plane packing of fgemm operands
  PC_TRSM,      // diagonal-block triangular solves
  PC_PERM,      // row / column block gathers and copy-back
  PC_INDEX,     // index-vector kernels (iota, compose, shifts)
  PC_OTHER,     // range check, copies, profiles, RREF scatter
  PC_THIN,      // thin products on the CUDA cores
  PC_COUNT
};

struct ProfRec {
  int cls;
  int a, b;  // indices into the event pool
  double flops, bytes, tflops;
};

struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<ProfRec> recs;
};

struct pluq_ctx {
  Profiler prof;
  WsAccount ws_own;            // the user's context: its account
  WsAccount* ws = &ws_own;     // child contexts: the parent's account
  long long wait_cycles = 4000000000LL;  // bound of device waits (~2 s at 2 GHz)
  int64_t launches[PC_COUNT] = {0, 0, 0, 0, 0, 0, 0, 0};
  int device = 0;
  int sm_count = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;  // a child context's stream
  cudaEvent_t fork_ev = nullptr;      // recorded before F and G start
  cudaEvent_t side_ev[2] = {nullptr, nullptr};  // E ready, G updated (two-stream update)
  std::vector<cudaEvent_t> la_ev;    // look-ahead events, two a recursion depth
  int lookahead = 0;                 // PLUQ_OPT_LOOKAHEAD
  FieldP F{};
  int form = PLUQ_FORM_FP64;
  int bm = 128, bn = 128;  // base-case tile
  int trsm_block = 64;     // diagonal block of the triangular solves
  int strip_max = 0;       // largest triangle solved by one strip launch (0: none)
  int leaf_dim = 1024;     // cooperative leaves up to leaf_dim x leaf_dim (0: off)
  int leaf_kind = 2;       // 0: grid barrier per pivot, 1: wavefront, 2: chosen per leaf,
                           // 3: cluster barrier per pivot, 4: one-CTA 16-bit tile
  double leaf_density = 1.0;  // rank / min(m, n) of the last leaf of the current call
  int chain_rows = 0;      // rows per CTA of wavefront leaves (0: default)
  int64_t mmax = 0, nmax = 0;
  // workspace
  DevBuf scratch;          // uint32 gathers, packed GEMM operands
  DevBuf pack;             // packed limb / fp64 GEMM operands
  DevBuf perm_r, perm_c;   // int32 [depth_slots][mmax], [depth_slots][nmax]
  int depth_slots = kMaxDepth;  // recursion levels + one spare slot
  DevBuf tmp_i;            // int32 scratch for segment permutations
  DevBuf tri_inv;          // inverted diagonal blocks of a triangular solve
  DevBuf small;            // int32 / int64 scalars (rank, flags)
  DevBuf inv_table;        // uint32[p] inverses when p is small
  uint32_t inv_table_p = 0;
  DevBuf work;             // a copy of A for echelon / rank-profile calls
  DevBuf leaf;             // grid-barrier words and candidate rows of leaf launches
  DevBuf batch_dev;        // batched descriptors, order, ranks, status
  void* batch_host = nullptr;   // pinned mirror of batch_dev
  size_t batch_host_bytes = 0;
  cudaGraphExec_t batch_graph = nullptr;  // captured batched launch
  int batch_graph_count = -1;
  int64_t batch_graph_elems = 0;
  int batch_graph_maxn = 0;          // widest matrix the captured launch was sized for
  int batch_graph_slab = 0;          // buffer height the captured launch was made for
  int batch_slab = 0;                // batched buffer height (PLUQ_OPT_BATCH_SLAB), 0: by width
  uint32_t batch_graph_p = 0;        // field and inverse table baked into the graph
  const void* batch_graph_tab = nullptr;
  DevBuf batch_scratch;    // per-CTA gather scratch of the batched kernel
  DevBuf batch_pq;         // pivot vectors and profile descriptors of a batched rank profile
  const void* batch_graph_key = nullptr;
  int32_t* host_small = nullptr;  // pinned host scalars
  uint32_t limb_plan_p = 0;       // p of the cached limb fgemm plan
  uint64_t limb_plan[6] = {0, 0, 0, 0, 0, 0};
  int limb_variant = 0;           // tile variant of the limb fgemm (0, 1, 2)
  int64_t fused_kmax = 0;         // limb fgemms with K up to this split digits in the producer
  bool fgemm_beta0 = false;       // limb fgemm writes C = -A B (C's old values unread)
  // inverses of full-rank square diagonal leaves (negated, b x b each, slot
  // k for the leaf at rows and columns [k b, (k + 1) b) of the whole matrix):
  // the triangular solves of every ancestor apply them as one product each
  DevBuf dinv;                    // [slots][2][b][b]: -L^-1, -U^-1
  std::vector<char> dinv_valid;   // per slot
  int64_t dinv_b = 0;             // block size (the leaf cut-off), 0: cache off
  std::atomic<bool> dinv_ok{false};  // no node so far had a rank-deficient A1 (no shifts)
  int dinv_enable = 1;            // option
  // concurrent recursion (the independent calls on F and G): two child
  // contexts, each with its own stream, workspace and host thread; they share
  // the parent's index-vector slots and inverse table (disjoint ranges /
  // read-only) and cooperative leaves in a child use at most its sm_count
  int fork_depth = 2;             // levels of the recursion that run F and G concurrently
  int thin_gemm = 1;              // limb form: CUDA-core fgemm for K <= kThinMaxK
  // decomposition: 0 tile recursive (both dimensions halved); 1 tiled
  // iterative (row slabs of slab_rows rows of the Schur complement in turn,
  // each slab by column tiles of the leaf cut-off)
  int decomposition = 0;
  int slab_rows = 0;              // 0: the leaf cut-off
  int lane_depth = 0;             // 0 for the user's context
  pluq_ctx* parent = nullptr;
  pluq_ctx* lane[3] = {nullptr, nullptr, nullptr};  // F, G (and side updates), look-ahead
  // schedules chosen by pluq_autotune, per (p, m, n, form); applied by every
  // factorization of a matching shape unless use_tuned is 0
  struct Tuned {
    uint32_t p;
    int64_t m, n;
    int form, leaf_dim, leaf_kind, fork_depth, limb_variant;
    double ms;
  };
  std::vector<Tuned> tuned;
  int use_tuned = 1;
  bool tuning = false;            // inside pluq_autotune: candidates set explicitly
  DevBuf tune_src, tune_dst;      // the caller's matrix and a trial copy
  // Strassen-Winograd levels above the fgemm: applied while M, N, K are all at
  // least wino_min (0: never); pre-additions and partial sums in `wino`, one
  // region a level from offset wino_used
  int64_t wino_min = 0;
  DevBuf wino;
  int64_t wino_used = 0;
  // per-call statistics (host side)
  int64_t n_base = 0, n_nodes = 0, n_gemm = 0;
  // device error flag (int) lives in small at offset 0
};

// Points every workspace buffer of c at the account c->ws.
inline void bind_workspace(pluq_ctx* c) {
  for (DevBuf* b : {&c->scratch, &c->pack, &c->perm_r, &c->perm_c, &c->tmp_i, &c->tri_inv,
                    &c->small, &c->inv_table, &c->work, &c->leaf, &c->batch_dev,
                    &c->batch_scratch, &c->batch_pq, &c->tune_src, &c->tune_dst, &c->wino,
                    &c->dinv})
    b->acct = c->ws;
}

// Count a kernel launch of class `cls` and, when profiling, bracket it with a
// pair of CUDA events on the context stream (work = algorithmic flops/bytes).
struct ProfScope {
  pluq_ctx* c;
  int idx = -1;
  ProfScope(pluq_ctx* ctx, int cls, double flops = 0, double bytes = 0, int nlaunch = 1,
            double tflops = 0);
  ~ProfScope();
};

// kernels / helpers implemented in the .cu files
int launch_base_pluq(pluq_ctx* c, uint32_t* A, int64_t lda, int m, int n, int32_t* perm_r,
                     int32_t* perm_c, int32_t* rank_out);
int launch_leaf_pluq(pluq_ctx* c, uint32_t* X, int64_t ldx, int m, int n, int32_t* perm_r,
                     int32_t* perm_c, int32_t* rank_out);
int leaf_fits(pluq_ctx* c, int64_t m, int64_t n);
int launch_leaf_chain(pluq_ctx* c, uint32_t* X, int64_t ldx, int m, int n, int32_t* perm_r,
                      int32_t* perm_c, int32_t* rank_out);
int chain_fits(pluq_ctx* c, int64_t m, int64_t n);
int launch_leaf_cluster(pluq_ctx* c, uint32_t* X, int64_t ldx, int m, int n, int32_t* perm_r,
                        int32_t* perm_c, int32_t* rank_out);
int cluster_leaf_fits(pluq_ctx* c, int64_t m, int64_t n);
int launch_leaf_tile(pluq_ctx* c, uint32_t* X, int64_t ldx, int m, int n, int32_t* perm_r,
                     int32_t* perm_c, int32_t* rank_out);
int tile_leaf_fits(pluq_ctx* c, int64_t m, int64_t n);
int leaf_max_dim();
int launch_iota(pluq_ctx* c, int32_t* dst, int64_t count);
int batched_max_dim();
int batched_grid(pluq_ctx* c, int max_n);
int launch_batched(pluq_ctx* c, const void* descs, const int32_t* order, int count,
                   int64_t* ranks, int32_t* status, int max_elems, int max_n);
size_t batched_desc_size();
void batched_fill_desc(void* out, int i, uint32_t* A, int32_t* P, int32_t* Q, int64_t lda, int m,
                       int n);
int launch_compose(pluq_ctx* c, int32_t* base, const int32_t* perm, int64_t count);
// (base_r, perm_r) and (base_c, perm_c) composed in one launch when both fit
int launch_compose_pair(pluq_ctx* c, int32_t* base_r, const int32_t* perm_r, int64_t count_r,
                        int32_t* base_c, const int32_t* perm_c, int64_t count_c);
int launch_iota_pair(pluq_ctx* c, int32_t* dst_r, int64_t count_r, int32_t* dst_c,
                     int64_t count_c);
int launch_segperm(pluq_ctx* c, int32_t* out, const int64_t* seg_start, const int64_t* seg_len,
                   int nseg);
int permute_rows(pluq_ctx* c, uint32_t* A, int64_t lda, int64_t rows, int64_t cols,
                 const int32_t* perm);
int permute_cols(pluq_ctx* c, uint32_t* A, int64_t lda, int64_t rows, int64_t cols,
                 const int32_t* perm);
// rows of A permuted over columns [c0, c0 + n0) and [c1, c1 + n1) at once
int permute_rows2(pluq_ctx* c, uint32_t* A, int64_t lda, int64_t rows, int64_t c0, int64_t n0,
                  int64_t c1, int64_t n1, const int32_t* perm);
// columns of A permuted over rows [r0, r0 + m0) and [r1, r1 + m1) at once
int permute_cols2(pluq_ctx* c, uint32_t* A, int64_t lda, int64_t r0, int64_t m0, int64_t r1,
                  int64_t m1, int64_t cols, const int32_t* perm);
// diag0: the triangle's offset on the whole matrix's diagonal (-1: not on it),
// for the cached inverses of full-rank diagonal leaves
int trsm_left_lower_unit(pluq_ctx* c, const uint32_t* L, int64_t ldl, int64_t r, uint32_t* B,
                         int64_t ldb, int64_t ncols, int64_t diag0 = -1);
int trsm_right_upper(pluq_ctx* c, const uint32_t* U, int64_t ldu, int64_t r, uint32_t* B,
                     int64_t ldb, int64_t nrows, int64_t diag0 = -1);
// -L^{-1}, -U^{-1} of the full-rank dinv_b x dinv_b block T into cache slot `slot`
int cache_leaf_inverses(pluq_ctx* c, const uint32_t* T, int64_t ldt, int64_t slot);
int cache_leaf_inverse(pluq_ctx* w, pluq_ctx* c, bool upper, const uint32_t* T, int64_t ldt,
                       int64_t slot);
int trsm_left_upper(pluq_ctx* c, const uint32_t* U, int64_t ldu, int64_t r, uint32_t* B,
                    int64_t ldb, int64_t ncols);
// one-launch solves of a triangle of at most strip_rows(c, count) rows (its
// 64-blocks inverted beforehand, o the triangle's offset in those blocks)
int strip_rows(const pluq_ctx* c, int64_t count);
int trsm_llu_strip(pluq_ctx* c, const uint32_t* L, int64_t ldl, int64_t o, int64_t r,
                   uint32_t* B, int64_t ldb, int64_t ncols);
int trsm_ru_strip(pluq_ctx* c, const uint32_t* U, int64_t ldu, int64_t o, int64_t r, uint32_t* B,
                  int64_t ldb, int64_t nrows);
// C <- C - A B (mod p); A M x K, B K x N, C M x N, all row-major uint32.
int fgemm_sub(pluq_ctx* c, int64_t M, int64_t N, int64_t K, const uint32_t* A, int64_t lda,
              const uint32_t* B, int64_t ldb, uint32_t* C, int64_t ldc);
// fgemm_sub without the Winograd levels (thin, limb or FP64 by form)
int fgemm_sub_classical(pluq_ctx* c, int64_t M, int64_t N, int64_t K, const uint32_t* A,
                        int64_t lda, const uint32_t* B, int64_t ldb, uint32_t* C, int64_t ldc);
// one Strassen-Winograd level (then recursively while wino_applies) over
// fgemm_sub_classical; depth counts the levels above
int wino_applies(const pluq_ctx* c, int64_t M, int64_t N, int64_t K);
int fgemm_sub_wino(pluq_ctx* c, int64_t M, int64_t N, int64_t K, const uint32_t* A, int64_t lda,
                   const uint32_t* B, int64_t ldb, uint32_t* C, int64_t ldc, int depth);
// the same on the CUDA cores for a thin inner dimension (K <= kThinMaxK,
// K p < 2^31) and small total work
constexpr int64_t kThinMaxK = 128;
int thin_fgemm_ok(const pluq_ctx* c, int64_t M, int64_t N, int64_t K);
int fgemm_sub_thin(pluq_ctx* c, int64_t M, int64_t N, int64_t K, const uint32_t* A, int64_t lda,
                   const uint32_t* B, int64_t ldb, uint32_t* C, int64_t ldc);
int fgemm_sub_fp64(pluq_ctx* c, int64_t M, int64_t N, int64_t K, const uint32_t* A,
                   int64_t lda, const uint32_t* B, int64_t ldb, uint32_t* C, int64_t ldc);
int fgemm_sub_limb(pluq_ctx* c, int64_t M, int64_t N, int64_t K, const uint32_t* A,
                   int64_t lda, const uint32_t* B, int64_t ldb, uint32_t* C, int64_t ldc);
int limb_form_supported(uint32_t p);
// PLUQ_OK when p is a prime in [2, 2^31), else P_OUT_OF_RANGE / P_NOT_PRIME.
int check_prime_range(uint32_t p);
int fp64_form_supported(uint32_t p);
int ensure_inv_table(pluq_ctx* c);
const uint32_t* inv_table_ptr(pluq_ctx* c);
