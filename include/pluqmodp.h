/*
 * pluqmodp.h — C ABI of the GB300 (sm_103a) rank-profile-revealing PLUQ
 * library over a prime field GF(p).
 *
 * Method: Dumas, Gautier, Pernet, Sultan, "Parallel computation of echelon
 * forms" (arXiv:1402.3501).  The factorization is the tile-recursive
 * elimination of Sec. 4.1 ("Tiled recursive elimination": recursive splitting
 * into four quadrants, the bottom-left and top-right eliminations independent
 * once the top-left one is done), built on the routines of Sec. 2.1: fgemm
 * C <- alpha A B + beta C mod p with delayed modular reduction (Sec. 3.1),
 * ftrsm, flaswp and fgetrf, which computes (P, L, U, Q) with L and U stored
 * in place of A such that A = P L U Q.  The pivoting reveals both the row and
 * the column rank profile (Sec. 4.1).
 *
 * Conventions shared by every entry point
 *   - p is prime, 2 <= p < 2^31.  Matrix entries are uint32 residues in
 *     [0, p), row-major with a leading dimension (elements, >= columns).
 *   - Device pointers unless stated otherwise; the caller owns every buffer.
 *   - Permutations are int32 index vectors: (P^T A)[t,:] = A[P[t],:] and
 *     (A Q^T)[:,u] = A[:,Q[u]].  The first r entries of P and Q are the
 *     pivots: {(P[k], Q[k]) : k < r} is the rank profile matrix of A.
 *   - Compressed storage of B = P^T A Q^T: B[i,j] for i > j, j < r holds L
 *     (unit diagonal implicit); B[i,j] for i <= j, i < r holds U (non-zero
 *     diagonal); the trailing (m-r) x (n-r) block is zero.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls
 *     enqueue work on it; the recursion reads block ranks back to the host,
 *     so calls return once the factorization has been issued and its ranks
 *     are known.  A context is not thread-safe; use one per host thread.
 *   - m = 0 or n = 0 is valid: rank 0, identity permutations.
 *   - Every call returns PLUQ_OK (0) or a negative status below.
 */
#ifndef PLUQMODP_H
#define PLUQMODP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define PLUQ_OK 0
#define PLUQ_ERR_INVALID_ARG -1        /* negative size, ld < columns, NULL */
#define PLUQ_ERR_P_NOT_PRIME -2        /* p fails a deterministic primality test */
#define PLUQ_ERR_P_OUT_OF_RANGE -3     /* p < 2 or p >= 2^31 */
#define PLUQ_ERR_ENTRY_OUT_OF_RANGE -4 /* an input entry is >= p */
#define PLUQ_ERR_UNSUPPORTED_FORM -5   /* fgemm form unavailable for this p */
#define PLUQ_ERR_NO_WORKSPACE -6       /* device workspace allocation failed */
#define PLUQ_ERR_CUDA -7               /* a CUDA runtime call failed */
#define PLUQ_ERR_TIMEOUT -8            /* a bounded device wait ran out */
#define PLUQ_ERR_TOO_LARGE -9          /* exceeds the fixed scratch of fgemm_modp_noalloc */

/* fgemm forms for the Schur-complement updates (Sec. 3.1).  Both are exact
 * and both cover every p < 2^31.
 *   FP64:     residues embedded in doubles, products on FP64 DMMA tensor
 *             instructions, one reduction per k(p-1)^2 < 2^53 block (the
 *             paper's floating-point embedding); for p beyond about 2^24 the
 *             operands are split into 16-bit halves and four exact products
 *             are combined.
 *   LIMB_F16: residues balanced and split into L signed base-2^8 digits held
 *             exactly in FP16 (L = 1 below p = 512, 2 up to about 2^18, 3 up
 *             to about 2^25, 4 beyond), products on tcgen05 tensor cores with
 *             FP32 accumulation kept below 2^24, recombined and reduced once
 *             per block.
 *   AUTO:     LIMB_F16. */
#define PLUQ_FORM_AUTO 0
#define PLUQ_FORM_FP64 1
#define PLUQ_FORM_LIMB_F16 2

typedef struct pluq_ctx pluq_ctx;

/* Create a context bound to CUDA device `device`; *ctx receives it.
 * The context owns the device workspace (grown on demand, freed by
 * pluq_destroy).  Errors: INVALID_ARG (ctx NULL), CUDA. */
int pluq_create(pluq_ctx** ctx, int device);

/* Release a context and its workspace.  NULL is accepted. */
int pluq_destroy(pluq_ctx* ctx);

/* Rank-profile-revealing PLUQ (getrf of Sec. 2.1, tile-recursive as in
 * Sec. 4.1) of the m x n matrix A over GF(p), in place.
 *   A        device, m x n, leading dimension lda >= n; on return holds the
 *            compressed L\U of B = P^T A Q^T (see conventions).
 *   P, Q     device int32, length m and n; receive the permutations.
 *   rank_dev device int64 scalar (may be NULL); receives r.
 *   rrp, crp device int32, length >= min(m,n) (either may be NULL); receive
 *            the sorted row and column rank profiles in their first r entries.
 *   form     PLUQ_FORM_*.
 * Errors: INVALID_ARG, P_NOT_PRIME, P_OUT_OF_RANGE, ENTRY_OUT_OF_RANGE (A is
 * left unmodified), UNSUPPORTED_FORM, NO_WORKSPACE, CUDA. */
int pluq_modp(pluq_ctx* ctx, uint32_t p, int64_t m, int64_t n, uint32_t* A, int64_t lda,
              int32_t* P, int32_t* Q, int64_t* rank_dev, int32_t* rrp, int32_t* crp,
              int form, void* stream);

/* Reduced row echelon form of A over GF(p) (the echelon form of Sec. 4.1,
 * made canonical: pivots equal to 1, zeros above them, rows ordered by pivot
 * column).  Computed from the PLUQ as R = (U Q)[:, CRP]^{-1} (U Q).
 *   A        device, m x n, lda >= n; not modified (a workspace copy is
 *            factored).
 *   R        device, min(m,n) x n, ldr >= n; receives the r x n RREF in its
 *            first r rows (rows r.. are left untouched).
 *   rank_dev device int64 scalar (may be NULL).
 *   crp      device int32, length >= min(m,n) (may be NULL): pivot columns.
 * Errors: as pluq_modp. */
int echelon_modp(pluq_ctx* ctx, uint32_t p, int64_t m, int64_t n, const uint32_t* A,
                 int64_t lda, uint32_t* R, int64_t ldr, int64_t* rank_dev, int32_t* crp,
                 int form, void* stream);

/* Reduced column echelon form of A over GF(p): E = RREF(A^T)^T, the echelon
 * form by columns that the paper also names (Sec. 4.1): pivots equal to 1,
 * zeros to their left, columns ordered by pivot row, the pivot rows being the
 * row rank profile.  Computed as the RREF of the transpose (one transpose
 * pass into the workspace, then as echelon_modp).
 *   A        device, m x n, lda >= n; not modified.
 *   C        device, m x min(m,n), ldc >= min(m,n); receives the m x r form
 *            in its first r columns (columns r.. are left untouched).
 *   rank_dev device int64 scalar (may be NULL).
 *   rrp      device int32, length >= min(m,n) (may be NULL): pivot rows.
 * Errors: as pluq_modp. */
int column_echelon_modp(pluq_ctx* ctx, uint32_t p, int64_t m, int64_t n, const uint32_t* A,
                        int64_t lda, uint32_t* C, int64_t ldc, int64_t* rank_dev, int32_t* rrp,
                        int form, void* stream);

/* Rank and both rank profiles of A over GF(p) (Sec. 4.1), A unmodified.
 *   rank_dev       device int64 scalar (may be NULL).
 *   rrp, crp       device int32, length >= min(m,n) (may be NULL).
 *   rpm_col_of_row device int32, length m (may be NULL): the rank profile
 *                  matrix as a map row -> pivot column, -1 for rows outside
 *                  the row rank profile.
 * Errors: as pluq_modp. */
int rank_profile_modp(pluq_ctx* ctx, uint32_t p, int64_t m, int64_t n, const uint32_t* A,
                      int64_t lda, int64_t* rank_dev, int32_t* rrp, int32_t* crp,
                      int32_t* rpm_col_of_row, int form, void* stream);

/* Schur-complement update C <- C - A B mod p (fgemm of Sec. 2.1 with
 * alpha = -1, beta = 1, delayed reduction of Sec. 3.1), exposed for callers
 * and kernel-level checks.
 *   A  device, M x K, lda >= K;  B device, K x N, ldb >= N;
 *   C  device, M x N, ldc >= N, updated in place.  C may not overlap A or B.
 * The call reads the kernels' device error word back, so it returns once the
 * product is complete on `stream`.
 * Errors: INVALID_ARG, P_*, UNSUPPORTED_FORM, NO_WORKSPACE, CUDA, TIMEOUT (a
 * bounded device wait ran out; C is then left unchanged or partly updated). */
int fgemm_modp(pluq_ctx* ctx, uint32_t p, int64_t M, int64_t N, int64_t K, const uint32_t* A,
               int64_t lda, const uint32_t* B, int64_t ldb, uint32_t* C, int64_t ldc, int form,
               void* stream);

/* fgemm_modp for callers that cannot allocate device memory (no cudaMalloc,
 * cudaFree or allocating library call happens inside).  The paper has no
 * counterpart: this is a deployment variant of the limb form of fgemm_modp.
 *   Computes C <- C - A B mod p exactly, as fgemm_modp with
 *   PLUQ_FORM_LIMB_F16; same argument layout, no context.  The digit planes
 *   live in one 32 MiB device array inside the library that each GPU loading
 *   the library keeps until process exit; problems whose planes exceed it,
 *   2 L (ceil(M/128)*128 + ceil(N/T)*T) ceil(K/64)*64 bytes with L digits as
 *   for PLUQ_FORM_LIMB_F16 (T = 128 for L = 1, 80 for L = 2, else 64), return
 *   PLUQ_ERR_TOO_LARGE.
 *   The first call on a device looks up that array's device address (with
 *   the device current), so make it before any stream capture.  All calls
 *   share the array: calls that overlap on the GPU (other streams, other
 *   host threads) race; issue them on one stream.  The call reads the
 *   kernel's error word back into a host variable of its own (no
 *   allocation), so it returns once the product is complete on `stream`.
 * Errors: INVALID_ARG, P_*, UNSUPPORTED_FORM (no limb plan; not reached for
 * p < 2^31), TOO_LARGE (also for any dimension beyond the array), CUDA,
 * TIMEOUT (a bounded device wait ran out; C is then left unchanged or partly
 * updated). */
int fgemm_modp_noalloc(uint32_t p, int64_t M, int64_t N, int64_t K, const uint32_t* A,
                       int64_t lda, const uint32_t* B, int64_t ldb, uint32_t* C, int64_t ldc,
                       void* stream);

/* Batched PLUQ of `batch` independent matrices (each as pluq_modp, in place):
 * the batching of many small rank-deficient factorizations in one persistent,
 * graph-captured launch.  Matrices with m, n <= 1024 are taken by CTAs of one
 * persistent kernel from a work counter (largest first), one CTA per matrix,
 * each running the rank-profile-revealing elimination of Sec. 4.1 (rows in
 * order) blocked by slabs of pivots collected in shared memory, the rows below
 * each slab updated at once (tensor cores for p < 2^16).  The launch and its
 * descriptor / result copies are captured once in a CUDA graph per batch size
 * and replayed.  Larger matrices are factored one by one (`form` selects their
 * product form).
 *   m, n, lda   host int64 arrays of length batch.
 *   A, P, Q     host arrays of `batch` device pointers.
 *   ranks       host int64 array of length batch; receives the ranks.
 *   status      host int32 array of length batch (may be NULL): per-matrix
 *               status codes (ENTRY_OUT_OF_RANGE leaves that matrix as is).
 * The call returns after the results are on the host.  Returns the first
 * failing per-matrix status, else PLUQ_OK. */
int pluq_modp_batched(pluq_ctx* ctx, uint32_t p, int32_t batch, const int64_t* m,
                      const int64_t* n, uint32_t* const* A, const int64_t* lda,
                      int32_t* const* P, int32_t* const* Q, int64_t* ranks, int32_t* status,
                      int form, void* stream);

/* Rank and both rank profiles of every matrix of a batch (the batched form of
 * rank_profile_modp, Sec. 4.1): pluq_modp_batched on the matrices, then one
 * launch sorting each matrix's pivot rows and columns.  A[b] is overwritten
 * with its compressed L\U, as in pluq_modp_batched; the permutations go to a
 * workspace of the context.
 *   rrp, crp host arrays of batch device pointers (either array may be NULL;
 *            an entry may be NULL): int32, length >= min(m[b], n[b]); receive
 *            the sorted row and column rank profiles.
 *   ranks    host, batch entries; -1 for a matrix that failed.
 *   status   host, batch entries (may be NULL).
 * Other arguments and errors as pluq_modp_batched.  Synchronises the stream. */
int rank_profile_modp_batched(pluq_ctx* ctx, uint32_t p, int32_t batch, const int64_t* m,
                              const int64_t* n, uint32_t* const* A, const int64_t* lda,
                              int32_t* const* rrp, int32_t* const* crp, int64_t* ranks,
                              int32_t* status, int form, void* stream);

/* Reduced row echelon form of every matrix of a batch (the batched form of
 * echelon_modp, Sec. 4.1): each matrix is factored and solved in turn on the
 * stream (each needs its own triangular solve by its own rank).
 *   m, n, lda, ldr  host int64 arrays of length batch (lda[b], ldr[b] >= n[b]).
 *   A        host array of batch device pointers, not modified.
 *   R        host array of batch device pointers: min(m[b], n[b]) x n[b]; receive
 *            the r x n RREF in their first r rows.
 *   crp      host array of batch device pointers (the array or an entry may be
 *            NULL): int32, length >= min(m[b], n[b]); receive the pivot columns.
 *   ranks    host, batch entries; -1 for a matrix that failed.
 *   status   host, batch entries (may be NULL): per-matrix status codes.
 * Returns the first failing per-matrix status, else PLUQ_OK; a failure that is
 * not the matrix's own (prime, form, workspace, device) stops the batch and
 * marks the remaining matrices with it.  Each factorization synchronises the
 * stream, as in echelon_modp. */
int echelon_modp_batched(pluq_ctx* ctx, uint32_t p, int32_t batch, const int64_t* m,
                         const int64_t* n, const uint32_t* const* A, const int64_t* lda,
                         uint32_t* const* R, const int64_t* ldr, int32_t* const* crp,
                         int64_t* ranks, int32_t* status, int form, void* stream);

/* Host copy of the rank found by the last factorization on this context. */
int pluq_last_rank(pluq_ctx* ctx, int64_t* rank);

/* Waits for the work the context has issued on its stream (the stream of its
 * last call) and returns the device-side status of that work: the context's
 * device error word (PLUQ_ERR_TIMEOUT when a bounded device wait ran out), else
 * PLUQ_ERR_CUDA for an asynchronous CUDA error, else PLUQ_OK.  The entry points
 * above already return once their results are complete (the recursion reads
 * each leaf's rank on the host), so this is the check for callers that queue
 * their own work on the same stream after a call.  The error word is cleared by
 * the context's next call. */
int pluq_sync_status(pluq_ctx* ctx);

/* Tuning knobs of the recursion (base-case tile bm x bn, 1..128 each, and the
 * diagonal block of the triangular solves, 1..64).  0 keeps the current
 * value. */
int pluq_set_tuning(pluq_ctx* ctx, int bm, int bn, int trsm_block);

/* Options of the recursion (value ranges in brackets):
 *   PLUQ_OPT_LEAF_DIM    largest leaf block, rows and columns [0, 2048]
 *                        (default 1024); 0 sends the recursion down to
 *                        one-CTA tiles
 *   PLUQ_OPT_LEAF_KIND   leaf kernel [0, 4]: 0 one grid barrier per pivot
 *                        (rows dealt cyclically over the CTAs; rows that
 *                        reduce to zero cost nothing more), 1 block-row
 *                        wavefront (each CTA applies the earlier CTAs'
 *                        pivot rows as they are published, then factors its
 *                        own rows; one hand-off per CTA; faster on dense
 *                        blocks), 2 (default) wavefront while the previous
 *                        leaf of the call had rank density above 1/2, else
 *                        kind 3 where the block fits it, else barrier; 3 one
 *                        cluster barrier per pivot (the
 *                        block in the shared memory of one thread-block
 *                        cluster of up to 16 CTAs, candidates and the
 *                        elected row read from the other CTAs' shared
 *                        memory; blocks up to 1024 x 1024 for p < 2^24,
 *                        smaller ones above; larger blocks take kind 0);
 *                        4 one CTA with the block as 16-bit residues in its
 *                        shared memory, one block barrier per pivot (p < 2^16,
 *                        blocks up to 256 x 256; other blocks as kind 2).
 *                        Kind 2 also takes the kind-4 leaf for dense blocks
 *                        that fit it.
 *   PLUQ_OPT_TILE_M/N    one-CTA base-case tile [1, 128]
 *   PLUQ_OPT_TRSM_BLOCK  diagonal block of the triangular solves [1, 64]
 *                        (each block is inverted, then applied as a product)
 *   PLUQ_OPT_CHAIN_ROWS  rows per CTA of wavefront leaves [0, 64]; 0 (default)
 *                        spreads the leaf over all SMs
 *   PLUQ_OPT_FORK_DEPTH  recursion levels [0, 4] (default 2) at which the two
 *                        independent calls on F and G run concurrently, each
 *                        on its own stream, host thread and workspace with
 *                        half the SMs for its leaves; 0 runs them in turn.
 *                        Profiling (pluq_profile_enable) runs them in turn.
 *   PLUQ_OPT_THIN_GEMM   1 (default): in the limb form, Schur updates with an
 *                        inner dimension K <= 128 (and K p < 2^31) and at most
 *                        2^27 multiply-adds run on the CUDA cores (exact
 *                        64-bit sums, one reduction per entry) instead of
 *                        packing digits for the tensor cores; 0: every update
 *                        on the tensor cores.
 *   PLUQ_OPT_DECOMPOSITION  [0, 1]: 0 (default) tile recursive (Sec. 4.1,
 *                        "Tiled recursive elimination": both dimensions
 *                        halved, F and G independent); 1 tiled iterative
 *                        (Sec. 4.1, "Tiled iterative elimination" and the
 *                        panel PLUQ figure): the first SLAB_ROWS rows are
 *                        factored across all columns, by column tiles of the
 *                        leaf cut-off taken in turn, then the Schur
 *                        complement below them the same way.  Both give the
 *                        same rank, rank profiles and rank profile matrix
 *                        (the pivoting of the recursion recovers them for any
 *                        split); P, Q and L\U may differ (any valid factors).
 *   PLUQ_OPT_SLAB_ROWS   rows of a tiled-iterative slab [0, 2^31); 0
 *                        (default): the leaf cut-off
 *   PLUQ_OPT_USE_TUNED   1 (default): factorizations whose (p, m, n, form)
 *                        was autotuned use the tuned schedule in place of
 *                        LEAF_DIM, LEAF_KIND and FORK_DEPTH; 0: ignore it.
 *   PLUQ_OPT_WAIT_LIMIT_US  bound of every spin-wait of the cooperative leaf
 *                        kernels (kinds 0 and 1) on a memory word, in
 *                        microseconds at a 2 GHz SM clock [0, 6e7] (default
 *                        2e6): a wait that runs out records PLUQ_ERR_TIMEOUT,
 *                        every CTA of the launch returns, the call returns
 *                        that status and the context stays usable.  0 makes
 *                        any wait that is not satisfied at once run out.
 *   PLUQ_OPT_WINOGRAD_MIN  [0, 2^31): Schur updates whose M, N and K are all at
 *                        least this value take a Strassen-Winograd level
 *                        (Sec. 2.3 and Sec. 3.2: seven half-size products and
 *                        fifteen additions mod p instead of eight products),
 *                        recursively while the halves still qualify; 0
 *                        (default): classical products only.  Results are
 *                        identical (the pre-additions are reduced mod p).
 *   PLUQ_OPT_FGEMM_TILE  [0, 2] tile variant of the limb fgemm: 0 (default)
 *                        128 x 128 tiles (128 x 64 for three or four digits),
 *                        one set of weight-class accumulators in TMEM; 1 as 0
 *                        with the two middle-class products of two-digit plans
 *                        in accumulators of their own (exact K groups twice as
 *                        long where the digits allow it); 2 two accumulator
 *                        sets of 128 x 80 tiles (two digits) or 128 x 128 (one
 *                        digit), drained while the other fills.  Results are
 *                        identical; the autotuner picks among them.
 *   PLUQ_OPT_TRSM_STRIP  0 (default), 256 or 512: triangular solves finish a
 *                        triangle of up to this many rows in one launch (each
 *                        CTA runs the block substitution over its own strip of
 *                        32 columns or rows of the right-hand side); 0 keeps
 *                        one launch per 64-block and per update between them,
 *                        which measured faster on the 32768^2 factorization.
 *                        Takes effect with PLUQ_OPT_TRSM_BLOCK 64.
 *   PLUQ_OPT_FUSED_KMAX  [0, 2^31): limb-form products with an inner dimension
 *                        K up to this value run the fused kernel, whose producer
 *                        warps read the raw residues and split them into FP16
 *                        digits in shared memory themselves (no separate
 *                        packing launch; each element converted once per tile
 *                        that reads it); longer products pack their digit
 *                        planes once and stream them with TMA.  0: never.
 *   PLUQ_OPT_DIAG_INVERSES  1 (default): the inverses of the triangles of
 *                        every full-rank square leaf on the matrix's diagonal are
 *                        computed once (leaf cut-off squared each, kept in the
 *                        workspace), and the triangular solves of its ancestors
 *                        stop at that size and apply them as single tensor-core
 *                        products; used while no recursion node so far met a
 *                        rank-deficient leading block.  0: off.
 *   PLUQ_OPT_WORKSPACE_MB  cap on the device workspace the context (with its
 *                        child contexts) holds, in MiB [0, 2^31); 0 (default):
 *                        none.  A call whose workspace would exceed the cap
 *                        returns PLUQ_ERR_NO_WORKSPACE; buffers already held
 *                        stay allocated until the context is destroyed.
 *   PLUQ_OPT_BATCH_SLAB  0 (default), 16, 24 or 32: rows of the shared-memory
 *                        buffer in which the batched factorization collects a
 *                        slab's pivots (the most pivots one update of the rows
 *                        below carries); smaller buffers fit more CTAs an SM.
 *                        0: 16.
 *   PLUQ_OPT_LOOKAHEAD   0 (default) or 1: where A1 has full rank (F and G
 *                        empty) and R splits further, H's update is split at R's
 *                        first quarter: H11 first, the rest on a third stream
 *                        while R's recursion factors H11 (results are identical;
 *                        the third stream's workspace is sized for H).
 * Errors: INVALID_ARG for an unknown option or a value out of range. */
#define PLUQ_OPT_LEAF_DIM 1
#define PLUQ_OPT_LEAF_KIND 2
#define PLUQ_OPT_TILE_M 3
#define PLUQ_OPT_TILE_N 4
#define PLUQ_OPT_TRSM_BLOCK 5
#define PLUQ_OPT_CHAIN_ROWS 6
#define PLUQ_OPT_FORK_DEPTH 7
#define PLUQ_OPT_USE_TUNED 8
#define PLUQ_OPT_THIN_GEMM 9
#define PLUQ_OPT_DECOMPOSITION 10
#define PLUQ_OPT_SLAB_ROWS 11
#define PLUQ_OPT_WAIT_LIMIT_US 12
#define PLUQ_OPT_WORKSPACE_MB 13
#define PLUQ_OPT_WINOGRAD_MIN 14
#define PLUQ_OPT_FGEMM_TILE 15
#define PLUQ_OPT_TRSM_STRIP 16
#define PLUQ_OPT_FUSED_KMAX 17
#define PLUQ_OPT_DIAG_INVERSES 18
#define PLUQ_OPT_BATCH_SLAB 19
#define PLUQ_OPT_LOOKAHEAD 20
int pluq_set_option(pluq_ctx* ctx, int option, int value);

/* Largest block (rows and columns, 0..2048) factored as one leaf by a
 * cooperative grid (the same as PLUQ_OPT_LEAF_DIM); 0 disables leaves so the
 * recursion descends to one-CTA base-case tiles.  Default 1024. */
int pluq_set_leaf(pluq_ctx* ctx, int leaf_dim);

/* Counters of the last call: base-case launches, internal recursion nodes,
 * fgemm calls. */
int pluq_last_stats(pluq_ctx* ctx, int64_t* n_base, int64_t* n_nodes, int64_t* n_gemm);

/* Autotuner of the recursion schedule (no counterpart in the paper, which tunes
 * by hand for one machine): times pluq_modp on copies of A (device, m x n, row
 * stride lda, read only) under candidate schedules - leaf cut-off 1024, 512,
 * 2048 crossed with leaf kind per-leaf choice, barrier, wavefront, cluster
 * (fork depth 2), and for p < 2^16 cut-off 256 with the per-leaf choice and the
 * one-CTA tile leaf; then fork depth 0, 1, 3 for the best; then, for p < 2^18,
 * the limb fgemm's tile variants (PLUQ_OPT_FGEMM_TILE) - one warm run and the
 * best of two timed runs each, stopping once budget_ms (0: 10 s) is spent
 * after at least one schedule.  The fastest is stored in the context for
 * (p, m, n, form) and applied by later pluq_modp / echelon_modp /
 * rank_profile_modp calls of that shape (PLUQ_OPT_USE_TUNED); a new call for
 * the shape replaces it.  The timings depend on A's rank structure, so tune on
 * a representative matrix.
 * chosen (host, may be NULL, 4 entries): leaf cut-off, leaf kind, fork depth,
 * fgemm tile variant; best_ms (host, may be NULL): its time.  Synchronises the
 * stream.
 * Errors: as pluq_modp, NO_WORKSPACE (two m x n copies). */
int pluq_autotune(pluq_ctx* ctx, uint32_t p, int64_t m, int64_t n, const uint32_t* A,
                  int64_t lda, int form, void* stream, double budget_ms, int32_t* chosen,
                  double* best_ms);

/* Per-kernel-class timers.  pluq_profile_enable(ctx, 1) resets the counters
 * and brackets every later kernel launch with CUDA events on the call's
 * stream (0 stops recording; launches are counted either way).
 * pluq_profile_read(ctx, cls, ...) waits for the recorded events and returns,
 * for class cls (0 base-case tile, 1 fgemm tensor kernel, 2 operand packing,
 * 3 triangular diagonal blocks, 4 block gathers, 5 index vectors, 6 other,
 * 7 thin products on the CUDA cores),
 * the launch count, the summed device time in ms, the summed algorithmic
 * field operations (2 M N K for an fgemm) and bytes, and the summed tensor-pipe
 * flops actually issued (digit products included) of the timed launches.
 * Any output pointer may be NULL. */
int pluq_profile_enable(pluq_ctx* ctx, int enable);
int pluq_profile_read(pluq_ctx* ctx, int cls, int64_t* launches, double* ms, double* flops,
                      double* bytes, double* tensor_flops);

/* Human-readable name of a status code (static string). */
const char* pluq_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* PLUQMODP_H */
