/*
 * CPU oracle for rank-profile-revealing PLUQ over GF(p).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test-suite, the smoke check and the CPU baseline
 * leg of the benchmark do.  It shares no code, header, table or helper with the
 * CUDA path.
 *
 * What it computes (Dumas, Gautier, Pernet, Sultan, "Parallel computation of
 * echelon forms", arXiv:1402.3501):
 *   - getrf: A = P L U Q with L, U stored in place of A (Sec. 2.1);
 *   - the row rank profile via the row-major pivot search of Sec. 4.1: pivots
 *     are searched row by row, and the next row is only considered once the
 *     current one has no non-zero left;
 *   - delayed modular reduction (Sec. 3.1): products are accumulated in exact
 *     integers and reduced mod p only when the accumulated magnitude could
 *     leave the exact range of the accumulator (here int64 instead of the
 *     paper's double mantissa);
 *   - both rank profiles (Sec. 4.1, "both row and column rank profiles") and
 *     the reduced row echelon form.
 *
 * Algorithm (plain row-by-row right-looking Gaussian elimination mod p):
 *   W <- A as int64.  For each row i in increasing order: reduce row i mod p,
 *   take the first column j with W[i,j] != 0 as pivot (if none, row i is
 *   dependent), invert W[i,j] by the extended Euclidean algorithm and, for
 *   every later row l, record the multiplier c = W[l,j]/W[i,j] and subtract
 *   c * row i from row l.
 *
 * Output conventions (shared with the library boundary, restated here):
 *   P, Q are index vectors: (P^T A)[t,:] = A[P[t],:], (A Q^T)[:,u] = A[:,Q[u]].
 *   P = pivot rows in processing order, then the other rows ascending.
 *   Q = pivot columns in the same order, then the other columns ascending.
 *   LU (m x n) holds B = P^T A Q^T compressed: L strictly below the diagonal in
 *   the first r columns (unit diagonal implicit), U on and above the diagonal
 *   in the first r rows, the trailing (m-r) x (n-r) block zero.
 *
 * Pins: the test-suite checks this oracle against brute-force minors,
 * exhaustive enumeration of tiny matrices over GF(2), GF(3), GF(5), closed
 * forms (identity, zero, rank one, permutations, Vandermonde, L.R.U
 * constructions whose rank profile matrix is R by construction) and a library
 * RREF over GF(p).  Every function here is pinned that way.
 *
 * The `mutate` argument plants a known mistake (used only by the tests that
 * prove the pins catch such mistakes); 0 means the correct algorithm.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum {
  MUT_NONE = 0,
  MUT_LAST_NONZERO_PIVOT = 1,  /* pivot = last non-zero of the row */
  MUT_SKIP_LAST_ROW = 2,       /* elimination forgets the last row */
  MUT_SIGN = 3,                /* adds c*row instead of subtracting */
  MUT_NO_INVERSE = 4,          /* multiplier not divided by the pivot */
  MUT_RREF_NO_NORMALISE = 5,   /* RREF pivots left un-normalised */
  MUT_TRANSPOSE_INPUT = 6,     /* reads A^T */
  MUT_CRP_UNSORTED = 7,        /* column profile left in pivot order */
  MUT_NO_REDUCTION = 8         /* delayed reduction never reduces */
};

static int64_t mod_p(int64_t x, int64_t p) {
  int64_t r = x % p;
  return r < 0 ? r + p : r;
}

/* Inverse of a in [1, p) by the extended Euclidean algorithm. */
static int64_t inv_mod(int64_t a, int64_t p) {
  int64_t r0 = p, r1 = a, t0 = 0, t1 = 1;
  while (r1 != 0) {
    int64_t q = r0 / r1, tmp;
    tmp = r0 - q * r1; r0 = r1; r1 = tmp;
    tmp = t0 - q * t1; t0 = t1; t1 = tmp;
  }
  return mod_p(t0, p);
}

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/*
 * Largest number of un-reduced updates an int64 entry can absorb.  After a
 * reduction an entry lies in [0, p); each update subtracts c * w with
 * c, w in [0, p), i.e. at most (p-1)^2, so t updates keep it in
 * (-t (p-1)^2, p), exact while t (p-1)^2 <= 2^63 - p (Sec. 3.1, with int64
 * in place of the double mantissa).
 */
static int64_t update_bound(int64_t p) {
  if (p <= 2) return INT64_MAX;
  uint64_t sq = (uint64_t)(p - 1) * (uint64_t)(p - 1);
  uint64_t lim = ((uint64_t)1 << 63) - (uint64_t)p;
  return (int64_t)(lim / sq);
}

/*
 * oracle_pluq: see the file header.  Returns 0 on success, -1 on bad
 * arguments, -2 on allocation failure.
 *   A        m x n row-major, leading dimension lda, entries in [0, p)
 *   rank     out: r
 *   P, Q     out: length m and n index vectors
 *   LU       out (may be NULL): m x n, leading dimension ldlu
 *   piv_rows, piv_cols  out (may be NULL): length >= min(m,n), the pivots
 *            (i_k, j_k) in processing order = the rank profile matrix
 *   rrp, crp out (may be NULL): sorted row / column rank profiles
 */
int oracle_pluq(uint32_t p32, int64_t m, int64_t n, const uint32_t* A, int64_t lda,
                int64_t* rank, int32_t* P, int32_t* Q, uint32_t* LU, int64_t ldlu,
                int32_t* piv_rows, int32_t* piv_cols, int32_t* rrp, int32_t* crp,
                int nthreads, int mutate) {
  const int64_t p = (int64_t)p32;
  if (p < 2 || m < 0 || n < 0 || !rank || !P || !Q) return -1;
  if (m > 0 && n > 0 && (!A || lda < (mutate == MUT_TRANSPOSE_INPUT ? m : n))) return -1;
  if (mutate == MUT_TRANSPOSE_INPUT && m != n) return -1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  const int64_t rmax = m < n ? m : n;
  int64_t* W = (int64_t*)malloc((size_t)(m * n > 0 ? m * n : 1) * sizeof(int64_t));
  int32_t* Lm = (int32_t*)calloc((size_t)(m * rmax > 0 ? m * rmax : 1), sizeof(int32_t));
  int64_t* cnt = (int64_t*)calloc((size_t)(m > 0 ? m : 1), sizeof(int64_t));
  int32_t* pr = (int32_t*)malloc((size_t)(rmax > 0 ? rmax : 1) * sizeof(int32_t));
  int32_t* pc = (int32_t*)malloc((size_t)(rmax > 0 ? rmax : 1) * sizeof(int32_t));
  char* rowpiv = (char*)calloc((size_t)(m > 0 ? m : 1), 1);
  char* colpiv = (char*)calloc((size_t)(n > 0 ? n : 1), 1);
  if (!W || !Lm || !cnt || !pr || !pc || !rowpiv || !colpiv) {
    free(W); free(Lm); free(cnt); free(pr); free(pc); free(rowpiv); free(colpiv);
    return -2;
  }
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j)
      W[i * n + j] = (mutate == MUT_TRANSPOSE_INPUT) ? (int64_t)A[j * lda + i]
                                                     : (int64_t)A[i * lda + j];
  const int64_t bound = (mutate == MUT_NO_REDUCTION) ? INT64_MAX : update_bound(p);

  int64_t r = 0;
  for (int64_t i = 0; i < m; ++i) {
    int64_t* wi = W + i * n;
    for (int64_t j = 0; j < n; ++j) wi[j] = mod_p(wi[j], p);
    cnt[i] = 0;
    int64_t jp = -1;
    if (mutate == MUT_LAST_NONZERO_PIVOT) {
      for (int64_t j = n - 1; j >= 0; --j) if (wi[j] != 0) { jp = j; break; }
    } else {
      for (int64_t j = 0; j < n; ++j) if (wi[j] != 0) { jp = j; break; }
    }
    if (jp < 0) continue;
    if (colpiv[jp] || r >= rmax) {
      /* A reduced row is zero on every earlier pivot column; reaching this
         means the arithmetic went wrong (only with a planted mistake). */
      free(W); free(Lm); free(cnt); free(pr); free(pc); free(rowpiv); free(colpiv);
      return -3;
    }
    const int64_t inv = (mutate == MUT_NO_INVERSE) ? 1 : inv_mod(wi[jp], p);
    const int64_t k = r;
    pr[k] = (int32_t)i;
    pc[k] = (int32_t)jp;
    rowpiv[i] = 1;
    colpiv[jp] = 1;
    r++;
    const int64_t lend = (mutate == MUT_SKIP_LAST_ROW) ? m - 1 : m;
#pragma omp parallel for schedule(static) if (m - i > 64 && n > 64)
    for (int64_t l = i + 1; l < lend; ++l) {
      int64_t* wl = W + l * n;
      const int64_t c = mod_p(mod_p(wl[jp], p) * inv, p);
      Lm[l * rmax + k] = (int32_t)c;
      if (c == 0) continue;
      if (cnt[l] >= bound) {
        for (int64_t j = 0; j < n; ++j) wl[j] = mod_p(wl[j], p);
        cnt[l] = 0;
      }
      if (mutate == MUT_SIGN) {
        for (int64_t j = jp; j < n; ++j) wl[j] += c * wi[j];
      } else {
        for (int64_t j = jp; j < n; ++j) wl[j] -= c * wi[j];
      }
      cnt[l] += 1;
    }
  }

  /* P, Q: pivots in processing order, then the rest ascending. */
  int64_t t = 0;
  for (int64_t k = 0; k < r; ++k) P[t++] = pr[k];
  for (int64_t i = 0; i < m; ++i) if (!rowpiv[i]) P[t++] = (int32_t)i;
  t = 0;
  for (int64_t k = 0; k < r; ++k) Q[t++] = pc[k];
  for (int64_t j = 0; j < n; ++j) if (!colpiv[j]) Q[t++] = (int32_t)j;

  if (LU) {
    for (int64_t a = 0; a < m; ++a) {
      const int64_t row = P[a];
      for (int64_t u = 0; u < n; ++u) {
        uint32_t v = 0;
        if (a < r && u >= a) {
          v = (uint32_t)mod_p(W[pr[a] * n + Q[u]], p); /* U: reduced pivot row */
        } else if (u < r && u < a) {
          v = (uint32_t)Lm[row * rmax + u]; /* L: multiplier of pivot u */
        }
        LU[a * ldlu + u] = v;
      }
    }
  }
  if (piv_rows) for (int64_t k = 0; k < r; ++k) piv_rows[k] = pr[k];
  if (piv_cols) for (int64_t k = 0; k < r; ++k) piv_cols[k] = pc[k];
  if (rrp) for (int64_t k = 0; k < r; ++k) rrp[k] = pr[k];
  if (crp) {
    for (int64_t k = 0; k < r; ++k) crp[k] = pc[k];
    if (mutate != MUT_CRP_UNSORTED) qsort(crp, (size_t)r, sizeof(int32_t), cmp_i32);
  }
  *rank = r;
  free(W); free(Lm); free(cnt); free(pr); free(pc); free(rowpiv); free(colpiv);
  return 0;
}

/*
 * oracle_rref: reduced row echelon form of A over GF(p) (the canonical
 * echelon form whose pivot columns are the column rank profile, Sec. 4.1).
 * Runs oracle_pluq, then Gauss-Jordan on the r pivot rows: sort them by pivot
 * column, scale each pivot to 1, clear the entries above each pivot.
 *   R  out: r x n, leading dimension ldr (caller sizes it min(m,n) x n)
 */
int oracle_rref(uint32_t p32, int64_t m, int64_t n, const uint32_t* A, int64_t lda,
                int64_t* rank, uint32_t* R, int64_t ldr, int nthreads, int mutate) {
  const int64_t p = (int64_t)p32;
  if (p < 2 || m < 0 || n < 0 || !rank) return -1;
  const int64_t rmax = m < n ? m : n;
  int32_t* P = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
  int32_t* Q = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  int32_t* pr = (int32_t*)malloc((size_t)(rmax > 0 ? rmax : 1) * sizeof(int32_t));
  int32_t* pc = (int32_t*)malloc((size_t)(rmax > 0 ? rmax : 1) * sizeof(int32_t));
  uint32_t* LU = (uint32_t*)malloc((size_t)(m * n > 0 ? m * n : 1) * sizeof(uint32_t));
  if (!P || !Q || !pr || !pc || !LU) { free(P); free(Q); free(pr); free(pc); free(LU); return -2; }
  int64_t r = 0;
  int pm = (mutate == MUT_RREF_NO_NORMALISE) ? 0 : mutate;
  int st = oracle_pluq(p32, m, n, A, lda, &r, P, Q, LU, n, pr, pc, NULL, NULL, nthreads, pm);
  if (st != 0) { free(P); free(Q); free(pr); free(pc); free(LU); return st; }
  /* Pivot row k in the original column order: U[k, u] sits at column Q[u]. */
  int64_t* rows = (int64_t*)calloc((size_t)(r * n > 0 ? r * n : 1), sizeof(int64_t));
  int64_t* order = (int64_t*)malloc((size_t)(r > 0 ? r : 1) * sizeof(int64_t));
  if (!rows || !order) { free(P); free(Q); free(pr); free(pc); free(LU); free(rows); free(order); return -2; }
  for (int64_t k = 0; k < r; ++k)
    for (int64_t u = k; u < n; ++u) rows[k * n + Q[u]] = LU[k * n + u];
  /* order = pivot indices sorted by pivot column (insertion sort on r keys). */
  for (int64_t k = 0; k < r; ++k) order[k] = k;
  for (int64_t a = 1; a < r; ++a) {
    int64_t key = order[a], b = a - 1;
    while (b >= 0 && pc[order[b]] > pc[key]) { order[b + 1] = order[b]; --b; }
    order[b + 1] = key;
  }
  for (int64_t t = 0; t < r; ++t) {
    int64_t* rt = rows + order[t] * n;
    const int64_t jt = pc[order[t]];
    if (mutate != MUT_RREF_NO_NORMALISE) {
      const int64_t inv = inv_mod(rt[jt], p);
      for (int64_t u = 0; u < n; ++u) rt[u] = mod_p(rt[u] * inv, p);
    }
    for (int64_t s = 0; s < t; ++s) {
      int64_t* rs = rows + order[s] * n;
      const int64_t c = rs[jt];
      if (c == 0) continue;
      for (int64_t u = 0; u < n; ++u) rs[u] = mod_p(rs[u] - mod_p(c * rt[u], p), p);
    }
  }
  for (int64_t t = 0; t < r; ++t)
    for (int64_t u = 0; u < n; ++u) R[t * ldr + u] = (uint32_t)rows[order[t] * n + u];
  *rank = r;
  free(P); free(Q); free(pr); free(pc); free(LU); free(rows); free(order);
  return 0;
}

/*
 * oracle_pluq_batch: oracle_pluq over `count` matrices of one shape stored
 * back to back (each m x n, dense), for exhaustive enumeration of tiny
 * matrices.  ranks: count entries; piv_rows / piv_cols: count * min(m,n)
 * entries, -1 past the rank.
 */
int oracle_pluq_batch(uint32_t p, int64_t count, int64_t m, int64_t n, const uint32_t* A,
                      int64_t* ranks, int32_t* piv_rows, int32_t* piv_cols, int mutate) {
  const int64_t rmax = m < n ? m : n;
  int32_t* P = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
  int32_t* Q = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  if (!P || !Q) { free(P); free(Q); return -2; }
  for (int64_t b = 0; b < count; ++b) {
    int32_t* prb = piv_rows + b * rmax;
    int32_t* pcb = piv_cols + b * rmax;
    for (int64_t k = 0; k < rmax; ++k) { prb[k] = -1; pcb[k] = -1; }
    int st = oracle_pluq(p, m, n, A + b * m * n, n, &ranks[b], P, Q, NULL, 0, prb, pcb,
                         NULL, NULL, 1, mutate);
    if (st != 0) { free(P); free(Q); return st; }
  }
  free(P); free(Q);
  return 0;
}
