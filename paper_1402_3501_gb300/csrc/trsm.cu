// Triangular solves mod p (the ftrsm of Sec. 2.1): block recursive, the
// off-diagonal work reduced to fgemm calls and the diagonal blocks (at most
// kTB x kTB) solved by one CTA in shared memory.
//
//   trsm_left_lower_unit : B <- L^{-1} B   (L unit lower, r x r)   D, O
//   trsm_right_upper     : B <- B U^{-1}   (U upper, r x r)        E, [I; K]
//   trsm_left_upper      : B <- U^{-1} B   (U upper, r x r)        RREF
//
// Non-unit triangles are first made unit by scaling with the inverses of
// their diagonal (U = D U' with U' unit upper), so the substitution loop
// needs no division: X U = B  <=>  (X D) U' = B, and U X = B  <=>
// U'' X = D^{-1} B with U'' = D^{-1} U.
#include "common.cuh"

namespace {

constexpr int kTB = 64;       // diagonal block
constexpr int kStrip = 64;    // columns (or rows) of B per CTA
constexpr int kTrsmThreads = 256;

// B (r x ncols) <- L^{-1} B, L unit lower r x r, r <= kTB; one CTA per strip
// of kStrip columns.
__global__ void __launch_bounds__(kTrsmThreads)
    k_trsm_llu_small(const uint32_t* __restrict__ L, int64_t ldl, int r, uint32_t* __restrict__ B,
                     int64_t ldb, int64_t ncols, FieldP F) {
  __shared__ uint32_t Lm[kTB][kTB + 1];
  __shared__ uint32_t X[kTB][kStrip];
  const int tid = threadIdx.x, tx = tid % kStrip, ty = tid / kStrip;
  const int64_t c0 = (int64_t)blockIdx.x * kStrip;
  for (int idx = tid; idx < r * r; idx += kTrsmThreads) {
    const int i = idx / r, k = idx % r;
    Lm[i][k] = (k < i) ? f_to_mont(L[(int64_t)i * ldl + k], F) : 0u;
  }
  const bool colok = c0 + tx < ncols;
  for (int i = ty; i < r; i += kTrsmThreads / kStrip)
    X[i][tx] = colok ? B[(int64_t)i * ldb + c0 + tx] : 0u;
  __syncthreads();
  for (int k = 0; k + 1 < r; ++k) {
    const uint32_t xk = X[k][tx];
    for (int i = ty; i < r; i += kTrsmThreads / kStrip)
      if (i > k) X[i][tx] = f_sub(X[i][tx], f_mul_mont(Lm[i][k], xk, F), F);
    __syncthreads();
  }
  if (colok)
    for (int i = ty; i < r; i += kTrsmThreads / kStrip) B[(int64_t)i * ldb + c0 + tx] = X[i][tx];
}

// B (nrows x r) <- B U^{-1}, U upper r x r, r <= kTB; one CTA per strip of
// kStrip rows.  Threads own columns (tx) of B.
__global__ void __launch_bounds__(kTrsmThreads)
    k_trsm_ru_small(const uint32_t* __restrict__ U, int64_t ldu, int r, uint32_t* __restrict__ B,
                    int64_t ldb, int64_t nrows, FieldP F, const uint32_t* __restrict__ inv_table) {
  __shared__ uint32_t Um[kTB][kTB + 1];  // U' = D^{-1} U (unit upper), Montgomery form
  __shared__ uint32_t dinv[kTB];
  __shared__ uint32_t Y[kStrip][kTB + 1];
  const int tid = threadIdx.x, tx = tid % kTB, ty = tid / kTB;
  const int64_t r0 = (int64_t)blockIdx.x * kStrip;
  if (tid < r) dinv[tid] = f_inv(U[(int64_t)tid * ldu + tid], F, inv_table);
  for (int idx = tid; idx < kStrip * r; idx += kTrsmThreads) {
    const int i = idx / r, j = idx % r;
    Y[i][j] = (r0 + i < nrows) ? B[(r0 + i) * ldb + j] : 0u;
  }
  __syncthreads();
  for (int idx = tid; idx < r * r; idx += kTrsmThreads) {
    const int j = idx / r, k = idx % r;
    Um[j][k] = (k > j) ? f_to_mont(f_mul(U[(int64_t)j * ldu + k], dinv[j], F), F) : 0u;
  }
  __syncthreads();
  // Y <- Y U'^{-1}: column k of Y loses Y[:, j] U'[j, k] for every j < k
  for (int j = 0; j + 1 < r; ++j) {
    if (tx > j && tx < r) {
      const uint32_t u = Um[j][tx];
      for (int i = ty; i < kStrip; i += kTrsmThreads / kTB)
        Y[i][tx] = f_sub(Y[i][tx], f_mul_mont(u, Y[i][j], F), F);
    }
    __syncthreads();
  }
  // X = Y D^{-1}
  for (int idx = tid; idx < kStrip * r; idx += kTrsmThreads) {
    const int i = idx / r, j = idx % r;
    if (r0 + i < nrows) B[(r0 + i) * ldb + j] = f_mul(Y[i][j], dinv[j], F);
  }
}

// B (r x ncols) <- U^{-1} B, U upper r x r, r <= kTB.
__global__ void __launch_bounds__(kTrsmThreads)
    k_trsm_lu_small(const uint32_t* __restrict__ U, int64_t ldu, int r, uint32_t* __restrict__ B,
                    int64_t ldb, int64_t ncols, FieldP F, const uint32_t* __restrict__ inv_table) {
  __shared__ uint32_t Um[kTB][kTB + 1];  // U'' = D^{-1} U, Montgomery form
  __shared__ uint32_t dinv[kTB];
  __shared__ uint32_t X[kTB][kStrip];
  const int tid = threadIdx.x, tx = tid % kStrip, ty = tid / kStrip;
  const int64_t c0 = (int64_t)blockIdx.x * kStrip;
  if (tid < r) dinv[tid] = f_inv(U[(int64_t)tid * ldu + tid], F, inv_table);
  __syncthreads();
  for (int idx = tid; idx < r * r; idx += kTrsmThreads) {
    const int l = idx / r, k = idx % r;
    Um[l][k] = (k > l) ? f_to_mont(f_mul(U[(int64_t)l * ldu + k], dinv[l], F), F) : 0u;
  }
  const bool colok = c0 + tx < ncols;
  for (int i = ty; i < r; i += kTrsmThreads / kStrip)
    X[i][tx] = colok ? f_mul(B[(int64_t)i * ldb + c0 + tx], dinv[i], F) : 0u;
  __syncthreads();
  for (int k = r - 1; k > 0; --k) {
    const uint32_t xk = X[k][tx];
    for (int l = ty; l < k; l += kTrsmThreads / kStrip)
      X[l][tx] = f_sub(X[l][tx], f_mul_mont(Um[l][k], xk, F), F);
    __syncthreads();
  }
  if (colok)
    for (int i = ty; i < r; i += kTrsmThreads / kStrip) B[(int64_t)i * ldb + c0 + tx] = X[i][tx];
}

int64_t split_point(int64_t r, int64_t tb) {
  int64_t h = (r / 2 + tb - 1) / tb * tb;
  if (h <= 0 || h >= r) h = tb;
  return h;
}

}  // namespace

int trsm_left_lower_unit(pluq_ctx* c, const uint32_t* L, int64_t ldl, int64_t r, uint32_t* B,
                         int64_t ldb, int64_t ncols) {
  if (r <= 1 || ncols <= 0) return PLUQ_OK;  // a unit 1x1 triangle is the identity
  const int64_t tb = c->trsm_block < kTB ? c->trsm_block : kTB;
  if (r <= tb) {
    ProfScope ps(c, PC_TRSM, (double)r * r * ncols, 8.0 * r * ncols);
    k_trsm_llu_small<<<(unsigned)cdiv(ncols, kStrip), kTrsmThreads, 0, c->stream>>>(
        L, ldl, (int)r, B, ldb, ncols, c->F);
    PLUQ_CUDA(cudaGetLastError());
    return PLUQ_OK;
  }
  const int64_t r1 = split_point(r, tb);
  PLUQ_TRY(trsm_left_lower_unit(c, L, ldl, r1, B, ldb, ncols));
  PLUQ_TRY(fgemm_sub(c, r - r1, ncols, r1, L + r1 * ldl, ldl, B, ldb, B + r1 * ldb, ldb));
  return trsm_left_lower_unit(c, L + r1 * ldl + r1, ldl, r - r1, B + r1 * ldb, ldb, ncols);
}

int trsm_right_upper(pluq_ctx* c, const uint32_t* U, int64_t ldu, int64_t r, uint32_t* B,
                     int64_t ldb, int64_t nrows) {
  if (r <= 0 || nrows <= 0) return PLUQ_OK;
  const int64_t tb = c->trsm_block < kTB ? c->trsm_block : kTB;
  if (r <= tb) {
    ProfScope ps(c, PC_TRSM, (double)r * r * nrows, 8.0 * r * nrows);
    k_trsm_ru_small<<<(unsigned)cdiv(nrows, kStrip), kTrsmThreads, 0, c->stream>>>(
        U, ldu, (int)r, B, ldb, nrows, c->F, inv_table_ptr(c));
    PLUQ_CUDA(cudaGetLastError());
    return PLUQ_OK;
  }
  const int64_t r1 = split_point(r, tb);
  PLUQ_TRY(trsm_right_upper(c, U, ldu, r1, B, ldb, nrows));
  PLUQ_TRY(fgemm_sub(c, nrows, r - r1, r1, B, ldb, U + r1, ldu, B + r1, ldb));
  return trsm_right_upper(c, U + r1 * ldu + r1, ldu, r - r1, B + r1, ldb, nrows);
}

int trsm_left_upper(pluq_ctx* c, const uint32_t* U, int64_t ldu, int64_t r, uint32_t* B,
                    int64_t ldb, int64_t ncols) {
  if (r <= 0 || ncols <= 0) return PLUQ_OK;
  const int64_t tb = c->trsm_block < kTB ? c->trsm_block : kTB;
  if (r <= tb) {
    ProfScope ps(c, PC_TRSM, (double)r * r * ncols, 8.0 * r * ncols);
    k_trsm_lu_small<<<(unsigned)cdiv(ncols, kStrip), kTrsmThreads, 0, c->stream>>>(
        U, ldu, (int)r, B, ldb, ncols, c->F, inv_table_ptr(c));
    PLUQ_CUDA(cudaGetLastError());
    return PLUQ_OK;
  }
  const int64_t r1 = split_point(r, tb);
  // U = [U11 U12; 0 U22]: X2 = U22^{-1} B2, B1 -= U12 X2, X1 = U11^{-1} B1
  PLUQ_TRY(trsm_left_upper(c, U + r1 * ldu + r1, ldu, r - r1, B + r1 * ldb, ldb, ncols));
  PLUQ_TRY(fgemm_sub(c, r1, ncols, r - r1, U + r1, ldu, B + r1 * ldb, ldb, B, ldb));
  return trsm_left_upper(c, U, ldu, r1, B, ldb, ncols);
}
