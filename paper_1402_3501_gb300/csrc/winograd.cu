// Strassen-Winograd levels above the fgemm (Sec. 2.3, "Parallel matrix
// multiplication", and the Winograd crossover of Sec. 3.2): C <- C - A B mod p
// with seven half-size products instead of eight.
//
// With A = [A11 A12; A21 A22], B = [B11 B12; B21 B22] (h x k and k x w
// quadrants) Winograd's form uses the pre-additions
//   S1 = A21 + A22, S2 = S1 - A11, S3 = A11 - A21, S4 = A12 - S2,
//   T1 = B12 - B11, T2 = B22 - T1, T3 = B22 - B12, T4 = T2 - B21,
// the products P1 = A11 B11, P2 = A12 B21, P3 = S4 B22, P4 = A22 T4,
// P5 = S1 T1, P6 = S2 T2, P7 = S3 T3, and the sums
//   C11 = P1 + P2, C12 = P1 + P6 + P5 + P3, C21 = P1 + P6 + P7 - P4,
//   C22 = P1 + P6 + P7 + P5.
// Here every product is taken by the subtracting fgemm (X <- X - Y Z) into the
// C quadrants or into two h x w temporaries holding negated partial sums:
//   Z1 = -P1;          C11 += Z1, C11 -= A12 B21;
//   Z1 -= S2 T2        (Z1 = -(P1 + P6));
//   Z2 = -P5;          C12 += Z1 + Z2, C12 -= S4 B22;
//   Z1 -= S3 T3        (Z1 = -(P1 + P6 + P7));
//   C22 += Z1 + Z2;    C21 += Z1, C21 -= A22 (-T4).
// Every pre-addition is reduced mod p, so the operands of the seven products
// are residues in [0, p) like the original ones: the exact-accumulation bounds
// of either fgemm form (block depth, digit ranges) are unchanged.  Odd
// dimensions are peeled: the even leading part takes the Winograd level, the
// last row, column or inner index a classical update.
#include "common.cuh"

namespace {

__device__ __forceinline__ uint32_t wadd(uint32_t a, uint32_t b, uint32_t p) {
  const uint32_t s = a + b;  // < 2^32 for a, b < 2^31
  return s >= p ? s - p : s;
}
__device__ __forceinline__ uint32_t wsub(uint32_t a, uint32_t b, uint32_t p) {
  return a >= b ? a - b : a + p - b;
}

// S1..S4 (rows x cols each, stored one after another, leading dimension cols)
// from the quadrants of A (rows x cols each, leading dimension lda).
__global__ void k_wino_pre_a(const uint32_t* __restrict__ A, int64_t lda, int64_t rows,
                             int64_t cols, uint32_t* __restrict__ S, uint32_t p) {
  const int64_t plane = rows * cols;
  for (int64_t i = blockIdx.y; i < rows; i += gridDim.y) {
    const uint32_t* a1 = A + i * lda;
    const uint32_t* a2 = A + (i + rows) * lda;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < cols;
         j += (int64_t)gridDim.x * blockDim.x) {
      const uint32_t a11 = a1[j], a12 = a1[cols + j], a21 = a2[j], a22 = a2[cols + j];
      const uint32_t s1 = wadd(a21, a22, p), s2 = wsub(s1, a11, p);
      const int64_t o = i * cols + j;
      S[o] = s1;
      S[plane + o] = s2;
      S[2 * plane + o] = wsub(a11, a21, p);
      S[3 * plane + o] = wsub(a12, s2, p);
    }
  }
}

// T1, T2, T3 and -T4 = B21 - T2 from the quadrants of B.
__global__ void k_wino_pre_b(const uint32_t* __restrict__ B, int64_t ldb, int64_t rows,
                             int64_t cols, uint32_t* __restrict__ T, uint32_t p) {
  const int64_t plane = rows * cols;
  for (int64_t i = blockIdx.y; i < rows; i += gridDim.y) {
    const uint32_t* b1 = B + i * ldb;
    const uint32_t* b2 = B + (i + rows) * ldb;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < cols;
         j += (int64_t)gridDim.x * blockDim.x) {
      const uint32_t b11 = b1[j], b12 = b1[cols + j], b21 = b2[j], b22 = b2[cols + j];
      const uint32_t t1 = wsub(b12, b11, p), t2 = wsub(b22, t1, p);
      const int64_t o = i * cols + j;
      T[o] = t1;
      T[plane + o] = t2;
      T[2 * plane + o] = wsub(b22, b12, p);
      T[3 * plane + o] = wsub(b21, t2, p);
    }
  }
}

// C0 += X (+ Y when Y is given); with C1 non-null also C1 += X (the fused
// C22 += Z1 + Z2, C21 += Z1 step).  X, Y dense rows x cols.
__global__ void k_wino_acc(uint32_t* __restrict__ C0, uint32_t* __restrict__ C1, int64_t ldc,
                           const uint32_t* __restrict__ X, const uint32_t* __restrict__ Y,
                           int64_t rows, int64_t cols, uint32_t p) {
  for (int64_t i = blockIdx.y; i < rows; i += gridDim.y) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < cols;
         j += (int64_t)gridDim.x * blockDim.x) {
      const uint32_t x = X[i * cols + j];
      const uint32_t xy = Y ? wadd(x, Y[i * cols + j], p) : x;
      C0[i * ldc + j] = wadd(C0[i * ldc + j], xy, p);
      if (C1) C1[i * ldc + j] = wadd(C1[i * ldc + j], x, p);
    }
  }
}

dim3 wgrid(int64_t rows, int64_t cols) {
  int64_t gx = cdiv(cols, 256);
  if (gx > 32) gx = 32;
  int64_t gy = rows < 65535 ? rows : 65535;
  return dim3((unsigned)(gx < 1 ? 1 : gx), (unsigned)(gy < 1 ? 1 : gy), 1);
}

constexpr int kMaxWinoDepth = 4;

// uint32 words of one level's temporaries for an even M x N x K product
int64_t level_words(int64_t M, int64_t N, int64_t K) {
  const int64_t h = M / 2, w = N / 2, k = K / 2;
  return 4 * h * k + 4 * k * w + 2 * h * w;
}

int wino_level(pluq_ctx* c, int64_t M, int64_t N, int64_t K, const uint32_t* A, int64_t lda,
               const uint32_t* B, int64_t ldb, uint32_t* C, int64_t ldc, int depth) {
  const int64_t h = M / 2, w = N / 2, k = K / 2;
  const uint32_t p = c->F.p;
  // workspace of this level: S (4 h k), T (4 k w), Z1, Z2 (h w); deeper levels
  // take the space after it (sized by the top level, never regrown below it)
  const int64_t need = level_words(M, N, K);
  const int64_t base = c->wino_used;
  if (depth == 0) {
    int64_t total = 0;
    for (int64_t m = M, n = N, kk = K, d = 0; d < kMaxWinoDepth && wino_applies(c, m, n, kk);
         m /= 2, n /= 2, kk /= 2, ++d)
      total += level_words(m & ~1LL, n & ~1LL, kk & ~1LL);
    PLUQ_TRY(c->wino.ensure(sizeof(uint32_t) * (size_t)total));
  }
  if ((size_t)(base + need) * sizeof(uint32_t) > c->wino.bytes) return PLUQ_ERR_NO_WORKSPACE;
  uint32_t* S = c->wino.as<uint32_t>() + base;
  uint32_t* T = S + 4 * h * k;
  uint32_t* Z1 = T + 4 * k * w;
  uint32_t* Z2 = Z1 + h * w;
  c->wino_used = base + need;
  const uint32_t* A11 = A;
  const uint32_t* A12 = A + k;
  const uint32_t* A22 = A + h * lda + k;
  const uint32_t* B11 = B;
  const uint32_t* B21 = B + k * ldb;
  const uint32_t* B22 = B + k * ldb + w;
  uint32_t* C11 = C;
  uint32_t* C12 = C + w;
  uint32_t* C21 = C + h * ldc;
  uint32_t* C22 = C + h * ldc + w;
  const uint32_t* S1 = S;
  const uint32_t* S2 = S + h * k;
  const uint32_t* S3 = S + 2 * h * k;
  const uint32_t* S4 = S + 3 * h * k;
  const uint32_t* T1 = T;
  const uint32_t* T2 = T + k * w;
  const uint32_t* T3 = T + 2 * k * w;
  const uint32_t* T4n = T + 3 * k * w;
  {
    ProfScope ps(c, PC_OTHER, 0, 32.0 * (h * k + k * w), 2);
    k_wino_pre_a<<<wgrid(h, k), 256, 0, c->stream>>>(A, lda, h, k, S, p);
    k_wino_pre_b<<<wgrid(k, w), 256, 0, c->stream>>>(B, ldb, k, w, T, p);
    PLUQ_CUDA(cudaGetLastError());
  }
  PLUQ_CUDA(cudaMemsetAsync(Z1, 0, sizeof(uint32_t) * 2 * h * w, c->stream));
  auto prod = [&](int64_t ldx, const uint32_t* X, int64_t ldy, const uint32_t* Y, uint32_t* Z,
                  int64_t ldz) {
    return fgemm_sub_wino(c, h, w, k, X, ldx, Y, ldy, Z, ldz, depth + 1);
  };
  auto acc = [&](uint32_t* C0, uint32_t* C1, const uint32_t* X, const uint32_t* Y) -> int {
    ProfScope ps(c, PC_OTHER, 0, (Y ? 16.0 : 12.0) * h * w + (C1 ? 8.0 * h * w : 0.0));
    k_wino_acc<<<wgrid(h, w), 256, 0, c->stream>>>(C0, C1, ldc, X, Y, h, w, p);
    PLUQ_CUDA(cudaGetLastError());
    return PLUQ_OK;
  };
  PLUQ_TRY(prod(lda, A11, ldb, B11, Z1, w));    // Z1 = -P1
  PLUQ_TRY(acc(C11, nullptr, Z1, nullptr));    // C11 -= P1
  PLUQ_TRY(prod(lda, A12, ldb, B21, C11, ldc));  // C11 -= P2
  PLUQ_TRY(prod(k, S2, w, T2, Z1, w));          // Z1 = -(P1 + P6)
  PLUQ_TRY(prod(k, S1, w, T1, Z2, w));          // Z2 = -P5
  PLUQ_TRY(acc(C12, nullptr, Z1, Z2));          // C12 -= P1 + P6 + P5
  PLUQ_TRY(prod(k, S4, ldb, B22, C12, ldc));    // C12 -= P3
  PLUQ_TRY(prod(k, S3, w, T3, Z1, w));          // Z1 = -(P1 + P6 + P7)
  PLUQ_TRY(acc(C22, C21, Z1, Z2));              // C22 -= .. + P5, C21 -= P1 + P6 + P7
  PLUQ_TRY(prod(lda, A22, w, T4n, C21, ldc));   // C21 += P4
  c->wino_used = base;
  return PLUQ_OK;
}

}  // namespace

int wino_applies(const pluq_ctx* c, int64_t M, int64_t N, int64_t K) {
  return c->wino_min > 0 && M >= c->wino_min && N >= c->wino_min && K >= c->wino_min;
}

int fgemm_sub_wino(pluq_ctx* c, int64_t M, int64_t N, int64_t K, const uint32_t* A, int64_t lda,
                   const uint32_t* B, int64_t ldb, uint32_t* C, int64_t ldc, int depth) {
  if (M <= 0 || N <= 0 || K <= 0) return PLUQ_OK;
  if (!wino_applies(c, M, N, K) || depth >= kMaxWinoDepth)
    return fgemm_sub_classical(c, M, N, K, A, lda, B, ldb, C, ldc);
  const int64_t Me = M & ~1LL, Ne = N & ~1LL, Ke = K & ~1LL;
  if (depth == 0) c->wino_used = 0;
  PLUQ_TRY(wino_level(c, Me, Ne, Ke, A, lda, B, ldb, C, ldc, depth));
  // peeled remainders: the last inner index, then the last row and column
  if (Ke < K)
    PLUQ_TRY(fgemm_sub_classical(c, Me, Ne, 1, A + Ke, lda, B + Ke * ldb, ldb, C, ldc));
  if (Me < M)
    PLUQ_TRY(fgemm_sub_classical(c, 1, N, K, A + Me * lda, lda, B, ldb, C + Me * ldc, ldc));
  if (Ne < N)
    PLUQ_TRY(fgemm_sub_classical(c, Me, 1, K, A, lda, B + Ne, ldb, C + Ne, ldc));
  return PLUQ_OK;
}
