// fgemm for a thin inner dimension: C <- C - A B mod p with K <= kThinMaxK on
// the CUDA cores.  The tile recursion produces many such products (updates by
// a rank-deficient leaf's few pivots, the innermost steps of the triangular
// solves); on the tensor-core limb form each would pay a digit-packing pass
// and a pipeline fill for one or two K blocks.
//
// Delayed reduction (Sec. 3.1) in 64-bit integers: the K products of plain
// residues are summed exactly (K (p-1)^2 < p 2^32 when K p < 2^31) and reduced
// once per output by two Montgomery steps: REDC(REDC(sum) * R^2 mod p) = sum
// mod p.  p = 2: the parity of the sum.
//
// One CTA per 64 x 64 block of C, 256 threads, each accumulating a 4 x 4
// micro-tile; A and B staged through shared memory 32 columns of K at a time.
#include "common.cuh"

namespace {

constexpr int kThinTile = 64;
constexpr int kThinK = 32;
constexpr int kThinThreads = 256;

__global__ void __launch_bounds__(kThinThreads)
    k_fgemm_thin(int64_t M, int64_t N, int64_t K, const uint32_t* __restrict__ A, int64_t lda,
                 const uint32_t* __restrict__ B, int64_t ldb, uint32_t* __restrict__ C,
                 int64_t ldc, FieldP F) {
  __shared__ uint32_t As[kThinK][kThinTile + 1];  // As[k][row]
  __shared__ uint32_t Bs[kThinK][kThinTile];      // Bs[k][col]
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int64_t r0 = (int64_t)blockIdx.y * kThinTile, c0 = (int64_t)blockIdx.x * kThinTile;
  uint64_t acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0;
  for (int64_t k0 = 0; k0 < K; k0 += kThinK) {
    // A block (64 rows x 32 k): thread loads 8 elements, k fastest within a row
#pragma unroll
    for (int q = 0; q < (kThinTile * kThinK) / kThinThreads; ++q) {
      const int idx = tid + q * kThinThreads, rr = idx / kThinK, kk = idx % kThinK;
      const int64_t gr = r0 + rr, gk = k0 + kk;
      As[kk][rr] = (gr < M && gk < K) ? A[gr * lda + gk] : 0u;
    }
    // B block (32 k x 64 cols)
#pragma unroll
    for (int q = 0; q < (kThinTile * kThinK) / kThinThreads; ++q) {
      const int idx = tid + q * kThinThreads, kk = idx / kThinTile, cc = idx % kThinTile;
      const int64_t gk = k0 + kk, gc = c0 + cc;
      Bs[kk][cc] = (gk < K && gc < N) ? B[gk * ldb + gc] : 0u;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < kThinK; ++kk) {
      uint32_t a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += (uint64_t)a[i] * b[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gr = r0 + ty + 16 * i;
    if (gr >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gc = c0 + tx + 16 * j;
      if (gc >= N) continue;
      const uint32_t v = F.is2 ? (uint32_t)(acc[i][j] & 1u)
                               : f_redc((uint64_t)f_redc(acc[i][j], F) * F.r2, F);
      uint32_t* cp = C + gr * ldc + gc;
      *cp = f_sub(*cp, v, F);
    }
  }
}

}  // namespace

// Worth it while the CUDA-core work stays below the tensor path's fixed cost
// (a packing pass and a pipeline fill, about 20 us): about 2^27 multiply-adds.
int thin_fgemm_ok(const pluq_ctx* c, int64_t M, int64_t N, int64_t K) {
  return K > 0 && K <= kThinMaxK && (uint64_t)K * c->F.p < (1ull << 31) &&
         (double)M * N * K <= 134217728.0;
}

int fgemm_sub_thin(pluq_ctx* c, int64_t M, int64_t N, int64_t K, const uint32_t* A, int64_t lda,
                   const uint32_t* B, int64_t ldb, uint32_t* C, int64_t ldc) {
  if (M <= 0 || N <= 0 || K <= 0) return PLUQ_OK;
  if (cdiv(M, kThinTile) > 65535) return PLUQ_ERR_INVALID_ARG;
  ProfScope ps(c, PC_THIN, 2.0 * M * N * K, 4.0 * (M * K + K * N + 2 * M * N), 1, 0.0);
  const dim3 grid((unsigned)cdiv(N, kThinTile), (unsigned)cdiv(M, kThinTile));
  k_fgemm_thin<<<grid, kThinThreads, 0, c->stream>>>(M, N, K, A, lda, B, ldb, C, ldc, c->F);
  PLUQ_CUDA(cudaGetLastError());
  return PLUQ_OK;
}
