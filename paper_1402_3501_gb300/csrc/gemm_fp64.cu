// fgemm, FP64 embedding form: C <- C - A B mod p with the residues embedded
// in doubles and the products on FP64 DMMA tensor instructions
// (mma.sync m8n8k4 .f64), accumulated exactly and reduced mod p only when the
// accumulated magnitude could leave the 53-bit mantissa (Sec. 3.1: sums of
// k products of residues in [0, p) stay exact while k (p-1)^2 < 2^53; the
// reduction is delayed to that k).  When even one 16-deep block of products
// of residues would not be exact ((p-1)^2 beyond 2^49), each operand is
// split into 16-bit halves, A = 2^16 Ah + Al, and the four products
// Ah Bh, Ah Bl, Al Bh, Al Bl are accumulated exactly in separate passes,
// each reduced and weighted by 2^32, 2^16, 2^16, 1 mod p.
#include "common.cuh"

namespace {

constexpr int kBMf = 64, kBNf = 64, kBKf = 16;
constexpr int kThreadsF = 128;

__device__ __forceinline__ void dmma_m8n8k4(double (&d)[2], double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d[0]), "+d"(d[1])
               : "d"(a), "d"(b));
}

// x mod p for an exact non-negative integer x < 2^53 held in a double.
__device__ __forceinline__ double dmod(double x, double p, double pinv) {
  double q = floor(x * pinv);
  double r = fma(-q, p, x);
  if (r < 0.0) r += p;
  if (r >= p) r -= p;
  return r;
}

// half_a / half_b: -1 whole residue, 0 low 16 bits, 1 high bits; the reduced
// product is multiplied by `scale` (mod p) before it is subtracted from C.
__device__ __forceinline__ uint32_t pick_half(uint32_t v, int half) {
  return half < 0 ? v : (half == 0 ? (v & 0xFFFFu) : (v >> 16));
}

__global__ void __launch_bounds__(kThreadsF)
    k_fgemm_fp64(int64_t M, int64_t N, int64_t K, const uint32_t* __restrict__ A, int64_t lda,
                 const uint32_t* __restrict__ B, int64_t ldb, uint32_t* __restrict__ C,
                 int64_t ldc, uint32_t p, double pd, double pinv, int ktiles_per_reduce,
                 int half_a, int half_b, uint32_t scale) {
  __shared__ double As[kBMf][kBKf + 1];
  __shared__ double Bs[kBKf][kBNf + 1];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t bm = (int64_t)blockIdx.y * kBMf, bn = (int64_t)blockIdx.x * kBNf;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int g = lane >> 2, q = lane & 3;
  double acc[4][4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;

  int ktile = 0;
  for (int64_t k0 = 0; k0 < K; k0 += kBKf, ++ktile) {
    for (int idx = tid; idx < kBMf * kBKf; idx += kThreadsF) {
      const int i = idx / kBKf, kk = idx % kBKf;
      const int64_t gi = bm + i, gk = k0 + kk;
      As[i][kk] = (gi < M && gk < K) ? (double)pick_half(A[gi * lda + gk], half_a) : 0.0;
    }
    for (int idx = tid; idx < kBKf * kBNf; idx += kThreadsF) {
      const int kk = idx / kBNf, j = idx % kBNf;
      const int64_t gk = k0 + kk, gj = bn + j;
      Bs[kk][j] = (gk < K && gj < N) ? (double)pick_half(B[gk * ldb + gj], half_b) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < kBKf; ks += 4) {
      double a[4], b[4];
#pragma unroll
      for (int mi = 0; mi < 4; ++mi) a[mi] = As[wm + mi * 8 + g][ks + q];
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) b[ni] = Bs[ks + q][wn + ni * 8 + g];
#pragma unroll
      for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) dmma_m8n8k4(acc[mi][ni], a[mi], b[ni]);
    }
    __syncthreads();
    if (ktiles_per_reduce > 0 && (ktile + 1) % ktiles_per_reduce == 0) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j][0] = dmod(acc[i][j][0], pd, pinv);
          acc[i][j][1] = dmod(acc[i][j][1], pd, pinv);
        }
    }
  }
#pragma unroll
  for (int mi = 0; mi < 4; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int64_t row = bm + wm + mi * 8 + g;
        const int64_t col = bn + wn + ni * 8 + q * 2 + e;
        if (row < M && col < N) {
          uint32_t v = (uint32_t)dmod(acc[mi][ni][e], pd, pinv);
          if (scale != 1u) v = (uint32_t)((uint64_t)v * scale % p);
          uint32_t* cp = C + row * ldc + col;
          const uint32_t cv = *cp;
          *cp = cv >= v ? cv - v : cv + p - v;
        }
      }
}

// Number of 16-deep k tiles whose products of operands bounded by `bound` can
// be summed exactly on top of a reduced value: p + kt*16*bound^2 < 2^53.  0
// when not even one tile fits.
int64_t fp64_ktiles_bound(uint32_t p, double bound) {
  const double lim = 9007199254740992.0;  // 2^53
  const double sq = bound * bound;
  if (sq == 0.0) return INT64_MAX;
  const double kt = floor((lim - (double)p) / (sq * kBKf));
  return kt >= 1.0 ? (int64_t)(kt > 1e15 ? 1e15 : kt) : 0;
}

int64_t fp64_ktiles(uint32_t p) { return fp64_ktiles_bound(p, (double)(p - 1)); }

int launch_fp64(pluq_ctx* c, int64_t M, int64_t N, int64_t K, const uint32_t* A, int64_t lda,
                const uint32_t* B, int64_t ldb, uint32_t* C, int64_t ldc, int64_t kt, int ha,
                int hb, uint32_t scale) {
  const int64_t total_kt = cdiv(K, kBKf);
  const int per_reduce = kt >= total_kt ? 0 : (int)kt;
  const dim3 grid((unsigned)cdiv(N, kBNf), (unsigned)cdiv(M, kBMf), 1);
  if (grid.y > 65535) return PLUQ_ERR_INVALID_ARG;
  ProfScope ps(c, PC_FGEMM, 2.0 * M * N * K, 4.0 * (M * K + K * N + 2 * M * N), 1,
               2.0 * cdiv(M, kBMf) * kBMf * cdiv(N, kBNf) * kBNf * cdiv(K, kBKf) * kBKf);
  k_fgemm_fp64<<<grid, kThreadsF, 0, c->stream>>>(M, N, K, A, lda, B, ldb, C, ldc, c->F.p,
                                                  (double)c->F.p, 1.0 / (double)c->F.p,
                                                  per_reduce, ha, hb, scale);
  PLUQ_CUDA(cudaGetLastError());
  return PLUQ_OK;
}

}  // namespace

// Every p < 2^31 has an FP64 form: direct, or with 16-bit halves.
int fp64_form_supported(uint32_t p) {
  return fp64_ktiles(p) > 0 || fp64_ktiles_bound(p, 65535.0) > 0;
}

int fgemm_sub_fp64(pluq_ctx* c, int64_t M, int64_t N, int64_t K, const uint32_t* A, int64_t lda,
                   const uint32_t* B, int64_t ldb, uint32_t* C, int64_t ldc) {
  if (M <= 0 || N <= 0 || K <= 0) return PLUQ_OK;
  const uint32_t p = c->F.p;
  const int64_t kt = fp64_ktiles(p);
  if (kt > 0) return launch_fp64(c, M, N, K, A, lda, B, ldb, C, ldc, kt, -1, -1, 1u);
  const int64_t kth = fp64_ktiles_bound(p, 65535.0);
  if (kth <= 0) return PLUQ_ERR_UNSUPPORTED_FORM;
  const uint32_t w16 = (uint32_t)((1ull << 16) % p), w32 = (uint32_t)((1ull << 32) % p);
  PLUQ_TRY(launch_fp64(c, M, N, K, A, lda, B, ldb, C, ldc, kth, 1, 1, w32));
  PLUQ_TRY(launch_fp64(c, M, N, K, A, lda, B, ldb, C, ldc, kth, 1, 0, w16));
  PLUQ_TRY(launch_fp64(c, M, N, K, A, lda, B, ldb, C, ldc, kth, 0, 1, w16));
  return launch_fp64(c, M, N, K, A, lda, B, ldb, C, ldc, kth, 0, 0, 1u);
}
