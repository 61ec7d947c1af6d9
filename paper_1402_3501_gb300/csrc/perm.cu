// Permutation kernels of the recursion (the flaswp of Sec. 2.1 / Sec. 2.3):
// row and column gathers of rectangular blocks, composition of index vectors
// and the block-cyclic shifts that gather the pivots of the four recursive
// calls at the front of a block.
//
// A block permutation is applied out of place into the context scratch (one
// coalesced read and write per element) and copied back, because the
// permutations of the recursion are arbitrary (pivots interleaved with the
// rest) and in-place cycle following does not vectorise.
#include <algorithm>

#include "common.cuh"

namespace {

__global__ void k_iota(int32_t* __restrict__ dst, int64_t count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) dst[i] = (int32_t)i;
}

// base[t] = base[perm[t]], t < count, through shared memory (count small).
__global__ void k_compose_smem(int32_t* __restrict__ base, const int32_t* __restrict__ perm,
                               int count) {
  extern __shared__ int32_t s[];
  for (int t = threadIdx.x; t < count; t += blockDim.x) s[t] = base[perm[t]];
  __syncthreads();
  for (int t = threadIdx.x; t < count; t += blockDim.x) base[t] = s[t];
}

// The row and the column index vectors of a node in one launch: block 0
// composes (base_r, perm_r), block 1 (base_c, perm_c); each <= 12288 entries.
__global__ void k_compose_pair(int32_t* __restrict__ base_r, const int32_t* __restrict__ perm_r,
                               int count_r, int32_t* __restrict__ base_c,
                               const int32_t* __restrict__ perm_c, int count_c) {
  extern __shared__ int32_t s[];
  int32_t* base = blockIdx.x == 0 ? base_r : base_c;
  const int32_t* perm = blockIdx.x == 0 ? perm_r : perm_c;
  const int count = blockIdx.x == 0 ? count_r : count_c;
  for (int t = threadIdx.x; t < count; t += blockDim.x) s[t] = base[perm[t]];
  __syncthreads();
  for (int t = threadIdx.x; t < count; t += blockDim.x) base[t] = s[t];
}

// dst_r[i] = i (i < count_r) and dst_c[j] = j (j < count_c) in one launch
__global__ void k_iota_pair(int32_t* __restrict__ dst_r, int64_t count_r,
                            int32_t* __restrict__ dst_c, int64_t count_c) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count_r) dst_r[i] = (int32_t)i;
  if (i < count_c) dst_c[i] = (int32_t)i;
}

__global__ void k_compose_gather(int32_t* __restrict__ out, const int32_t* __restrict__ base,
                                 const int32_t* __restrict__ perm, int64_t count) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < count) out[t] = base[perm[t]];
}

__global__ void k_copy_i32(int32_t* __restrict__ dst, const int32_t* __restrict__ src,
                           int64_t count) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < count) dst[t] = src[t];
}

struct Segs {
  int64_t start[4];
  int64_t len[4];
  int n;
};

__global__ void k_segperm(int32_t* __restrict__ out, Segs sg, int64_t total) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  int64_t acc = 0;
  for (int k = 0; k < sg.n; ++k) {
    if (t < acc + sg.len[k]) {
      out[t] = (int32_t)(sg.start[k] + (t - acc));
      return;
    }
    acc += sg.len[k];
  }
}

// Two segments of one index range: index i < len0 maps to off0 + i, index
// i >= len0 to off1 + (i - len0).  A permutation applied to two disjoint
// column (or row) ranges of the same rows (columns) takes one pass.
struct Seg2 {
  int64_t len0, off0, off1;
  __device__ __forceinline__ int64_t at(int64_t i) const {
    return i < len0 ? off0 + i : off1 + (i - len0);
  }
};

// S[t, u] = A[perm[t], cs.at(u)]: rows permuted, over two column segments
__global__ void k_gather_rows(uint32_t* __restrict__ S, const uint32_t* __restrict__ A, int64_t lda,
                              int64_t rows, int64_t cols, Seg2 cs,
                              const int32_t* __restrict__ perm) {
  for (int64_t t = blockIdx.y; t < rows; t += gridDim.y) {
    const uint32_t* s = A + (int64_t)perm[t] * lda;
    uint32_t* d = S + t * cols;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < cols;
         u += (int64_t)gridDim.x * blockDim.x)
      d[u] = s[cs.at(u)];
  }
}

// S[t, u] = A[rs.at(t), perm[u]]: columns permuted, over two row segments
__global__ void k_gather_cols(uint32_t* __restrict__ S, const uint32_t* __restrict__ A, int64_t lda,
                              int64_t rows, int64_t cols, Seg2 rs,
                              const int32_t* __restrict__ perm) {
  for (int64_t t = blockIdx.y; t < rows; t += gridDim.y) {
    const uint32_t* s = A + rs.at(t) * lda;
    uint32_t* d = S + t * cols;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < cols;
         u += (int64_t)gridDim.x * blockDim.x)
      d[u] = s[perm[u]];
  }
}

// A[rs.at(t), cs.at(u)] = S[t, u]
__global__ void k_scatter_back(uint32_t* __restrict__ A, int64_t lda, const uint32_t* __restrict__ S,
                               int64_t rows, int64_t cols, Seg2 rs, Seg2 cs) {
  for (int64_t t = blockIdx.y; t < rows; t += gridDim.y) {
    const uint32_t* s = S + t * cols;
    uint32_t* d = A + rs.at(t) * lda;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < cols;
         u += (int64_t)gridDim.x * blockDim.x)
      d[cs.at(u)] = s[u];
  }
}

dim3 grid2d(int64_t rows, int64_t cols, int threads) {
  int64_t gx = cdiv(cols, threads);
  if (gx > 64) gx = 64;
  int64_t gy = rows;
  if (gy > 65535) gy = 65535;
  return dim3((unsigned)gx, (unsigned)gy, 1);
}

}  // namespace

int launch_iota(pluq_ctx* c, int32_t* dst, int64_t count) {
  if (count <= 0) return PLUQ_OK;
  ProfScope ps(c, PC_INDEX, 0, 4.0 * count);
  k_iota<<<(unsigned)cdiv(count, 256), 256, 0, c->stream>>>(dst, count);
  PLUQ_CUDA(cudaGetLastError());
  return PLUQ_OK;
}

int launch_compose(pluq_ctx* c, int32_t* base, const int32_t* perm, int64_t count) {
  if (count <= 1) return PLUQ_OK;
  ProfScope ps(c, PC_INDEX, 0, 12.0 * count, count <= 12288 ? 1 : 2);
  if (count <= 12288) {
    k_compose_smem<<<1, 1024, sizeof(int32_t) * count, c->stream>>>(base, perm, (int)count);
  } else {
    PLUQ_TRY(c->tmp_i.ensure(sizeof(int32_t) * count));
    int32_t* tmp = c->tmp_i.as<int32_t>();
    k_compose_gather<<<(unsigned)cdiv(count, 256), 256, 0, c->stream>>>(tmp, base, perm, count);
    k_copy_i32<<<(unsigned)cdiv(count, 256), 256, 0, c->stream>>>(base, tmp, count);
  }
  PLUQ_CUDA(cudaGetLastError());
  return PLUQ_OK;
}

int launch_compose_pair(pluq_ctx* c, int32_t* base_r, const int32_t* perm_r, int64_t count_r,
                        int32_t* base_c, const int32_t* perm_c, int64_t count_c) {
  if (count_r > 12288 || count_c > 12288 || count_r <= 1 || count_c <= 1) {
    PLUQ_TRY(launch_compose(c, base_r, perm_r, count_r));
    return launch_compose(c, base_c, perm_c, count_c);
  }
  ProfScope ps(c, PC_INDEX, 0, 12.0 * (count_r + count_c));
  const size_t smem = sizeof(int32_t) * (size_t)std::max(count_r, count_c);
  k_compose_pair<<<2, 1024, smem, c->stream>>>(base_r, perm_r, (int)count_r, base_c, perm_c,
                                               (int)count_c);
  PLUQ_CUDA(cudaGetLastError());
  return PLUQ_OK;
}

int launch_iota_pair(pluq_ctx* c, int32_t* dst_r, int64_t count_r, int32_t* dst_c,
                     int64_t count_c) {
  const int64_t count = std::max(count_r, count_c);
  if (count <= 0) return PLUQ_OK;
  ProfScope ps(c, PC_INDEX, 0, 4.0 * (count_r + count_c));
  k_iota_pair<<<(unsigned)cdiv(count, 256), 256, 0, c->stream>>>(dst_r, count_r, dst_c, count_c);
  PLUQ_CUDA(cudaGetLastError());
  return PLUQ_OK;
}

int launch_segperm(pluq_ctx* c, int32_t* out, const int64_t* seg_start, const int64_t* seg_len,
                   int nseg) {
  Segs sg{};
  int64_t total = 0;
  sg.n = nseg;
  for (int k = 0; k < nseg; ++k) {
    sg.start[k] = seg_start[k];
    sg.len[k] = seg_len[k];
    total += seg_len[k];
  }
  if (total <= 0) return PLUQ_OK;
  ProfScope ps(c, PC_INDEX, 0, 4.0 * total);
  k_segperm<<<(unsigned)cdiv(total, 256), 256, 0, c->stream>>>(out, sg, total);
  PLUQ_CUDA(cudaGetLastError());
  return PLUQ_OK;
}

int permute_rows2(pluq_ctx* c, uint32_t* A, int64_t lda, int64_t rows, int64_t c0, int64_t n0,
                  int64_t c1, int64_t n1, const int32_t* perm) {
  const int64_t cols = n0 + n1;
  if (rows <= 1 || cols <= 0) return PLUQ_OK;
  PLUQ_TRY(c->scratch.ensure(sizeof(uint32_t) * rows * cols));
  uint32_t* S = c->scratch.as<uint32_t>();
  const Seg2 cs{n0, c0, c1}, rs{rows, 0, 0};
  const dim3 g = grid2d(rows, cols, 256);
  ProfScope ps(c, PC_PERM, 0, 8.0 * rows * cols, 2);
  k_gather_rows<<<g, 256, 0, c->stream>>>(S, A, lda, rows, cols, cs, perm);
  k_scatter_back<<<g, 256, 0, c->stream>>>(A, lda, S, rows, cols, rs, cs);
  PLUQ_CUDA(cudaGetLastError());
  return PLUQ_OK;
}

int permute_cols2(pluq_ctx* c, uint32_t* A, int64_t lda, int64_t r0, int64_t m0, int64_t r1,
                  int64_t m1, int64_t cols, const int32_t* perm) {
  const int64_t rows = m0 + m1;
  if (rows <= 0 || cols <= 1) return PLUQ_OK;
  PLUQ_TRY(c->scratch.ensure(sizeof(uint32_t) * rows * cols));
  uint32_t* S = c->scratch.as<uint32_t>();
  const Seg2 rs{m0, r0, r1}, cs{cols, 0, 0};
  const dim3 g = grid2d(rows, cols, 256);
  ProfScope ps(c, PC_PERM, 0, 8.0 * rows * cols, 2);
  k_gather_cols<<<g, 256, 0, c->stream>>>(S, A, lda, rows, cols, rs, perm);
  k_scatter_back<<<g, 256, 0, c->stream>>>(A, lda, S, rows, cols, rs, cs);
  PLUQ_CUDA(cudaGetLastError());
  return PLUQ_OK;
}

int permute_rows(pluq_ctx* c, uint32_t* A, int64_t lda, int64_t rows, int64_t cols,
                 const int32_t* perm) {
  return permute_rows2(c, A, lda, rows, 0, cols, 0, 0, perm);
}

int permute_cols(pluq_ctx* c, uint32_t* A, int64_t lda, int64_t rows, int64_t cols,
                 const int32_t* perm) {
  return permute_cols2(c, A, lda, 0, rows, 0, 0, cols, perm);
}
