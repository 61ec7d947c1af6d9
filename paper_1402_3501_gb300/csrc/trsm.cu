// Triangular solves mod p (the ftrsm of Sec. 2.1): block recursive, the
// off-diagonal work reduced to fgemm calls.  The kTB x kTB diagonal blocks
// are first inverted together (one launch, one CTA per block); each diagonal
// solve is then a small dense product with its inverse, parallel over all the
// right-hand sides and their rows (no sequential substitution chain).
//
//   trsm_left_lower_unit : B <- L^{-1} B   (L unit lower, r x r)   D, O
//   trsm_right_upper     : B <- B U^{-1}   (U upper, r x r)        E, [I; K]
//   trsm_left_upper      : B <- U^{-1} B   (U upper, r x r)        RREF

#include "common.cuh"

namespace {

constexpr int kTB = 64;  // diagonal block

// ------------------------------------------------- diagonal-block inverses --
//
// One CTA inverts one diagonal block T of the triangle (rows and columns
// [b tb, b tb + s), s <= tb <= kTB); the block is padded to kTB x kTB with
// the identity.  An
// upper block is inverted as the lower block T^T and stored transposed back
// ((T^T)^{-1} = (T^{-1})^T).  Recursive doubling: with the inverses of the
// two h x h diagonal blocks A, B of a 2h x 2h lower block [A 0; C B] known,
// its inverse is [A^{-1} 0; -B^{-1} C A^{-1}  B^{-1}]; h = 1, 2, ..., kTB/2.
// The result is written in Montgomery form (t R mod p) for the apply kernels.
constexpr int kInvThreads = 256;

template <bool kUpper, bool kUnit>
__global__ void __launch_bounds__(kInvThreads)
    k_tri_inv(const uint32_t* __restrict__ T, int64_t ldt, int r, int tb,
              uint32_t* __restrict__ out, FieldP F, const uint32_t* __restrict__ inv_table) {
  // M and Y hold Montgomery forms (x R mod p): a sum of h <= 32 products of
  // two such forms, reduced once by REDC, is the Montgomery form of the sum of
  // the plain products (exact while the sum stays below p R: p < 2^26), else
  // one REDC per product.  p = 2: plain bits, the parity of the sum.
  __shared__ uint32_t M[kTB][kTB + 1];
  __shared__ uint32_t Y[kTB][kTB + 1];
  const int b = blockIdx.x, tid = threadIdx.x;
  const int o = b * tb;
  const int s = min(tb, r - o);
  const bool big = F.p >= (1u << 26);
  const uint32_t one_m = f_to_mont(1u, F);
  // M = lower form of the block (T, or T^T for an upper block), identity padded
  for (int idx0 = tid; idx0 < kTB * kTB; idx0 += 4 * kInvThreads) {
    uint32_t v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = idx0 + q * kInvThreads, i = idx / kTB, k = idx % kTB;
      v[q] = 0;
      if (idx < kTB * kTB && i < s && k < s && k <= i)
        v[q] = kUpper ? T[(int64_t)(o + k) * ldt + o + i] : T[(int64_t)(o + i) * ldt + o + k];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = idx0 + q * kInvThreads, i = idx / kTB, k = idx % kTB;
      if (idx >= kTB * kTB) continue;
      uint32_t w;
      if (i == k)
        w = (i >= s || kUnit) ? one_m : f_to_mont(f_inv(v[q], F, inv_table), F);
      else
        w = f_to_mont(v[q], F);
      M[i][k] = w;
    }
  }
  __syncthreads();
  auto dot = [&](const uint32_t* a, int sa, const uint32_t* x, int sx, int len) -> uint32_t {
    if (!big) {
      uint64_t acc = 0;
      for (int k = 0; k < len; ++k) acc += (uint64_t)a[k * sa] * x[k * sx];
      return F.is2 ? (uint32_t)(acc & 1u) : f_redc(acc, F);
    }
    uint32_t acc = 0;
    for (int k = 0; k < len; ++k) acc = f_add(acc, f_redc((uint64_t)a[k * sa] * x[k * sx], F), F);
    return acc;
  };
  for (int h = 1; h < kTB; h <<= 1) {
    // Y = C A^{-1} for every pair; C = M[B rows, A cols] (original entries)
    const int npairs = kTB / (2 * h), outs = npairs * h * h;
    for (int idx = tid; idx < outs; idx += kInvThreads) {
      const int q = idx / (h * h), rem = idx % (h * h), i = rem / h, j = rem % h;
      const int a0 = 2 * q * h, b0 = a0 + h;
      // A^{-1} is lower: only k >= j contribute
      Y[b0 + i][a0 + j] = dot(&M[b0 + i][a0 + j], 1, &M[a0 + j][a0 + j], kTB + 1, h - j);
    }
    __syncthreads();
    // X = -B^{-1} Y into C's place (B^{-1} lower: k <= i)
    for (int idx = tid; idx < outs; idx += kInvThreads) {
      const int q = idx / (h * h), rem = idx % (h * h), i = rem / h, j = rem % h;
      const int a0 = 2 * q * h, b0 = a0 + h;
      M[b0 + i][a0 + j] = f_sub(0u, dot(&M[b0 + i][b0], 1, &Y[b0][a0 + j], kTB + 1, i + 1), F);
    }
    __syncthreads();
  }
  uint32_t* dst = out + (size_t)b * kTB * kTB;
  for (int idx = tid; idx < kTB * kTB; idx += kInvThreads) {
    const int i = idx / kTB, k = idx % kTB;
    dst[idx] = kUpper ? M[k][i] : M[i][k];
  }
}

// ----------------------------------------------------------- apply kernels --
//
// X = Tinv Bblk (left; Bblk s x count) or X = Bblk Tinv (right; count x s),
// in place, with Tinv (kTB x kTB, Montgomery form, zero outside the s x s
// triangle) in shared memory.  Each CTA owns a strip of kStrip columns (left)
// or rows (right) of the block, staged in shared memory before it is
// overwritten.  An output is sum_k tinv_ik b_k: summed exactly in 64 bits and
// reduced by one REDC (exact while the sum stays below p R: p < 2^26), else
// one REDC per product.
constexpr int kStrip = 32;
constexpr int kApplyThreads = 256;

template <bool kBig>
__device__ __forceinline__ uint32_t mont_dot(const uint32_t* a, int sa, const uint32_t* x, int sx,
                                             int len, const FieldP& F) {
  if (!kBig) {
    uint64_t s0 = 0, s1 = 0;
    int k = 0;
    for (; k + 1 < len; k += 2) {
      s0 += (uint64_t)a[k * sa] * x[k * sx];
      s1 += (uint64_t)a[(k + 1) * sa] * x[(k + 1) * sx];
    }
    if (k < len) s0 += (uint64_t)a[k * sa] * x[k * sx];
    return F.is2 ? (uint32_t)((s0 + s1) & 1u) : f_redc(s0 + s1, F);
  }
  uint32_t acc = 0;
  for (int k = 0; k < len; ++k) acc = f_add(acc, f_redc((uint64_t)a[k * sa] * x[k * sx], F), F);
  return acc;
}

template <bool kBig>
__global__ void __launch_bounds__(kApplyThreads)
    k_tri_apply_left(const uint32_t* __restrict__ tinv, int s, uint32_t* __restrict__ B,
                     int64_t ldb, int64_t count, FieldP F) {
  __shared__ uint32_t Ti[kTB][kTB];
  __shared__ uint32_t Xs[kTB][kStrip + 1];
  const int tid = threadIdx.x;
  const int64_t c0 = (int64_t)blockIdx.x * kStrip;
  const int w = (int)(count - c0 < kStrip ? count - c0 : kStrip);
  copy_g2s(&Ti[0][0], tinv, kTB * kTB, tid, kApplyThreads);
  for (int idx0 = tid; idx0 < s * kStrip; idx0 += 8 * kApplyThreads) {
    uint32_t v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int idx = idx0 + q * kApplyThreads, k = idx / kStrip, j = idx % kStrip;
      v[q] = (idx < s * kStrip && j < w) ? B[(int64_t)k * ldb + c0 + j] : 0u;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int idx = idx0 + q * kApplyThreads, k = idx / kStrip, j = idx % kStrip;
      if (idx < s * kStrip) Xs[k][j] = v[q];
    }
  }
  __syncthreads();
  // thread: column j = tid % kStrip, rows i = tid / kStrip + 8 t
  const int j = tid % kStrip;
  uint32_t res[kTB / 8];
#pragma unroll
  for (int t = 0; t < kTB / 8; ++t) {
    const int i = tid / kStrip + 8 * t;
    res[t] = i < s ? mont_dot<kBig>(&Ti[i][0], 1, &Xs[0][j], kStrip + 1, s, F) : 0u;
  }
  if (j < w) {
#pragma unroll
    for (int t = 0; t < kTB / 8; ++t) {
      const int i = tid / kStrip + 8 * t;
      if (i < s) B[(int64_t)i * ldb + c0 + j] = res[t];
    }
  }
}

template <bool kBig>
__global__ void __launch_bounds__(kApplyThreads)
    k_tri_apply_right(const uint32_t* __restrict__ tinv, int s, uint32_t* __restrict__ B,
                      int64_t ldb, int64_t count, FieldP F) {
  __shared__ uint32_t Ti[kTB][kTB];
  __shared__ uint32_t Xs[kStrip][kTB + 1];
  const int tid = threadIdx.x;
  const int64_t t0 = (int64_t)blockIdx.x * kStrip;
  const int h = (int)(count - t0 < kStrip ? count - t0 : kStrip);
  copy_g2s(&Ti[0][0], tinv, kTB * kTB, tid, kApplyThreads);
  for (int idx0 = tid; idx0 < kStrip * s; idx0 += 8 * kApplyThreads) {
    uint32_t v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int idx = idx0 + q * kApplyThreads, rr = idx / s, k = idx % s;
      v[q] = (idx < kStrip * s && rr < h) ? B[(t0 + rr) * ldb + k] : 0u;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int idx = idx0 + q * kApplyThreads, rr = idx / s, k = idx % s;
      if (idx < kStrip * s) Xs[rr][k] = v[q];
    }
  }
  __syncthreads();
  // thread: output column jj = tid % kTB, rows rr = tid / kTB + 4 t
  const int jj = tid % kTB;
  uint32_t res[kStrip / 4];
#pragma unroll
  for (int t = 0; t < kStrip / 4; ++t) {
    const int rr = tid / kTB + 4 * t;
    res[t] = jj < s ? mont_dot<kBig>(&Ti[0][jj], kTB, &Xs[rr][0], 1, s, F) : 0u;
  }
  __syncthreads();
  if (jj < s) {
#pragma unroll
    for (int t = 0; t < kStrip / 4; ++t) Xs[tid / kTB + 4 * t][jj] = res[t];
  }
  __syncthreads();
  for (int idx = tid; idx < h * s; idx += kApplyThreads) {
    const int rr = idx / s, k = idx % s;
    B[(t0 + rr) * ldb + k] = Xs[rr][k];
  }
}

enum TriKind { kLowerUnitLeft, kUpperLeft, kUpperRight };

// Inverses of every diagonal block (size c->trsm_block) of the r x r
// triangle into c->tri_inv.
int invert_diag_blocks(pluq_ctx* c, TriKind kind, const uint32_t* T, int64_t ldt, int64_t r) {
  const int tb = c->trsm_block;
  const int64_t nb = cdiv(r, tb);
  PLUQ_TRY(c->tri_inv.ensure(sizeof(uint32_t) * nb * kTB * kTB));
  ProfScope ps(c, PC_TRSM, (double)nb * tb * tb * tb / 3.0, 8.0 * r * tb);
  uint32_t* out = c->tri_inv.as<uint32_t>();
  if (kind == kLowerUnitLeft)
    k_tri_inv<false, true><<<(unsigned)nb, kInvThreads, 0, c->stream>>>(T, ldt, (int)r, tb, out,
                                                                         c->F, inv_table_ptr(c));
  else
    k_tri_inv<true, false><<<(unsigned)nb, kInvThreads, 0, c->stream>>>(T, ldt, (int)r, tb, out,
                                                                         c->F, inv_table_ptr(c));
  PLUQ_CUDA(cudaGetLastError());
  return PLUQ_OK;
}

// Diagonal block `blk` (size s <= kTB) applied to `count` columns (rows for
// kUpperRight) of B.
int apply_diag_block(pluq_ctx* c, TriKind kind, int64_t blk, int64_t s, uint32_t* B, int64_t ldb,
                     int64_t count) {
  if (s <= 0 || count <= 0) return PLUQ_OK;
  ProfScope ps(c, PC_TRSM, (double)s * s * count, 8.0 * s * count);
  const uint32_t* tinv = c->tri_inv.as<uint32_t>() + blk * kTB * kTB;
  const unsigned g = (unsigned)cdiv(count, kStrip);
  const bool big = c->F.p >= (1u << 26);
  if (kind == kUpperRight) {
    if (big)
      k_tri_apply_right<true><<<g, kApplyThreads, 0, c->stream>>>(tinv, (int)s, B, ldb, count, c->F);
    else
      k_tri_apply_right<false><<<g, kApplyThreads, 0, c->stream>>>(tinv, (int)s, B, ldb, count, c->F);
  } else {
    if (big)
      k_tri_apply_left<true><<<g, kApplyThreads, 0, c->stream>>>(tinv, (int)s, B, ldb, count, c->F);
    else
      k_tri_apply_left<false><<<g, kApplyThreads, 0, c->stream>>>(tinv, (int)s, B, ldb, count, c->F);
  }
  PLUQ_CUDA(cudaGetLastError());
  return PLUQ_OK;
}

int64_t split_point(int64_t r, int64_t tb) {
  int64_t h = (r / 2 + tb - 1) / tb * tb;
  if (h <= 0 || h >= r) h = tb;
  return h;
}

// Recursive solves over the diagonal blocks [o, o + r) of the triangle (o a
// multiple of the block size tb); the diagonal blocks were inverted
// beforehand.
int llu_rec(pluq_ctx* c, const uint32_t* L, int64_t ldl, int64_t o, int64_t r, uint32_t* B,
            int64_t ldb, int64_t ncols) {
  const int64_t tb = c->trsm_block;
  if (r > tb && r <= strip_rows(c, ncols)) return trsm_llu_strip(c, L, ldl, o, r, B, ldb, ncols);
  if (r <= tb) return apply_diag_block(c, kLowerUnitLeft, o / tb, r, B, ldb, ncols);
  const int64_t r1 = split_point(r, tb);
  PLUQ_TRY(llu_rec(c, L, ldl, o, r1, B, ldb, ncols));
  PLUQ_TRY(fgemm_sub(c, r - r1, ncols, r1, L + r1 * ldl, ldl, B, ldb, B + r1 * ldb, ldb));
  return llu_rec(c, L + r1 * ldl + r1, ldl, o + r1, r - r1, B + r1 * ldb, ldb, ncols);
}

int ru_rec(pluq_ctx* c, const uint32_t* U, int64_t ldu, int64_t o, int64_t r, uint32_t* B,
           int64_t ldb, int64_t nrows) {
  const int64_t tb = c->trsm_block;
  if (r > tb && r <= strip_rows(c, nrows)) return trsm_ru_strip(c, U, ldu, o, r, B, ldb, nrows);
  if (r <= tb) return apply_diag_block(c, kUpperRight, o / tb, r, B, ldb, nrows);
  const int64_t r1 = split_point(r, tb);
  PLUQ_TRY(ru_rec(c, U, ldu, o, r1, B, ldb, nrows));
  PLUQ_TRY(fgemm_sub(c, nrows, r - r1, r1, B, ldb, U + r1, ldu, B + r1, ldb));
  return ru_rec(c, U + r1 * ldu + r1, ldu, o + r1, r - r1, B + r1, ldb, nrows);
}

int lu_rec(pluq_ctx* c, const uint32_t* U, int64_t ldu, int64_t o, int64_t r, uint32_t* B,
           int64_t ldb, int64_t ncols) {
  const int64_t tb = c->trsm_block;
  if (r <= tb) return apply_diag_block(c, kUpperLeft, o / tb, r, B, ldb, ncols);
  const int64_t r1 = split_point(r, tb);
  // U = [U11 U12; 0 U22]: X2 = U22^{-1} B2, B1 -= U12 X2, X1 = U11^{-1} B1
  PLUQ_TRY(lu_rec(c, U + r1 * ldu + r1, ldu, o + r1, r - r1, B + r1 * ldb, ldb, ncols));
  PLUQ_TRY(fgemm_sub(c, r1, ncols, r - r1, U + r1, ldu, B + r1 * ldb, ldb, B, ldb));
  return lu_rec(c, U, ldu, o, r1, B, ldb, ncols);
}

// ---------------------------------------------- cached diagonal inverses --
//
// When the diagonal b x b blocks of a triangle are full-rank square leaves of
// the recursion, their inverses were computed once when the leaf was factored
// (negated: -L^{-1}, -U^{-1}); every ancestor's solve then recurses only down
// to b and applies each diagonal block as one product X = Inv B with the
// product overwriting B (the limb fgemm's operands are packed before it writes,
// so the update is in place; the other forms go through scratch).

__global__ void k_copy_block(uint32_t* __restrict__ dst, int64_t ldd, const uint32_t* __restrict__ src,
                             int64_t lds, int64_t rows, int64_t cols) {
  for (int64_t t = blockIdx.y; t < rows; t += gridDim.y)
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < cols;
         u += (int64_t)gridDim.x * blockDim.x)
      dst[t * ldd + u] = src ? src[t * lds + u] : 0u;
}

dim3 block_grid(int64_t rows, int64_t cols) {
  int64_t gx = cdiv(cols, 256);
  if (gx > 32) gx = 32;
  const int64_t gy = rows < 65535 ? rows : 65535;
  return dim3((unsigned)(gx < 1 ? 1 : gx), (unsigned)(gy < 1 ? 1 : gy), 1);
}

// C (rows x cols) <- -(X Y) mod p, X rows x k, Y k x cols; C may be X or Y.
int product_overwrite(pluq_ctx* c, int64_t rows, int64_t cols, int64_t k, const uint32_t* X,
                      int64_t ldx, const uint32_t* Y, int64_t ldy, uint32_t* C, int64_t ldc) {
  if (c->form == PLUQ_FORM_LIMB_F16) {
    c->fgemm_beta0 = true;
    const int st = fgemm_sub_limb(c, rows, cols, k, X, ldx, Y, ldy, C, ldc);
    c->fgemm_beta0 = false;
    return st;
  }
  // the other forms read C: copy the operand C aliases to scratch, zero C
  PLUQ_TRY(c->scratch.ensure(sizeof(uint32_t) * rows * cols));
  uint32_t* S = c->scratch.as<uint32_t>();
  const bool left = (const uint32_t*)C == Y;  // C is Y (rows = k) or X (cols = k)
  {
    ProfScope ps(c, PC_TRSM, 0, 12.0 * rows * cols, 2);
    k_copy_block<<<block_grid(rows, cols), 256, 0, c->stream>>>(S, cols, C, ldc, rows, cols);
    k_copy_block<<<block_grid(rows, cols), 256, 0, c->stream>>>(C, ldc, nullptr, 0, rows, cols);
    PLUQ_CUDA(cudaGetLastError());
  }
  if (left) return fgemm_sub_classical(c, rows, cols, k, X, ldx, S, cols, C, ldc);
  return fgemm_sub_classical(c, rows, cols, k, S, cols, Y, ldy, C, ldc);
}

const uint32_t* cached_inv(const pluq_ctx* owner, int64_t slot, int which) {
  const int64_t b = owner->dinv_b;
  return owner->dinv.as<uint32_t>() + (slot * 2 + which) * b * b;
}

int llu_cached(pluq_ctx* c, const pluq_ctx* owner, const uint32_t* L, int64_t ldl, int64_t slot,
               int64_t r, uint32_t* B, int64_t ldb, int64_t ncols) {
  const int64_t b = owner->dinv_b;
  if (r == b) return product_overwrite(c, b, ncols, b, cached_inv(owner, slot, 0), b, B, ldb, B, ldb);
  const int64_t r1 = (r / 2 + b - 1) / b * b;
  PLUQ_TRY(llu_cached(c, owner, L, ldl, slot, r1, B, ldb, ncols));
  PLUQ_TRY(fgemm_sub(c, r - r1, ncols, r1, L + r1 * ldl, ldl, B, ldb, B + r1 * ldb, ldb));
  return llu_cached(c, owner, L + r1 * ldl + r1, ldl, slot + r1 / b, r - r1, B + r1 * ldb, ldb,
                    ncols);
}

int ru_cached(pluq_ctx* c, const pluq_ctx* owner, const uint32_t* U, int64_t ldu, int64_t slot,
              int64_t r, uint32_t* B, int64_t ldb, int64_t nrows) {
  const int64_t b = owner->dinv_b;
  if (r == b) return product_overwrite(c, nrows, b, b, B, ldb, cached_inv(owner, slot, 1), b, B, ldb);
  const int64_t r1 = (r / 2 + b - 1) / b * b;
  PLUQ_TRY(ru_cached(c, owner, U, ldu, slot, r1, B, ldb, nrows));
  PLUQ_TRY(fgemm_sub(c, nrows, r - r1, r1, B, ldb, U + r1, ldu, B + r1, ldb));
  return ru_cached(c, owner, U + r1 * ldu + r1, ldu, slot + r1 / b, r - r1, B + r1, ldb, nrows);
}

// The context holding cached inverses for the r x r triangle at diagonal
// offset diag0 (c or its ancestors), or null when a block is missing.
const pluq_ctx* cache_owner(const pluq_ctx* c, int64_t diag0, int64_t r) {
  for (const pluq_ctx* o = c; o; o = o->parent) {
    const int64_t b = o->dinv_b;
    if (b <= 0 || !o->dinv_ok || diag0 < 0 || r <= 0 || diag0 % b || r % b) continue;
    const int64_t s0 = diag0 / b, s1 = s0 + r / b;
    if (s1 > (int64_t)o->dinv_valid.size()) continue;
    bool all = true;
    for (int64_t s = s0; s < s1 && all; ++s) all = o->dinv_valid[s] != 0;
    if (all) return o;
  }
  return nullptr;
}

}  // namespace

int trsm_left_lower_unit(pluq_ctx* c, const uint32_t* L, int64_t ldl, int64_t r, uint32_t* B,
                         int64_t ldb, int64_t ncols, int64_t diag0) {
  if (r <= 1 || ncols <= 0) return PLUQ_OK;  // a unit 1x1 triangle is the identity
  if (const pluq_ctx* o = cache_owner(c, diag0, r))
    return llu_cached(c, o, L, ldl, diag0 / o->dinv_b, r, B, ldb, ncols);
  PLUQ_TRY(invert_diag_blocks(c, kLowerUnitLeft, L, ldl, r));
  return llu_rec(c, L, ldl, 0, r, B, ldb, ncols);
}

int trsm_right_upper(pluq_ctx* c, const uint32_t* U, int64_t ldu, int64_t r, uint32_t* B,
                     int64_t ldb, int64_t nrows, int64_t diag0) {
  if (r <= 0 || nrows <= 0) return PLUQ_OK;
  if (const pluq_ctx* o = cache_owner(c, diag0, r))
    return ru_cached(c, o, U, ldu, diag0 / o->dinv_b, r, B, ldb, nrows);
  PLUQ_TRY(invert_diag_blocks(c, kUpperRight, U, ldu, r));
  return ru_rec(c, U, ldu, 0, r, B, ldb, nrows);
}

// -(L^{-1}) and -(U^{-1}) of the b x b full-rank block T (compressed L\U) into
// cache slot `slot` of c: the identity solved against each triangle, negated.
__global__ void k_identity(uint32_t* __restrict__ X, int64_t b) {
  for (int64_t i = blockIdx.y; i < b; i += gridDim.y)
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < b;
         j += (int64_t)gridDim.x * blockDim.x)
      X[i * b + j] = i == j ? 1u : 0u;
}

__global__ void k_negate(uint32_t* __restrict__ X, int64_t count, uint32_t p) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x)
    X[t] = X[t] == 0u ? 0u : p - X[t];
}

// One of the two: -(L^{-1}) (upper = false) or -(U^{-1}) into c's slot, the work
// issued on w's stream with w's workspace (w = c, or a child context of c so
// that the two triangles are inverted at once).
int cache_leaf_inverse(pluq_ctx* w, pluq_ctx* c, bool upper, const uint32_t* T, int64_t ldt,
                       int64_t slot) {
  const int64_t b = c->dinv_b;
  uint32_t* X = c->dinv.as<uint32_t>() + (slot * 2 + (upper ? 1 : 0)) * b * b;
  {
    ProfScope ps(w, PC_TRSM, 0, 4.0 * b * b);
    k_identity<<<block_grid(b, b), 256, 0, w->stream>>>(X, b);
    PLUQ_CUDA(cudaGetLastError());
  }
  if (upper)
    PLUQ_TRY(trsm_right_upper(w, T, ldt, b, X, b, b, -1));
  else
    PLUQ_TRY(trsm_left_lower_unit(w, T, ldt, b, X, b, b, -1));
  {
    ProfScope ps(w, PC_TRSM, 0, 8.0 * b * b);
    k_negate<<<(unsigned)cdiv(b * b, 256 * 8), 256, 0, w->stream>>>(X, b * b, c->F.p);
    PLUQ_CUDA(cudaGetLastError());
  }
  return PLUQ_OK;
}

int cache_leaf_inverses(pluq_ctx* c, const uint32_t* T, int64_t ldt, int64_t slot) {
  PLUQ_TRY(cache_leaf_inverse(c, c, false, T, ldt, slot));
  return cache_leaf_inverse(c, c, true, T, ldt, slot);
}

int trsm_left_upper(pluq_ctx* c, const uint32_t* U, int64_t ldu, int64_t r, uint32_t* B,
                    int64_t ldb, int64_t ncols) {
  if (r <= 0 || ncols <= 0) return PLUQ_OK;
  PLUQ_TRY(invert_diag_blocks(c, kUpperLeft, U, ldu, r));
  return lu_rec(c, U, ldu, 0, r, B, ldb, ncols);
}

// ---------------------------------------------------------------------------
// Strip solves: a whole triangle of up to NB diagonal blocks (NB * 64 rows)
// in one launch.  Columns of B (left solves) or rows of B (right solves) are
// independent, so each CTA takes a strip of 32 of them into shared memory and
// runs the block forward substitution on it alone: X_k = T_kk^{-1} B_k with the
// inverted diagonal block, then B_j -= T_jk X_k for the later blocks j.  The
// 64 x 64 operand of each product is staged in shared memory in Montgomery
// form; a 64-term dot product of a Montgomery value and a plain residue is
// summed exactly in 64 bits and reduced by one REDC (p < 2^26), else one REDC
// per product.  One launch replaces the 2 NB - 1 launches (diagonal products
// and the thin updates between them) of the block recursion below NB * 64.
namespace {

constexpr int kStripW = 32;        // columns (left) or rows (right) per CTA
constexpr int kStripThreads = 256;

template <bool kBig>
__device__ __forceinline__ uint32_t dot64(const uint32_t* a, int sa, const uint32_t* x, int sx,
                                          int len, const FieldP& F) {
  return mont_dot<kBig>(a, sa, x, sx, len, F);
}

// Left solve X = L^{-1} B with L unit lower (r x r, r <= NB * 64): CTA owns
// columns [c0, c0 + 32) of B.
template <int NB, bool kBig>
__global__ void __launch_bounds__(kStripThreads)
    k_trsm_llu_strip(const uint32_t* __restrict__ L, int64_t ldl, int r,
                     const uint32_t* __restrict__ tinv, uint32_t* __restrict__ B, int64_t ldb,
                     int64_t ncols, FieldP F) {
  extern __shared__ uint32_t strip_smem[];
  uint32_t* Xs = strip_smem;                          // [NB * 64][kStripW + 1]
  uint32_t* Ws = Xs + NB * kTB * (kStripW + 1);       // [64][65]
  constexpr int XS = kStripW + 1, WS = kTB + 1;
  const int tid = threadIdx.x;
  const int64_t c0 = (int64_t)blockIdx.x * kStripW;
  const int w = (int)(ncols - c0 < kStripW ? ncols - c0 : kStripW);
  for (int idx = tid; idx < r * kStripW; idx += kStripThreads) {
    const int i = idx / kStripW, j = idx % kStripW;
    Xs[i * XS + j] = j < w ? B[(int64_t)i * ldb + c0 + j] : 0u;
  }
  const int nb = (r + kTB - 1) / kTB;
  const int col = tid % kStripW, rb = tid / kStripW;  // outputs rows rb + 8 q
  for (int k = 0; k < nb; ++k) {
    const int sk = min(kTB, r - k * kTB);
    for (int j = k; j < nb; ++j) {
      const int sj = min(kTB, r - j * kTB);
      __syncthreads();  // the previous product's writes to Xs and reads of Ws are done
      // Ws = T_jk in Montgomery form: the inverted diagonal block for j = k
      // (already Montgomery), else the block of L
      if (j == k) {
        for (int idx = tid; idx < kTB * kTB; idx += kStripThreads)
          Ws[(idx / kTB) * WS + idx % kTB] = tinv[(size_t)k * kTB * kTB + idx];
      } else {
        for (int idx = tid; idx < sj * sk; idx += kStripThreads) {
          const int i = idx / sk, q = idx % sk;
          Ws[i * WS + q] = f_to_mont(L[(int64_t)(j * kTB + i) * ldl + k * kTB + q], F);
        }
      }
      __syncthreads();
      uint32_t res[kTB / 8];
#pragma unroll
      for (int t = 0; t < kTB / 8; ++t) {
        const int i = rb + 8 * t;
        res[t] = i < sj ? dot64<kBig>(&Ws[i * WS], 1, &Xs[(k * kTB) * XS + col], XS, sk, F) : 0u;
      }
      __syncthreads();
#pragma unroll
      for (int t = 0; t < kTB / 8; ++t) {
        const int i = rb + 8 * t;
        if (i >= sj) continue;
        uint32_t* xp = &Xs[(j * kTB + i) * XS + col];
        *xp = j == k ? res[t] : f_sub(*xp, res[t], F);
      }
    }
  }
  __syncthreads();
  for (int idx = tid; idx < r * kStripW; idx += kStripThreads) {
    const int i = idx / kStripW, j = idx % kStripW;
    if (j < w) B[(int64_t)i * ldb + c0 + j] = Xs[i * XS + j];
  }
}

// Right solve X = B U^{-1} with U upper (r x r, r <= NB * 64): CTA owns rows
// [t0, t0 + 32) of B; X_k = B_k Uinv_k, then B_j -= X_k U_kj for j > k.
template <int NB, bool kBig>
__global__ void __launch_bounds__(kStripThreads)
    k_trsm_ru_strip(const uint32_t* __restrict__ U, int64_t ldu, int r,
                    const uint32_t* __restrict__ tinv, uint32_t* __restrict__ B, int64_t ldb,
                    int64_t nrows, FieldP F) {
  extern __shared__ uint32_t strip_smem[];
  constexpr int XS = NB * kTB + 1, WS = kTB + 1;
  uint32_t* Xs = strip_smem;                  // [32][NB * 64 + 1]
  uint32_t* Ws = Xs + kStripW * XS;           // [64][65]: Ws[q][c] = T[q][c] (Montgomery)
  const int tid = threadIdx.x;
  const int64_t t0 = (int64_t)blockIdx.x * kStripW;
  const int h = (int)(nrows - t0 < kStripW ? nrows - t0 : kStripW);
  for (int idx = tid; idx < kStripW * r; idx += kStripThreads) {
    const int i = idx / r, q = idx % r;
    Xs[i * XS + q] = i < h ? B[(t0 + i) * ldb + q] : 0u;
  }
  const int nb = (r + kTB - 1) / kTB;
  const int c = tid % kTB, rb = tid / kTB;  // output column c, rows rb + 4 q
  for (int k = 0; k < nb; ++k) {
    const int sk = min(kTB, r - k * kTB);
    for (int j = k; j < nb; ++j) {
      const int sj = min(kTB, r - j * kTB);
      __syncthreads();
      if (j == k) {
        for (int idx = tid; idx < kTB * kTB; idx += kStripThreads)
          Ws[(idx / kTB) * WS + idx % kTB] = tinv[(size_t)k * kTB * kTB + idx];
      } else {
        for (int idx = tid; idx < sk * sj; idx += kStripThreads) {
          const int q = idx / sj, cc = idx % sj;
          Ws[q * WS + cc] = f_to_mont(U[(int64_t)(k * kTB + q) * ldu + j * kTB + cc], F);
        }
      }
      __syncthreads();
      uint32_t res[kStripW / 4];
#pragma unroll
      for (int t = 0; t < kStripW / 4; ++t) {
        const int i = rb + 4 * t;
        res[t] = c < sj ? dot64<kBig>(&Ws[c], WS, &Xs[i * XS + k * kTB], 1, sk, F) : 0u;
      }
      __syncthreads();
      if (c < sj) {
#pragma unroll
        for (int t = 0; t < kStripW / 4; ++t) {
          uint32_t* xp = &Xs[(rb + 4 * t) * XS + j * kTB + c];
          *xp = j == k ? res[t] : f_sub(*xp, res[t], F);
        }
      }
    }
  }
  __syncthreads();
  for (int idx = tid; idx < kStripW * r; idx += kStripThreads) {
    const int i = idx / r, q = idx % r;
    if (i < h) B[(t0 + i) * ldb + q] = Xs[i * XS + q];
  }
}

template <int NB>
size_t strip_smem_llu() { return sizeof(uint32_t) * (NB * kTB * (kStripW + 1) + kTB * (kTB + 1)); }
template <int NB>
size_t strip_smem_ru() { return sizeof(uint32_t) * (kStripW * (NB * kTB + 1) + kTB * (kTB + 1)); }

template <int NB>
int launch_llu_strip(pluq_ctx* c, const uint32_t* L, int64_t ldl, int64_t r,
                     const uint32_t* tinv, uint32_t* B, int64_t ldb, int64_t ncols) {
  const size_t smem = strip_smem_llu<NB>();
  static const cudaError_t a0 = cudaFuncSetAttribute(
      k_trsm_llu_strip<NB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  static const cudaError_t a1 = cudaFuncSetAttribute(
      k_trsm_llu_strip<NB, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  PLUQ_CUDA(a0);
  PLUQ_CUDA(a1);
  const unsigned g = (unsigned)cdiv(ncols, kStripW);
  ProfScope ps(c, PC_TRSM, (double)r * r * ncols, 8.0 * r * ncols);
  if (c->F.p >= (1u << 26))
    k_trsm_llu_strip<NB, true><<<g, kStripThreads, smem, c->stream>>>(L, ldl, (int)r, tinv, B, ldb,
                                                                      ncols, c->F);
  else
    k_trsm_llu_strip<NB, false><<<g, kStripThreads, smem, c->stream>>>(L, ldl, (int)r, tinv, B,
                                                                       ldb, ncols, c->F);
  PLUQ_CUDA(cudaGetLastError());
  return PLUQ_OK;
}

template <int NB>
int launch_ru_strip(pluq_ctx* c, const uint32_t* U, int64_t ldu, int64_t r, const uint32_t* tinv,
                    uint32_t* B, int64_t ldb, int64_t nrows) {
  const size_t smem = strip_smem_ru<NB>();
  static const cudaError_t a0 = cudaFuncSetAttribute(
      k_trsm_ru_strip<NB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  static const cudaError_t a1 = cudaFuncSetAttribute(
      k_trsm_ru_strip<NB, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  PLUQ_CUDA(a0);
  PLUQ_CUDA(a1);
  const unsigned g = (unsigned)cdiv(nrows, kStripW);
  ProfScope ps(c, PC_TRSM, (double)r * r * nrows, 8.0 * r * nrows);
  if (c->F.p >= (1u << 26))
    k_trsm_ru_strip<NB, true><<<g, kStripThreads, smem, c->stream>>>(U, ldu, (int)r, tinv, B, ldb,
                                                                     nrows, c->F);
  else
    k_trsm_ru_strip<NB, false><<<g, kStripThreads, smem, c->stream>>>(U, ldu, (int)r, tinv, B,
                                                                      ldb, nrows, c->F);
  PLUQ_CUDA(cudaGetLastError());
  return PLUQ_OK;
}

}  // namespace

// Largest triangle a strip launch takes for `count` right-hand sides: more
// diagonal blocks while there are few strips (the launch is latency-bound), fewer
// when the CUDA-core work of the triangle's blocks would dominate.
int strip_rows(const pluq_ctx* c, int64_t count) {
  if (c->trsm_block != kTB || c->strip_max <= 0) return 0;
  const int rows = count <= 4096 ? 8 * kTB : 4 * kTB;
  return rows < c->strip_max ? rows : c->strip_max;
}

int trsm_llu_strip(pluq_ctx* c, const uint32_t* L, int64_t ldl, int64_t o, int64_t r,
                   uint32_t* B, int64_t ldb, int64_t ncols) {
  const uint32_t* tinv = c->tri_inv.as<uint32_t>() + (o / kTB) * kTB * kTB;
  if (r <= 4 * kTB) return launch_llu_strip<4>(c, L, ldl, r, tinv, B, ldb, ncols);
  return launch_llu_strip<8>(c, L, ldl, r, tinv, B, ldb, ncols);
}

int trsm_ru_strip(pluq_ctx* c, const uint32_t* U, int64_t ldu, int64_t o, int64_t r, uint32_t* B,
                  int64_t ldb, int64_t nrows) {
  const uint32_t* tinv = c->tri_inv.as<uint32_t>() + (o / kTB) * kTB * kTB;
  if (r <= 4 * kTB) return launch_ru_strip<4>(c, U, ldu, r, tinv, B, ldb, nrows);
  return launch_ru_strip<8>(c, U, ldu, r, tinv, B, ldb, nrows);
}
