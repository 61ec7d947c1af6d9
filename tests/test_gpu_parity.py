"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bit-exact on every seeded input: rank, rank profile matrix (pivots of P, Q),
row and column rank profiles, reduced echelon form, and the factor identity
P L U Q = A mod p with the library's storage conventions.  Sizes span several
base-case tiles with ragged tails; the recursion is also driven deep with
small tiles so every block of the recursion (F, G, H, R, shifts) is exercised.
"""
import numpy as np
import pytest

import oracle
import workloads
from pluq_checks import check_pluq, check_rpm_from_pq, check_rref, exact_identity, matmul_mod

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU-only containers
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1402_3501_gb300 as pq  # noqa: E402

FORMS = ["fp64", "limb"]


@pytest.fixture(scope="module")
def ctx():
    c = pq.Context(0)
    yield c
    c.close()


class leaf_mode:
    """Temporarily set the leaf size and kind (leaf 0: one-CTA tiles) and base tiles.

    `leaf` is an int (wavefront leaves of that size) or a (size, kind) pair.
    """

    def __init__(self, ctx, leaf, tiles=(128, 128), trsm_block=64):
        self.leaf, self.kind = (leaf if isinstance(leaf, tuple) else (leaf, 1))
        self.ctx, self.tiles, self.tb = ctx, tiles, trsm_block

    def __enter__(self):
        self.ctx.set_option("leaf_dim", self.leaf)
        self.ctx.set_option("leaf_kind", self.kind)
        self.ctx.set_tuning(self.tiles[0], self.tiles[1], self.tb)

    def __exit__(self, *exc):
        self.ctx.set_option("leaf_dim", 1024)
        self.ctx.set_option("leaf_kind", 2)
        self.ctx.set_tuning(128, 128, 64)


def to_dev(A):
    return torch.from_numpy(np.ascontiguousarray(A).astype(np.int32)).cuda()


def run_pluq(ctx, A, p, form):
    res = pq.pluq_modp(to_dev(A), p, form=form, ctx=ctx)
    torch.cuda.synchronize()
    return (res.rank, res.P.cpu().numpy(), res.Q.cpu().numpy(), res.LU.cpu().numpy(),
            res.rrp.cpu().numpy(), res.crp.cpu().numpy())


def assert_parity(ctx, A, p, form="auto", expect=None):
    r, P, Q, LU, rrp, crp = run_pluq(ctx, A, p, form)
    ref = oracle.pluq(A, p) if expect is None else expect
    assert r == ref.rank
    check_rpm_from_pq(P, Q, r, ref.rpm)
    assert rrp.tolist() == ref.rrp.tolist()
    assert crp.tolist() == ref.crp.tolist()
    check_pluq(A, p, P, Q, LU.astype(np.int64), r)
    return r


# ---------------------------------------------------------------- fgemm ----

@pytest.mark.parametrize("thin", [1, 0])
def test_fgemm_thin_and_tensor_paths(ctx, thin):
    """Inner dimensions around the CUDA-core / tensor-core switch (K = 128), both
    paths forced in turn, ragged tiles, extreme residues."""
    ctx.set_option("thin_gemm", thin)
    try:
        for p in (2, 65521, 131071, 16777213):
            for (M, N, K) in [(1, 1, 1), (65, 63, 31), (200, 130, 127), (129, 257, 128),
                              (70, 300, 129)]:
                rng = np.random.default_rng(M + 3 * N + 7 * K + p % 89)
                A = rng.integers(0, p, (M, K), dtype=np.int64)
                B = rng.integers(0, p, (K, N), dtype=np.int64)
                C = rng.integers(0, p, (M, N), dtype=np.int64)
                A[0, :] = p - 1
                B[:, 0] = p - 1
                expect = (C - matmul_mod(A, B, p)) % p
                Cd = to_dev(C)
                pq.fgemm_modp(Cd, to_dev(A), to_dev(B), p, form="limb", ctx=ctx)
                torch.cuda.synchronize()
                assert np.array_equal(Cd.cpu().numpy().astype(np.int64), expect), (p, M, N, K)
    finally:
        ctx.set_option("thin_gemm", 1)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("p", [2, 3, 251, 65521, 131071])
@pytest.mark.parametrize("mnk", [(1, 1, 1), (70, 33, 17), (129, 257, 100), (300, 200, 700),
                                 (64, 64, 1024)])
def test_fgemm_parity(ctx, form, p, mnk):
    M, N, K = mnk
    rng = np.random.default_rng(M * 7 + N * 3 + K + p % 97)
    A = rng.integers(0, p, (M, K), dtype=np.int64)
    B = rng.integers(0, p, (K, N), dtype=np.int64)
    C = rng.integers(0, p, (M, N), dtype=np.int64)
    expect = (C - matmul_mod(A, B, p)) % p
    Cd = to_dev(C)
    pq.fgemm_modp(Cd, to_dev(A), to_dev(B), p, form=form, ctx=ctx)
    torch.cuda.synchronize()
    assert np.array_equal(Cd.cpu().numpy().astype(np.int64), expect)


@pytest.mark.parametrize("tile", [0, 1, 2])
@pytest.mark.parametrize("p", [2, 251, 65521, 131071, 1048573])
@pytest.mark.parametrize("mnk", [(70, 33, 17), (129, 257, 1100), (300, 200, 2100)])
def test_fgemm_tile_variants(ctx, tile, p, mnk):
    """Every tile variant of the limb fgemm gives exactly C - A B mod p, with
    K spanning several exact accumulation groups and operands at p - 1."""
    M, N, K = mnk
    rng = np.random.default_rng(M + 3 * N + K + p % 89 + tile)
    A = rng.integers(0, p, (M, K), dtype=np.int64)
    B = rng.integers(0, p, (K, N), dtype=np.int64)
    C = rng.integers(0, p, (M, N), dtype=np.int64)
    A[: M // 2, :] = p - 1
    B[:, : N // 3] = p - 1
    expect = (C - matmul_mod(A, B, p)) % p
    ctx.set_option("fgemm_tile", tile)
    ctx.set_option("thin_gemm", 0)
    try:
        Cd = to_dev(C)
        pq.fgemm_modp(Cd, to_dev(A), to_dev(B), p, form="limb", ctx=ctx)
        torch.cuda.synchronize()
    finally:
        ctx.set_option("fgemm_tile", 0)
        ctx.set_option("thin_gemm", 1)
    assert np.array_equal(Cd.cpu().numpy().astype(np.int64), expect)


@pytest.mark.parametrize("p", [2, 251, 65521, 131071, 1048573, 2147483647])
@pytest.mark.parametrize("mnk", [(1, 1, 1), (70, 33, 17), (129, 257, 64), (300, 200, 130),
                                 (200, 300, 2100)])
def test_fgemm_fused_split(ctx, p, mnk):
    """The fgemm whose producer warps split the digits (no packing pass) gives
    exactly C - A B mod p: every digit count, ragged tiles, K spanning several
    exact groups, operands at p - 1, and strided (unaligned) views."""
    M, N, K = mnk
    rng = np.random.default_rng(M + 5 * N + K + p % 83)
    A = rng.integers(0, p, (M, K), dtype=np.int64)
    B = rng.integers(0, p, (K, N), dtype=np.int64)
    C = rng.integers(0, p, (M, N), dtype=np.int64)
    A[: (M + 1) // 2, :] = p - 1
    B[:, : (N + 2) // 3] = p - 1
    expect = (C - matmul_mod(A, B, p)) % p
    ctx.set_option("fused_kmax", 1 << 30)
    ctx.set_option("thin_gemm", 0)
    try:
        Cd = to_dev(C)
        pq.fgemm_modp(Cd, to_dev(A), to_dev(B), p, form="limb", ctx=ctx)
        # the same product on views with odd leading dimensions
        big = torch.zeros((M + 3, K + N + 7), dtype=torch.int32, device="cuda")
        Av = big[1:M + 1, 3:K + 3]
        Av.copy_(to_dev(A))
        bigb = torch.zeros((K + 2, N + 5), dtype=torch.int32, device="cuda")
        Bv = bigb[1:K + 1, 1:N + 1]
        Bv.copy_(to_dev(B))
        Cv = to_dev(C)
        pq.fgemm_modp(Cv, Av, Bv, p, form="limb", ctx=ctx)
        torch.cuda.synchronize()
    finally:
        ctx.set_option("fused_kmax", 0)
        ctx.set_option("thin_gemm", 1)
    assert np.array_equal(Cd.cpu().numpy().astype(np.int64) % (1 << 32), expect)
    assert np.array_equal(Cv.cpu().numpy().astype(np.int64) % (1 << 32), expect)


@pytest.mark.parametrize("kmax", [128, 512])
@pytest.mark.parametrize("p,shape,frac", [(65521, (1100, 900), 1.0), (131071, (777, 700), 0.6),
                                          (2147483647, (600, 650), 0.8)])
def test_pluq_fused_split(ctx, kmax, p, shape, frac):
    m, n = shape
    g = workloads.prescribed_rank_matrix(m, n, int(frac * min(m, n)), p, seed=16)
    ctx.set_option("fused_kmax", kmax)
    try:
        with leaf_mode(ctx, (128, 2)):
            assert_parity(ctx, g.A, p, "limb")
    finally:
        ctx.set_option("fused_kmax", 0)


@pytest.mark.parametrize("tile", [1, 2])
@pytest.mark.parametrize("p,shape,frac", [(65521, (1100, 900), 1.0), (131071, (777, 700), 0.6)])
def test_pluq_tile_variants(ctx, tile, p, shape, frac):
    m, n = shape
    g = workloads.prescribed_rank_matrix(m, n, int(frac * min(m, n)), p, seed=14)
    ctx.set_option("fgemm_tile", tile)
    try:
        with leaf_mode(ctx, (256, 2)):
            assert_parity(ctx, g.A, p, "limb")
    finally:
        ctx.set_option("fgemm_tile", 0)


@pytest.mark.parametrize("form", FORMS)
def test_fgemm_adversarial_extremes(ctx, form):
    # all entries p-1: the largest products the delayed reduction must absorb
    for p in [65521, 131071]:
        for K in [255, 256, 257, 1024, 4099]:
            A = np.full((130, K), p - 1, dtype=np.int64)
            B = np.full((K, 70), p - 1, dtype=np.int64)
            C = np.zeros((130, 70), dtype=np.int64)
            expect = (C - matmul_mod(A, B, p)) % p
            Cd = to_dev(C)
            pq.fgemm_modp(Cd, to_dev(A), to_dev(B), p, form=form, ctx=ctx)
            torch.cuda.synchronize()
            assert np.array_equal(Cd.cpu().numpy().astype(np.int64), expect), (p, K)


# primes past the 17-bit range: the FP64 form splits into 16-bit halves (four
# exact passes); the limb form takes three (p < 2^25) or four base-2^8 digits
LARGE_PRIMES = [1048573, 16777213, 33554393, 268435399, 1073741789, 2147483647]


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("p", LARGE_PRIMES)
@pytest.mark.parametrize("mnk", [(70, 33, 17), (129, 257, 300), (130, 70, 2000)])
def test_fgemm_large_primes(ctx, form, p, mnk):
    M, N, K = mnk
    rng = np.random.default_rng(M + N + K + p % 1000)
    A = rng.integers(0, p, (M, K), dtype=np.int64)
    B = rng.integers(0, p, (K, N), dtype=np.int64)
    C = rng.integers(0, p, (M, N), dtype=np.int64)
    A[0, :] = p - 1
    B[:, 0] = p - 1
    expect = (C - matmul_mod(A, B, p)) % p
    Cd = to_dev(C)
    pq.fgemm_modp(Cd, to_dev(A), to_dev(B), p, form=form, ctx=ctx)
    torch.cuda.synchronize()
    assert np.array_equal(Cd.cpu().numpy().astype(np.int64), expect)


@pytest.mark.parametrize("p", [16777213, 33554393, 2147483647])
def test_fgemm_large_primes_extremes(ctx, p):
    # the balanced extremes +-(p-1)/2 maximise every digit-class sum of the limb form
    h = (p - 1) // 2
    for a, b in [(h, h), (h, h + 1), (h + 1, h + 1), (p - 1, p - 1)]:
        for K in [319, 320, 321, 1281]:
            A = np.full((130, K), a, dtype=np.int64)
            B = np.full((K, 70), b, dtype=np.int64)
            C = np.zeros((130, 70), dtype=np.int64)
            expect = (C - matmul_mod(A, B, p)) % p
            for form in FORMS:
                Cd = to_dev(C)
                pq.fgemm_modp(Cd, to_dev(A), to_dev(B), p, form=form, ctx=ctx)
                torch.cuda.synchronize()
                assert np.array_equal(Cd.cpu().numpy().astype(np.int64), expect), (form, a, b, K)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("p", [2, 65521, 131071, 2147483647])
@pytest.mark.parametrize("mnk", [(256, 256, 256), (301, 259, 333), (520, 130, 777)])
def test_fgemm_winograd_levels(ctx, form, p, mnk):
    """Strassen-Winograd levels (forced down to small sizes, odd dimensions
    peeled) give exactly C - A B mod p, as the classical product does."""
    M, N, K = mnk
    rng = np.random.default_rng(M + N + K + p % 101)
    A = rng.integers(0, p, (M, K), dtype=np.int64)
    B = rng.integers(0, p, (K, N), dtype=np.int64)
    C = rng.integers(0, p, (M, N), dtype=np.int64)
    A[0, :] = p - 1
    B[:, -1] = p - 1
    expect = (C - matmul_mod(A, B, p)) % p
    for wmin in (64, 100):
        ctx.set_option("winograd_min", wmin)
        try:
            Cd = to_dev(C)
            pq.fgemm_modp(Cd, to_dev(A), to_dev(B), p, form=form, ctx=ctx)
            torch.cuda.synchronize()
        finally:
            ctx.set_option("winograd_min", 0)
        assert np.array_equal(Cd.cpu().numpy().astype(np.int64), expect), wmin


@pytest.mark.parametrize("p,shape,frac", [(65521, (900, 900), 1.0), (131071, (777, 700), 0.6)])
def test_pluq_winograd_levels(ctx, p, shape, frac):
    """The factorization with Winograd levels in its Schur updates equals the oracle."""
    m, n = shape
    g = workloads.prescribed_rank_matrix(m, n, int(frac * min(m, n)), p, seed=8)
    ctx.set_option("winograd_min", 96)
    try:
        with leaf_mode(ctx, (128, 3)):
            assert_parity(ctx, g.A, p, "limb")
            assert_parity(ctx, g.A, p, "fp64")
    finally:
        ctx.set_option("winograd_min", 0)


def test_fgemm_strided_views(ctx):
    p = 131071
    rng = np.random.default_rng(3)
    big = to_dev(rng.integers(0, p, (300, 400)))
    A = big[10:110, 5:77]
    B = big[120:192, 200:333]
    C = big[200:300, 0:133].clone()
    expect = (C.cpu().numpy().astype(np.int64)
              - matmul_mod(A.cpu().numpy(), B.cpu().numpy(), p)) % p
    pq.fgemm_modp(C, A, B, p, ctx=ctx)
    torch.cuda.synchronize()
    assert np.array_equal(C.cpu().numpy().astype(np.int64), expect)


# ------------------------------------------------------------- pluq ----

SHAPES = [(1, 1), (1, 40), (40, 1), (17, 33), (128, 128), (129, 130), (200, 300), (300, 200),
          (513, 257)]


@pytest.mark.parametrize("leaf", [(2048, 1), (2048, 0), (1024, 2), (1024, 3), (256, 4), (0, 0)])
@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("p", [2, 3, 65521, 131071])
@pytest.mark.parametrize("shape", SHAPES)
def test_pluq_uniform(ctx, leaf, form, p, shape):
    m, n = shape
    A = workloads.uniform_matrix(m, n, p, seed=1)
    with leaf_mode(ctx, leaf):
        assert_parity(ctx, A, p, form)


@pytest.mark.parametrize("leaf", [(2048, 1), (2048, 0), (1024, 3), (96, 1), (96, 0), (96, 2),
                                  (96, 3), (96, 4), (256, 4), (256, 2), (0, 0)])
@pytest.mark.parametrize("p", [3, 131071])
@pytest.mark.parametrize("shape", [(64, 64), (150, 200), (300, 260), (513, 257), (700, 700)])
@pytest.mark.parametrize("frac", [0.0, 0.1, 0.5, 0.9])
def test_pluq_prescribed_rank(ctx, leaf, p, shape, frac):
    m, n = shape
    r = int(min(m, n) * frac)
    g = workloads.prescribed_rank_matrix(m, n, r, p, seed=2)
    with leaf_mode(ctx, leaf):
        got = assert_parity(ctx, g.A, p)
    assert got == r


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("p", [1048573, 2147483647])
@pytest.mark.parametrize("shape,frac", [((129, 130), 1.0), ((300, 200), 1.0), ((513, 257), 0.5),
                                        ((700, 700), 0.9)])
def test_pluq_large_primes(ctx, form, p, shape, frac):
    m, n = shape
    r = int(frac * min(m, n))
    with leaf_mode(ctx, 96, tiles=(64, 64)):
        if frac == 1.0:
            assert_parity(ctx, workloads.uniform_matrix(m, n, p, 5), p, form)
        else:
            A = workloads.prescribed_rank_matrix(m, n, r, p, 5).A
            assert assert_parity(ctx, A, p, form) == r


@pytest.mark.parametrize("thin", [0, 1])
def test_pluq_thin_gemm_switch(ctx, thin):
    """The factorization is the same whether thin Schur updates use the CUDA cores."""
    g = workloads.prescribed_rank_matrix(700, 650, 300, 131071, 12)
    ctx.set_option("thin_gemm", thin)
    try:
        with leaf_mode(ctx, 96, tiles=(64, 64)):
            assert assert_parity(ctx, g.A, 131071, "limb") == 300
    finally:
        ctx.set_option("thin_gemm", 1)


@pytest.mark.parametrize("fork_depth", [0, 1, 4])
@pytest.mark.parametrize("leaf", [(96, 0), (96, 1), (96, 3), (96, 4), (0, 0)])
@pytest.mark.parametrize("p,shape,frac", [(3, (700, 700), 0.5), (131071, (513, 777), 0.8),
                                          (65521, (600, 450), 1.0)])
def test_pluq_concurrent_branches(ctx, fork_depth, leaf, p, shape, frac):
    """F and G factored concurrently on child contexts give the same result."""
    m, n = shape
    r = int(frac * min(m, n))
    A = workloads.prescribed_rank_matrix(m, n, r, p, 9).A
    ctx.set_option("fork_depth", fork_depth)
    try:
        with leaf_mode(ctx, leaf, tiles=(64, 64)):
            assert assert_parity(ctx, A, p, "limb") == r
    finally:
        ctx.set_option("fork_depth", 2)


def test_pluq_leaf_too_large_for_child_context(ctx):
    """A block within the leaf cut-off that no leaf kernel of a child context (half
    the SMs) can hold is split further instead of recursing on itself."""
    m = n = 4096  # F and G are about 2000 x 2048 in contexts of half the SMs
    g = workloads.prescribed_rank_matrix(m, n, 600, 131071, 3, device="cuda")
    ctx.set_option("fork_depth", 2)
    try:
        with leaf_mode(ctx, (2048, 1)):
            r, P, Q, LU, rrp, crp = run_pluq(ctx, g.A, 131071, "limb")
    finally:
        ctx.set_option("fork_depth", 2)
    assert r == g.rank
    check_rpm_from_pq(P, Q, r, g.rpm)
    assert rrp.tolist() == g.rrp.tolist() and crp.tolist() == g.crp.tolist()


@pytest.mark.parametrize("mode", [(0, (8, 8)), (0, (16, 8)), (0, (5, 13)), (0, (32, 32)),
                                  (0, (128, 64)), ((9, 0), (8, 8)), ((24, 0), (8, 8)),
                                  ((40, 0), (8, 8)), ((9, 1), (8, 8)), ((24, 1), (8, 8)),
                                  ((40, 1), (8, 8)), ((1, 1), (8, 8)), ((9, 3), (8, 8)),
                                  ((40, 3), (8, 8))])
@pytest.mark.parametrize("seed", [1, 2])
def test_pluq_deep_recursion(ctx, mode, seed):
    # small leaves / base tiles drive many recursion levels through every block step
    p = 131071
    with leaf_mode(ctx, mode[0], mode[1]):
        for m, n, frac in [(90, 70, 0.5), (64, 100, 0.3), (133, 133, 1.0)]:
            g = workloads.prescribed_rank_matrix(m, n, int(min(m, n) * frac), p, seed)
            assert_parity(ctx, g.A, p)
        A = workloads.uniform_matrix(77, 91, 5, seed)
        assert_parity(ctx, A, 5)


# cluster leaves: 16-bit storage (p < 2^16), 16 + 8-bit planes (p < 2^24) and
# 32-bit words, from a single row to the 1024 x 1024 limit, fewer rows than
# CTAs, zero and full rank
@pytest.mark.parametrize("p", [2, 3, 65521, 131071, 1048573, 2147483647])
@pytest.mark.parametrize("shape,frac", [((1024, 1024), 1.0), ((1024, 1024), 0.06),
                                        ((1000, 1024), 0.5), ((1024, 600), 0.3),
                                        ((700, 700), 0.9), ((15, 1024), 1.0), ((1, 1024), 1.0),
                                        ((1024, 1), 1.0), ((300, 300), 0.0), ((513, 1000), 1.0)])
def test_pluq_cluster_leaf(ctx, p, shape, frac):
    m, n = shape
    r = int(frac * min(m, n))
    if frac == 1.0:
        A = workloads.uniform_matrix(m, n, p, 7)
    else:
        A = workloads.prescribed_rank_matrix(m, n, r, p, 7).A
    with leaf_mode(ctx, (1024, 3)):
        got = assert_parity(ctx, A, p, "limb")
    if frac < 1.0:
        assert got == r


# tiled-iterative decomposition (row slabs, each by column tiles): the same
# rank, profiles and RPM as the oracle, valid factors; slabs of the leaf
# cut-off and other heights, several leaf kinds, rank-deficient and full rank
@pytest.mark.parametrize("slab", [0, 40, 150, 300])
@pytest.mark.parametrize("leaf", [(96, 3), (96, 0), (96, 1), (96, 4), (0, 0)])
@pytest.mark.parametrize("p,shape,frac", [(3, (700, 700), 0.5), (131071, (513, 777), 0.8),
                                          (65521, (600, 450), 1.0), (131071, (450, 600), 0.1),
                                          (2147483647, (300, 260), 0.7)])
def test_pluq_tiled_iterative(ctx, slab, leaf, p, shape, frac):
    m, n = shape
    r = int(frac * min(m, n))
    A = workloads.prescribed_rank_matrix(m, n, r, p, 11).A
    ctx.set_option("decomposition", 1)
    ctx.set_option("slab_rows", slab)
    try:
        with leaf_mode(ctx, leaf, tiles=(64, 64)):
            assert assert_parity(ctx, A, p, "limb") == r
    finally:
        ctx.set_option("decomposition", 0)
        ctx.set_option("slab_rows", 0)


@pytest.mark.parametrize("form", FORMS)
def test_pluq_tiled_iterative_bench_shape(ctx, form):
    """The 8192 x 8192 rank-4096 workload under tiled iteration (slabs and tiles
    of the leaf cut-off): rank, profiles and RPM as constructed, factors checked
    by Freivalds' test."""
    cfg = workloads.CONFIGS["lru-8192-r4096-p131071"]
    g = workloads.prescribed_rank_matrix(cfg.m, cfg.n, cfg.r, cfg.p, 1, device="cuda")
    ctx.set_option("decomposition", 1)
    try:
        r, P, Q, LU, rrp, crp = run_pluq(ctx, g.A, cfg.p, form)
    finally:
        ctx.set_option("decomposition", 0)
    assert r == g.rank
    check_rpm_from_pq(P, Q, r, g.rpm)
    assert rrp.tolist() == g.rrp.tolist() and crp.tolist() == g.crp.tolist()
    assert not np.any(LU[r:, r:])
    assert np.all(np.diag(LU[:r, :r]) != 0)
    exact_identity(g.A, cfg.p, P, Q, LU.astype(np.int64), r)


@pytest.mark.parametrize("p", [2, 3, 251, 65521])
@pytest.mark.parametrize("shape,frac", [((256, 256), 1.0), ((256, 256), 0.3), ((255, 256), 1.0),
                                        ((256, 130), 1.0), ((1, 256), 1.0), ((256, 1), 1.0),
                                        ((200, 256), 0.0), ((513, 700), 0.9)])
def test_pluq_tile_leaf(ctx, p, shape, frac):
    """The one-CTA 16-bit leaf (blocks up to 256 x 256, p < 2^16): exact against
    the oracle on full, ragged, degenerate and zero blocks, and inside a recursion."""
    m, n = shape
    g = workloads.prescribed_rank_matrix(m, n, int(frac * min(m, n)), p, seed=12)
    with leaf_mode(ctx, (256, 4)):
        assert_parity(ctx, g.A, p, "limb")
    A = workloads.uniform_matrix(m, n, p, 13)
    with leaf_mode(ctx, (256, 4)):
        assert_parity(ctx, A, p, "limb")


@pytest.mark.parametrize("strip", [0, 256, 512])
@pytest.mark.parametrize("p,shape,frac", [(65521, (1500, 1400), 1.0), (131071, (900, 1300), 0.7),
                                          (2147483647, (700, 650), 0.9), (3, (800, 800), 0.5)])
def test_pluq_trsm_strips(ctx, strip, p, shape, frac):
    """Triangular solves finished by strip launches (whole triangles of up to 256
    or 512 rows per launch, ragged last blocks) equal the oracle, as the one-launch-
    per-block path does."""
    m, n = shape
    g = workloads.prescribed_rank_matrix(m, n, int(frac * min(m, n)), p, seed=15)
    ctx.set_option("trsm_strip", strip)
    try:
        with leaf_mode(ctx, (96, 2)):
            assert_parity(ctx, g.A, p, "limb")
        with leaf_mode(ctx, (512, 2)):
            assert_parity(ctx, g.A, p, "fp64")
    finally:
        ctx.set_option("trsm_strip", 0)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("fork_depth", [0, 2])
@pytest.mark.parametrize("leaf", [(128, 1), (96, 3), (256, 2)])
@pytest.mark.parametrize("p,shape,kind", [(65521, (1024, 1024), "uniform"),
                                          (131071, (1000, 1100), "uniform"),
                                          (3, (900, 900), "uniform"),
                                          (65521, (1024, 1024), "lru")])
def test_pluq_cached_diagonal_inverses(ctx, form, fork_depth, leaf, p, shape, kind):
    """Triangular solves that apply the cached inverses of full-rank diagonal
    leaves (one product per leaf-sized block, in place) equal the oracle; ragged
    edges, rank-deficient blocks (p = 3, prescribed rank) and concurrent branches
    fall back where a block is missing."""
    m, n = shape
    A = (workloads.uniform_matrix(m, n, p, 17) if kind == "uniform"
         else workloads.prescribed_rank_matrix(m, n, m // 2, p, 17).A)
    ctx.set_option("fork_depth", fork_depth)
    try:
        for on in (1, 0):
            ctx.set_option("diag_inverses", on)
            with leaf_mode(ctx, leaf):
                assert_parity(ctx, A, p, form)
    finally:
        ctx.set_option("diag_inverses", 1)
        ctx.set_option("fork_depth", 2)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("fork_depth", [1, 2])
@pytest.mark.parametrize("p,shape,kind", [(65521, (1536, 1536), "uniform"),
                                          (131071, (1300, 1700), "uniform"),
                                          (3, (1100, 1000), "uniform"),
                                          (65521, (1536, 1536), "lru")])
def test_pluq_lookahead(ctx, form, fork_depth, p, shape, kind):
    """The look-ahead split of H's update (H11 on the main stream, the rest on a
    third stream while R's recursion factors H11) gives the oracle's result, with
    it on and off, on full-rank leading blocks (where it applies), ragged shapes
    and rank-deficient ones (where it does not)."""
    m, n = shape
    A = (workloads.uniform_matrix(m, n, p, 23) if kind == "uniform"
         else workloads.prescribed_rank_matrix(m, n, m // 2, p, 23).A)
    ctx.set_option("fork_depth", fork_depth)
    try:
        for on in (1, 0):
            ctx.set_option("lookahead", on)
            with leaf_mode(ctx, (128, 1)):
                assert_parity(ctx, A, p, form)
    finally:
        ctx.set_option("lookahead", 0)
        ctx.set_option("fork_depth", 2)


@pytest.mark.parametrize("tb", [1, 7, 16, 64])
def test_pluq_trsm_blocks(ctx, tb):
    p = 65521
    with leaf_mode(ctx, 40, (32, 32), tb):
        g = workloads.prescribed_rank_matrix(260, 240, 180, p, seed=4)
        assert_parity(ctx, g.A, p)


def test_pluq_special_matrices(ctx):
    p = 131071
    for n in [1, 5, 129, 300]:
        assert_parity(ctx, np.eye(n, dtype=np.uint32), p)
        assert_parity(ctx, np.zeros((n, n + 7), dtype=np.uint32), p)
        perm = np.random.default_rng(n).permutation(n)
        Pm = np.zeros((n, n), dtype=np.uint32)
        Pm[np.arange(n), perm] = 1
        assert_parity(ctx, Pm, p)
    u = np.arange(1, 301, dtype=np.int64)
    v = np.arange(7, 207, dtype=np.int64)
    u[:50] = 0
    v[:120] = 0
    assert_parity(ctx, matmul_mod(u[:, None], v[None, :], p).astype(np.uint32), p)


def test_pluq_strided_lda(ctx):
    p = 131071
    g = workloads.prescribed_rank_matrix(200, 150, 90, p, seed=7)
    big = torch.zeros((200, 180), dtype=torch.int32, device="cuda")
    big[:, :150] = to_dev(g.A)
    big[:, 150:] = 12345
    view = big[:, :150]
    res = pq.pluq_modp(view, p, ctx=ctx)
    torch.cuda.synchronize()
    assert res.rank == 90
    assert torch.all(big[:, 150:] == 12345)
    check_pluq(g.A, p, res.P.cpu().numpy(), res.Q.cpu().numpy(),
               view.cpu().numpy().astype(np.int64), res.rank)
    check_rpm_from_pq(res.P.cpu().numpy(), res.Q.cpu().numpy(), 90, g.rpm)


def test_pluq_empty(ctx):
    for shape in [(0, 5), (5, 0), (0, 0)]:
        A = torch.zeros(shape, dtype=torch.int32, device="cuda")
        res = pq.pluq_modp(A, 131071, ctx=ctx)
        assert res.rank == 0
        assert res.P.cpu().tolist() == list(range(shape[0]))
        assert res.Q.cpu().tolist() == list(range(shape[1]))


# ----------------------------------------------------- echelon / profiles --

@pytest.mark.parametrize("p", [3, 65521, 131071])
@pytest.mark.parametrize("shape,frac", [((40, 60), 0.5), ((257, 300), 0.7), ((300, 257), 1.0),
                                        ((129, 129), 0.0)])
def test_echelon_parity(ctx, p, shape, frac):
    m, n = shape
    g = workloads.prescribed_rank_matrix(m, n, int(min(m, n) * frac), p, seed=5)
    r, R, crp = pq.echelon_modp(to_dev(g.A), p, ctx=ctx)
    torch.cuda.synchronize()
    rr, Rref = oracle.rref(g.A, p)
    assert r == rr == g.rank
    assert crp.cpu().tolist() == g.crp.tolist()
    assert np.array_equal(R.cpu().numpy().astype(np.int64), Rref.astype(np.int64))
    check_rref(g.A, p, R.cpu().numpy(), crp.cpu().numpy())


@pytest.mark.parametrize("p", [2, 65521, 131071, 2147483647])
@pytest.mark.parametrize("shape,frac", [((40, 60), 0.5), ((257, 300), 0.7), ((300, 257), 1.0),
                                        ((1, 5), 1.0), ((700, 130), 0.4)])
def test_column_echelon_parity(ctx, p, shape, frac):
    """Reduced column echelon form = RREF(A^T)^T; its pivot rows are the row rank profile."""
    m, n = shape
    g = workloads.prescribed_rank_matrix(m, n, int(min(m, n) * frac), p, seed=7)
    r, E, rrp = pq.column_echelon_modp(to_dev(g.A), p, ctx=ctx)
    torch.cuda.synchronize()
    rr, Rt = oracle.rref(np.ascontiguousarray(g.A.T), p)
    assert r == rr == g.rank
    assert rrp.cpu().tolist() == g.rrp.tolist()
    assert np.array_equal(E.cpu().numpy().astype(np.int64), Rt.T.astype(np.int64))


@pytest.mark.parametrize("p", [2, 131071])
def test_rank_profile_parity(ctx, p):
    g = workloads.prescribed_rank_matrix(333, 222, 111, p, seed=6)
    A = to_dev(g.A)
    before = A.clone()
    r, rrp, crp, rpm = pq.rank_profile_modp(A, p, ctx=ctx)
    torch.cuda.synchronize()
    assert torch.equal(A, before)
    assert r == g.rank
    assert rrp.cpu().tolist() == g.rrp.tolist()
    assert crp.cpu().tolist() == g.crp.tolist()
    expect = np.full(333, -1)
    expect[g.rows] = g.cols
    assert rpm.cpu().numpy().tolist() == expect.tolist()


@pytest.mark.parametrize("leaf", [(96, 3), (96, 0), (96, 1), (96, 4), (0, 0)])
@pytest.mark.parametrize("fork_depth", [0, 2])
@pytest.mark.parametrize("p,shape,frac", [(3, (700, 700), 0.5), (131071, (513, 777), 0.8),
                                          (65521, (900, 500), 0.3)])
def test_rank_and_echelon_fast_paths_deep(ctx, leaf, fork_depth, p, shape, frac):
    """rank_profile_modp (no L or U kept) and echelon_modp (U only) skip the
    permutations of blocks whose factors they never read; through a deep
    recursion with rank-deficient blocks both still equal the oracle."""
    m, n = shape
    g = workloads.prescribed_rank_matrix(m, n, int(frac * min(m, n)), p, seed=11)
    ctx.set_option("fork_depth", fork_depth)
    try:
        with leaf_mode(ctx, leaf, tiles=(32, 32)):
            r, rrp, crp, rpm = pq.rank_profile_modp(to_dev(g.A), p, ctx=ctx)
            r2, R, crp2 = pq.echelon_modp(to_dev(g.A), p, ctx=ctx)
            torch.cuda.synchronize()
    finally:
        ctx.set_option("fork_depth", 2)
    assert r == r2 == g.rank
    assert rrp.cpu().tolist() == g.rrp.tolist() and crp.cpu().tolist() == g.crp.tolist()
    expect = np.full(m, -1)
    expect[g.rows] = g.cols
    assert rpm.cpu().numpy().tolist() == expect.tolist()
    rr, Rref = oracle.rref(g.A, p)
    assert crp2.cpu().tolist() == g.crp.tolist()
    assert np.array_equal(R.cpu().numpy().astype(np.int64), Rref.astype(np.int64))


# ------------------------------------------------------------- errors --

@pytest.mark.parametrize("kind", [0, 1])
def test_wait_limit_runs_out(kind):
    """A cooperative leaf whose spin-waits are given no time returns
    PLUQ_ERR_TIMEOUT (every CTA leaves, nothing faults), and the same context
    then factors the matrix exactly once the limit is restored."""
    c = pq.Context(0)
    try:
        p = 131071
        A = workloads.uniform_matrix(700, 700, p, 9)
        c.set_option("leaf_dim", 1024)
        c.set_option("leaf_kind", kind)
        c.set_option("wait_limit_us", 0)
        with pytest.raises(pq.PluqError) as e:
            pq.pluq_modp(to_dev(A), p, ctx=c)
        assert e.value.status == -8  # PLUQ_ERR_TIMEOUT
        assert pq.sync_status(c) == -8  # the device error word until the next call
        c.set_option("wait_limit_us", 2000000)
        assert_parity(c, A, p)
        assert pq.sync_status(c) == 0
    finally:
        c.close()


def test_workspace_cap():
    """A workspace cap below what a call needs gives PLUQ_ERR_NO_WORKSPACE; lifting it
    lets the same context factor the matrix."""
    c = pq.Context(0)
    try:
        p = 65521
        A = workloads.uniform_matrix(1500, 1400, p, 4)
        c.set_option("workspace_mb", 1)
        with pytest.raises(pq.PluqError) as e:
            pq.pluq_modp(to_dev(A), p, ctx=c)
        assert e.value.status == -6  # PLUQ_ERR_NO_WORKSPACE
        c.set_option("workspace_mb", 0)
        assert_parity(c, A, p)
    finally:
        c.close()


def test_status_codes(ctx):
    A = to_dev(np.ones((4, 4)))
    with pytest.raises(pq.PluqError) as e:
        pq.pluq_modp(A.clone(), 15, ctx=ctx)
    assert e.value.status == -2
    with pytest.raises(pq.PluqError) as e:
        pq.pluq_modp(A.clone(), 2 ** 31 + 11, ctx=ctx)
    assert e.value.status == -3
    bad = to_dev(np.full((4, 4), 7))
    keep = bad.clone()
    with pytest.raises(pq.PluqError) as e:
        pq.pluq_modp(bad, 5, ctx=ctx)
    assert e.value.status == -4
    assert torch.equal(bad, keep)
    # the context stays usable after errors
    assert_parity(ctx, workloads.uniform_matrix(50, 50, 131071, 1), 131071)


# ------------------------------------------------------------- batched --

def _batch_cases(p, seed):
    rng = np.random.default_rng(seed)
    cases = []
    for _ in range(40):
        m, n = (int(v) for v in rng.integers(1, 300, 2))
        r = int(rng.integers(0, min(m, n) + 1))
        cases.append(workloads.prescribed_rank_matrix(m, n, r, p, seed=int(rng.integers(1 << 30))).A)
    cases += [np.zeros((5, 7), np.uint32), np.eye(1, dtype=np.uint32), np.zeros((0, 4), np.uint32),
              workloads.uniform_matrix(1, 300, p, seed), workloads.uniform_matrix(300, 1, p, seed),
              workloads.uniform_matrix(1024, 64, p, seed), workloads.uniform_matrix(1100, 40, p, seed),
              workloads.uniform_matrix(1000, 1024, p, seed),
              workloads.prescribed_rank_matrix(700, 900, 333, p, seed=seed).A]
    return cases


@pytest.mark.parametrize("p", [2, 3, 65521, 131071, 134217757, 2147483647])
def test_batched_parity(ctx, p):
    """Every matrix of a mixed batch (empty, one-row, one-column, rank-deficient,
    the widest the persistent kernel takes, one past it) against the oracle, for
    each of the slab kernel's field modes: p = 2, p < 2^16 (the update below a
    slab on the tensor cores, 8-bit digits), p < 2^27 (one reduction per dot
    product) and larger p (a reduction per product)."""
    cases = _batch_cases(p, 3)
    As = [to_dev(A) for A in cases]
    for rep in range(2):  # the second call replays the captured graph
        As = [to_dev(A) for A in cases]
        ranks, Ps, Qs = pq.pluq_modp_batched(As, p, ctx=ctx)
        torch.cuda.synchronize()
        for A, Ad, r, P, Q in zip(cases, As, ranks, Ps, Qs):
            ref = oracle.pluq(A, p)
            assert r == ref.rank
            P, Q = P.cpu().numpy(), Q.cpu().numpy()
            check_rpm_from_pq(P, Q, r, ref.rpm)
            check_pluq(A, p, P, Q, Ad.cpu().numpy().astype(np.int64), r)


@pytest.mark.parametrize("p", [2, 65521, 131071, 2147483647])
@pytest.mark.parametrize("slab", [16, 24, 32])
def test_batched_slab_heights(slab, p):
    """Each buffer height of the batched kernel (pivots a slab collects before
    updating the rows below) against the oracle on the mixed batch, in every
    field mode (bits, 16-bit buffer and tensor-core updates, one reduction per
    dot product, a reduction per product)."""
    c = pq.Context(0)
    try:
        c.set_option("batch_slab", slab)
        cases = _batch_cases(p, 5)
        As = [to_dev(A) for A in cases]
        ranks, Ps, Qs = pq.pluq_modp_batched(As, p, ctx=c)
        torch.cuda.synchronize()
        for A, Ad, r, P, Q in zip(cases, As, ranks, Ps, Qs):
            ref = oracle.pluq(A, p)
            assert r == ref.rank
            P, Q = P.cpu().numpy(), Q.cpu().numpy()
            check_rpm_from_pq(P, Q, r, ref.rpm)
            check_pluq(A, p, P, Q, Ad.cpu().numpy().astype(np.int64), r)
    finally:
        c.close()


@pytest.mark.parametrize("p", [2, 65521])
def test_rank_profile_batched(ctx, p):
    """Batched ranks and sorted profiles equal the construction's, matrix by matrix,
    including matrices past the persistent kernel's size (factored one by one)."""
    shapes = [(40, 60, 20), (512, 300, 250), (33, 33, 33), (1, 7, 1), (600, 700, 100),
              (128, 96, 0)]
    gens = [workloads.prescribed_rank_matrix(m, n, r, p, 30 + i) for i, (m, n, r) in
            enumerate(shapes)]
    As = [to_dev(g.A) for g in gens]
    ranks, rrps, crps = pq.rank_profile_modp_batched(As, p, ctx=ctx)
    torch.cuda.synchronize()
    for g, r, rr, cc in zip(gens, ranks, rrps, crps):
        assert r == g.rank
        assert rr.cpu().tolist() == g.rrp.tolist()
        assert cc.cpu().tolist() == g.crp.tolist()


@pytest.mark.parametrize("p", [2, 65521, 131071, 2147483647])
def test_echelon_batched(ctx, p):
    """Batched RREF equals the oracle's, matrix by matrix (rank, pivot columns and
    the reduced rows), with an empty matrix and one whose entry is out of range
    (its own status, the others unaffected)."""
    shapes = [(40, 60, 20), (300, 257, 200), (33, 33, 33), (1, 7, 1), (700, 130, 52), (96, 128, 0)]
    gens = [workloads.prescribed_rank_matrix(m, n, r, p, 50 + i) for i, (m, n, r) in
            enumerate(shapes)]
    As = [to_dev(g.A) for g in gens]
    bad = np.zeros((8, 9), np.int64)
    bad[3, 4] = p  # p <= 2^31 - 1: still an int32
    As.insert(2, to_dev(bad))
    As.append(torch.zeros((0, 5), dtype=torch.int32, device="cuda"))
    ranks, Rs, crps, status = pq.echelon_modp_batched(As, p, ctx=ctx, return_status=True)
    torch.cuda.synchronize()
    assert status[2] == -4 and ranks[2] == -1  # PLUQ_ERR_ENTRY_OUT_OF_RANGE
    assert status[-1] == 0 and ranks[-1] == 0
    for i, g in zip([0, 1, 3, 4, 5, 6], gens):
        rr, Rref = oracle.rref(g.A, p)
        assert status[i] == 0 and ranks[i] == rr == g.rank
        assert crps[i].cpu().tolist() == g.crp.tolist()
        assert np.array_equal(Rs[i].cpu().numpy().astype(np.int64), Rref.astype(np.int64))


def test_batched_bad_entry_status(ctx):
    p = 65521
    good = workloads.prescribed_rank_matrix(50, 60, 20, p, seed=1).A
    bad = good.copy()
    bad[3, 4] = p + 5
    As = [to_dev(good), to_dev(bad), to_dev(good)]
    keep = As[1].clone()
    ranks, Ps, Qs, status = pq.pluq_modp_batched(As, p, ctx=ctx, return_status=True)
    torch.cuda.synchronize()
    assert status == [0, -4, 0] and ranks[0] == ranks[2] == 20
    assert torch.equal(As[1], keep)


# ------------------------------------------------------------- autotuner --

@pytest.mark.parametrize("p,shape,frac", [(131071, (700, 700), 0.3), (65521, (1100, 900), 1.0)])
def test_autotune_schedule_parity(ctx, p, shape, frac):
    """The autotuned schedule is applied to later calls of the shape and stays exact."""
    m, n = shape
    r = int(frac * min(m, n))
    A = workloads.prescribed_rank_matrix(m, n, r, p, 21).A
    Ad = to_dev(A)
    keep = Ad.clone()
    ch = ctx.autotune(Ad, p, form="limb", budget_ms=3000)
    torch.cuda.synchronize()
    assert torch.equal(Ad, keep)  # the tuner works on copies
    assert ch["leaf_dim"] in (256, 512, 1024, 2048)
    assert ch["leaf_kind"] in ("barrier", "wavefront", "per-leaf", "cluster", "tile")
    assert ch["fork_depth"] in (0, 1, 2, 3) and ch["ms"] > 0
    assert ch["fgemm_tile"] in (0, 1, 2)
    try:
        assert assert_parity(ctx, A, p, "limb") == r
        ctx.set_option("use_tuned", 0)
        assert assert_parity(ctx, A, p, "limb") == r
    finally:
        ctx.set_option("use_tuned", 1)
