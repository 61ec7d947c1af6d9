"""Bit-exact parity of the CUDA path on the five workloads at their full sizes.

For every seeded input: rank, the rank profile matrix (pivots of P and Q), both
sorted rank profiles, the factor identity P L U Q = A mod p and the storage
structure; the reduced echelon form where the oracle can produce it.  What
decides each case:

  * uniform 1024^2 over GF(131071), seeds 1-3: the CPU oracle (rank profile
    matrix, profiles, RREF) and an exact host product for the factor identity;
  * 8192^2 rank 4096 over GF(131071), seeds 1-3: the L R U construction, whose
    rank profile matrix is R (Sec. 4.1), an exact float64 host product of L U
    (every partial sum below 2^53) for both forms, and the oracle's RREF (seed 1);
  * uniform 32768^2 over GF(65521): the oracle's rank profile matrix stored by
    tests/golden/make_oracle_goldens.py, an exact product of L U computed with
    cuBLAS float64 on the GPU (a library product, independent of this
    library's kernels), and a 3-trial Freivalds check on the host, both forms;
  * 16384 x 20480 rank 16320 over GF(2^31 - 1): the construction, the exact
    GPU product in 16-bit halves and 3-trial Freivalds, both forms;
  * the batch of 4096 matrices (m, n uniform in [32, 512], p = 65521): the
    construction for every matrix, L U = the permuted A exactly for every
    matrix, and the oracle on every 8th matrix.
"""
import os

import numpy as np
import pytest

import oracle
import workloads
from pluq_checks import check_pluq, check_rpm_from_pq

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU-only containers
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1402_3501_gb300 as pq  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def ctx():
    c = pq.Context(0)
    yield c
    c.close()


def to_dev(A):
    return torch.from_numpy(np.ascontiguousarray(A).astype(np.int64).astype(np.int32)).cuda()


def factor(ctx, A_dev, p, form):
    """pluq_modp on a copy; (rank, P, Q, LU (device), rrp, crp) with host vectors."""
    X = A_dev.clone()
    res = pq.pluq_modp(X, p, form=form, ctx=ctx)
    torch.cuda.synchronize()
    return (res.rank, res.P.cpu().numpy(), res.Q.cpu().numpy(), X,
            res.rrp.cpu().numpy().tolist(), res.crp.cpu().numpy().tolist())


def check_structure(LU, r):
    """Trailing (m - r) x (n - r) block zero and U's diagonal non-zero (device)."""
    assert not torch.any(LU[r:, r:] != 0), "trailing block not zero"
    assert torch.all(torch.diagonal(LU[:r, :r]) != 0), "zero on U's diagonal"


def _lu_block_f64(LU, r, i0, i1):
    """Rows i0..i1 of the unit lower trapezoidal L (m x r) as float64 (device)."""
    Lb = LU[i0:i1, :r].to(torch.float64)
    rows = torch.arange(i0, i1, device=LU.device)[:, None]
    cols = torch.arange(r, device=LU.device)[None, :]
    Lb = torch.where(cols < rows, Lb, torch.zeros_like(Lb))
    return Lb + (cols == rows).to(torch.float64)


def exact_identity_gpu(A_dev, p, P, Q, LU, r, block=4096):
    """A[P][:, Q] == L U mod p, entry by entry, with cuBLAS float64 products.

    Every float64 product of integers is exact while its sums stay below 2^53:
    r (p-1)^2 < 2^53 for p < 2^17 and r <= 2^19; larger p are split into 16-bit
    halves (four products, each sum below r 2^32).
    """
    m, n = A_dev.shape
    dev = A_dev.device
    Pt = torch.from_numpy(P.astype(np.int64)).to(dev)
    Qt = torch.from_numpy(Q.astype(np.int64)).to(dev)
    if r == 0:
        assert not torch.any(A_dev != 0)
        return
    U = torch.triu(LU[:r, :].to(torch.int64))
    split = r * (p - 1) ** 2 >= 2 ** 53
    if split:
        Uh, Ul = (U >> 16).to(torch.float64), (U & 0xFFFF).to(torch.float64)
        c16, c32 = pow(2, 16, p), pow(2, 32, p)
    else:
        Uf = U.to(torch.float64)
    del U
    for i0 in range(0, m, block):
        i1 = min(m, i0 + block)
        Lb = _lu_block_f64(LU, r, i0, i1)
        if not split:
            got = torch.remainder(Lb @ Uf, p).to(torch.int64)
        else:
            Li = Lb.to(torch.int64)
            Lh, Ll = (Li >> 16).to(torch.float64), (Li & 0xFFFF).to(torch.float64)
            hh = torch.remainder(Lh @ Uh, p).to(torch.int64)
            mid = torch.remainder(torch.remainder(Lh @ Ul, p) + torch.remainder(Ll @ Uh, p),
                                  p).to(torch.int64)
            ll = torch.remainder(Ll @ Ul, p).to(torch.int64)
            got = (hh * c32 % p + mid * c16 % p + ll) % p
        want = A_dev[Pt[i0:i1]][:, Qt].to(torch.int64) % (1 << 32)
        assert torch.equal(got, want), f"P L U Q != A in rows {i0}..{i1}"


def freivalds_host(A, p, P, Q, LU_host, r, trials=3, seed=0, step=2048):
    """Host Freivalds check of A[P][:, Q] = L U mod p with exact int64 sums (chunks of
    the inner dimension keep every partial sum below 2^63); error below p^-trials."""
    rng = np.random.default_rng(seed)
    m, n = A.shape

    def mv_part(X, v, xmax):
        # sums of at most `chunk` products below xmax * p stay below 2^62
        chunk = max(1, (2 ** 62) // max(1, xmax * p))
        out = np.zeros(X.shape[0], dtype=np.int64)
        for s in range(0, X.shape[1], chunk):
            out = (out + (X[:, s:s + chunk] @ v[s:s + chunk]) % p) % p
        return out

    def mv(X, v):
        X = X.astype(np.int64)
        if p < 2 ** 20:
            return mv_part(X, v, p)
        # 16-bit halves of X: X v = 2^16 (X_hi v) + X_lo v
        hi = mv_part(X >> 16, v, p >> 16)
        lo = mv_part(X & 0xFFFF, v, 1 << 16)
        return (hi * (1 << 16) % p + lo) % p

    for _ in range(trials):
        x = rng.integers(0, p, n, dtype=np.int64)
        z = np.zeros(n, dtype=np.int64)
        z[Q] = x
        lhs = np.concatenate([mv(A[i:i + step], z) for i in range(0, m, step)])[P]
        ux = (np.concatenate([mv(np.triu(LU_host[i:min(r, i + step)].astype(np.int64), i), x)
                              for i in range(0, r, step)]) if r else np.zeros(0, np.int64))
        rhs = np.zeros(m, dtype=np.int64)
        for i in range(0, m, step):
            rows = np.arange(i, min(m, i + step))
            Lb = np.where(np.arange(r)[None, :] < rows[:, None],
                          LU_host[i:i + step, :r].astype(np.int64), 0)
            on_diag = rows < r
            Lb[np.nonzero(on_diag)[0], rows[on_diag]] = 1
            rhs[i:i + step] = mv(Lb, ux)
        assert np.array_equal(lhs, rhs), "Freivalds check of P L U Q = A failed"


def exact_identity_host_f64(A, p, P, Q, LU_host, r, step=2048):
    """A[P][:, Q] == L U mod p with float64 host products (exact: r (p-1)^2 < 2^53)."""
    assert r * (p - 1) ** 2 < 2 ** 53
    m, n = A.shape
    U = np.triu(LU_host[:r, :].astype(np.float64))
    for i in range(0, m, step):
        rows = np.arange(i, min(m, i + step))
        Lb = np.where(np.arange(r)[None, :] < rows[:, None],
                      LU_host[i:i + step, :r].astype(np.float64), 0.0)
        on_diag = rows < r
        Lb[np.nonzero(on_diag)[0], rows[on_diag]] = 1.0
        got = np.mod(Lb @ U, p).astype(np.int64)
        want = A[P[i:i + step]][:, Q].astype(np.int64)
        assert np.array_equal(got, want), f"P L U Q != A in rows {i}..{i + len(rows)}"


# ------------------------------------------------------- uniform 1024^2 --

@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("form", ["limb", "fp64"])
def test_uniform_1024(ctx, seed, form):
    cfg = workloads.CONFIGS["uniform-1024-p131071"]
    A = workloads.uniform_matrix(cfg.m, cfg.n, cfg.p, seed)
    ref = oracle.pluq(A, cfg.p)
    r, P, Q, LU, rrp, crp = factor(ctx, to_dev(A), cfg.p, form)
    assert r == ref.rank
    check_rpm_from_pq(P, Q, r, ref.rpm)
    assert rrp == ref.rrp.tolist() and crp == ref.crp.tolist()
    check_pluq(A, cfg.p, P, Q, LU.cpu().numpy().astype(np.int64), r)
    # the reduced echelon form equals the oracle's, entry by entry
    rr, Rref = oracle.rref(A, cfg.p)
    r2, R, crp2 = pq.echelon_modp(to_dev(A), cfg.p, form=form, ctx=ctx)
    torch.cuda.synchronize()
    assert r2 == rr
    assert crp2.cpu().tolist() == ref.crp.tolist()
    assert np.array_equal(R.cpu().numpy().astype(np.int64), Rref.astype(np.int64))


# ----------------------------------------------- 8192^2 rank 4096 (L R U) --

@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("form", ["limb", "fp64"])
def test_lru_8192(ctx, seed, form):
    cfg = workloads.CONFIGS["lru-8192-r4096-p131071"]
    g = workloads.prescribed_rank_matrix(cfg.m, cfg.n, cfg.r, cfg.p, seed=seed, device="cuda")
    Ad = to_dev(g.A)
    r, P, Q, LU, rrp, crp = factor(ctx, Ad, cfg.p, form)
    assert r == cfg.r
    check_rpm_from_pq(P, Q, r, g.rpm)
    assert rrp == g.rrp.tolist() and crp == g.crp.tolist()
    check_structure(LU, r)
    exact_identity_host_f64(g.A, cfg.p, P, Q, LU.cpu().numpy(), r)


def test_lru_8192_rref(ctx):
    """The reduced echelon form at full size equals the oracle's (both forms)."""
    cfg = workloads.CONFIGS["lru-8192-r4096-p131071"]
    g = workloads.prescribed_rank_matrix(cfg.m, cfg.n, cfg.r, cfg.p, seed=1, device="cuda")
    rr, Rref = oracle.rref(g.A, cfg.p, threads=os.cpu_count() or 1)
    assert rr == cfg.r
    Ad = to_dev(g.A)
    for form in ("limb", "fp64"):
        r, R, crp = pq.echelon_modp(Ad, cfg.p, form=form, ctx=ctx)
        torch.cuda.synchronize()
        assert r == rr and crp.cpu().tolist() == g.crp.tolist()
        assert np.array_equal(R.cpu().numpy().astype(np.int64), Rref.astype(np.int64)), form


# ------------------------------------------------------ uniform 32768^2 --

def _golden_32768():
    path = os.path.join(GOLDEN, "oracle_rpm_uniform-32768-p65521_seed1.npz")
    assert os.path.exists(path), "oracle golden of the 32768^2 workload is missing"
    return np.load(path)


@pytest.mark.parametrize("form", ["limb", "fp64"])
def test_uniform_32768(ctx, form):
    cfg = workloads.CONFIGS["uniform-32768-p65521"]
    gold = _golden_32768()
    A = workloads.uniform_matrix(cfg.m, cfg.n, cfg.p, seed=1)
    import hashlib
    assert hashlib.sha256(A.tobytes()).hexdigest() == str(gold["sha256"][0])
    Ad = to_dev(A)
    r, P, Q, LU, rrp, crp = factor(ctx, Ad, cfg.p, form)
    # the oracle's rank profile matrix, rank and profiles, in full
    assert r == int(gold["rank"][0])
    check_rpm_from_pq(P, Q, r, set(zip(gold["piv_rows"].tolist(), gold["piv_cols"].tolist())))
    assert rrp == gold["rrp"].tolist() and crp == gold["crp"].tolist()
    check_structure(LU, r)
    # factor identity: exact library product on the GPU (limb form; the FP64
    # form takes the host check alone) and 3-trial Freivalds on the host
    if form == "limb":
        exact_identity_gpu(Ad, cfg.p, P, Q, LU, r)
    LU_host = LU.cpu().numpy().view(np.uint32)
    del LU
    torch.cuda.empty_cache()
    freivalds_host(A, cfg.p, P, Q, LU_host, r, trials=3)


# --------------------------------- 16384 x 20480 rank 16320 over 2^31 - 1 --

@pytest.mark.parametrize("form", ["limb", "fp64"])
def test_lru_16384x20480_p31(ctx, form):
    cfg = workloads.CONFIGS["lru-16384x20480-r16320-p2147483647"]
    g = workloads.prescribed_rank_matrix(cfg.m, cfg.n, cfg.r, cfg.p, seed=1, device="cuda")
    Ad = to_dev(g.A)
    r, P, Q, LU, rrp, crp = factor(ctx, Ad, cfg.p, form)
    assert r == cfg.r
    check_rpm_from_pq(P, Q, r, g.rpm)
    assert rrp == g.rrp.tolist() and crp == g.crp.tolist()
    check_structure(LU, r)
    if form == "limb":
        exact_identity_gpu(Ad, cfg.p, P, Q, LU, r)
    LU_host = LU.cpu().numpy().view(np.uint32)
    del LU
    torch.cuda.empty_cache()
    freivalds_host(g.A, cfg.p, P, Q, LU_host, r, trials=3)


# ------------------------------------------------- batch of 4096 matrices --

def test_batched_4096(ctx):
    cfg = workloads.CONFIGS["batched-4096-lru-p65521"]
    p = cfg.p
    ms, ns, rs = workloads.batched_shapes(cfg.count, cfg.lo, cfg.hi, seed=1)
    gens = [workloads.prescribed_rank_matrix(int(ms[b]), int(ns[b]), int(rs[b]), p, seed=1,
                                             tag=f"batched:{b}", device="cuda")
            for b in range(cfg.count)]
    As = [to_dev(g.A) for g in gens]
    ranks, Ps, Qs = pq.pluq_modp_batched(As, p, ctx=ctx)
    torch.cuda.synchronize()
    rr_in = [to_dev(g.A) for g in gens]
    ranks2, rrps, crps = pq.rank_profile_modp_batched(rr_in, p, ctx=ctx)
    torch.cuda.synchronize()
    for b, g in enumerate(gens):
        r = ranks[b]
        assert r == g.rank == ranks2[b], b
        P, Q = Ps[b].cpu().numpy(), Qs[b].cpu().numpy()
        check_rpm_from_pq(P, Q, r, g.rpm)
        assert rrps[b].cpu().tolist() == g.rrp.tolist(), b
        assert crps[b].cpu().tolist() == g.crp.tolist(), b
        LU = As[b].cpu().numpy().astype(np.int64)
        assert not np.any(LU[r:, r:]) and np.all(np.diag(LU[:r, :r]) != 0), b
        # L U = A[P][:, Q] exactly: float64 sums of at most 512 products < 2^32
        L = np.tril(LU[:, :r], -1).astype(np.float64)
        L[np.arange(r), np.arange(r)] = 1.0
        U = np.triu(LU[:r, :]).astype(np.float64)
        assert np.array_equal(np.mod(L @ U, p).astype(np.int64),
                              g.A.astype(np.int64)[P][:, Q]), b
        if b % 8 == 0:
            ref = oracle.pluq(g.A, p, want_lu=False)
            assert ref.rank == r and ref.rpm == g.rpm, b
