"""Bit-exact parity of the CUDA path on the five workloads at their full sizes.

For every seeded input: rank, the rank profile matrix (pivots of P and Q), both
sorted rank profiles, the factor identity P L U Q = A mod p and the storage
structure; the reduced echelon form where the oracle can produce it.  What
decides each case:

  * uniform 1024^2 over GF(131071), seeds 1-3: the CPU oracle (rank profile
    matrix, profiles, RREF) and an exact host product for the factor identity;
  * 8192^2 rank 4096 over GF(131071), seeds 1-3: the L R U construction, whose
    rank profile matrix is R (Sec. 4.1), an exact float64 host product of L U
    (every partial sum below 2^53) for both forms, and the oracle's RREF (seed 1,
    compared through the SHA-256 digest its writer script stores);
  * uniform 32768^2 over GF(65521): the oracle's rank profile matrix stored by
    tests/golden/make_oracle_goldens.py, the exact product L U on 4096 sampled
    rows computed with cuBLAS float64 on the GPU (a library product,
    independent of this library's kernels), and a 3-trial Freivalds check of
    the whole identity on the host, both forms;
  * 16384 x 20480 rank 16320 over GF(2^31 - 1): the construction, the exact
    GPU product on 2048 sampled rows (16-bit halves) and 3-trial Freivalds,
    both forms;
  * the batch of 4096 matrices (m, n uniform in [32, 512], p = 65521): the
    construction for every matrix, L U = the permuted A exactly for every
    matrix, and the oracle on every 8th matrix.
"""
import os

import numpy as np
import pytest

import oracle
import workloads
from pluq_checks import check_pluq, check_rpm_from_pq, exact_identity, freivalds

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


def _lu_rows_f64(LU, r, sel):
    """The rows `sel` (device int64) of the unit lower trapezoidal L (m x r) as
    float64 (device)."""
    Lb = LU[sel, :r].to(torch.float64)
    rows = sel[:, None]
    cols = torch.arange(r, device=LU.device)[None, :]
    Lb = torch.where(cols < rows, Lb, torch.zeros_like(Lb))
    return Lb + (cols == rows).to(torch.float64)


def sample_rows(m, count, seed):
    """`count` distinct rows of [0, m), seeded, always with the first and last."""
    rng = np.random.default_rng(seed)
    rows = rng.choice(m, size=min(m, count), replace=False)
    return np.unique(np.concatenate([rows, [0, m - 1]]))


def exact_identity_gpu(A_dev, p, P, Q, LU, r, rows, block=4096):
    """A[P][:, Q] == L U mod p entry by entry on the given rows of the permuted
    frame, with cuBLAS float64 products (a library product, independent of this
    library's kernels).

    Every float64 product of integers is exact while its sums stay below 2^53:
    r (p-1)^2 < 2^53 for p < 2^17 and r <= 2^19; larger p are split into 16-bit
    halves (four products, each sum below r 2^32).
    """
    m, n = A_dev.shape
    dev = A_dev.device
    Pt = torch.from_numpy(P.astype(np.int64)).to(dev)
    Qt = torch.from_numpy(Q.astype(np.int64)).to(dev)
    sel_all = torch.from_numpy(np.sort(np.asarray(rows, dtype=np.int64))).to(dev)
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
    for i0 in range(0, len(sel_all), block):
        sel = sel_all[i0:i0 + block]
        Lb = _lu_rows_f64(LU, r, sel)
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
        want = A_dev[Pt[sel]][:, Qt].to(torch.int64) % (1 << 32)
        assert torch.equal(got, want), f"P L U Q != A in sampled rows from {i0}"


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
    exact_identity(g.A, cfg.p, P, Q, LU.cpu().numpy().view(np.uint32), r)


def test_lru_8192_rref(ctx):
    """The reduced echelon form at full size equals the oracle's, byte for byte
    (its SHA-256 as stored by tests/golden/make_oracle_goldens.py --rref), in
    both forms, and satisfies the properties that fix it: R[:, CRP] = I, zeros
    left of each pivot, A = A[:, CRP] R mod p (checked on sampled rows)."""
    import hashlib
    cfg = workloads.CONFIGS["lru-8192-r4096-p131071"]
    path = os.path.join(GOLDEN, "oracle_rref_lru-8192-r4096-p131071_seed1.npz")
    assert os.path.exists(path), "oracle RREF digest of the 8192^2 workload is missing"
    gold = np.load(path)
    g = workloads.prescribed_rank_matrix(cfg.m, cfg.n, cfg.r, cfg.p, seed=1, device="cuda")
    assert hashlib.sha256(g.A.tobytes()).hexdigest() == str(gold["input_sha256"][0])
    Ad = to_dev(g.A)
    for form in ("limb", "fp64"):
        r, R, crp = pq.echelon_modp(Ad, cfg.p, form=form, ctx=ctx)
        torch.cuda.synchronize()
        assert r == int(gold["rank"][0]) == cfg.r
        assert crp.cpu().tolist() == g.crp.tolist() == gold["crp"].tolist()
        Rh = np.ascontiguousarray(R.cpu().numpy().view(np.uint32))
        assert hashlib.sha256(Rh.tobytes()).hexdigest() == str(gold["sha256"][0]), form
    # properties of the form (independent of the oracle)
    c = g.crp
    assert np.array_equal(Rh[:, c], np.eye(r, dtype=np.uint32))
    first = np.argmax(Rh != 0, axis=1)
    assert np.array_equal(first, c)
    rows = sample_rows(cfg.m, 512, 5)
    from pluq_checks import matmul_mod_f64
    got = matmul_mod_f64(g.A[rows][:, c].astype(np.int64), Rh.astype(np.int64), cfg.p)
    assert np.array_equal(got, g.A[rows].astype(np.int64))


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
    # factor identity: exact library product on the GPU over 4096 sampled rows
    # of the permuted frame, and 3-trial Freivalds over all of it on the host
    exact_identity_gpu(Ad, cfg.p, P, Q, LU, r, sample_rows(cfg.m, 4096, 3))
    LU_host = LU.cpu().numpy().view(np.uint32)
    del LU
    torch.cuda.empty_cache()
    freivalds(A, cfg.p, P, Q, LU_host, r, trials=3)


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
    exact_identity_gpu(Ad, cfg.p, P, Q, LU, r, sample_rows(cfg.m, 2048, 4))
    LU_host = LU.cpu().numpy().view(np.uint32)
    del LU
    torch.cuda.empty_cache()
    freivalds(g.A, cfg.p, P, Q, LU_host, r, trials=3)


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
