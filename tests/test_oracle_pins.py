"""Pins of the CPU oracle against what the paper and the mathematics fix.

The oracle is plain row-by-row elimination mod p (Sec. 4.1 row-major pivot
search, Sec. 3.1 delayed reduction).  Each test below checks it against
something other than itself:
  * brute force: rank = largest non-vanishing minor, rank profile matrix from
    the ranks of all leading blocks (definition, Sec. 4.1), on <= 6 x 6;
  * exhaustive enumeration of all 2x2, 2x3, 3x2, 3x3 matrices over GF(2),
    GF(3), GF(5) against closed-form leading-block ranks;
  * closed forms: identity, zero, rank one u v^T, permutation matrices,
    Vandermonde, L.R.U constructions (rank profile matrix = R by
    construction);
  * a library routine: sympy's RREF and rank over GF(p);
  * planted mistakes: every mutation of the oracle fails at least one pin.
"""
import numpy as np
import pytest

import oracle
import workloads
from pluq_checks import (brute_rank, brute_rpm, check_pluq, check_rpm_from_pq, check_rref,
                         matmul_mod, rpm_from_leading_ranks)

PRIMES = [2, 3, 5, 7, 251, 65521, 131071, 2147483647]


def _rand(rng, m, n, p):
    return rng.integers(0, p, size=(m, n), dtype=np.int64).astype(np.uint32)


def _low_rank(rng, m, n, r, p):
    X = rng.integers(0, p, size=(m, r), dtype=np.int64)
    Y = rng.integers(0, p, size=(r, n), dtype=np.int64)
    return matmul_mod(X, Y, p).astype(np.uint32)


def _sparse(rng, m, n, p, density=0.3):
    A = _rand(rng, m, n, p)
    A[rng.random((m, n)) > density] = 0
    return A


def _check_all(A, p, res):
    check_pluq(A, p, res.P, res.Q, res.LU, res.rank)
    check_rpm_from_pq(res.P, res.Q, res.rank, res.rpm)
    assert res.rrp.tolist() == sorted(res.piv_rows.tolist())
    assert res.crp.tolist() == sorted(res.piv_cols.tolist())


@pytest.mark.parametrize("p", PRIMES)
def test_brute_force_minors(p):
    rng = np.random.default_rng(1000 + p % 1000)
    cases = []
    for m in range(1, 7):
        for n in range(1, 7):
            if m * n > 25 and p > 7:
                continue
            cases.append(_rand(rng, m, n, p))
            cases.append(_low_rank(rng, m, n, max(1, min(m, n) // 2), p))
            cases.append(_sparse(rng, m, n, p))
    for A in cases:
        res = oracle.pluq(A, p)
        assert res.rank == brute_rank(A, p)
        assert res.rpm == brute_rpm(A, p)
        _check_all(A, p, res)


def _leading_ranks_tiny(As: np.ndarray, p: int):
    """Vectorised ranks of every leading block of many <= 3 x 3 matrices."""
    count, m, n = As.shape
    A = As.astype(np.int64)

    def rank_block(i, j):
        B = A[:, :i, :j]
        rk = np.zeros(count, dtype=np.int64)
        rk[np.any(B.reshape(count, -1) % p != 0, axis=1)] = 1
        if min(i, j) >= 2:
            for r0, r1 in [(a, b) for a in range(i) for b in range(a + 1, i)]:
                for c0, c1 in [(a, b) for a in range(j) for b in range(a + 1, j)]:
                    d = (B[:, r0, c0] * B[:, r1, c1] - B[:, r0, c1] * B[:, r1, c0]) % p
                    rk[(d != 0) & (rk < 2)] = 2
        if min(i, j) >= 3:
            M = B[:, :3, :3]
            d = (M[:, 0, 0] * (M[:, 1, 1] * M[:, 2, 2] - M[:, 1, 2] * M[:, 2, 1])
                 - M[:, 0, 1] * (M[:, 1, 0] * M[:, 2, 2] - M[:, 1, 2] * M[:, 2, 0])
                 + M[:, 0, 2] * (M[:, 1, 0] * M[:, 2, 1] - M[:, 1, 1] * M[:, 2, 0])) % p
            rk[d != 0] = 3
        return rk

    rk = np.zeros((count, m + 1, n + 1), dtype=np.int64)
    for i in range(1, m + 1):
        for j in range(1, n + 1):
            rk[:, i, j] = rank_block(i, j)
    return rk


@pytest.mark.parametrize("p", [2, 3, 5])
@pytest.mark.parametrize("shape", [(2, 2), (2, 3), (3, 2), (3, 3)])
def test_exhaustive_tiny(p, shape):
    m, n = shape
    count = p ** (m * n)
    idx = np.arange(count, dtype=np.int64)
    digits = np.stack([(idx // p ** k) % p for k in range(m * n)], axis=1)
    As = digits.reshape(count, m, n).astype(np.uint32)
    ranks, pr, pc = oracle.pluq_batch(As, p)
    rk = _leading_ranks_tiny(As, p)
    assert np.array_equal(ranks, rk[:, m, n])
    # rank profile matrix from the leading-block ranks, as a dense 0/1 array
    R = rk[:, 1:, 1:] - rk[:, :-1, 1:] - rk[:, 1:, :-1] + rk[:, :-1, :-1]
    assert set(np.unique(R).tolist()) <= {0, 1}
    got = np.zeros((count, m, n), dtype=np.int64)
    b_idx, k_idx = np.nonzero(pr >= 0)
    got[b_idx, pr[b_idx, k_idx], pc[b_idx, k_idx]] = 1
    assert np.array_equal(got, R)


@pytest.mark.parametrize("p", [3, 131071, 2147483647])
@pytest.mark.parametrize("n", [1, 7, 64])
def test_identity_zero_permutation(p, n):
    I = np.eye(n, dtype=np.uint32)
    res = oracle.pluq(I, p)
    assert res.rank == n and res.rpm == {(i, i) for i in range(n)}
    r, R = oracle.rref(I, p)
    assert r == n and np.array_equal(R, I)
    Z = np.zeros((n, n + 3), dtype=np.uint32)
    res = oracle.pluq(Z, p)
    assert res.rank == 0 and res.P.tolist() == list(range(n)) and res.Q.tolist() == list(range(n + 3))
    rng = np.random.default_rng(n)
    perm = rng.permutation(n)
    Pm = np.zeros((n, n), dtype=np.uint32)
    Pm[np.arange(n), perm] = 1
    res = oracle.pluq(Pm, p)
    assert res.rank == n and res.rpm == {(i, int(perm[i])) for i in range(n)}
    _check_all(Pm, p, res)


@pytest.mark.parametrize("p", [5, 65521, 2147483647])
def test_rank_one_outer_product(p):
    rng = np.random.default_rng(7)
    for m, n in [(1, 1), (5, 9), (40, 33)]:
        u = rng.integers(1, p, size=m, dtype=np.int64)
        v = rng.integers(1, p, size=n, dtype=np.int64)
        u[: m // 3] = 0
        v[: n // 2] = 0
        if not u.any():
            u[-1] = 1
        if not v.any():
            v[-1] = 1
        A = matmul_mod(u[:, None], v[None, :], p).astype(np.uint32)
        res = oracle.pluq(A, p)
        i0 = int(np.flatnonzero(u)[0])
        j0 = int(np.flatnonzero(v)[0])
        assert res.rank == 1 and res.rpm == {(i0, j0)}
        r, R = oracle.rref(A, p)
        expect = (v * pow(int(v[j0]), p - 2, p)) % p
        assert r == 1 and np.array_equal(R[0].astype(np.int64), expect)
        _check_all(A, p, res)


@pytest.mark.parametrize("p", [131071, 2147483647])
def test_vandermonde_generic_rank_profile(p):
    # distinct nodes: every leading minor is a Vandermonde determinant != 0
    n = 24
    x = np.arange(2, 2 + n, dtype=np.int64)
    V = np.array([[pow(int(xi), j, p) for j in range(n)] for xi in x], dtype=np.uint32)
    res = oracle.pluq(V, p)
    assert res.rank == n and res.rpm == {(i, i) for i in range(n)}
    _check_all(V, p, res)


@pytest.mark.parametrize("p", [2, 3, 131071, 65521, 2147483647])
@pytest.mark.parametrize("shape", [(1, 9), (9, 1), (17, 33), (64, 48), (150, 200)])
def test_prescribed_rank_profile(p, shape):
    m, n = shape
    for seed, frac in [(1, 0.5), (2, 1.0), (3, 0.1)]:
        r = max(0, int(min(m, n) * frac))
        g = workloads.prescribed_rank_matrix(m, n, r, p, seed)
        res = oracle.pluq(g.A, p)
        assert res.rank == r
        assert res.rpm == g.rpm
        assert res.rrp.tolist() == g.rrp.tolist()
        assert res.crp.tolist() == g.crp.tolist()
        _check_all(g.A, p, res)


@pytest.mark.parametrize("p", [3, 251, 131071])
def test_rref_against_sympy(p):
    sympy = pytest.importorskip("sympy")
    from sympy.polys.domains import GF
    from sympy.polys.matrices import DomainMatrix
    rng = np.random.default_rng(p)
    for m, n, r in [(12, 20, 7), (30, 25, 25), (25, 30, 3), (8, 8, 8)]:
        A = _low_rank(rng, m, n, r, p)
        dm = DomainMatrix([[GF(p)(int(v)) for v in row] for row in A.tolist()], (m, n), GF(p))
        Rs, pivots = dm.rref()
        Rs = np.array([[int(v) % p for v in row] for row in Rs.to_Matrix().tolist()],
                      dtype=np.int64)
        rank, R = oracle.rref(A, p)
        assert rank == len(pivots) == dm.rank()
        assert np.array_equal(R.astype(np.int64), Rs[:rank])
        res = oracle.pluq(A, p)
        assert res.crp.tolist() == list(pivots)
        check_rref(A, p, R, res.crp)


def test_delayed_reduction_bound_large_p():
    # p = 2^31 - 1: an int64 entry absorbs only two updates of (p-1)^2.
    p = 2147483647
    rng = np.random.default_rng(5)
    A = rng.integers(p - 50, p, size=(40, 40), dtype=np.int64).astype(np.uint32)
    res = oracle.pluq(A, p)
    _check_all(A, p, res)


def test_generator_determinism():
    a = workloads.uniform_matrix(33, 17, 131071, 1)
    b = workloads.uniform_matrix(33, 17, 131071, 1)
    c = workloads.uniform_matrix(33, 17, 131071, 2)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.max() < 131071
    g1 = workloads.prescribed_rank_matrix(40, 30, 12, 65521, 3)
    g2 = workloads.prescribed_rank_matrix(40, 30, 12, 65521, 3)
    assert np.array_equal(g1.A, g2.A) and g1.rpm == g2.rpm


def _pins_fail(mutation: int) -> bool:
    """Run a compact version of the pins against a mutated oracle."""
    checks = []
    rng = np.random.default_rng(11)
    for p in [3, 131071, 2147483647]:
        for m, n in [(5, 5), (6, 4), (4, 6)]:
            for A in (_rand(rng, m, n, p), _low_rank(rng, m, n, 2, p), _sparse(rng, m, n, p)):
                checks.append((A, p))
        # large entries exercise the delayed-reduction bound
        checks.append((rng.integers(p - 9, p, size=(24, 24), dtype=np.int64).astype(np.uint32), p))
    for A, p in checks:
        try:
            res = oracle.pluq(A, p, mutate=mutation)
            if res.rank != brute_rank(A, p) if A.shape[0] <= 6 else False:
                return True
            if A.shape[0] <= 6 and res.rpm != brute_rpm(A, p):
                return True
            _check_all(A, p, res)
            rank, R = oracle.rref(A, p, mutate=mutation)
            check_rref(A, p, R, res.crp)
        except (AssertionError, RuntimeError):
            return True
    return False


@pytest.mark.parametrize("name", sorted(oracle.MUTATIONS))
def test_planted_mistakes_are_caught(name):
    assert not _pins_fail(0)
    assert _pins_fail(oracle.MUTATIONS[name]), f"mutation {name} slipped through the pins"


def test_golden_hand_worked_example():
    from golden_io import load
    g = load("rpm_4x5_gf5.txt")
    res = oracle.pluq(g["A"], g["p"])
    assert res.rank == g["rank"] and res.rpm == g["rpm"]
    assert res.rrp.tolist() == g["rrp"] and res.crp.tolist() == g["crp"]
    r, R = oracle.rref(g["A"], g["p"])
    assert np.array_equal(R, g["rref"])
