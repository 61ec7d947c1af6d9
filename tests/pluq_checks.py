"""Definition-level checks of a PLUQ / echelon result over GF(p) (test helpers).

Independent of both the CPU oracle and the CUDA path: every check restates a
definition (A = P L U Q with L unit lower and U upper trapezoidal, Sec. 2.1;
rank profiles and the rank profile matrix, Sec. 4.1; the reduced echelon form)
using plain Python/numpy integer arithmetic.
"""
from __future__ import annotations

import itertools

import numpy as np


def matmul_mod(X: np.ndarray, Y: np.ndarray, p: int) -> np.ndarray:
    """Exact X @ Y mod p for residues in [0, p): 16-bit halves, int64 sums."""
    X = np.asarray(X, dtype=np.int64)
    Y = np.asarray(Y, dtype=np.int64)
    k = X.shape[1]
    if k == 0:
        return np.zeros((X.shape[0], Y.shape[1]), dtype=np.int64)
    if (p - 1) ** 2 * k < 2 ** 62:
        # chunk the inner dimension so that every partial sum stays < 2^63
        out = np.zeros((X.shape[0], Y.shape[1]), dtype=np.int64)
        step = max(1, (2 ** 62) // max(1, (p - 1) ** 2))
        for s in range(0, k, step):
            out = (out + (X[:, s:s + step] @ Y[s:s + step, :]) % p) % p
        return out
    Xh, Xl = X >> 16, X & 0xFFFF
    Yh, Yl = Y >> 16, Y & 0xFFFF
    c16, c32 = pow(2, 16, p), pow(2, 32, p)

    def mm(a, b):
        out = np.zeros((a.shape[0], b.shape[1]), dtype=np.int64)
        step = 1 << 20
        for s in range(0, k, step):
            out = (out + (a[:, s:s + step] @ b[s:s + step, :]) % p) % p
        return out

    hh, hl, lh, ll = mm(Xh, Yh), mm(Xh, Yl), mm(Xl, Yh), mm(Xl, Yl)
    return ((hh * c32) % p + ((hl + lh) % p * c16) % p + ll) % p


def split_lu(LU: np.ndarray, r: int):
    """Compressed L\\U (m x n) -> L (m x r, unit lower), U (r x n, upper)."""
    LU = np.asarray(LU, dtype=np.int64)
    m, n = LU.shape
    L = np.tril(LU[:, :r], k=-1)
    L[np.arange(r), np.arange(r)] = 1
    U = np.triu(LU[:r, :], k=0)
    return L, U


def check_pluq(A: np.ndarray, p: int, P, Q, LU, r: int) -> None:
    """Assert A = P L U Q mod p with the storage conventions of the library.

    (P^T A)[t,:] = A[P[t],:], (A Q^T)[:,u] = A[:,Q[u]]; L unit lower
    trapezoidal m x r, U upper trapezoidal r x n with non-zero diagonal,
    trailing (m-r) x (n-r) block of the compressed storage zero.
    """
    A = np.asarray(A, dtype=np.int64)
    m, n = A.shape
    P = np.asarray(P, dtype=np.int64)
    Q = np.asarray(Q, dtype=np.int64)
    LU = np.asarray(LU, dtype=np.int64)
    assert sorted(P.tolist()) == list(range(m)), "P is not a permutation"
    assert sorted(Q.tolist()) == list(range(n)), "Q is not a permutation"
    assert LU.shape == (m, n)
    assert 0 <= r <= min(m, n)
    assert np.all((LU >= 0) & (LU < p)), "entries outside [0, p)"
    assert not np.any(LU[r:, r:]), "trailing block not zero"
    L, U = split_lu(LU, r)
    if r:
        assert np.all(np.diag(U[:, :r]) != 0), "U has a zero on its diagonal"
    B = A[P][:, Q]
    assert np.array_equal(matmul_mod(L, U, p), B % p), "P L U Q != A"


def check_rpm_from_pq(P, Q, r: int, rpm: set) -> None:
    """P [I_r 0; 0 0] Q equals the rank profile matrix given as pairs."""
    got = set(zip(np.asarray(P)[:r].tolist(), np.asarray(Q)[:r].tolist()))
    assert got == set(rpm), "pivots of P, Q differ from the rank profile matrix"


def det_mod(M: np.ndarray, p: int) -> int:
    """Determinant mod p by the Leibniz formula (tiny matrices only)."""
    k = M.shape[0]
    if k == 0:
        return 1
    total = 0
    for perm in itertools.permutations(range(k)):
        inv = sum(1 for a in range(k) for b in range(a + 1, k) if perm[a] > perm[b])
        prod = 1
        for i in range(k):
            prod = prod * int(M[i, perm[i]]) % p
        total += -prod if inv % 2 else prod
    return total % p


def brute_rank(M: np.ndarray, p: int) -> int:
    """Largest k with a non-zero k x k minor (definition of rank)."""
    M = np.asarray(M, dtype=np.int64) % p
    m, n = M.shape
    for k in range(min(m, n), 0, -1):
        for rows in itertools.combinations(range(m), k):
            for cols in itertools.combinations(range(n), k):
                if det_mod(M[np.ix_(rows, cols)], p):
                    return k
    return 0


def rpm_from_leading_ranks(rank_of, m: int, n: int) -> set:
    """Rank profile matrix from rk(i, j) = rank of the leading i x j block.

    R[i-1, j-1] = rk(i,j) - rk(i-1,j) - rk(i,j-1) + rk(i-1,j-1) (Sec. 4.1: the
    row and column rank profiles are read off the leading blocks).
    """
    rk = np.zeros((m + 1, n + 1), dtype=np.int64)
    for i in range(1, m + 1):
        for j in range(1, n + 1):
            rk[i, j] = rank_of(i, j)
    out = set()
    for i in range(1, m + 1):
        for j in range(1, n + 1):
            d = rk[i, j] - rk[i - 1, j] - rk[i, j - 1] + rk[i - 1, j - 1]
            assert d in (0, 1)
            if d:
                out.add((i - 1, j - 1))
    return out


def brute_rpm(A: np.ndarray, p: int) -> set:
    A = np.asarray(A, dtype=np.int64)
    m, n = A.shape
    return rpm_from_leading_ranks(lambda i, j: brute_rank(A[:i, :j], p), m, n)


def check_rref(A: np.ndarray, p: int, R: np.ndarray, crp) -> None:
    """R is the reduced echelon form of A with pivot columns crp.

    R[:, crp] = I_r, each row is zero left of its pivot, and
    A = A[:, crp] R mod p.  A[:, crp] has full column rank, so these
    properties fix R uniquely.
    """
    A = np.asarray(A, dtype=np.int64)
    R = np.asarray(R, dtype=np.int64)
    crp = np.asarray(crp, dtype=np.int64)
    r = len(crp)
    assert R.shape == (r, A.shape[1])
    assert np.array_equal(R[:, crp], np.eye(r, dtype=np.int64)), "R[:, crp] != I"
    for t in range(r):
        assert not np.any(R[t, :crp[t]]), "non-zero left of a pivot"
    assert np.array_equal(matmul_mod(A[:, crp], R, p), A % p), "A != A[:, crp] R"


def _split16(X: np.ndarray, p: int):
    """X as a list of (weight mod p, float64 part) with every part below 2^16 when
    p >= 2^20 (16-bit halves), else the whole of X."""
    X = np.asarray(X, dtype=np.int64)
    if p < 2 ** 20:
        return [(1, X.astype(np.float64))]
    return [(pow(2, 16, p), (X >> 16).astype(np.float64)), (1, (X & 0xFFFF).astype(np.float64))]


def matmul_mod_f64(X: np.ndarray, Y: np.ndarray, p: int) -> np.ndarray:
    """Exact X @ Y mod p by float64 BLAS products: operands split into 16-bit
    halves for p >= 2^20 so that every sum stays below 2^53 (inner dimension up
    to 2^20)."""
    k = np.asarray(X).shape[1]
    out = np.zeros((np.asarray(X).shape[0], np.asarray(Y).shape[1]), dtype=np.int64)
    for wx, xs in _split16(X, p):
        for wy, ys in _split16(Y, p):
            bound = float(xs.max(initial=0.0)) * float(ys.max(initial=0.0)) * k
            assert bound < 2.0 ** 53, "float64 sums would not be exact"
            part = np.mod(xs @ ys, p).astype(np.int64)
            out = (out + part * (wx * wy % p)) % p
    return out


def unit_lower_rows(LU: np.ndarray, r: int, i0: int, i1: int) -> np.ndarray:
    """Rows i0..i1 of the unit lower trapezoidal L (m x r) of a compressed L\\U."""
    rows = np.arange(i0, i1)
    Lb = np.where(np.arange(r)[None, :] < rows[:, None],
                  np.asarray(LU[i0:i1, :r], dtype=np.int64), 0)
    on_diag = rows < r
    Lb[np.nonzero(on_diag)[0], rows[on_diag]] = 1
    return Lb


def freivalds(A: np.ndarray, p: int, P, Q, LU: np.ndarray, r: int, trials: int = 3,
              seed: int = 0, step: int = 2048) -> None:
    """Freivalds' test of A[P][:, Q] = L U mod p with `trials` random vectors at once
    (a wrong factorization passes with probability at most p^-trials); exact
    float64 BLAS products, row blocks of `step` rows."""
    rng = np.random.default_rng(seed)
    m, n = A.shape
    P = np.asarray(P, dtype=np.int64)
    Q = np.asarray(Q, dtype=np.int64)
    X = rng.integers(0, p, (n, trials), dtype=np.int64)
    Z = np.zeros((n, trials), dtype=np.int64)
    Z[Q] = X  # (A Q^T) X = A Z
    AZ = np.concatenate([matmul_mod_f64(A[i:i + step], Z, p) for i in range(0, m, step)])
    lhs = AZ[P]
    UX = (np.concatenate([matmul_mod_f64(np.triu(np.asarray(LU[i:min(r, i + step)],
                                                            dtype=np.int64), i), X, p)
                          for i in range(0, r, step)]) if r else np.zeros((0, trials), np.int64))
    rhs = np.concatenate([matmul_mod_f64(unit_lower_rows(LU, r, i, min(m, i + step)), UX, p)
                          for i in range(0, m, step)])
    assert np.array_equal(lhs, rhs), "Freivalds check of P L U Q = A failed"


def exact_identity(A: np.ndarray, p: int, P, Q, LU: np.ndarray, r: int, rows=None,
                   step: int = 2048) -> None:
    """A[P][:, Q] = L U mod p entry by entry (exact float64 BLAS products), over
    every row or over the given rows of the permuted frame."""
    m, n = A.shape
    P = np.asarray(P, dtype=np.int64)
    Q = np.asarray(Q, dtype=np.int64)
    U = np.triu(np.asarray(LU[:r, :], dtype=np.int64))
    idx = np.arange(m) if rows is None else np.sort(np.asarray(rows, dtype=np.int64))
    for s in range(0, len(idx), step):
        sel = idx[s:s + step]
        Lb = np.concatenate([unit_lower_rows(LU, r, i, i + 1) for i in sel]) if rows is not None \
            else unit_lower_rows(LU, r, int(sel[0]), int(sel[-1]) + 1)
        got = matmul_mod_f64(Lb, U, p) if r else np.zeros((len(sel), n), np.int64)
        want = np.asarray(A, dtype=np.int64)[P[sel]][:, Q] % p
        assert np.array_equal(got, want), f"P L U Q != A in rows {sel[0]}..{sel[-1]}"
