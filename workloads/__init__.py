"""Seeded synthetic inputs shaped like the paper's workloads.

This module serves both the CUDA path's tests/benchmark and the CPU oracle; it
holds none of the factorization's arithmetic.  Inputs are drawn with
SplitMix64 (S. Vigna's published generator, one counter per element) and
mapped to [0, p) by a 64-bit multiply-shift (bias below p / 2^64).

Two matrix families, after the paper's experiments:
  * dense uniform residues, full rank with high probability (Sec. 3, Table 3);
  * prescribed rank with random row and column rank profiles, like the S16K
    matrix of Sec. 4.1 whose independent rows and columns are spread
    uniformly: A = L R U with L unit lower triangular, U unit upper
    triangular (entries below / above the diagonal uniform) and R an
    r-permutation matrix.  Leading blocks satisfy
    A[:i,:j] = L[:i,:i] R[:i,:j] U[:j,:j] with invertible triangular factors,
    so the rank profile matrix of A is R exactly.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied elementwise (uint64, wrapping)."""
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _fnv1a64(text: str) -> int:
    h = 0xCBF29CE484222325
    for b in text.encode():
        h ^= b
        h = (h * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h


class Stream:
    """Counter-based SplitMix64 stream keyed by (seed, tag)."""

    def __init__(self, seed: int, tag: str):
        base = (_fnv1a64(tag) ^ ((int(seed) * 0xD1B54A32D192ED03) & 0xFFFFFFFFFFFFFFFF))
        self.state = np.uint64(base & 0xFFFFFFFFFFFFFFFF)
        self.counter = 0

    def u64(self, count: int) -> np.ndarray:
        idx = np.arange(self.counter + 1, self.counter + 1 + count, dtype=np.uint64)
        self.counter += count
        with np.errstate(over="ignore"):
            return _mix(self.state + idx * _GAMMA)

    def below(self, bound: int, count: int) -> np.ndarray:
        """count integers uniform in [0, bound) (bound < 2^32), as uint64."""
        z = self.u64(count)
        b = np.uint64(bound)
        hi = z >> np.uint64(32)
        lo = z & np.uint64(0xFFFFFFFF)
        with np.errstate(over="ignore"):
            return (hi * b + ((lo * b) >> np.uint64(32))) >> np.uint64(32)

    def subset(self, universe: int, k: int) -> np.ndarray:
        """Sorted uniformly random k-subset of range(universe)."""
        keys = self.u64(universe)
        return np.sort(np.argsort(keys, kind="stable")[:k]).astype(np.int64)

    def permutation(self, k: int) -> np.ndarray:
        return np.argsort(self.u64(k), kind="stable").astype(np.int64)


def uniform_matrix(m: int, n: int, p: int, seed: int, tag: str = "uniform") -> np.ndarray:
    """m x n residues i.i.d. uniform in [0, p), uint32 row-major.

    Drawn in row blocks (one counter sequence), so large matrices need no
    64-bit temporaries of their full size.
    """
    s = Stream(seed, f"{tag}:{m}x{n}:p{p}")
    out = np.empty((m, n), dtype=np.uint32)
    rows = max(1, (1 << 24) // max(n, 1))
    for r0 in range(0, m, rows):
        r1 = min(m, r0 + rows)
        out[r0:r1] = s.below(p, (r1 - r0) * n).astype(np.uint32).reshape(r1 - r0, n)
    return out


@dataclass
class PrescribedRank:
    A: np.ndarray          # uint32 m x n
    rows: np.ndarray       # int64, rank profile matrix rows (sorted, = row rank profile)
    cols: np.ndarray       # int64, column of the pivot in each of those rows
    p: int

    @property
    def rank(self) -> int:
        return int(self.rows.shape[0])

    @property
    def rrp(self) -> np.ndarray:
        return self.rows

    @property
    def crp(self) -> np.ndarray:
        return np.sort(self.cols)

    @property
    def rpm(self) -> set:
        return set(zip(self.rows.tolist(), self.cols.tolist()))


def _matmul_mod(X: np.ndarray, Y: np.ndarray, p: int, device=None) -> np.ndarray:
    """X @ Y mod p for uint64 residues, exact via float64 products.

    Each float64 product is exact while k * max|x| * max|y| < 2^53; larger
    moduli are split into 16-bit halves first.  ``device`` (a torch device)
    runs the float64 products with torch instead of numpy; the result is the
    same exact integer matrix.
    """
    k = X.shape[1]

    def fmm(a, b):
        if device is None:
            return a.astype(np.float64) @ b.astype(np.float64)
        import torch
        ta = torch.from_numpy(a.astype(np.float64)).to(device)
        tb = torch.from_numpy(b.astype(np.float64)).to(device)
        return (ta @ tb).cpu().numpy()

    def exact_mod(f):
        return np.mod(f.astype(np.int64), p).astype(np.uint64)

    if k * (p - 1) ** 2 < 2 ** 53:
        return exact_mod(fmm(X, Y))
    assert k * (2 ** 16 - 1) ** 2 < 2 ** 53, "inner dimension too large"
    mask = np.uint64(0xFFFF)
    Xh, Xl = X >> np.uint64(16), X & mask
    Yh, Yl = Y >> np.uint64(16), Y & mask
    hh = exact_mod(fmm(Xh, Yh))
    mid = (exact_mod(fmm(Xh, Yl)) + exact_mod(fmm(Xl, Yh))) % np.uint64(p)
    ll = exact_mod(fmm(Xl, Yl))
    c16 = np.uint64(pow(2, 16, p))
    c32 = np.uint64(pow(2, 32, p))
    return ((hh * c32) % np.uint64(p) + (mid * c16) % np.uint64(p) + ll) % np.uint64(p)


def prescribed_rank_matrix(m: int, n: int, r: int, p: int, seed: int,
                           tag: str = "lru", device=None) -> PrescribedRank:
    """A = L R U with a random r-permutation matrix R (see module docstring).

    Only the r columns of L and rows of U that R selects matter:
    A = sum_k L[:, i_k] U[j_k, :], with L[:, i] zero above i, one at i and
    uniform below; U[j, :] zero left of j, one at j and uniform right of it.
    """
    assert 0 <= r <= min(m, n)
    s = Stream(seed, f"{tag}:{m}x{n}:r{r}:p{p}")
    rows = s.subset(m, r)
    cols_sorted = s.subset(n, r)
    cols = cols_sorted[s.permutation(r)]
    if r == 0:
        return PrescribedRank(np.zeros((m, n), np.uint32), rows, cols, p)
    Lsel = s.below(p, m * r).reshape(m, r)
    ii = np.arange(m)[:, None]
    Lsel[ii < rows[None, :]] = 0
    Lsel[rows, np.arange(r)] = 1
    Usel = s.below(p, r * n).reshape(r, n)
    jj = np.arange(n)[None, :]
    Usel[jj < cols[:, None]] = 0
    Usel[np.arange(r), cols] = 1
    A = _matmul_mod(Lsel, Usel, p, device=device).astype(np.uint32)
    return PrescribedRank(A, rows, cols, p)


@dataclass
class Config:
    key: str
    kind: str            # "uniform" | "lru" | "batched"
    m: int
    n: int
    p: int
    r: int | None = None
    count: int = 1
    lo: int = 0
    hi: int = 0


# The workloads the measurements and parity tests are quoted on.
CONFIGS = {
    "uniform-1024-p131071": Config("uniform-1024-p131071", "uniform", 1024, 1024, 131071),
    "lru-8192-r4096-p131071": Config("lru-8192-r4096-p131071", "lru", 8192, 8192, 131071, r=4096),
    "uniform-32768-p65521": Config("uniform-32768-p65521", "uniform", 32768, 32768, 65521),
    "lru-16384x20480-r16320-p2147483647": Config("lru-16384x20480-r16320-p2147483647", "lru",
                                                 16384, 20480, 2147483647, r=16320),
    "batched-4096-lru-p65521": Config("batched-4096-lru-p65521", "batched", 512, 512, 65521,
                                      count=4096, lo=32, hi=512),
}


def batched_shapes(count: int, lo: int, hi: int, seed: int, tag: str = "batched"):
    """(m, n, r) per matrix: m, n uniform in [lo, hi], r uniform in [1, min(m, n)]."""
    s = Stream(seed, f"{tag}:shapes:{count}:{lo}:{hi}")
    m = s.below(hi - lo + 1, count).astype(np.int64) + lo
    n = s.below(hi - lo + 1, count).astype(np.int64) + lo
    u = s.below(2 ** 31, count).astype(np.int64)
    r = 1 + (u % np.minimum(m, n))
    return m, n, r


def batched_matrices(count: int, lo: int, hi: int, p: int, seed: int, tag: str = "batched"):
    """List of PrescribedRank matrices for the batched workload."""
    ms, ns, rs = batched_shapes(count, lo, hi, seed, tag)
    return [prescribed_rank_matrix(int(ms[b]), int(ns[b]), int(rs[b]), p, seed,
                                   tag=f"{tag}:{b}") for b in range(count)]
