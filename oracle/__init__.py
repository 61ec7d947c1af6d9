"""CPU oracle for rank-profile-revealing PLUQ over GF(p) (test infrastructure).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it, and
it shares no code with the CUDA path.

The arithmetic lives in ``pluq_oracle.c`` (plain row-by-row Gaussian
elimination mod p in int64 with delayed reduction, Sec. 3.1 and Sec. 4.1 of
Dumas, Gautier, Pernet, Sultan, arXiv:1402.3501).  This module compiles it
with gcc and marshals numpy arrays through ctypes; it adds no arithmetic.

Pins (in ``tests/test_oracle_pins.py``): brute-force minors, exhaustive tiny
fields, closed forms, L.R.U constructions and a library RREF over GF(p).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pluq_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

# Planted-mistake codes understood by pluq_oracle.c (0 = correct algorithm).
MUTATIONS = {
    "last_nonzero_pivot": 1,
    "skip_last_row": 2,
    "sign": 3,
    "no_inverse": 4,
    "rref_no_normalise": 5,
    "transpose_input": 6,
    "crp_unsorted": 7,
    "no_reduction": 8,
}


def build(force: bool = False) -> str:
    """Compile pluq_oracle.c into liboracle.so (gcc, OpenMP) if stale."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        lib.oracle_pluq.argtypes = [ctypes.c_uint32, i64, i64, P, i64, P, P, P, P, i64,
                                    P, P, P, P, ctypes.c_int, ctypes.c_int]
        lib.oracle_pluq.restype = ctypes.c_int
        lib.oracle_rref.argtypes = [ctypes.c_uint32, i64, i64, P, i64, P, P, i64,
                                    ctypes.c_int, ctypes.c_int]
        lib.oracle_rref.restype = ctypes.c_int
        lib.oracle_pluq_batch.argtypes = [ctypes.c_uint32, i64, i64, i64, P, P, P, P,
                                          ctypes.c_int]
        lib.oracle_pluq_batch.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class PLUQ:
    rank: int
    P: np.ndarray        # int32, length m: (P^T A)[t,:] = A[P[t],:]
    Q: np.ndarray        # int32, length n: (A Q^T)[:,u] = A[:,Q[u]]
    LU: np.ndarray       # uint32 m x n, compressed L\U in the (P, Q) frame
    piv_rows: np.ndarray  # int32, length r: rank profile matrix rows
    piv_cols: np.ndarray  # int32, length r: rank profile matrix columns
    rrp: np.ndarray      # int32 sorted row rank profile
    crp: np.ndarray      # int32 sorted column rank profile

    @property
    def rpm(self) -> set:
        """Rank profile matrix as a set of (row, column) pairs."""
        return set(zip(self.piv_rows.tolist(), self.piv_cols.tolist()))


def pluq(A: np.ndarray, p: int, threads: int = 0, mutate: int = 0,
         want_lu: bool = True) -> PLUQ:
    """Row-by-row elimination of A (uint32, entries in [0,p)) over GF(p)."""
    lib = _load()
    A = np.ascontiguousarray(A, dtype=np.uint32)
    m, n = A.shape
    rmax = min(m, n)
    rank = np.zeros(1, dtype=np.int64)
    P = np.zeros(max(m, 1), dtype=np.int32)
    Q = np.zeros(max(n, 1), dtype=np.int32)
    LU = np.zeros((m, n), dtype=np.uint32) if want_lu else None
    pr = np.zeros(max(rmax, 1), dtype=np.int32)
    pc = np.zeros(max(rmax, 1), dtype=np.int32)
    rrp = np.zeros(max(rmax, 1), dtype=np.int32)
    crp = np.zeros(max(rmax, 1), dtype=np.int32)
    st = lib.oracle_pluq(int(p), m, n, _ptr(A), max(n, 1), _ptr(rank), _ptr(P), _ptr(Q),
                         _ptr(LU), max(n, 1), _ptr(pr), _ptr(pc), _ptr(rrp), _ptr(crp),
                         int(threads), int(mutate))
    if st != 0:
        raise RuntimeError(f"oracle_pluq failed with status {st}")
    r = int(rank[0])
    return PLUQ(r, P[:m].copy(), Q[:n].copy(),
                LU if LU is not None else np.zeros((0, 0), np.uint32),
                pr[:r].copy(), pc[:r].copy(), rrp[:r].copy(), crp[:r].copy())


def rref(A: np.ndarray, p: int, threads: int = 0, mutate: int = 0) -> tuple[int, np.ndarray]:
    """Reduced row echelon form (rank, r x n uint32) of A over GF(p)."""
    lib = _load()
    A = np.ascontiguousarray(A, dtype=np.uint32)
    m, n = A.shape
    rmax = min(m, n)
    rank = np.zeros(1, dtype=np.int64)
    R = np.zeros((max(rmax, 1), max(n, 1)), dtype=np.uint32)
    st = lib.oracle_rref(int(p), m, n, _ptr(A), max(n, 1), _ptr(rank), _ptr(R), max(n, 1),
                         int(threads), int(mutate))
    if st != 0:
        raise RuntimeError(f"oracle_rref failed with status {st}")
    r = int(rank[0])
    return r, R[:r, :n].copy()


def pluq_batch(As: np.ndarray, p: int, mutate: int = 0):
    """Pivots of many tiny matrices (count x m x n): ranks, piv_rows, piv_cols."""
    lib = _load()
    As = np.ascontiguousarray(As, dtype=np.uint32)
    count, m, n = As.shape
    rmax = min(m, n)
    ranks = np.zeros(count, dtype=np.int64)
    pr = np.zeros((count, rmax), dtype=np.int32)
    pc = np.zeros((count, rmax), dtype=np.int32)
    st = lib.oracle_pluq_batch(int(p), count, m, n, _ptr(As), _ptr(ranks), _ptr(pr), _ptr(pc),
                               int(mutate))
    if st != 0:
        raise RuntimeError(f"oracle_pluq_batch failed with status {st}")
    return ranks, pr, pc
