"""Write the oracle's rank profile matrices of large workloads into tests/golden/.

Calls only the CPU oracle (oracle/) and the seeded input generators
(workloads/); nothing here touches the CUDA path.  The uniform 32768 x 32768
matrix over GF(65521) has no construction that fixes its rank profile matrix
(a leading block is singular with probability about 1 - (1 - 1/p)^n, roughly
0.39 at this size), so its pivots are recorded from a full oracle run: plain
row-by-row elimination with the row-major first-non-zero pivot search of
Sec. 4.1.  That run takes hours on a few cores and is done once.

Output: <key>_seed<s>.npz with arrays rank (1), piv_rows, piv_cols (int32, in
the oracle's processing order), rrp, crp (sorted) and the input's shape, p and
seed, plus a SHA-256 of the input bytes so a test can tell that the matrix it
regenerates is the one that was factored.

  python tests/golden/make_oracle_goldens.py [--threads T] [--key KEY] [--seed S]
  python tests/golden/make_oracle_goldens.py --rref --key lru-8192-r4096-p131071

--rref instead records the oracle's reduced row echelon form of a prescribed-rank
workload as a digest (rank, pivot columns, SHA-256 of its bytes).
"""
from __future__ import annotations

import argparse
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads  # noqa: E402


def golden_path(key: str, seed: int) -> str:
    return os.path.join(HERE, f"oracle_rpm_{key}_seed{seed}.npz")


def input_digest(A: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(A, dtype=np.uint32).tobytes()).hexdigest()


def write(key: str, seed: int, threads: int) -> str:
    cfg = workloads.CONFIGS[key]
    assert cfg.kind == "uniform", "prescribed-rank workloads are fixed by their construction"
    A = workloads.uniform_matrix(cfg.m, cfg.n, cfg.p, seed)
    t = time.time()
    ref = oracle.pluq(A, cfg.p, threads=threads, want_lu=False)
    dt = time.time() - t
    out = golden_path(key, seed)
    np.savez_compressed(
        out, rank=np.array([ref.rank], np.int64), piv_rows=ref.piv_rows.astype(np.int32),
        piv_cols=ref.piv_cols.astype(np.int32), rrp=ref.rrp.astype(np.int32),
        crp=ref.crp.astype(np.int32), shape=np.array([cfg.m, cfg.n], np.int64),
        p=np.array([cfg.p], np.int64), seed=np.array([seed], np.int64),
        sha256=np.array([input_digest(A)]))
    print(f"{key} seed {seed}: rank {ref.rank}, oracle {dt:.0f} s on {threads} threads -> {out}")
    return out


def rref_path(key: str, seed: int) -> str:
    return os.path.join(HERE, f"oracle_rref_{key}_seed{seed}.npz")


def write_rref(key: str, seed: int, threads: int) -> str:
    """The oracle's reduced row echelon form of a prescribed-rank workload, kept as
    its rank, pivot columns and the SHA-256 of its r x n uint32 bytes (the form
    itself is too large to store): a result is equal to it iff its digest is."""
    cfg = workloads.CONFIGS[key]
    assert cfg.kind == "lru"
    A = workloads.prescribed_rank_matrix(cfg.m, cfg.n, cfg.r, cfg.p, seed=seed).A
    t = time.time()
    r, R = oracle.rref(A, cfg.p, threads=threads)
    dt = time.time() - t
    R = np.ascontiguousarray(R, dtype=np.uint32)
    pivots = np.array([int(np.flatnonzero(R[i])[0]) for i in range(r)], np.int32)
    out = rref_path(key, seed)
    np.savez_compressed(
        out, rank=np.array([r], np.int64), crp=pivots, shape=np.array([cfg.m, cfg.n], np.int64),
        p=np.array([cfg.p], np.int64), seed=np.array([seed], np.int64),
        sha256=np.array([hashlib.sha256(R.tobytes()).hexdigest()]),
        input_sha256=np.array([input_digest(A)]))
    print(f"{key} seed {seed}: RREF rank {r}, oracle {dt:.0f} s on {threads} threads -> {out}")
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--key", default="uniform-32768-p65521")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--rref", action="store_true",
                    help="write the digest of the oracle's RREF of a prescribed-rank workload")
    a = ap.parse_args()
    if a.rref:
        write_rref(a.key, a.seed, a.threads)
    else:
        write(a.key, a.seed, a.threads)


if __name__ == "__main__":
    main()
