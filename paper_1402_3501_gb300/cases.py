"""Single-call cases for profiling one kernel under ncu.

  python -m paper_1402_3501_gb300.cases fgemm --m 8192 --n 8192 --k 4096 --p 65521 [--form limb]
  python -m paper_1402_3501_gb300.cases pluq --workload lru-8192-r4096-p131071 [--leaf 1024 --kind 0 --fork 2]

Each case builds its inputs with the seeded generators (workloads/), runs the
library call `--repeat` times and prints one line; nothing is checked here (the
parity tests do that).  Inputs for pluq are the workload matrices; fgemm takes
uniform residues.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np


def main(argv=None):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch
    import workloads
    import paper_1402_3501_gb300 as pq

    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["fgemm", "pluq"])
    ap.add_argument("--m", type=int, default=8192)
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--k", type=int, default=4096)
    ap.add_argument("--p", type=int, default=65521)
    ap.add_argument("--form", default="limb")
    ap.add_argument("--workload", default="lru-8192-r4096-p131071", choices=list(workloads.CONFIGS))
    ap.add_argument("--leaf", type=int, default=1024)
    ap.add_argument("--kind", type=int, default=2)
    ap.add_argument("--fork", type=int, default=2)
    ap.add_argument("--repeat", type=int, default=2)
    a = ap.parse_args(argv)
    ctx = pq.Context(0)
    if a.case == "fgemm":
        A = torch.from_numpy(workloads.uniform_matrix(a.m, a.k, a.p, 1, "casea").astype(np.int32)).cuda()
        B = torch.from_numpy(workloads.uniform_matrix(a.k, a.n, a.p, 1, "caseb").astype(np.int32)).cuda()
        C = torch.from_numpy(workloads.uniform_matrix(a.m, a.n, a.p, 1, "casec").astype(np.int32)).cuda()
        for _ in range(a.repeat):
            torch.cuda.synchronize()
            t = time.time()
            pq.fgemm_modp(C, A, B, a.p, form=a.form, ctx=ctx)
            torch.cuda.synchronize()
        print(f"fgemm {a.m}x{a.n}x{a.k} p={a.p} {a.form}: {1e3 * (time.time() - t):.3f} ms")
        return
    cfg = workloads.CONFIGS[a.workload]
    if cfg.kind == "uniform":
        A = workloads.uniform_matrix(cfg.m, cfg.n, cfg.p, seed=1)
    else:
        A = workloads.prescribed_rank_matrix(cfg.m, cfg.n, cfg.r, cfg.p, seed=1, device="cuda").A
    A0 = torch.from_numpy(A.astype(np.int32)).cuda()
    ctx.set_option("leaf_dim", a.leaf)
    ctx.set_option("leaf_kind", a.kind)
    ctx.set_option("fork_depth", a.fork)
    for _ in range(a.repeat):
        X = A0.clone()
        torch.cuda.synchronize()
        t = time.time()
        res = pq.pluq_modp(X, cfg.p, form=a.form, ctx=ctx)
        torch.cuda.synchronize()
    print(f"pluq {a.workload} rank {res.rank}: {1e3 * (time.time() - t):.3f} ms")


if __name__ == "__main__":
    main()
