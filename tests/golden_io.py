"""Reader for the hand-worked fixtures under tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name: str) -> dict:
    lines = [ln.strip() for ln in open(os.path.join(GOLDEN, name)) if ln.strip()
             and not ln.startswith("#")]
    out, i = {}, 0
    while i < len(lines):
        key, *rest = lines[i].split()
        if key in ("A", "rref"):
            rows = []
            i += 1
            while i < len(lines) and lines[i].split()[0].isdigit():
                rows.append([int(v) for v in lines[i].split()])
                i += 1
            out[key] = np.array(rows, dtype=np.uint32)
            continue
        if key == "rpm":
            out[key] = {tuple(int(x) for x in pr.split(",")) for pr in rest}
        elif key in ("rrp", "crp"):
            out[key] = [int(v) for v in rest]
        else:
            out[key] = int(rest[0])
        i += 1
    return out
