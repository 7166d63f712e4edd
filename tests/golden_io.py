"""Reader for the worked-example fixtures under tests/golden/ (letters a..g = vertices 0..6)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    meta, rows = {}, []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0] in ("r", "s", "n_s", "rho", "decs"):
                meta[parts[0]] = int(parts[1])
            elif parts[0] in ("sizes", "levels"):
                meta[parts[0]] = [int(x) for x in parts[1:]]
            else:
                tup = tuple(ord(ch) - ord("a") for ch in parts[0])
                rows.append((tup, int(parts[1]), int(parts[2]), int(parts[3])))
    rows.sort()
    meta["tuples"] = np.array([r[0] for r in rows], np.int32)
    meta["count"] = np.array([r[1] for r in rows], np.int64)
    meta["core"] = np.array([r[2] for r in rows], np.int32)
    meta["round"] = np.array([r[3] for r in rows], np.int32)
    return meta
