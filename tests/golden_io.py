"""Readers for the text fixtures under tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def philox_kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            w = [int(t, 16) for t in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def contract_example():
    d = {}
    with open(os.path.join(GOLDEN, "contract_example.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            d[key] = vals
    n = int(d["n"][0])
    e = d["edges"]
    trip = [(int(e[i]), int(e[i + 1]), float(e[i + 2])) for i in range(0, len(e), 3)]
    # symmetric CSR with sorted rows and the per-entry omega
    ent = sorted([(u, v, w) for u, v, w in trip] + [(v, u, w) for u, v, w in trip])
    rp = np.zeros(n + 1, dtype=np.int64)
    for u, _, _ in ent:
        rp[u + 1] += 1
    rp = np.cumsum(rp)
    col = np.array([v for _, v, _ in ent], dtype=np.int32)
    ew = np.array([w for _, _, w in ent], dtype=np.float64)
    out = dict(
        n=n, rp=rp, col=col, ew=ew,
        labels=np.array([int(t) for t in d["labels"]], dtype=np.int32),
        map=np.array([int(t) for t in d["map"]], dtype=np.int32),
        c=np.array([float(t) for t in d["c"]]),
        crp=np.array([int(t) for t in d["row_ptr"]], dtype=np.int64),
        ccol=np.array([int(t) for t in d["col"]], dtype=np.int32),
        cew=np.array([float(t) for t in d["omega"]]),
    )
    return out
