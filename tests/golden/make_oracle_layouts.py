#!/usr/bin/env python3
"""Writes oracle_layouts.json: the FP64 oracle's multilevel layouts of the
bench workloads, summarised by their objective (Eq. 1 at alpha = 0.008).

For each workload the oracle builds its own hierarchy (Sec. 3.1), lays the
graph out (Sec. 3, Barnes-Hut entropy sum with the workload's theta, the
exact sum on the coarsest level) and evaluates M with the stress over S
exact and the ln-sum over pairs outside S estimated from random pairs
(oracle.objective_sampled, fixed seed; the standard error is stored).  The
GPU side is later compared with these values on the same hierarchy (the
oracle's levels fed to the device) and on its own.

Calls only oracle/ and the seeded input generators.  Run from the repository
root:  python tests/golden/make_oracle_layouts.py [workload ...]
(del20 takes several minutes of CPU time).
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1506_04383_gb300 import graphs  # noqa: E402

OUT = os.path.join(HERE, "oracle_layouts.json")

# workload name -> (generator call, oracle parameters); the same graphs and
# parameters as the benchmark's workloads of these names
WORKLOADS = {
    "rgg100k": (lambda: graphs.rgg(100000, 8.0, 1506)[:2],
                dict(k=2, theta=0.5, coarsest_n=100)),
    "del20": (lambda: graphs.delaunay(1 << 20, 1506)[:2],
              dict(k=1, theta=0.6, coarsest_n=100)),
}
SAMPLES = 20_000_000
SAMPLE_SEED = 1506


def summarise(name):
    make, kw = WORKLOADS[name]
    t0 = time.time()
    rp, col = make()
    p = oracle.params(**kw)
    levels = oracle.build_hierarchy(rp, col, p)
    x, info = oracle.layout(rp, col, p, levels=levels)
    est = oracle.objective_sampled(x, levels[0]["S"], 0.008, samples=SAMPLES, seed=SAMPLE_SEED)
    return {
        "n": int(len(rp) - 1), "m": int(len(col) // 2), "params": kw,
        "level_n": [int(L["n"]) for L in levels], "level_sweeps": [int(s) for s in info["sweeps"]],
        "stress": est["stress"], "lnsum": est["lnsum"], "M": est["M"],
        "se_lnsum": est["se_lnsum"], "se_M": est["se_M"], "samples": SAMPLES,
        "samples_kept": est["kept"], "sample_seed": SAMPLE_SEED, "alpha": 0.008,
        "oracle_threads": oracle.num_threads(), "seconds": round(time.time() - t0, 1),
    }


def main(names):
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as fh:
            data = json.load(fh)
    for name in names:
        data[name] = summarise(name)
        print(name, json.dumps(data[name]), flush=True)
        with open(OUT, "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)
            fh.write("\n")


if __name__ == "__main__":
    main(sys.argv[1:] or sorted(WORKLOADS))
