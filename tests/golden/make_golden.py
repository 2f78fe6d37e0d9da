"""Write the stored expected values under tests/golden/ from the CPU oracle only.

    python tests/golden/make_golden.py n32      # config: n=32 int, dense and 50% sparse

Every value here comes from ``oracle`` (natural-order brute force, exact int64);
nothing is taken from the GPU path.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2310_19373_gb300 import inputs  # noqa: E402


def n32():
    out = {"citation": "Eq. 1 minimised by exhaustive natural-order enumeration (the naive method "
                       "of Section 3) in exact int64 by the CPU oracle; ties -> lowest index.",
           "generator": "paper_2310_19373_gb300.inputs.config_n32_int(seed=0, sparse=...)"}
    for sparse in (False, True):
        Q = inputs.config_n32_int(0, sparse=sparse)
        t = time.time()
        v, am = oracle.brute_min(Q)
        vals, ix = oracle.brute_topk(Q, 8)
        out["sparse" if sparse else "dense"] = {
            "min": int(v), "argmin": int(am),
            "top8": [[int(a), int(b)] for a, b in zip(vals, ix)],
            "oracle_seconds": round(time.time() - t, 1),
        }
        print(sparse, v, am, time.time() - t, flush=True)
    with open(os.path.join(HERE, "config_n32_int.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    {"n32": n32}[sys.argv[1]]()
