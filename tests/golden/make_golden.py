"""Write the stored expected values under tests/golden/ from the CPU oracle only.

    python tests/golden/make_golden.py n32      # n=32 int32, dense and 50% sparse (literal oracle)
    python tests/golden/make_golden.py n40      # n=40 FP32 headline instance: min, argmin, top-8
    python tests/golden/make_golden.py batched  # every n >= 26 instance of the 4096-instance batch
    python tests/golden/make_golden.py n44      # the n=44 FP32 instance of the chunked solver
    python tests/golden/make_golden.py logz     # 4 of the 64 n=28 log Z instances in full

Every value here comes from ``oracle`` (natural-order enumeration; exact int64
for integer Q, canonical FP64 for float Q); nothing is taken from the GPU
path.  n32 uses the literal loop; the others use the blocked natural-order
walk (oracle.blocked_topk), which returns the literal loop's answer bit for
bit (pinned in tests/test_oracle_pins.py) and runs at about 1e10 states/s on
eight x86 cores (n=40 in about two minutes, the batch in about fifteen, n=44
in about half an hour).
"""
import json
import os
import sys
import time

import numpy as np

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


BLOCKED_CITATION = ("Eq. 1 minimised by exhaustive natural-order enumeration (the naive method "
                    "of Section 3) by the CPU oracle's blocked walk; float values in canonical "
                    "FP64 order, integer values exact in int64; ties -> lowest index.")


def _topk_entry(Q, k):
    t = time.time()
    vals, ix, ncand = oracle.blocked_topk(Q, k, return_candidates=True)
    is_int = np.issubdtype(np.asarray(Q).dtype, np.integer)
    conv = int if is_int else float
    return {"min": conv(vals[0]), "argmin": int(ix[0]),
            "topk": [[conv(a), int(b)] for a, b in zip(vals, ix)],
            "oracle_candidates": ncand,
            "oracle_seconds": round(time.time() - t, 1)}


def n40():
    Q = inputs.config_n40_f32(0)
    out = {"citation": BLOCKED_CITATION, "generator": "paper_2310_19373_gb300.inputs.config_n40_f32(0)",
           "dtype": "float32", "n": 40}
    out.update(_topk_entry(Q, 8))
    print(out, flush=True)
    with open(os.path.join(HERE, "config_n40_f32.json"), "w") as f:
        json.dump(out, f, indent=1)


def n44():
    Q = inputs.gaussian_f32(44, seed=44)
    out = {"citation": BLOCKED_CITATION, "generator": "paper_2310_19373_gb300.inputs.gaussian_f32(44, seed=44)",
           "dtype": "float32", "n": 44}
    out.update(_topk_entry(Q, 8))
    print(out, flush=True)
    with open(os.path.join(HERE, "gaussian_n44_f32.json"), "w") as f:
        json.dump(out, f, indent=1)


def batched(n_min=26):
    Qs = inputs.config_batched()
    out = {"citation": BLOCKED_CITATION,
           "generator": "paper_2310_19373_gb300.inputs.config_batched() (4096 instances, seed 0)",
           "n_min": n_min, "instances": []}
    t0 = time.time()
    for i, Q in enumerate(Qs):
        n = Q.shape[0]
        if n < n_min:
            continue
        v, am = oracle.blocked_min(Q)
        out["instances"].append({"index": i, "n": n, "dtype": str(Q.dtype),
                                 "min": int(v) if np.issubdtype(Q.dtype, np.integer) else float(v),
                                 "argmin": int(am)})
        if len(out["instances"]) % 100 == 0:
            print(len(out["instances"]), i, round(time.time() - t0), flush=True)
    out["oracle_seconds"] = round(time.time() - t0, 1)
    with open(os.path.join(HERE, "config_batched_n26up.json"), "w") as f:
        json.dump(out, f, indent=0)


LOGZ_INSTANCES = (0, 21, 42, 63)
LOGZ_FD_ENTRIES = ((0, 0), (3, 17), (10, 27), (27, 27), (14, 2), (5, 6))
LOGZ_FD_H = 1e-3


def logz():
    """log Z(beta) and E_beta[x x^T] of four instances of the n=28 log Z workload
    (literal FP64 oracle, Kahan sums), and central differences of the oracle's
    log Z for six entries of instance 0 (h = 1e-3)."""
    Qs = inputs.config_logz()
    betas = list(inputs.LOGZ_BETAS)
    out = {"citation": "log Z(beta) = log sum_x exp(-beta x^T Q x) over all x (Eq. 1's objective) "
                       "and E_beta[x_i x_j] by the CPU oracle's natural-order enumeration in FP64; "
                       "central differences of the oracle's log Z.",
           "generator": "paper_2310_19373_gb300.inputs.config_logz() (64 x n=28, seed 0)",
           "betas": betas, "instances": []}
    t0 = time.time()
    for b in LOGZ_INSTANCES:
        lz, E, vmin, am = oracle.logz(Qs[b], betas)
        out["instances"].append({"index": b, "logz": [float(v) for v in lz],
                                 "moment": [[[float(v) for v in row] for row in Eb] for Eb in E],
                                 "min": float(vmin), "argmin": int(am)})
        print(b, lz, round(time.time() - t0), flush=True)
    fd = []
    Q0 = Qs[0].astype(np.float64)
    for (i, j) in LOGZ_FD_ENTRIES:
        Qp, Qm = Q0.copy(), Q0.copy()
        Qp[i, j] += LOGZ_FD_H
        Qm[i, j] -= LOGZ_FD_H
        lp, _, _, _ = oracle.logz(Qp, betas, moment=False)
        lm, _, _, _ = oracle.logz(Qm, betas, moment=False)
        fd.append({"i": i, "j": j,
                   "dlogz": [float((a - c) / (2 * LOGZ_FD_H)) for a, c in zip(lp, lm)]})
        print(i, j, fd[-1]["dlogz"], round(time.time() - t0), flush=True)
    out["central_differences"] = {"instance": 0, "h": LOGZ_FD_H,
                                  "note": "Q perturbed in FP64 (the FP32 instance widened)",
                                  "entries": fd}
    out["oracle_seconds"] = round(time.time() - t0, 1)
    with open(os.path.join(HERE, "config_logz_n28.json"), "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    {"n32": n32, "n40": n40, "n44": n44, "batched": batched, "logz": logz}[sys.argv[1]]()
