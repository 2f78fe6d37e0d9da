#!/usr/bin/env python
"""Benchmark: certified exhaustive minimisation of one n=40 QUBO on one GB300.

A step is one full solve through the C ABI (qbf_solve): fixed-point image of
Q, walk tables, the Gray-code walk over all 2^40 states, candidate re-walk,
FP64 rescoring and the top-1 selection, with the result read back to the
host.  Input: n=40, FP32, off-diagonal N(0,1), diagonal N(-0.5,1), upper
triangular, seed 0 (synthetic; the paper names no dataset).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.  Under torchrun every rank solves its own
copy of the instance (replicas, no data-path collective); the value is the
states all ranks processed over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "QUBO states evaluated/sec at n=40 (1 GB300) and % of ALU peak; batched & TC form vs plain"
N_VARS = 40
WORKLOAD = ("single QUBO n=40, FP32 upper triangular, off-diagonal N(0,1), diagonal N(-0.5,1), "
            "seed 0; certified min + lowest-index argmin")
# bytes the end-to-end call moves per step: Q in (n*n*4) and the result out
# (device result block: 64 doubles + 64 uint64 + 16 B, plus the 48-byte plan head)
E2E_D2H_BYTES = 64 * 8 + 64 * 8 + 16 + 48
# value operations every visited state needs in a Gray walk once the flipped
# variable's field is at hand: one add (the delta of Eq. 2) and one min input.
# The forms differ only in how they come by that field: the split walks share
# its lane-invariant part across lanes, the two-pipe walk then adds it once
# per value (3 operations per state), the deferred walk once per eight values
# (2.25 per state)
ALGO_OPS_PER_STATE = 2
# per SM and clock: 128 FP32 lanes (FADD / packed f32x2 add) and 128 INT32/ALU
# lanes (IADD3, IMNMX, FMNMX and their three-input forms)
PIPE_LANES_PER_SM = 128 + 128
WALK_KERNELS = {0: "walk_split_kernel<6, MIN>", 1: "field_min_kernel", 2: "walk_split_kernel<6, MIN>",
                6: "naive_min_kernel",
                3: "tc_min_kernel", 4: "walk_f32x2_min_kernel<6>", 5: "walk_mix_min_kernel<6>",
                7: "walk_defer2_min_kernel<7>"}


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        loaded = [c for c in sm if mx and c > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def cpu_model():
    """The host CPU's model name and core count (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def random_windows(n, bits, count, seed):
    """`count` distinct aligned windows of 2^bits natural indices at random high
    prefixes: the sample spans the whole index range, so the set bits per
    state (which the oracle's per-state cost follows) match the full walk."""
    import numpy as np

    rng = np.random.default_rng(seed)
    hi = 1 << (n - bits)
    w = rng.choice(hi, size=min(count, hi), replace=False)
    return [(int(v) << bits, (int(v) + 1) << bits) for v in w]


def cpu_baseline(Q, target_s=12.0, seed=0):
    """Time the CPU oracle (as it stands) on a bounded sample of the same instance:
    whole 2^22-state windows at random high prefixes, until about target_s."""
    import oracle

    cores = oracle.threads_default()
    bits = 22
    wins = random_windows(N_VARS, bits, 4096, seed)
    done, dt = 0, 0.0
    for lo, hi in wins:
        t0 = time.perf_counter()
        oracle.brute_min(Q, lo, hi)
        dt += time.perf_counter() - t0
        done += 1
        if dt >= target_s:
            break
    return {"value": done * (1 << bits) / dt, "unit": "states/s", "cores": cores, "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": f"natural-order FP64 brute force over {done} windows of 2^{bits} states at "
                      f"random high prefixes of the n=40 instance (seed {seed}), {dt:.1f} s"}


def cpu_gray_baseline(Q, target_s=6.0):
    """The paper's CPU design on the same cores: Algorithm 1 (Eq. 2's O(n) delta
    from the row of the flipped variable) with the prefix threads of Section
    3.1, FP64, written fresh (cpu_baseline/cpu_gray.c).  Timed on random
    prefixes of the n=40 instance; the paper's own figure is n = 30 in under
    4 s on an Intel i7-8700 (at least 2.7e8 states/s)."""
    import numpy as np

    import cpu_baseline as cg

    m = 16
    rng = np.random.default_rng(1)
    pre = rng.choice(1 << m, size=16, replace=False)
    t0 = time.perf_counter()
    _, _, T = cg.walk(Q, m, pre)
    dt = time.perf_counter() - t0
    per = 16 * 2.0 ** (N_VARS - m) / dt
    count = max(16, min(1 << m, int(16 * target_s / max(dt, 1e-3))))
    pre = rng.choice(1 << m, size=count, replace=False)
    t0 = time.perf_counter()
    _, _, T = cg.walk(Q, m, pre)
    dt = time.perf_counter() - t0
    rate = count * 2.0 ** (N_VARS - m) / dt
    return {"value": rate, "unit": "states/s", "cores": T, "cpu_model": cpu_model(),
            "kind": "Algorithm 1 + Section 3.1 prefix threads, FP64 (the paper's CPU design)",
            "sample": f"{count} prefixes of the top {m} variables (2^{N_VARS - m} states each) of "
                      f"the n=40 instance, {dt:.1f} s",
            "n30_seconds_at_this_rate": 2.0 ** 30 / rate,
            "paper_context": "n=30 in < 4 s on an Intel i7-8700 (Section 4): >= 2.7e8 states/s"}


def oracle_timings():
    """The CPU oracle on the other configurations, on the host cores: n=20 FP64
    top-8 in full (literal loop); n=32 int32 dense and 50% sparse in full
    (blocked walk) and the literal loop's rate on random windows; the literal
    loop's rate on an n=28 log Z instance, scaled to the 64-instance, 3-beta
    forward pass; the blocked walk at n=40 on a 2^34-state sample scaled to
    the whole space."""
    import oracle
    from paper_2310_19373_gb300 import inputs

    out = {"cores": oracle.threads_default(), "cpu_model": cpu_model()}
    t0 = time.perf_counter()
    oracle.brute_topk(inputs.config_n20_f64(0), 8)
    out["n20_f64_top8_literal_s"] = time.perf_counter() - t0
    for sparse in (False, True):
        Q = inputs.config_n32_int(0, sparse=sparse)
        key = "n32_int32_sparse" if sparse else "n32_int32"
        t0 = time.perf_counter()
        oracle.blocked_topk(Q, 8)
        out[key + "_blocked_s"] = time.perf_counter() - t0
        wins = random_windows(32, 22, 4, 2)
        t0 = time.perf_counter()
        for lo, hi in wins:
            oracle.brute_min(Q, lo, hi)
        rate = len(wins) * 2.0 ** 22 / (time.perf_counter() - t0)
        out[key + "_literal_states_per_s"] = rate
        out[key + "_literal_s_extrapolated"] = 2.0 ** 32 / rate
    # log Z: the oracle evaluates Eq. 1 for every state once for the minimum and
    # once per beta; its rate on random windows of one n = 28 instance gives a
    # lower bound for the 64-instance, 3-beta forward pass (exp not counted)
    QL = inputs.config_logz(count=1)[0]
    wins = random_windows(28, 22, 4, 3)
    t0 = time.perf_counter()
    for lo, hi in wins:
        oracle.brute_min(QL, lo, hi)
    rate = len(wins) * 2.0 ** 22 / (time.perf_counter() - t0)
    out["logz_n28_literal_states_per_s"] = rate
    out["logz_64x28_3beta_forward_s_lower_bound"] = 64 * 2.0 ** 28 * (1 + 3) / rate
    Q40 = inputs.config_n40_f32(0)
    lo = 0b100101 << 34
    t0 = time.perf_counter()
    oracle.blocked_min(Q40, lo, lo + (1 << 34))
    dt = time.perf_counter() - t0
    out["n40_blocked_states_per_s"] = 2.0 ** 34 / dt
    out["n40_blocked_s_extrapolated"] = 2.0 ** 40 * dt / 2.0 ** 34
    return out


def init_ranks(world):
    """torch.distributed over gloo for N > 1 replicas (host-side timing reduce
    only: the path itself has no collective); None for one process."""
    if world <= 1:
        return None
    import torch.distributed as dist

    dist.init_process_group("gloo")
    return dist


def max_over_ranks(x, pg):
    """The largest per-rank value over all ranks (the slowest replica sets the
    time); x itself without a process group."""
    if pg is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, states_per_replica, seconds):
    """Whole-job states/s: every rank walks its own full instance in `seconds`."""
    return world * states_per_replica / seconds


def run_reference(args, rank):
    if rank != 0:
        return
    from paper_2310_19373_gb300 import inputs

    Q = inputs.config_n40_f32(0)
    per_step = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    for w in range(args.warmup):
        cpu_baseline(Q, target_s=per_step / 4, seed=100 + w)
    vals = []
    last = None
    for st in range(args.steps):
        last = cpu_baseline(Q, target_s=per_step, seed=st)
        vals.append(last["value"])
    v = statistics.median(vals)
    ms = (1 << N_VARS) / v * 1e3
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "states/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "n": N_VARS},
        "cpu_baseline": {"value": v, "unit": "states/s", "cores": last["cores"],
                         "kind": "oracle", "cpu_model": last["cpu_model"],
                         "sample": last["sample"]},
        "e2e": {"value": v, "unit": "states/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


VARIANTS = {"auto": 0, "field": 1, "split": 2, "tc": 3, "f32": 4, "mix": 5, "naive": 6, "defer": 7}


def run_profile_case(n, variant=0, prefix_bits=-1):
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2310_19373_gb300 import _binding as qb
    from paper_2310_19373_gb300 import inputs

    Q = torch.from_numpy(inputs.gaussian_f32(n, seed=0)).cuda()
    for _ in range(2):
        sol = qb.solve(Q, timing=True, variant=variant, prefix_bits=prefix_bits)
    torch.cuda.synchronize()
    print(json.dumps({"profile_n": n, "prefix_bits": sol.prefix_bits, "min_value": sol.min_value,
                      "argmin": sol.argmin, "walk_ms": sol.walk_seconds * 1e3}))


def run_prefix_sweep(ns):
    """MIN walk time of the table-driven deferred walk over prefix widths, for
    FP32 Gaussian instances of each n (the planner's width reported beside)."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2310_19373_gb300 import _binding as qb
    from paper_2310_19373_gb300 import inputs

    for n in ns:
        Q = torch.from_numpy(inputs.config_n40_f32(0) if n == 40 else
                             inputs.gaussian_f32(n, seed=n)).cuda()
        auto = qb.solve(Q, timing=True)
        row = {"n": n, "planner_prefix_bits": auto.prefix_bits, "walk_ms": {}}
        for k in range(max(10, n - 24), min(28, n - 8) + 1):
            ts = []
            for _ in range(3):
                s = qb.solve(Q, variant=qb.QBF_VARIANT_SPLIT_DEFER, prefix_bits=k, timing=True)
                ts.append(s.walk_seconds)
            if (s.min_value, s.argmin) != (auto.min_value, auto.argmin):
                raise SystemExit(f"prefix sweep: n={n} k={k} changed the answer")
            row["walk_ms"][k] = round(min(ts) * 1e3, 4)
        print(json.dumps(row), flush=True)


def run_profile_small():
    """Three solves each of the n = 32 int32 instance (top-1) and the n = 20
    FP64 instance (top-8): small solves, whose time the fixed kernels around
    the walk set (a case for an ncu launch list)."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2310_19373_gb300 import _binding as qb
    from paper_2310_19373_gb300 import inputs

    Q32 = torch.from_numpy(inputs.config_n32_int(0)).cuda()
    Q20 = torch.from_numpy(inputs.config_n20_f64(0)).cuda()
    for _ in range(3):
        s32 = qb.solve(Q32)
        s20 = qb.solve(Q20, top_k=8)
    torch.cuda.synchronize()
    print(json.dumps({"profile_small": True, "n32_prefix_bits": s32.prefix_bits,
                      "n20_prefix_bits": s20.prefix_bits, "n20_top8": s20.topk_indices}))


def run_profile_batched(count, variant=0):
    """Two batched solves on the first `count` instances of the 4096-instance
    workload (a small case for ncu)."""
    import numpy as np
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2310_19373_gb300 import _binding as qb
    from paper_2310_19373_gb300 import inputs

    Qs = [torch.from_numpy(np.ascontiguousarray(q)).cuda()
          for q in inputs.config_batched(count=count)]
    for _ in range(2):
        t0 = time.perf_counter()
        vmin, am = qb.solve_batched(Qs, variant=variant)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    states = float(sum(2 ** q.shape[0] for q in Qs))
    print(json.dumps({"profile_batched": count, "seconds": dt, "states_per_s": states / dt}))


def run_profile_logz(count):
    """log Z forward and backward (3 betas) on the first `count` instances of
    the log Z workload (n = 28), twice each (a small case for ncu)."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2310_19373_gb300 import _binding as qb
    from paper_2310_19373_gb300 import inputs

    QL = torch.from_numpy(inputs.config_logz(count=count)).cuda()
    betas = list(inputs.LOGZ_BETAS)
    sp = torch.cuda.current_stream().cuda_stream
    grad = torch.empty((count, 28, 28), dtype=torch.float64, device="cuda")
    for _ in range(2):
        t0 = time.perf_counter()
        qb.qbf_logz(QL.data_ptr(), 28, qb.QBF_F32, count, betas, sp)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        qb.qbf_logz_backward(QL.data_ptr(), 28, qb.QBF_F32, count, betas, None, grad.data_ptr(),
                             None, sp)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
    print(json.dumps({"profile_logz": count, "forward_seconds": t1 - t0,
                      "backward_seconds": t2 - t1}))


ALU_OPS = ["IADD3", "IMNMX", "3-input integer min", "FADD", "FFMA", "FMNMX", "3-input FMNMX",
           "packed FADD (f32x2)", "IADD3 + IMNMX pair", "FADD + FMNMX pair", "EX2 (ex2.approx)",
           "DADD (FP64)", "IMAD", "I2F + F2I pair", "deferred-walk step mix (value-ops)"]


def run_alu_microbench():
    """Lane-op/s of each ALU instruction class; per-clock figures use the sampled SM clock."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2310_19373_gb300 import _binding as qb

    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    clk = ClockSampler(0)
    clk.start()
    rows = []
    for rep in range(2):
        for op, name in enumerate(ALU_OPS):
            ops, mhz, sec = qb.qbf_alu_microbench(op)
            if rep == 1:
                rows.append((op, name, ops * nsm * mhz * 1e6))
    c = clk.stop() or {}
    f = c.get("sm_mhz") or float(measured_peaks().get("sm_max_mhz", 2070.0))
    for op, name, rate in rows:
        print(json.dumps({"op": op, "name": name, "lane_ops_per_s": rate,
                          "lane_ops_per_clk_per_sm": rate / (nsm * f * 1e6), "sm_mhz": f}))


def run_variants(dev, flush):
    """Other workloads of the path, timed with CUDA events (reported beside the headline)."""
    import numpy as np
    import torch

    from paper_2310_19373_gb300 import _binding as qb
    from paper_2310_19373_gb300 import inputs

    out = {}
    stream = torch.cuda.current_stream(dev)

    def timed(fn, reps=3):
        fn()
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e-3)
        return statistics.median(ts)

    # batched: 4096 instances, n ~ U{16..34}, half FP32 uniform[-1,1], half int16;
    # timed with the library defaults, then again after qbf_tune has chosen the
    # suffix width and CTAs per SM for every n of both element classes
    Qs = [torch.from_numpy(np.ascontiguousarray(q)).to(dev) for q in inputs.config_batched()]
    states = float(sum(2 ** q.shape[0] for q in Qs))
    t_default = timed(lambda: qb.solve_batched(Qs))
    cache = os.path.join(tempfile.mkdtemp(), "qbf_tune.txt")
    t0 = time.perf_counter()
    qb.qbf_tune(16, 34, qb.QBF_F32, cache)
    qb.qbf_tune(16, 34, qb.QBF_I16, cache)
    t_tune = time.perf_counter() - t0
    t = timed(lambda: qb.solve_batched(Qs))
    tuned = {cls: {n: list(qb.qbf_tuned_params(n, code)) for n in range(16, 35)}
             for cls, code in (("f32", qb.QBF_F32), ("i16", qb.QBF_I16))}
    _, _, info = qb.solve_batched_info(Qs)
    out["batched_4096"] = {"workload": "4096 QUBOs, n ~ U{16..34}, half FP32 uniform[-1,1], "
                                       "half int16 uniform{-50..50}, seed 0; one persistent walk "
                                       "under a CUDA graph",
                           "states": states, "seconds": t, "states_per_s": states / t,
                           "default_seconds": t_default,
                           "tuned": {"by": "qbf_tune(16, 34) per element class",
                                     "seconds_to_tune": t_tune,
                                     "suffix_bits_ctas_per_sm_by_n": tuned},
                           "n_candidates": int(sum(x.n_candidates for x in info))}
    # log Z forward and backward: 64 instances, n = 28, N(0, 1/n), beta in {0.1, 1, 10}
    QL = torch.from_numpy(inputs.config_logz()).to(dev)
    betas = list(inputs.LOGZ_BETAS)
    sp = stream.cuda_stream
    grad = torch.empty((64, 28, 28), dtype=torch.float64, device=dev)
    t_f = timed(lambda: qb.qbf_logz(QL.data_ptr(), 28, qb.QBF_F32, 64, betas, sp), reps=2)
    t_b = timed(lambda: qb.qbf_logz_backward(QL.data_ptr(), 28, qb.QBF_F32, 64, betas, None,
                                             grad.data_ptr(), None, sp), reps=2)
    st = 64.0 * 2 ** 28
    out["logz_64x28"] = {"workload": "64 QUBOs n=28 FP32 N(0,1/n), beta in {0.1,1,10}; forward "
                                     "= certified min + log Z for 3 betas, backward = -beta "
                                     "E[xx^T] for 3 betas",
                         "states": st, "forward_seconds": t_f, "backward_seconds": t_b,
                         "forward_states_per_s": st / t_f}
    # the kernel forms of the n = 40 headline solve, side by side
    Q40 = torch.from_numpy(inputs.config_n40_f32(0)).to(dev)
    for name, var in (("deferred_walk_n40", 7), ("two_pipe_walk_n40", 5), ("packed_f32_walk_n40", 4),
                      ("int32_walk_n40", 2), ("tc_blocked_n40", 3)):
        walk = []

        def one(var=var, walk=walk):
            walk.append(qb.solve(Q40, variant=var, timing=True).walk_seconds)

        t = timed(one)
        out[name] = {"workload": "n=40 FP32 (headline instance), certified min",
                     "seconds": t, "states_per_s": 2.0 ** 40 / t,
                     "min_kernel_ms": statistics.median(walk[1:]) * 1e3}
    # the paper's comparison on this GPU (MIN kernel times, one n = 32 FP32 instance):
    # naive O(n^2) evaluation per state, the plain Gray walk (n_s + 1 adds per state,
    # Algorithm 1), and the split walks of this library
    Qg = torch.from_numpy(inputs.gaussian_f32(32, seed=0)).to(dev)
    forms = {}
    for name, var in (("naive", 6), ("gray_field", 1), ("int32_split", 2), ("two_pipe", 5),
                      ("deferred", 7)):
        walk = []

        def one(var=var, walk=walk):
            walk.append(qb.solve(Qg, variant=var, timing=True).walk_seconds)

        t = timed(one, reps=2)
        kms = statistics.median(walk[1:]) * 1e3
        forms[name] = {"seconds": t, "min_kernel_ms": kms, "states_per_s": 2.0 ** 32 / (kms * 1e-3)}
    out["naive_vs_gray_n32"] = {
        "workload": "n=32 FP32 off-diagonal N(0,1), diagonal N(-0.5,1), seed 0; certified min",
        "forms": forms,
        "gray_over_naive": forms["naive"]["min_kernel_ms"] / forms["gray_field"]["min_kernel_ms"],
        "two_pipe_over_gray": forms["gray_field"]["min_kernel_ms"] / forms["two_pipe"]["min_kernel_ms"],
        "deferred_over_gray": forms["gray_field"]["min_kernel_ms"] / forms["deferred"]["min_kernel_ms"]}
    # beyond n = 40: n = 44 through the chunked, resumable API (16 chunks of 2^40)
    Q44 = torch.from_numpy(inputs.gaussian_f32(44, seed=44)).to(dev)
    holder = {}

    def chunked():
        c = qb.Chunked.start(Q44, chunk_bits=4)
        c.step(Q44, max_chunks=16)
        holder["r"] = c.result()

    t = timed(chunked, reps=1)
    out["chunked_n44"] = {"workload": "n=44 FP32 off-diagonal N(0,1), diagonal N(-0.5,1), seed 44; "
                                      "qbf_chunked_* in 16 chunks of 2^40 states, certified min",
                          "seconds": t, "states_per_s": 2.0 ** 44 / t,
                          "min_value": holder["r"].min_value, "argmin": holder["r"].argmin}
    # n = 32 int32 (dense), exact
    Q32 = torch.from_numpy(inputs.config_n32_int(0)).to(dev)
    t = timed(lambda: qb.solve(Q32))
    out["n32_int32"] = {"workload": "n=32 int32 uniform[-100,100], seed 0, exact",
                        "seconds": t, "states_per_s": 2.0 ** 32 / t}
    # the same with each off-diagonal entry zeroed with p = 0.5: the split walk's
    # per-state work does not read Q, so density should not change the time
    Q32s = torch.from_numpy(inputs.config_n32_int(0, sparse=True)).to(dev)
    walk = []

    def sparse_one():
        walk.append(qb.solve(Q32s, timing=True).walk_seconds)

    t = timed(sparse_one)
    dense_walk = []
    timed(lambda: dense_walk.append(qb.solve(Q32, timing=True).walk_seconds))
    out["n32_int32_sparse"] = {"workload": "n=32 int32 uniform[-100,100], seed 0, off-diagonal "
                                           "zeroed with p=0.5 (mask seed 1), exact",
                               "seconds": t, "states_per_s": 2.0 ** 32 / t,
                               "min_kernel_ms": statistics.median(walk[1:]) * 1e3,
                               "dense_min_kernel_ms": statistics.median(dense_walk[1:]) * 1e3}
    # n = 20 FP64 top-8 (latency)
    Q20 = torch.from_numpy(inputs.config_n20_f64(0)).to(dev)
    t = timed(lambda: qb.solve(Q20, top_k=8), reps=10)
    out["n20_f64_top8"] = {"workload": "n=20 FP64 uniform[-1,1], seed 0, top-8",
                           "seconds": t, "states_per_s": 2.0 ** 20 / t}
    return out


def load_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if its
    source files are unchanged since the counters were taken (else None)."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)[kernel]
        h = hashlib.sha256()
        for src in t.get("sources") or [t["source"]]:
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
        if h.hexdigest() != t["source_sha256"]:
            return None
        return t["bytes_per_full_launch"]
    except (OSError, KeyError, ValueError, TypeError):
        return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the batched / n=32 / n=20 lines reported beside the headline")
    ap.add_argument("--profile-small", action="store_true",
                    help="run three n=32 int32 and three n=20 FP64 top-8 solves and exit")
    ap.add_argument("--prefix-sweep", default="",
                    help="comma-separated n: time the deferred MIN walk over prefix widths and exit")
    ap.add_argument("--profile-n", type=int, default=0,
                    help="profiling target: two solves of an n-variable Gaussian FP32 instance, "
                         "no timing (for ncu)")
    ap.add_argument("--prefix-bits", type=int, default=-1,
                    help="with --profile-n: prefix bits of the solve (-1: the planner's choice)")
    ap.add_argument("--variant", default="auto", choices=list(VARIANTS),
                    help="kernel form of the headline solve (auto: the library's choice)")
    ap.add_argument("--profile-batched", type=int, default=0,
                    help="run two batched solves on this many instances of the batched workload")
    ap.add_argument("--profile-logz", type=int, default=0,
                    help="run log Z forward and backward on this many instances of the log Z workload")
    ap.add_argument("--alu-microbench", action="store_true",
                    help="print the ALU throughput table (roofline denominators) and exit")
    args = ap.parse_args()
    world = env_int("WORLD_SIZE", 1)
    rank = env_int("RANK", 0)
    local = env_int("LOCAL_RANK", 0)
    if args.warmup < 3:
        args.warmup = 3

    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.profile_small:
        run_profile_small()
        return
    if args.prefix_sweep:
        run_prefix_sweep([int(x) for x in args.prefix_sweep.split(",")])
        return
    if args.profile_n:
        run_profile_case(args.profile_n, VARIANTS[args.variant], args.prefix_bits)
        return
    if args.alu_microbench:
        run_alu_microbench()
        return
    if args.profile_batched:
        run_profile_batched(args.profile_batched, VARIANTS[args.variant])
        return
    if args.profile_logz:
        run_profile_logz(args.profile_logz)
        return

    import numpy as np
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2310_19373_gb300 import _binding as qb
    from paper_2310_19373_gb300 import inputs

    pg = init_ranks(world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    Qnp = inputs.config_n40_f32(0)
    Qd = torch.from_numpy(Qnp).to(dev)
    Qh = torch.from_numpy(Qnp).pin_memory()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    stream = torch.cuda.current_stream(dev)

    variant = VARIANTS[args.variant]
    for _ in range(args.warmup):
        qb.solve(Qd, timing=True, variant=variant)
    torch.cuda.synchronize(dev)

    clocks = ClockSampler(local)
    clocks.start()
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    step_ms, walk_s = [], []
    launches = 0
    sol = None
    for _ in range(args.steps):
        flush.zero_()  # evict L2 between steps (outside the timed events)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sol = qb.solve(Qd, timing=True, variant=variant)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        walk_s.append(sol.walk_seconds)
        launches += sol.kernel_launches
    torch.cuda.synchronize(dev)
    if pg:
        pg.barrier()
    clk = clocks.stop()

    ms = max_over_ranks(sum(step_ms) / len(step_ms), pg)
    states = float(1 << N_VARS)
    value = replica_throughput(world, states, ms * 1e-3)

    # end to end: Q from pinned host memory, result back to the host, every step
    e2e_s = []
    for _ in range(max(3, min(args.steps, 5))):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        qb.solve(Qh, variant=variant)
        e2e_s.append(time.perf_counter() - t0)
    e2e_t = max_over_ranks(statistics.median(e2e_s), pg)

    # roofline of the dominant kernel (the MIN walk): algorithmic value-ops / device time,
    # against both 128-lane pipes of every SM at the maximum SM clock
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = measured_peaks()
    fmax = float(peaks.get("sm_max_mhz", 2070.0))
    peak_ops = nsm * PIPE_LANES_PER_SM * fmax * 1e6
    walk_t = statistics.median(walk_s)
    achieved = ALGO_OPS_PER_STATE * states / walk_t
    kernel = WALK_KERNELS.get(sol.variant, "walk")
    # arithmetic types of the MIN walk (all on exact integers; certification rescoring is FP64)
    path_dtype = {3: "f16/f32", 4: "f32", 5: "f32+i32", 7: "f32"}.get(sol.variant, "i32")

    line = {
        "metric": METRIC, "value": value, "unit": "states/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": path_dtype,
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N_VARS, "top_k": 1,
                   "prefix_bits": sol.prefix_bits, "suffix_bits": sol.suffix_bits,
                   "l2": "flushed between steps (256 MiB device write outside the timed events)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "result": {"min_value": sol.min_value, "argmin": sol.argmin,
                   "n_candidates": sol.n_candidates, "error_bound": sol.error_bound,
                   "scale_bits": sol.scale_bits},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                     "unit": "Tvalue-op/s", "frac": achieved / peak_ops,
                     "traffic": load_traffic(kernel), "kernel": kernel,
                     "kernel_ms": walk_t * 1e3,
                     "peak_basis": (f"{nsm} SMs x (128 FP32 + 128 INT32/ALU lanes) x {fmax:.0f} MHz "
                                    "(unit counts and clock; measured: FADD 126, IMNMX 127.5, "
                                    "packed/three-input forms 127 values per clk per SM)"),
                     "ops_per_state": ALGO_OPS_PER_STATE,
                     "metric_normalised_ops_per_s": states * N_VARS / (ms * 1e-3),
                     "metric_normalised_frac": states * N_VARS / (ms * 1e-3) / peak_ops},
        "e2e": {"value": replica_throughput(world, states, e2e_t), "unit": "states/s",
                "h2d_bytes_per_step": N_VARS * N_VARS * 4,
                "d2h_bytes_per_step": E2E_D2H_BYTES},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_variants:
        line["variants"] = run_variants(dev, flush)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(Qnp)
        line["cpu_gray"] = cpu_gray_baseline(Qnp)
        line["oracle_timings"] = oracle_timings()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
