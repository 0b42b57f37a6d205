"""Benchmark of the semisort hot path on GB300.

Workload (one "step" = one semisort_= call over one n = 10^9 batch):
  semisort_= on n = 10^9 records (uint64 key, uint64 value = index); steps
  cycle over the ten key distributions of the paper's Table 2 uniform/Zipf
  rows: uniform with exactly {10, 10^3, 10^5, 10^7, 10^9} distinct keys and
  Zipf s in {0.6, 0.8, 1.0, 1.2, 1.5} over 10^9 ranks (synthetic, seeded).
  Inputs are device resident and larger than L2, so no flush is needed.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle (the
plain stable sort that defines a valid output) on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_DEFAULT = 10**9
DISTS = [("uniform", 10), ("uniform", 10**3), ("uniform", 10**5), ("uniform", 10**7), ("uniform", 10**9),
         ("zipf", 0.6), ("zipf", 0.8), ("zipf", 1.0), ("zipf", 1.2), ("zipf", 1.5)]
SEED = 0x5EED0002
METRIC = "semisort Grecords/s & HBM roofline % at n=1e9; learned/batched vs plain form"
UNIT = "Grecords/s"


def dist_name(d):
    return f"{d[0]}-{d[1]:g}"


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, gpu_index: int):
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"semisort_bench_clocks_{os.getpid()}_{gpu_index}.csv")
        self.gpu = gpu_index

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_keys(sg, d, n, out):
    kind, p = d
    if kind == "uniform":
        return sg.uniform_exact(SEED, n, int(p), out=out)
    return sg.zipf(SEED, n, float(p), N=10**9, out=out)


def cpu_oracle_sample(sample_n: int, dists) -> dict:
    """Single-thread scale point: the oracle's std::stable_sort (the stable
    sort that defines a valid semisort_= output) on one host core, on the
    first sample_n records of each distribution (numpy generators, same seed
    as the GPU workload)."""
    import numpy as np

    import oracle
    import synth
    oracle.build()
    total_n, total_t = 0, 0.0
    for d in dists:
        keys = synth.uniform_exact(SEED, N_DEFAULT, int(d[1]), 0, sample_n) if d[0] == "uniform" else \
            synth.zipf(SEED, sample_n, float(d[1]), N=10**9)
        vals = np.arange(sample_n, dtype=np.uint64)
        t0 = time.perf_counter()
        oracle.stable_sort(keys, vals)
        total_t += time.perf_counter() - t0
        total_n += sample_n
    return {"value": total_n / total_t / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {sample_n} records of {', '.join(dist_name(d) for d in dists)} "
                      f"(same generators and seed as the GPU workload); std::stable_sort, 1 thread"}


def cpu_oracle_all_cores(torch, keys, vals, dists, sample_n: int) -> dict:
    """The oracle's stable sort on all host cores (libstdc++ parallel mode,
    OpenMP), on the first sample_n records of every headline distribution,
    copied from the GPU-generated inputs."""
    import numpy as np

    import oracle
    total_n, total_t, used = 0, 0.0, 0
    for k in keys:
        kh = k[:sample_n].view(torch.int64).cpu().numpy().view(np.uint64)
        vh = vals[:sample_n].view(torch.int64).cpu().numpy().view(np.uint64)
        t0 = time.perf_counter()
        _, _, used = oracle.stable_sort_parallel(kh, vh, 0)
        total_t += time.perf_counter() - t0
        total_n += len(kh)
    return {"value": total_n / total_t / 1e9, "unit": UNIT, "cores": used, "nproc": os.cpu_count(),
            "kind": "oracle",
            "sample": f"first {sample_n} records of each of {', '.join(dist_name(d) for d in dists)} "
                      f"(copied from the GPU inputs); __gnu_parallel::stable_sort on {used} threads"}


def headline_config(n, dists, world):
    return {"workload": f"semisort_equal n={n} (u64 key, u64 value=index), steps cycle over "
                        + ", ".join(dist_name(d) for d in dists),
            "parallelism": "replicas" if world > 1 else "single GPU",
            "l2": f"inputs ({16 * n / 1e9:.3g} GB per step) larger than L2; no flush"}


def run_reference(args, rank, world):
    """The reference arm: the oracle (the stable sort that defines a valid
    semisort_= output) on all host cores, each step a bounded sample -- the
    first ref_sample records -- of the step's distribution of the headline
    workload (same generators and seed), cycling over the same ten
    distributions.  Sample generation is outside the timed steps."""
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    import synth
    dists = [DISTS[int(i)] for i in args.dists.split(",")] if args.dists else DISTS
    sample_n = args.ref_sample
    samples = {}
    t_steps, used = [], 0
    for i in range(args.warmup + args.steps):
        d = dists[i % len(dists)]
        if d not in samples:
            samples[d] = synth.uniform_exact(SEED, N_DEFAULT, int(d[1]), 0, sample_n) if d[0] == "uniform" else \
                synth.zipf(SEED, sample_n, float(d[1]), N=10**9)
        keys = samples[d]
        vals = np.arange(sample_n, dtype=np.uint64)
        t0 = time.perf_counter()
        _, _, used = oracle.stable_sort_parallel(keys, vals, 0)
        if i >= args.warmup:
            t_steps.append(time.perf_counter() - t0)
    total_t = sum(t_steps)
    value = args.steps * sample_n / total_t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": headline_config(args.n, dists, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "nproc": os.cpu_count(), "kind": "oracle",
                             "sample": f"first {sample_n} records of each step's distribution; "
                                       f"__gnu_parallel::stable_sort on {used} threads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def alg_bytes(st: dict) -> int:
    """Compulsory bytes of the method's passes for one call (u64 key + u64
    value): per record and distribution level 8 B (count: key) + 32 B
    (distribute: read and write key and value); per refined or copied record
    32 B (read and write)."""
    dist = sum(st.get(f"dist_l{i}", 0) for i in range(4))
    return 40 * dist + 32 * st.get("refined", 0) + 32 * st.get("copied", 0)


def max_over_ranks(ms, world, device):
    """The slowest rank's time: with N replicas, the job ends with the last one."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, n, steps, ms):
    """Whole-job records per second (Grec/s): every replica processes n
    records per step, all within the slowest rank's time."""
    return world * n * steps / (ms / 1000.0) / 1e9


DIST_REGION = ("paper_2304_10078_gb300/csrc/ss_kernels.cuh",
               "// distribute: the second pass of Blocked Distributing",
               "static __global__ void __launch_bounds__(1024) k_scan_items")


def kernel_source_hash():
    """sha256 of the source the distribute kernel is built from: its section of
    the kernels file (the kernel and its helpers) and the shared primitives."""
    import hashlib
    h = hashlib.sha256()
    path, start, end = DIST_REGION
    with open(os.path.join(ROOT, path)) as f:
        text = f.read()
    a = text.index(start)
    h.update(text[a:text.index(end, a)].encode())
    with open(os.path.join(ROOT, "paper_2304_10078_gb300/csrc/ss_common.cuh"), "rb") as f:
        h.update(f.read())
    return h.hexdigest()


def dram_traffic_per_launch(n):
    """DRAM bytes (read + write) of one distribute.L0 launch on n records,
    from the committed ncu counters scaled by records; None when the kernel's
    source changed after the counters were taken."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)["distribute.L0"]
        if kernel_source_hash() != t["kernel_source_sha256"]:
            return None
        return t["bytes_per_record"] * n
    except (OSError, KeyError, ValueError):
        return None


LESS_EXTRA = [("exponential", 1e-6), ("gaussian_mixture", 8)]


def time_op(ss, sg, torch, name, keys, dists, vals, kout, vout, ws, n, stream):
    """One warm-up call, then one timed call per input distribution (CUDA
    events on the launching stream), for an operation other than the headline.
    collect-reduce and histogram run on the ten headline distributions;
    semisort_< on uniform-10^9, Zipf-1.2, floor(Exp(10^-6)) and an 8-component
    Gaussian mixture."""
    learned = name == "semisort_less_learned"
    flags = (ss.FLAG_IDENTITY_HASH if name == "semisort_equal_identity" else 0) | \
        (ss.FLAG_HASH_BUCKETS if name == "semisort_less_hash" else 0) | \
        (ss.FLAG_SWAP_OUTPUT if name == "semisort_equal_swap" else 0)
    opt_plain = ss.make_options(seed=1, flags=flags, splitter_mode=1 if learned else 0)
    opt_timed = ss.make_options(seed=1, flags=flags | ss.FLAG_PHASE_TIMING, splitter_mode=1 if learned else 0)
    nu = torch.zeros(1, dtype=torch.uint64, device="cuda")
    names = [dist_name(d) for d in dists]
    inputs = list(keys)
    extra = []
    if name.startswith("semisort_less"):
        pick = [i for i, d in enumerate(dists) if d in (("uniform", 10**9), ("zipf", 1.2))]
        inputs = [keys[i] for i in pick]
        names = [names[i] for i in pick]
        for kind, p in LESS_EXTRA:
            t = sg.exponential(SEED, n, p) if kind == "exponential" else sg.gaussian_mixture(SEED, n, int(p))
            extra.append(t)
            inputs.append(t)
            names.append(f"{kind}-{p:g}")

    def call(k, opt=opt_plain):
        if name.startswith("semisort_equal"):
            ss.semisort_equal(k, vals, keys_out=kout, vals_out=vout, workspace=ws, options=opt)
        elif name.startswith("semisort_less"):
            ss.semisort_less(k, vals, keys_out=kout, vals_out=vout, workspace=ws, options=opt)
        elif name == "collect_reduce":
            ss.collect_reduce(k, vals, capacity=n, ukeys_out=kout, sums_out=vout, num_unique=nu, workspace=ws,
                              options=opt)
        else:
            ss.histogram(k, capacity=n, ukeys_out=kout, counts_out=vout.view(torch.uint32)[:n], num_unique=nu,
                         workspace=ws, options=opt)

    call(inputs[0])
    torch.cuda.synchronize()
    per, phases, total, balance = {}, {}, 0.0, {}
    for k, nm in zip(inputs, names):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        call(k)
        b.record(stream)
        b.synchronize()
        per[nm] = a.elapsed_time(b)
        total += per[nm]
        call(k, opt_timed)  # a second, instrumented call for the phase split
        torch.cuda.synchronize()
        for pn, pm in ss.phase_times():
            phases[pn] = phases.get(pn, 0.0) + pm / len(inputs)
        if name in ("semisort_less", "semisort_less_learned"):
            st = ss.stats(ws)
            balance[nm] = {"splitters": ["sampled", "learned", "learned rejected"][st["l0_splitters"]],
                           "max_light_bucket_over_mean": st["l0_max_light_bucket"] / (n / max(1, st["l0_light_buckets"])),
                           "records_at_level3": st["dist_l2"], "learn_steps": st["learn_steps"]}
    err = ss.last_device_error(ws)
    del extra
    out = {"value": n * len(inputs) / (total / 1000.0) / 1e9, "unit": UNIT, "device_error": err,
           "per_distribution_ms": per, "phase_ms": phases}
    if balance:
        out["top_level_balance"] = balance
    return out


BATCH_SEED = 0x5EED0004


def batched_workload(sg, torch, ni=4096, lo=8, hi=22):
    """4096 instances of floor(2^U[8,22]) records; instance i draws Zipf keys
    with s ~ U[0.6, 1.5] over D ~ floor(exp(U[ln 10, ln size])) ranks, ranks
    hashed with the instance's own seed (keys differ across instances)."""
    import numpy as np

    import synth
    idx = np.arange(ni, dtype=np.uint64)
    sizes = np.floor(2.0 ** (lo + (hi - lo) * synth.unit(synth.rand64(BATCH_SEED, 0x1A, idx)))).astype(np.int64)
    s_i = 0.6 + 0.9 * synth.unit(synth.rand64(BATCH_SEED, 0x1B, idx))
    ud = synth.unit(synth.rand64(BATCH_SEED, 0x1C, idx))
    d_i = np.maximum(2, np.floor(np.exp(np.log(10) + (np.log(np.maximum(sizes, 10)) - np.log(10)) * ud)))
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(off[-1])
    keys = torch.empty(n, dtype=torch.uint64, device="cuda")
    for i in range(ni):
        if sizes[i]:
            sg.zipf(BATCH_SEED + 1 + i, int(sizes[i]), float(s_i[i]), N=int(d_i[i]), out=keys[off[i]:off[i + 1]])
    return off, keys, n


def bench_batched(ss, sg, torch, stream, reps=3):
    """The batched forms on the 4096-instance workload: one autotuned call
    (eager, and captured once in a CUDA graph and replayed) against one plain
    call per instance, for semisort_= and collect-reduce."""
    import numpy as np

    from paper_2304_10078_gb300.autotune import CANDIDATES, Tuner
    off_h, keys, n = batched_workload(sg, torch)
    ni = len(off_h) - 1
    off = torch.from_numpy(off_h).cuda().view(torch.uint64)
    vals = sg.iota(n)
    kout, vout = torch.empty_like(keys), torch.empty_like(vals)
    nu = torch.zeros(ni, dtype=torch.uint64, device="cuda")
    oo = torch.zeros(ni + 1, dtype=torch.uint64, device="cuda")
    tuner = Tuner()
    big = int(np.max(np.diff(off_h)))
    res = {"workload": f"{ni} instances, {n} records (u64 key, u64 value = index), sizes floor(2^U[8,22]), "
                       "per-instance Zipf s ~ U[0.6,1.5] over floor(exp(U[ln 10, ln size])) ranks"}

    def timed(fn, k):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / k

    for op in ("semisort_equal", "collect_reduce"):
        code = ss.OP_EQUAL if op == "semisort_equal" else ss.OP_REDUCE
        ws_bytes = max(ss.workspace_size_batched(code, ss.SS_U64, ss.SS_U64, n, ni, ss.make_options(**c))
                       for c in CANDIDATES + [{}])
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")

        def run(opt, st=None):
            if op == "semisort_equal":
                ss.semisort_equal_batched(keys, vals, off, keys_out=kout, vals_out=vout, workspace=ws, options=opt,
                                          stream=st)
            else:
                ss.collect_reduce_batched(keys, vals, off, capacity=n, ukeys_out=kout, sums_out=vout, num_unique=nu,
                                          out_offsets=oo, workspace=ws, options=opt, stream=st)

        opt, tune_ms = tuner.best(op + "_batched", n, ni, run)
        eager_ms = timed(lambda: run(opt), reps)
        launches = ss.kernel_launches()
        assert ss.last_device_error(ws) == 0
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            run(opt, side)
        torch.cuda.synchronize()
        graph_ms = timed(g.replay, reps)
        assert ss.last_device_error(ws) == 0
        del g
        # one plain call per instance (untuned defaults), on the same stream
        plain = ss.make_options(seed=1)
        ws1 = ss.alloc_workspace(code, keys[:big], vals[:big], plain)
        nu1 = torch.zeros(1, dtype=torch.uint64, device="cuda")

        def per_instance():
            for i in range(ni):
                a, b = int(off_h[i]), int(off_h[i + 1])
                if a == b:
                    continue
                if op == "semisort_equal":
                    ss.semisort_equal(keys[a:b], vals[a:b], keys_out=kout[a:b], vals_out=vout[a:b], workspace=ws1,
                                      options=plain)
                else:
                    ss.collect_reduce(keys[a:b], vals[a:b], capacity=b - a, ukeys_out=kout[a:b], sums_out=vout[a:b],
                                      num_unique=nu1, workspace=ws1, options=plain)
        per_ms = timed(per_instance, 1)
        assert ss.last_device_error(ws1) == 0
        del ws, ws1
        res[op] = {"unit": UNIT, "batched_graph": n / (graph_ms / 1000) / 1e9,
                   "batched_eager": n / (eager_ms / 1000) / 1e9, "per_instance_calls": n / (per_ms / 1000) / 1e9,
                   "ms": {"batched_graph": graph_ms, "batched_eager": eager_ms, "per_instance_calls": per_ms},
                   "kernel_launches_per_batched_call": launches,
                   "tuned_options": {k: getattr(opt, k) for k in ("subarray", "alpha", "n_light_log2")},
                   "tuning_ms": tune_ms}
    return res


RMAT_SEED = 0x5EED0005


def rmat_partitions(m, parts=64):
    """Contiguous edge ranges with seeded log-uniform sizes 2^U[0,4], scaled to m."""
    import numpy as np

    import synth
    w = 2.0 ** (4.0 * synth.unit(synth.rand64(RMAT_SEED, 0x9A, np.arange(parts, dtype=np.uint64))))
    cut = np.floor(np.cumsum(w) / w.sum() * m).astype(np.int64)
    cut[-1] = m
    return np.concatenate([[0], cut]).astype(np.int64)


def bench_rmat_csr(ss, sg, torch, stream, reps=3, scale=26, m=1 << 30):
    """CSR build of an R-MAT graph (2^26 vertices, 2^30 edges, u32 src / u32
    dst) over 64 uneven edge partitions: semisort_< on src with dst as value
    plus the degree histogram.  One batched call of each, against one call
    per partition (sampled splitters) and per partition with learned
    splitters.  Records = edges."""
    import numpy as np
    src, dst = sg.rmat_edges(RMAT_SEED, m, scale)
    off_h = rmat_partitions(m)
    parts = len(off_h) - 1
    off = torch.from_numpy(off_h).cuda().view(torch.uint64)
    ks, vs = torch.empty_like(src), torch.empty_like(dst)
    uk = torch.empty_like(src)
    cnt = torch.empty(m, dtype=torch.uint32, device="cuda")
    nu = torch.zeros(parts, dtype=torch.uint64, device="cuda")
    oo = torch.zeros(parts + 1, dtype=torch.uint64, device="cuda")
    plain = ss.make_options(seed=1)
    learned_b = ss.make_options(seed=1, splitter_mode=1)
    ws_l = ss.alloc_workspace_batched(ss.OP_LESS, src, off, dst, learned_b)
    ws_h = ss.alloc_workspace_batched(ss.OP_HIST, src, off, None, plain)

    def batched(opt=plain):
        ss.semisort_less_batched(src, dst, off, keys_out=ks, vals_out=vs, workspace=ws_l, options=opt)
        ss.histogram_batched(src, off, capacity=m, ukeys_out=uk, counts_out=cnt, num_unique=nu, out_offsets=oo,
                             workspace=ws_h, options=plain)

    def timed(fn, k):
        fn()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / k

    t_b = timed(batched, reps)
    assert ss.last_device_error(ws_l) == 0 and ss.last_device_error(ws_h) == 0
    t_bl = timed(lambda: batched(learned_b), reps)
    assert ss.last_device_error(ws_l) == 0
    kept = ss.stats(ws_l)["l0_max_sample_range"]
    del ws_l, ws_h
    big = int(np.max(np.diff(off_h)))
    learned = ss.make_options(seed=1, splitter_mode=1)
    w1l = ss.alloc_workspace(ss.OP_LESS, src[:big], dst[:big], learned)
    w1h = ss.alloc_workspace(ss.OP_HIST, src[:big], None, plain)
    nu1 = torch.zeros(1, dtype=torch.uint64, device="cuda")
    out = {}
    for mode, opt in (("per_partition_sampled", plain), ("per_partition_learned", learned)):
        def per_part():
            for p in range(parts):
                a, b = int(off_h[p]), int(off_h[p + 1])
                ss.semisort_less(src[a:b], dst[a:b], keys_out=ks[a:b], vals_out=vs[a:b], workspace=w1l, options=opt)
                ss.histogram(src[a:b], capacity=b - a, ukeys_out=uk[a:b], counts_out=cnt[a:b], num_unique=nu1,
                             workspace=w1h, options=plain)
        out[mode] = timed(per_part, 1)
        assert ss.last_device_error(w1l) == 0
    return {"workload": f"R-MAT scale {scale}, {m} edges (u32 src, u32 dst), 64 partitions of sizes 2^U[0,4]",
            "unit": UNIT, "batched": m / (t_b / 1000) / 1e9, "batched_learned": m / (t_bl / 1000) / 1e9,
            "batched_learned_partitions_kept_model": kept,
            "per_partition_sampled": m / (out["per_partition_sampled"] / 1000) / 1e9,
            "per_partition_learned": m / (out["per_partition_learned"] / 1000) / 1e9,
            "ms": {"batched": t_b, "batched_learned": t_bl, **out}}


SWEEP_DISTS = [("zipf", 1.2), ("uniform", 10**7)]


def bench_sweeps(ss, sg, torch, stream, reps=3):
    """The paper's two scaling experiments (Sec. 5, input size scalability and
    varying key lengths) for semisort_= on one GPU:
    * input size: n = 10^7 .. 10^9 (u64 key, u64 value = index);
    * key width at n = 10^9: 32-bit keys with 32-bit values, 64-bit keys with
      64-bit values, 128-bit keys with 64-bit values (the library has no
      128-bit value type).  32-bit keys are the high halves of the 64-bit
      keys; a 128-bit key is (64-bit key, its SplitMix64 mix), so distinct
      64-bit keys stay distinct.
    Zipf 1.2 and uniform 10^7 (the paper's representative distributions).
    Device time of one call, median of `reps`, inputs resident in HBM."""
    out = {"unit": UNIT, "input_size": {}, "key_width": {}}

    def timed(fn):
        fn()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    for d in SWEEP_DISTS:
        row = {}
        for n in (10**7, 3 * 10**7, 10**8, 3 * 10**8, 10**9):
            k = make_keys(sg, d, n, None)
            v = sg.iota(n)
            ko, vo = torch.empty_like(k), torch.empty_like(v)
            ws = ss.alloc_workspace(ss.OP_EQUAL, k, v, ss.make_options(seed=1))
            ms = timed(lambda: ss.semisort_equal(k, v, keys_out=ko, vals_out=vo, workspace=ws,
                                                 options=ss.make_options(seed=1)))
            assert ss.last_device_error(ws) == 0
            row[str(n)] = n / (ms / 1000) / 1e9
            del k, v, ko, vo, ws
            torch.cuda.empty_cache()
        out["input_size"][dist_name(d)] = row
    n = 10**9
    for d in SWEEP_DISTS:
        row = {}
        k64 = make_keys(sg, d, n, None)
        for width in (32, 64, 128):
            if width == 32:
                k = (k64.view(torch.int64) >> 32).to(torch.int32).view(torch.uint32)
                v = sg.iota(n).view(torch.int64).to(torch.int32).view(torch.uint32)
            elif width == 64:
                k, v = k64, sg.iota(n)
            else:
                hi = ss.hash_u64(k64, 0x5EED)
                k = torch.stack([k64.view(torch.int64), hi.view(torch.int64)], dim=1).view(torch.uint64)
                v = sg.iota(n)
            ko, vo = torch.empty_like(k), torch.empty_like(v)
            ws = ss.alloc_workspace(ss.OP_EQUAL, k, v, ss.make_options(seed=1))
            ms = timed(lambda: ss.semisort_equal(k, v, keys_out=ko, vals_out=vo, workspace=ws,
                                                 options=ss.make_options(seed=1)))
            assert ss.last_device_error(ws) == 0
            row[f"{width}-bit"] = n / (ms / 1000) / 1e9
            del k, v, ko, vo, ws
            torch.cuda.empty_cache()
        out["key_width"][dist_name(d)] = row
        del k64
        torch.cuda.empty_cache()
    out["workload"] = ("semisort_= (value = index); input sizes 1e7..1e9 with u64/u64; key widths at n=1e9: "
                       "u32/u32, u64/u64, u128/u64; distributions " + ", ".join(dist_name(d) for d in SWEEP_DISTS))
    return out


def e2e_pipelined(ss, torch, hk, hv, n, steps, ws, opt, hko=None, hvo=None):
    """End to end through the public API with host buffers: every step copies
    its input (keys, values) from pinned host memory to the device, runs
    semisort_=, and copies the output back to pinned host memory.  Steps are
    pipelined on three streams with two device buffer sets, so step i+1's
    upload and step i-1's download overlap step i's call; all copies are
    inside the timed region.  One untimed step first warms the copy path."""
    u64 = torch.uint64
    s_cmp = torch.cuda.current_stream()
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    din = [(torch.empty(n, dtype=u64, device="cuda"), torch.empty(n, dtype=u64, device="cuda")) for _ in range(2)]
    dout = [(torch.empty(n, dtype=u64, device="cuda"), torch.empty(n, dtype=u64, device="cuda")) for _ in range(2)]
    if hko is None:
        hko = torch.empty(n, dtype=u64, pin_memory=True)
        hvo = torch.empty(n, dtype=u64, pin_memory=True)
    din[0][0].copy_(hk, non_blocking=True)
    din[0][1].copy_(hv, non_blocking=True)
    ss.semisort_equal(din[0][0], din[0][1], keys_out=dout[0][0], vals_out=dout[0][1], workspace=ws, options=opt)
    hko.copy_(dout[0][0], non_blocking=True)
    hvo.copy_(dout[0][1], non_blocking=True)
    ev = lambda: torch.cuda.Event()
    ev_in, ev_cmp, ev_out = [ev(), ev()], [ev(), ev()], [ev(), ev()]
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s_cmp)
    s_in.wait_event(e0)
    s_out.wait_event(e0)
    for i in range(steps):
        b = i % 2
        if i >= 2:
            s_in.wait_event(ev_cmp[b])   # step i-2 has consumed din[b]
        with torch.cuda.stream(s_in):
            din[b][0].copy_(hk, non_blocking=True)
            din[b][1].copy_(hv, non_blocking=True)
        ev_in[b].record(s_in)
        s_cmp.wait_event(ev_in[b])
        if i >= 2:
            s_cmp.wait_event(ev_out[b])  # step i-2's download has read dout[b]
        ss.semisort_equal(din[b][0], din[b][1], keys_out=dout[b][0], vals_out=dout[b][1], workspace=ws,
                          options=opt, stream=s_cmp)
        ev_cmp[b].record(s_cmp)
        s_out.wait_event(ev_cmp[b])
        with torch.cuda.stream(s_out):
            hko.copy_(dout[b][0], non_blocking=True)
            hvo.copy_(dout[b][1], non_blocking=True)
        ev_out[b].record(s_out)
    s_cmp.wait_event(ev_out[(steps - 1) % 2])
    e1.record(s_cmp)
    torch.cuda.synchronize()
    assert ss.last_device_error(ws) == 0
    t = e0.elapsed_time(e1) / 1000.0
    # the last step's output is the input's semisort: spot-check stability of the download
    ok = bool(torch.equal(hko[:1024], dout[(steps - 1) % 2][0][:1024].cpu()))
    del din, dout
    return n * steps / t / 1e9, t, ok


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--ref-sample", type=int, default=1 << 24)
    ap.add_argument("--cpu-sample", type=int, default=1 << 25,
                    help="records per distribution for the all-core oracle leg (0: skip both CPU legs)")
    ap.add_argument("--cpu-scale-sample", type=int, default=1 << 24,
                    help="records per distribution for the single-thread scale point (0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=8)
    ap.add_argument("--dists", default="", help="comma-separated indices into the distribution list")
    ap.add_argument("--ops", default="collect_reduce,histogram,semisort_equal_identity,semisort_equal_swap,"
                                      "semisort_less,"
                                      "semisort_less_learned,semisort_less_hash,batched,rmat_csr,sweeps",
                    help="further operations timed after the headline (empty: none)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist

    import paper_2304_10078_gb300 as ss
    import synth.gpu as sg

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    ss.lib()
    n = args.n
    dists = [DISTS[int(i)] for i in args.dists.split(",")] if args.dists else DISTS
    # pinned host buffers of the end-to-end leg, allocated before the large
    # device allocations (their placement then matches a standalone run)
    e2e_host = None
    if rank == 0 and args.e2e_steps > 0:
        e2e_host = [torch.empty(n, dtype=torch.uint64, pin_memory=True) for _ in range(4)]
    # device-resident inputs: one key array per distribution, one value array
    keys = []
    vals = sg.iota(n)
    for d in dists:
        keys.append(make_keys(sg, d, n, None))
    torch.cuda.synchronize()
    kout = torch.empty(n, dtype=torch.uint64, device="cuda")
    vout = torch.empty(n, dtype=torch.uint64, device="cuda")
    opt = ss.make_options(seed=1)
    opt_timed = ss.make_options(seed=1, flags=ss.FLAG_PHASE_TIMING)
    ops = [o for o in args.ops.split(",") if o]
    op_codes = {"semisort_equal": ss.OP_EQUAL, "collect_reduce": ss.OP_REDUCE, "histogram": ss.OP_HIST,
                "semisort_less": ss.OP_LESS, "semisort_less_learned": ss.OP_LESS, "semisort_less_hash": ss.OP_LESS,
                "semisort_equal_identity": ss.OP_EQUAL, "semisort_equal_swap": ss.OP_EQUAL}
    ws_bytes = max(ss.workspace_size(op_codes[o], ss.SS_U64, ss.SS_U64, n, opt)
                   for o in ["semisort_equal"] + ops if o in op_codes)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step(i, o=opt):
        ss.semisort_equal(keys[i % len(dists)], vals, keys_out=kout, vals_out=vout, workspace=ws, options=o)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    assert ss.last_device_error(ws) == 0

    # ---- timed region: the plain library calls back to back (no
    # instrumentation, no host synchronization between steps) ----
    launches = 0
    clocks = Clocks(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev_steps = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev_steps[0].record(stream)
    for i in range(args.steps):
        step(i)
        launches += ss.kernel_launches()
        ev_steps[i + 1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    elapsed_ms = ev_steps[0].elapsed_time(ev_steps[-1])
    if world > 1:
        dist.barrier()
    elapsed_ms = max_over_ranks(elapsed_ms, world, "cuda")
    assert ss.last_device_error(ws) == 0
    per_dist = {dist_name(d): [] for d in dists}
    for i in range(args.steps):
        per_dist[dist_name(dists[i % len(dists)])].append(ev_steps[i].elapsed_time(ev_steps[i + 1]))

    # ---- instrumented pass over the same K steps: per-kernel CUDA events
    # recorded by the library on the launching stream, and the exact record
    # classes of each call (for the byte model) ----
    phases = {}
    dominant, dom_bytes, alg_total, instr_ms = [], [], 0, 0.0
    for i in range(args.steps):
        e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e_a.record(stream)
        step(i, opt_timed)
        e_b.record(stream)
        e_b.synchronize()
        instr_ms += e_a.elapsed_time(e_b)
        ph = dict()
        for name, ms in ss.phase_times():
            ph[name] = ph.get(name, 0.0) + ms
        for name, ms in ph.items():
            phases.setdefault(name, []).append(ms)
        st = ss.stats(ws)
        alg_total += alg_bytes(st)
        dominant.append(ph.get("distribute.L0", float("nan")))
        dom_bytes.append(32 * st.get("dist_l0", 0))
    assert ss.last_device_error(ws) == 0

    value = job_throughput(world, n, args.steps, elapsed_ms)
    peak, peak_kind = load_peaks()
    dom_ms = [t for t in dominant if t == t]
    dom_avg = sum(dom_ms) / len(dom_ms) if dom_ms else float("nan")
    dom_b = sum(dom_bytes) / len(dom_bytes)
    achieved = dom_b / (dom_avg / 1000.0) / 1e9 if dom_ms else None
    traffic = dram_traffic_per_launch(n)

    by_op = {}
    for o in ops:
        if o not in ("batched", "rmat_csr", "sweeps"):
            by_op[o] = time_op(ss, sg, torch, o, keys, dists, vals, kout, vout, ws, n, stream)

    # end to end through the public API with host buffers (own staging buffers)
    e2e = None
    cpu = None
    if rank == 0 and args.e2e_steps > 0:
        d_i = next((i for i, d in enumerate(dists) if d == ("zipf", 1.2)), len(dists) - 1)
        hk, hv, hko, hvo = e2e_host
        hk.copy_(keys[d_i])
        hv.copy_(vals)
        del kout, vout
        torch.cuda.empty_cache()
        v_e2e, t_e2e, ok = e2e_pipelined(ss, torch, hk, hv, n, args.e2e_steps, ws, opt, hko, hvo)
        e2e = {"value": v_e2e, "unit": UNIT, "h2d_bytes_per_step": 16 * n, "d2h_bytes_per_step": 16 * n,
               "workload": f"semisort_equal n={n} {dist_name(dists[d_i])}, {args.e2e_steps} steps pipelined "
                           "(upload, call, download on three streams, two device buffer sets)",
               "seconds": t_e2e, "download_check": ok}
        del hk, hv, hko, hvo, e2e_host
    if rank == 0 and args.cpu_sample:
        cpu = cpu_oracle_all_cores(torch, keys, vals, dists, args.cpu_sample)
    if "batched" in ops or "rmat_csr" in ops or "sweeps" in ops:
        keys.clear()
        del ws, vals
        torch.cuda.empty_cache()
    if "batched" in ops:
        by_op["batched"] = bench_batched(ss, sg, torch, stream, reps=3)
        torch.cuda.empty_cache()
    if "rmat_csr" in ops:
        by_op["rmat_csr"] = bench_rmat_csr(ss, sg, torch, stream, reps=3)
        torch.cuda.empty_cache()
    if "sweeps" in ops:
        by_op["sweeps"] = bench_sweeps(ss, sg, torch, stream)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    if cpu is not None and args.cpu_scale_sample:
        cpu["single_thread_scale_point"] = cpu_oracle_sample(args.cpu_scale_sample, [dists[min(3, len(dists) - 1)],
                                                                                     dists[-2 if len(dists) > 1
                                                                                           else 0]])
    ms_step = elapsed_ms / args.steps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": headline_config(n, dists, world),
        "roofline": {"bound": "hbm", "kernel": "distribute.L0",
                     "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "alg_bytes_per_launch": dom_b, "avg_launch_ms": dom_avg,
                     "measured_in": "instrumented pass over the same steps (per-kernel CUDA events on the "
                                    "launching stream)"},
        "path_roofline": {"alg_bytes_per_step": alg_total / args.steps,
                          "achieved_gbs": alg_total / (elapsed_ms / 1000.0) / 1e9,
                          "frac": alg_total / (elapsed_ms / 1000.0) / 1e9 / peak},
        "instrumented_ms_per_step": instr_ms / args.steps,
        "per_distribution_ms": {k: (sum(v) / len(v) if v else None) for k, v in per_dist.items()},
        "phase_ms": {k: sum(v) / len(v) for k, v in phases.items()},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "other_ops": by_op,
    }
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
