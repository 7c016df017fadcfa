"""Benchmark of the FliX hot path on GB300 (one JSON line on stdout).

Workload (read-scale case): 2^26 distinct uniform uint64 keys bulk-loaded at node size 64 (32 keys
per node, 2^21 buckets).  One step runs every stage of the hot path once over fresh-from-HBM
batches:
    lookup 2^24 (30% misses) -> successor 2^24 (30% misses) -> range 2^18 (1..1000 keys each)
    -> insert 2^20 fresh keys -> delete the same 2^20 keys -> restructure.
Each batch is sorted on the GPU inside the timed region (the paper's unsorted-query mode, Sec. 6.4).
The insert/delete pair and the restructure return the index to its starting layout, so every step
does the same work.  Ops per step = 2^24 + 2^24 + 2^18 + 2^20 + 2^20.

`value` is whole-job Mops/s over device-resident inputs; `e2e` is the same step through the public
Python API from pinned host buffers with the host<->device copies inside the timed region.
`--impl reference` times the CPU oracle instead (a bounded sample per step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workload as W  # noqa: E402

LOG_LOAD = 26
LOG_Q = 24
LOG_R = 18
LOG_U = 20
NODE_SIZE = 64
KW = 64
METRIC = "Mops/s per op mix at 1 GB300 (bit-exact vs oracle), % HBM roofline; p50/p99 latency"
WORKLOAD = ("read-scale: 2^26 distinct uniform uint64 keys/values, node size 64; per step lookup 2^24 "
            "(30% miss) + successor 2^24 (30% miss) + range 2^18 (1-1000 keys) + insert 2^20 fresh + "
            "delete the same 2^20 + restructure")


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def make_inputs(seed, log_load=LOG_LOAD, log_q=LOG_Q, log_r=LOG_R, log_u=LOG_U):
    c = W.read_scale(seed=seed, n_load=1 << log_load, batch=1 << log_q, n_range=1 << log_r)
    n_load = 1 << log_load
    fresh = W.universe(KW, seed, n_load + (1 << log_q), n_load + (1 << log_q) + (1 << log_u))
    c["ins_keys"] = fresh
    c["ins_vals"] = W.values_for(KW, fresh, salt=9)
    # successor queries: a second seeded draw with the same recipe
    c2 = W.read_scale(seed=seed + 1, n_load=1 << log_load, batch=1 << log_q, n_range=0)
    c["succ_queries"] = c2["queries"]
    return c


def max_over_ranks(x: float, world: int) -> float:
    """The slowest rank's time (replicas run independently; the job ends with the last one)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mops(ops_per_rank_step: int, world: int, ms_per_step: float) -> float:
    """Whole-job throughput: every rank's ops over the slowest rank's step time."""
    return ops_per_rank_step * world / (ms_per_step * 1e-3) / 1e6


def ops_per_step(log_q=LOG_Q, log_r=LOG_R, log_u=LOG_U):
    return dict(lookup=1 << log_q, successor=1 << log_q, range=1 << log_r, insert=1 << log_u, delete=1 << log_u)


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu_id), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0=None, t1=None):
        """Samples taken between wall-clock times t0 and t1 (seconds since the epoch)."""
        import datetime
        rows = []
        for line in (getattr(self, "out", "") or "").splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                ts = datetime.datetime.strptime(p[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                ts = None
            if t0 is not None and ts is not None and not (t0 <= ts <= t1):
                continue
            try:
                rows.append(dict(sm=float(p[1]), smax=float(p[2]), power=float(p[3]) if p[3] not in ("[N/A]", "N/A") else 0.0,
                                 hw=p[5], hwt=p[6], swt=p[7], pcap=p[8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        reasons = set()
        for r in rows:
            if r["hw"] == "Active":
                reasons.add("hw_slowdown")
            if r["hwt"] == "Active":
                reasons.add("hw_thermal_slowdown")
            if r["swt"] == "Active":
                reasons.add("sw_thermal_slowdown")
            if r["pcap"] == "Active":
                reasons.add("sw_power_cap")
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["smax"] for r in rows),
                "power_w_max": max(r["power"] for r in rows), "samples": len(rows), "reasons": sorted(reasons)}


def gpu_id_for_smi(torch):
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
    except Exception:
        return os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def traffic_record(kernel):
    """ncu DRAM bytes per item for `kernel`, valid only while the source it was compiled from (the
    recorded file, or the part of it between the recorded markers) is unchanged."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            d = json.load(f)[kernel]
        src = open(os.path.join(ROOT, "paper_2604_16725_gb300", "csrc", d["source"]), "rb").read()
        if d.get("until"):                 # the record covers the source between two markers
            src = src[src.index(d["from"].encode()) if d.get("from") else 0:src.index(d["until"].encode())]
        if hashlib.sha256(src).hexdigest() != d["sha256"]:
            return None
        return d
    except Exception:
        return None


def step_bytes(rcap, log_load=None, log_q=None, log_r=LOG_R, log_u=LOG_U):
    """Algorithmic bytes per read-scale step of each search-and-apply kernel: what its job requires
    it to read and write, with uniform keys (ks = vs = 8 bytes, node size 64, half-full nodes after
    the step's restructure).  T = nb (1 - e^(-m / nb)) nodes are touched by m uniform keys; a hit or
    a successor reads one 32-byte value sector; rcap = the range pairs of the step."""
    log_load = LOG_LOAD if log_load is None else log_load
    log_q = LOG_Q if log_q is None else log_q
    ks = vs = 8
    h = NODE_SIZE // 2
    n, B, R, U = 1 << log_load, 1 << log_q, 1 << log_r, 1 << log_u
    nb = n // h
    T = lambda m: nb * (1.0 - np.exp(-m / nb))  # noqa: E731
    hits = 0.7 * B
    node = h * ks                                      # a node's key prefix
    part = lambda m, out: nb * ks + m * ks + out        # noqa: E731  (MKBA + sorted keys + bk or off)
    return {
        "partition": part(B, 4 * B) * 2 + part(R, 4 * R) + part(U, 4 * nb) * 2,
        # sorted key, position and bucket; touched node prefixes; value sectors; results
        "read_point": (B * (ks + 8) + T(B) * node + hits * 32 + B * vs)
                      + (B * (ks + 8) + T(B) * node + B * 32 + B * (ks + vs)),
        # windowed delivery: the position tag the read kernel writes beside each result, then
        # (position, result) read and the result written to its position
        "read_unsort": (B * 4 + B * (4 + vs) + B * vs) + (B * 4 + B * (4 + ks + vs) + B * (ks + vs)),
        # lower bound, position, bucket, upper bound; first node's prefix; start (3 words) and count out
        "range_count": R * (ks + 8) + R * ks + T(R) * node + R * (12 + 8),
        # the pairs copied (read and written), the start and the offsets per query
        "range_fill": rcap * 2 * (ks + vs) + R * (4 + 12 + 16),
        # net updates (key, op) and touched node prefixes, per insert and per delete batch
        "update_count": 2 * (U * (ks + 4) + T(U) * node + nb * (4 + 8)),
        # net updates (key, value, op); touched nodes' pairs read and written
        "update_apply": 2 * (U * (2 * ks + 4)) + 2 * (T(U) * 2 * h * (ks + vs)),
        # one-pass restructure: every pair read and written once
        "gather": n * 2 * (ks + vs),
        # histograms of every digit: one read of the keys of each sort
        "sort_hist": (2 * B + R + 2 * U) * ks,
    }


def apply_rooflines(prof, steps, peak, peak_kind, rcap):
    out = {"peak": peak, "peak_kind": peak_kind + " hbm copy", "unit": "GB/s",
           "timing": "per-launch CUDA events in a second pass of the same steps (profiling adds an event pair "
                     "per launch and reads each sort's pass plan back, so these times are slightly above "
                     "the unprofiled step's)"}
    for k, by in step_bytes(rcap).items():
        p = prof.get(k)
        if not p or not p["ms"]:
            continue
        ms = p["ms"] / steps
        ach = by / (ms * 1e-3) / 1e9
        out[k] = {"bytes_per_step": int(by), "ms_per_step": round(ms, 4), "achieved": round(ach, 1),
                  "frac": round(ach / peak, 3)}
    return out


def run_step(torch, idx, bufs, stream, events=None):
    """One step on device-resident inputs.  events: dict phase -> (start, end) CUDA events."""
    def ev(name, which):
        if events is not None:
            events[name][which].record(stream)

    ev("lookup", 0)
    idx.lookup(bufs["q"], stream=stream, out=bufs["lv"], found=False)
    ev("lookup", 1)
    ev("successor", 0)
    idx.successor(bufs["sq"], stream=stream)
    ev("successor", 1)
    ev("range", 0)
    idx.range(bufs["lo"], bufs["hi"], capacity=bufs["rcap"], stream=stream)
    ev("range", 1)
    ev("insert", 0)
    idx.insert(bufs["ik"], bufs["iv"], stream=stream)
    ev("insert", 1)
    ev("delete", 0)
    idx.delete(bufs["ik"], stream=stream)
    ev("delete", 1)
    ev("restructure", 0)
    idx.restructure(stream=stream)
    ev("restructure", 1)


def timed_span(torch, st, spans, fn):
    """Run fn() enqueueing work on stream st; with a list `spans`, bracket it by timing events."""
    if spans is None:
        return fn()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    r = fn()
    b.record(st)
    spans.append((a, b))
    return r


def upload_inputs(torch, host, h2d, spans=None):
    """One step's inputs, host -> device on the h2d stream; returns (tensors, ready event)."""
    with torch.cuda.stream(h2d):
        dev = timed_span(torch, h2d, spans, lambda: {k: host[k].to("cuda", non_blocking=True)
                                                      for k in ("q", "sq", "lo", "hi", "ik", "iv")})
        ready = torch.cuda.Event()
        ready.record(h2d)
    return dev, ready


def run_step_e2e(torch, idx, host, stream, h2d, d2h, outs, step, pending, spans=None):
    """The same step through the public API from pinned host buffers, results read back to host.
    Each step copies its own inputs host -> device, one step ahead on the h2d stream (`pending`
    holds this step's upload); each phase's results go device -> host on the d2h stream as soon as
    the phase has run; the phases run on `stream`.  Device results are double-buffered: a step
    writes buffer set step % 2 once the copies out of that set (two steps earlier) are done.
    Returns the next step's upload."""
    o = outs[step % 2]
    dev, ready = pending
    nxt = upload_inputs(torch, host, h2d, None if spans is None else spans["h2d"])
    for t in dev.values():
        t.record_stream(stream)
    stream.wait_event(ready)
    if o["copied"] is not None:
        stream.wait_event(o["copied"])

    def down(pairs):
        done = torch.cuda.Event()
        done.record(stream)
        d2h.wait_event(done)
        with torch.cuda.stream(d2h):
            timed_span(torch, d2h, None if spans is None else spans["d2h"],
                       lambda: [dst.copy_(src, non_blocking=True) for dst, src in pairs])

    with torch.cuda.stream(stream):
        v, _ = idx.lookup(dev["q"], stream=stream, out=o["lv"], found=False)
        down([(host["lv"], v)])
        sk, sv = idx.successor(dev["sq"], stream=stream, out=(o["sk"], o["sv"]))
        down([(host["sk"], sk), (host["sv"], sv)])
        off, rk, rv = idx.range(dev["lo"], dev["hi"], stream=stream, out=(o["roff"], o["rk"], o["rv"]))
        down([(host["roff"], off), (host["rk"][: rk.numel()], rk), (host["rv"][: rv.numel()], rv)])
        idx.insert(dev["ik"], dev["iv"], stream=stream)
        idx.delete(dev["ik"], stream=stream)
        idx.restructure(stream=stream)
    o["copied"] = torch.cuda.Event()
    o["copied"].record(d2h)
    return nxt


_ORACLE_MAP = {}


def oracle_map(c):
    """The oracle's map of the loaded keys, built once per process (its qsort of 2^26 pairs takes
    about 25 s); each sampled step inserts and then deletes the same fresh keys, which leaves it as
    it was."""
    import oracle
    key = id(c["load_keys"])
    if key not in _ORACLE_MAP:
        mp = oracle.Map(KW)
        mp.bulk_load(c["load_keys"], c["load_vals"])
        _ORACLE_MAP.clear()
        _ORACLE_MAP[key] = mp
    return _ORACLE_MAP[key]


def cpu_oracle_sample(c, scale_log=4):
    """The oracle, as it stands, on a bounded sample of the step: every batch 2^-scale_log of its size,
    against the full 2^26-key map.  Returns (Mops/s, seconds, description)."""
    mp = oracle_map(c)
    nq = c["queries"].size >> scale_log
    nr = c["range_lo"].size >> scale_log
    nu = c["ins_keys"].size >> scale_log
    t0 = time.perf_counter()
    mp.read(np.full(nq, W.OP_LOOKUP, np.uint8), c["queries"][:nq])
    mp.read(np.full(nq, W.OP_SUCC, np.uint8), c["succ_queries"][:nq])
    mp.read(np.full(nr, W.OP_RANGE, np.uint8), c["range_lo"][:nr], c["range_hi"][:nr])
    mp.update(np.full(nu, W.OP_INSERT, np.uint8), c["ins_keys"][:nu], c["ins_vals"][:nu])
    mp.update(np.full(nu, W.OP_DELETE, np.uint8), c["ins_keys"][:nu])
    dt = time.perf_counter() - t0
    ops = 2 * nq + nr + 2 * nu
    desc = ("oracle (plain C, 1 thread) on the full 2^26-key map; per step 2^%d lookups, 2^%d successors, "
            "2^%d ranges, 2^%d inserts, 2^%d deletes" % (LOG_Q - scale_log, LOG_Q - scale_log, LOG_R - scale_log,
                                                         LOG_U - scale_log, LOG_U - scale_log))
    return ops / dt / 1e6, dt, desc


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_oracle_sample_mt(c, scale_log=2, threads=None):
    """The batch-synchronous oracle (reads split over host threads on the snapshot, then the updates
    merged by key range on the same threads) on a bounded sample of the step: every batch
    2^-scale_log of its size, against the full 2^26-key map.  Returns (Mops/s, seconds, threads,
    description)."""
    threads = threads or host_cores()
    mp = oracle_map(c)
    nq = c["queries"].size >> scale_log
    nr = c["range_lo"].size >> scale_log
    nu = c["ins_keys"].size >> scale_log
    t0 = time.perf_counter()
    mp.read_mt(np.full(nq, W.OP_LOOKUP, np.uint8), c["queries"][:nq], threads=threads)
    mp.read_mt(np.full(nq, W.OP_SUCC, np.uint8), c["succ_queries"][:nq], threads=threads)
    mp.read_mt(np.full(nr, W.OP_RANGE, np.uint8), c["range_lo"][:nr], c["range_hi"][:nr], threads=threads)
    mp.update_mt(np.full(nu, W.OP_INSERT, np.uint8), c["ins_keys"][:nu], c["ins_vals"][:nu], threads=threads)
    mp.update_mt(np.full(nu, W.OP_DELETE, np.uint8), c["ins_keys"][:nu], threads=threads)
    dt = time.perf_counter() - t0
    ops = 2 * nq + nr + 2 * nu
    desc = ("batch-synchronous oracle (plain C, %d threads) on the full 2^26-key map; per step 2^%d lookups, "
            "2^%d successors, 2^%d ranges, 2^%d inserts, 2^%d deletes"
            % (threads, LOG_Q - scale_log, LOG_Q - scale_log, LOG_R - scale_log, LOG_U - scale_log,
               LOG_U - scale_log))
    return ops / dt / 1e6, dt, threads, desc


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    c = make_inputs(seed=2000)
    vals = []
    desc = ""
    cores = 1
    for s in range(args.warmup + args.steps):
        mops, dt, cores, desc = cpu_oracle_sample_mt(c, scale_log=5)
        if s >= args.warmup:
            vals.append((mops, dt))
    v = statistics.median(m for m, _ in vals)
    ms = statistics.median(d for _, d in vals) * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mops/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "each step: every batch at 1/32 of its size"},
            "cpu_baseline": {"value": v, "unit": "Mops/s", "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": v, "unit": "Mops/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    global LOG_LOAD, LOG_Q
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="flix", choices=["flix", "reference"])
    ap.add_argument("--form", default="plain", choices=["plain", "batched", "served", "update_heavy", "xy", "light"],
                    help="plain: the read-scale step (default); batched: mixed-batch stream through CUDA "
                         "graphs vs plain launches; served: continuous batching under Poisson arrivals")
    ap.add_argument("--batches", type=int, default=None,
                    help="batched form: stream length (default 10000); update_heavy form: insert batches per "
                         "distribution (default 64)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="plain form: leave out the short batched, update-heavy and serving forms after the step")
    ap.add_argument("--log-load", type=int, default=LOG_LOAD, help="log2 of the keys loaded (smaller cases)")
    ap.add_argument("--log-q", type=int, default=LOG_Q, help="log2 of the lookup/successor batch")
    ap.add_argument("--sort-variant", type=int, default=0, help="0 auto, 1 one-sweep, 2 reduce-then-scan")
    ap.add_argument("--xy-max-build", type=int, default=100_000_000,
                    help="xy form: largest build of the restructure accounting (1M, 33M, 100M)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return reference_arm(args)
    if args.form == "batched":
        return bench_batched(args)
    if args.form == "served":
        return bench_served(args)
    if args.form == "update_heavy":
        return bench_update_heavy(args)
    if args.form == "xy":
        return bench_xy(args)
    if args.form == "light":
        return bench_light(args)

    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    import paper_2604_16725_gb300 as fx

    LOG_LOAD, LOG_Q = args.log_load, args.log_q
    if (LOG_LOAD, LOG_Q) != (26, 24):
        args.no_cpu_baseline = True
    c = make_inputs(seed=2000 + 17 * rank, log_load=LOG_LOAD, log_q=LOG_Q)
    idx = fx.Index(key_bits=KW, node_size=NODE_SIZE, sort_variant=args.sort_variant)
    stream = torch.cuda.Stream()
    td = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()  # noqa: E731
    idx.bulk_load(td(c["load_keys"]), td(c["load_vals"]), stream=stream)
    bufs = dict(q=td(c["queries"]), sq=td(c["succ_queries"]), lo=td(c["range_lo"]), hi=td(c["range_hi"]),
                ik=td(c["ins_keys"]), iv=td(c["ins_vals"]), lv=torch.empty(1 << LOG_Q, dtype=torch.int64, device="cuda"))
    # size the range output once (counts), outside the timed region
    off, rk, rv = idx.range(bufs["lo"], bufs["hi"], stream=stream)
    bufs["rcap"] = int(rk.numel())
    del off, rk, rv
    stream.synchronize()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        run_step(torch, idx, bufs, stream)
    phases = ["lookup", "successor", "range", "insert", "delete", "restructure"]
    events = {p: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for p in phases}
    per_phase = {p: [] for p in phases}
    step_ms = []
    launches0 = idx.launch_count()
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(gpu_id_for_smi(torch)) as clk:
        time.sleep(1.0)            # let the sampler start before the timed region
        barrier()
        wall0 = time.time()
        t_start.record(stream)
        for _ in range(args.steps):
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            run_step(torch, idx, bufs, stream, events)
            s1.record(stream)
            s1.synchronize()
            step_ms.append(s0.elapsed_time(s1))
            for p in phases:
                per_phase[p].append(events[p][0].elapsed_time(events[p][1]))
        t_end.record(stream)
        barrier()
        wall1 = time.time()
        time.sleep(0.3)
    clocks = clk.summary(wall0 - 0.25, wall1 + 0.25)
    total_ms = t_start.elapsed_time(t_end)
    launches = idx.launch_count() - launches0
    total_ms = max_over_ranks(total_ms, world)
    ops = ops_per_step(log_q=LOG_Q)
    n_ops = sum(ops.values())
    ms_step = total_ms / args.steps
    value = whole_job_mops(n_ops, world, ms_step)

    # per-kernel durations: a second pass of the same steps with per-launch CUDA events
    idx.profile(True)
    idx.profile_reset()
    for _ in range(args.steps):
        run_step(torch, idx, bufs, stream)
    torch.cuda.synchronize()
    prof = idx.profile_read()
    idx.profile(False)

    # predecessor (not part of the step): 2^24 queries of the successor recipe, timed alone
    pred_ms = []
    for i in range(args.warmup + args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        idx.predecessor(bufs["sq"], stream=stream)
        b.record(stream)
        b.synchronize()
        if i >= args.warmup:
            pred_ms.append(a.elapsed_time(b))

    # config 2's smaller read batches (2^20 and 2^22: the first queries of the step's batches), each
    # timed alone, 10 repetitions after warm-up, median
    sizes_ms = {}
    sk_buf = torch.empty(1 << LOG_Q, dtype=torch.int64, device="cuda")
    sv_buf = torch.empty(1 << LOG_Q, dtype=torch.int64, device="cuda")
    for lg in sorted({lg_ for lg_ in (20, 22, LOG_Q) if lg_ <= LOG_Q}):
        m = 1 << lg
        for name, fn in (("lookup", lambda m=m: idx.lookup(bufs["q"][:m], stream=stream, out=bufs["lv"][:m],
                                                            found=False)),
                         ("successor", lambda m=m: idx.successor(bufs["sq"][:m], stream=stream,
                                                                 out=(sk_buf[:m], sv_buf[:m])))):
            t = []
            for i in range(args.warmup + 10):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                b.synchronize()
                if i >= args.warmup:
                    t.append(a.elapsed_time(b))
            med = statistics.median(t)
            sizes_ms["%s_2e%d" % (name, lg)] = {"ms_p50": round(med, 4), "mops": round(m / (med * 1e-3) / 1e6, 1)}
    del sk_buf, sv_buf

    # roofline of the dominant kernel: the radix-sort scatter pass
    peak, peak_kind = measured_peaks()
    down = prof.get("sort_onesweep", {"launches": 0, "ms": 0.0, "bytes": 0.0})
    # algorithmic bytes of the scatter passes the sort plans ran, as the library counts them per launch:
    # the first pass of a sort reads keys only (payload = position), later passes read key+payload, all
    # write key+payload (64-bit keys, 32-bit payload); passes the plan leaves out are "sort_pass_idle"
    ks = 8
    dom = max(prof.items(), key=lambda kv: kv[1]["ms"])[0] if prof else "sort_onesweep"
    achieved = down["bytes"] / (down["ms"] * 1e-3) / 1e9 if down["ms"] else 0.0
    tr = traffic_record("sort_onesweep")
    traffic = None
    if tr:
        traffic = tr["dram_bytes_per_item"] * (1 << LOG_Q)
    roofline = {"kernel": "sort_onesweep", "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_kind": peak_kind + " hbm copy", "traffic": traffic,
                "traffic_unit": "bytes per 2^24-item launch",
                "dominant_by_time": dom,
                "kernel_share": {k: round(v["ms"] / max(sum(x["ms"] for x in prof.values()), 1e-9), 4)
                                 for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])[:8]}}
    # the search-and-apply kernels: algorithmic bytes per step (the formulas of the design notes'
    # kernel table applied to this step's batches) over each kernel's CUDA-event time per step
    apply_roofline = apply_rooflines(prof, args.steps, peak, peak_kind, rcap=bufs["rcap"])

    line = {"metric": METRIC, "value": value, "unit": "Mops/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "node_size": NODE_SIZE, "key_bits": KW,
                       "restructure": "one pass into a second key/value node array",
                       "l2": "inputs larger than L2: 2.2 GB of nodes and >3 GB touched per step",
                       "parallelism": "replicas" if world > 1 else "single", "sort_variant": args.sort_variant},
            "per_op": {p: {"mops": (ops[p] / (statistics.median(per_phase[p]) * 1e-3) / 1e6) if p in ops else None,
                           "ms_p50": statistics.median(per_phase[p]),
                           "ms_p99": float(np.percentile(per_phase[p], 99))} for p in phases},
            "outside_step": {"predecessor": {"mops": (1 << LOG_Q) / (statistics.median(pred_ms) * 1e-3) / 1e6,
                                             "ms_p50": statistics.median(pred_ms), "queries": 1 << LOG_Q},
                             "read_batches": sizes_ms},
            "step_ms_p50": statistics.median(step_ms), "step_ms_p99": float(np.percentile(step_ms, 99)),
            "roofline": roofline, "apply_roofline": apply_roofline,
            # every kernel's CUDA-event time per step (profiled pass): apply-only times are the
            # non-sort entries (read_point, read_unsort, range_*, update_*, gather, ...)
            "kernel_ms_per_step": {k: round(v["ms"] / args.steps, 4)
                                   for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])},
            "gpu_launches": launches,
            "clocks": clocks}
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).pin_memory()  # noqa: E731
        host = dict(q=pin(c["queries"]), sq=pin(c["succ_queries"]), lo=pin(c["range_lo"]), hi=pin(c["range_hi"]),
                    ik=pin(c["ins_keys"]), iv=pin(c["ins_vals"]), rcap=bufs["rcap"])
        n = 1 << LOG_Q
        for k, shape, dt in (("lv", n, torch.int64), ("sk", n, torch.int64),
                             ("sv", n, torch.int64), ("roff", (1 << LOG_R) + 1, torch.int64),
                             ("rk", bufs["rcap"], torch.int64), ("rv", bufs["rcap"], torch.int64)):
            host[k] = torch.empty(shape, dtype=dt).pin_memory()
        h2d_st, d2h_st = torch.cuda.Stream(), torch.cuda.Stream()
        # this box's device-to-host link: one 1 GiB copy into pinned memory, the best of three (the
        # e2e step moves 2.5 GB of results down, so its time is bounded by this rate)
        lk_d = torch.empty(1 << 27, dtype=torch.int64, device="cuda")
        lk_h = torch.empty(1 << 27, dtype=torch.int64).pin_memory()
        lk = []
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(d2h_st)
            with torch.cuda.stream(d2h_st):
                lk_h.copy_(lk_d, non_blocking=True)
            b.record(d2h_st)
            b.synchronize()
            lk.append(a.elapsed_time(b))
        link_gbs = (1 << 30) / (min(lk) * 1e-3) / 1e9
        del lk_d, lk_h
        outs = [dict(lv=torch.empty(n, dtype=torch.int64, device="cuda"),
                     sk=torch.empty(n, dtype=torch.int64, device="cuda"),
                     sv=torch.empty(n, dtype=torch.int64, device="cuda"),
                     roff=torch.empty((1 << LOG_R) + 1, dtype=torch.int64, device="cuda"),
                     rk=torch.empty(bufs["rcap"], dtype=torch.int64, device="cuda"),
                     rv=torch.empty(bufs["rcap"], dtype=torch.int64, device="cuda"), copied=None) for _ in range(2)]
        pending = upload_inputs(torch, host, h2d_st)
        for s in range(3):
            pending = run_step_e2e(torch, idx, host, stream, h2d_st, d2h_st, outs, s, pending)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        spans = {"h2d": [], "d2h": []}
        pending = upload_inputs(torch, host, h2d_st, spans["h2d"])     # the first timed step's inputs
        for s in range(args.steps):
            pending = run_step_e2e(torch, idx, host, stream, h2d_st, d2h_st, outs, s, pending, spans)
        torch.cuda.synchronize()
        barrier()
        e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
        # time each copy engine direction was busy per step (the copies' own durations)
        busy = {k: sum(a.elapsed_time(b) for a, b in v) / args.steps for k, v in spans.items()}
        e2e_ms = max_over_ranks(e2e_ms, world)
        h2d = sum(host[k].numel() * host[k].element_size() for k in ("q", "sq", "lo", "hi", "ik", "iv"))
        d2h = sum(host[k].numel() * host[k].element_size() for k in ("lv", "sk", "sv", "roff", "rk", "rv"))
        line["e2e"] = {"value": n_ops * world / (e2e_ms * 1e-3) / 1e6, "unit": "Mops/s",
                       "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms,
                       "d2h_link_gbs": round(link_gbs, 1),
                       "d2h_link_bound_ms_per_step": round(d2h / (link_gbs * 1e9) * 1e3, 2),
                       "d2h_busy_ms_per_step": round(busy["d2h"], 2), "h2d_busy_ms_per_step": round(busy["h2d"], 2)}
    if rank == 0 and world == 1 and not args.no_forms:
        # the batched form beside the plain path on a short stream of small mixed batches (the full
        # config-4 stream is `--form batched`): 600 batches of log-uniform 2^4..2^11 ops on a 2^24-key
        # index, plain per-batch flix_apply against the persistent kernel taking each batch as it comes
        from paper_2604_16725_gb300.batched import BatchedRunner
        from workload import device as WD
        ss = WD.mixed_stream_device(seed=4100, n_preload=1 << 24, n_batches=600, lo_exp=4, hi_exp=11)
        sb = list(ss["batches"]())
        res = run_stream(torch, fx, BatchedRunner, sb, ss["preload_keys"], ss["preload_vals"], NODE_SIZE, 0, 0,
                         lambda m: None, queue_depth=1, modes=("plain", "persistent"))
        fin = res.pop("_finals")
        line["small_batch_stream"] = {
            "workload": "600 mixed batches of log-uniform 2^4..2^11 ops (60/15/5/10/10 lookup/successor/range/"
                        "insert/delete) on 2^24 preloaded uint64 keys; persistent = flix_apply_queue, one batch "
                        "per launch",
            "plain": {k: round(v, 4) if isinstance(v, float) else v for k, v in res["plain"].items()},
            "persistent": {k: round(v, 4) if isinstance(v, float) else v for k, v in res["persistent"].items()},
            "final_state_equal": bool(torch.equal(fin["plain"][0], fin["persistent"][0]) and
                                      torch.equal(fin["plain"][1], fin["persistent"][1]))}
        del ss, sb, fin
        torch.cuda.empty_cache()
        line["short_forms"] = mini_forms(torch, fx)
    if rank == 0 and not args.no_cpu_baseline:
        mops_mt, dt_mt, cores, desc_mt = cpu_oracle_sample_mt(c)
        mops, dt, desc = cpu_oracle_sample(c)
        line["cpu_baseline"] = {"value": mops_mt, "unit": "Mops/s", "cores": cores, "kind": "oracle",
                                "sample": desc_mt, "seconds": dt_mt,
                                "single_thread": {"value": mops, "unit": "Mops/s", "cores": 1, "sample": desc,
                                                  "seconds": dt}}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------------------------------------
# Batched and served forms (their own JSON lines; the default run is the plain read-scale step)
# ------------------------------------------------------------------------------------------------

def run_stream(torch, fx, BatchedRunner, batches, pre_k, pre_v, NS, sv, bt, log, queue_depth=1,
               modes=("plain", "graph", "persistent")):
    """One stream through plain per-batch flix_apply, the graph path and the persistent path.
    Per batch: latency from submission to completion (CUDA events); throughput = ops / wall time."""
    n_ops = sum(int(k.numel()) for _, k, _ in batches)
    sizes = np.array([int(k.numel()) for _, k, _ in batches])
    max_b = int(sizes.max())
    # free nodes held for the asynchronous paths: new nodes hold at least NS/2 keys, inserts are a
    # tenth of the ops, and the runner restructures every 50 batches when nodes exceed 2x buckets
    free_min = min(1 << 24, n_ops // 10 // max(NS // 4, 1) + (1 << 20))
    results = {}
    finals = {}
    for mode in modes:
        idx = fx.Index(key_bits=64, node_size=NS, sort_variant=sv, bucket_threads=bt)
        idx.bulk_load(pre_k, pre_v)
        log("%s: device memory free %.1f GB" % (mode, torch.cuda.mem_get_info()[0] / 1e9))
        st = torch.cuda.Stream()
        run = None
        if mode != "plain":
            run = BatchedRunner(idx, max_batch=max_b, min_log=8, range_per_op=64,
                                free_nodes_min=free_min, queue_depth=queue_depth if mode == "persistent" else 0)
            for o, k, a in batches:
                if mode == "graph" or int(k.numel()) > fx.QUEUE_BATCH_MAX:
                    run.graph_for(run.size_for(int(k.numel())))
            st = run.stream
        else:
            idx.reserve(max_b, free_min)
        torch.cuda.synchronize()
        sub = [torch.cuda.Event(enable_timing=True) for _ in batches]
        done = [None] * len(batches)
        pend = []

        def flushed():
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(st)
            for j in pend:
                done[j] = ev
            pend.clear()

        if run is not None:
            run.on_flush = flushed
        t0 = time.perf_counter()
        for i, (o, k, a) in enumerate(batches):
            sub[i].record(st)
            queued = mode == "persistent" and int(k.numel()) <= fx.QUEUE_BATCH_MAX
            if queued:
                pend.append(i)
            try:
                if run is None:
                    with torch.cuda.stream(st):
                        idx.apply(o, k, a, range_capacity=max(64 * int(k.numel()), 1 << 18), stream=st)
                else:
                    run.run(o, k, a)
            except fx.FlixError:
                free_b, total_b = torch.cuda.mem_get_info()
                log("%s: batch %d of %d ops failed; index %s; device memory free %.1f of %.1f GB"
                    % (mode, i, int(k.numel()), idx.stats(stream=st), free_b / 1e9, total_b / 1e9))
                raise
            if not queued:
                done[i] = torch.cuda.Event(enable_timing=True)
                done[i].record(st)
            if (i + 1) % 50 == 0:
                if run is not None:
                    run.restructure_if_needed()
                else:
                    s_ = idx.stats(stream=st)
                    if s_["nodes_used"] > 2 * s_["buckets"] or s_["max_chain"] > 64:
                        idx.restructure(stream=st)
        if run is not None:
            run.synchronize()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        lat = np.array([sub[i].elapsed_time(done[i]) for i in range(len(batches))])
        small = sizes <= fx.QUEUE_BATCH_MAX
        results[mode] = {"mops": n_ops / wall / 1e6, "wall_s": wall,
                         "batch_ms_p50": float(np.median(lat)), "batch_ms_p99": float(np.percentile(lat, 99)),
                         "small_batch_ms_p50": float(np.median(lat[small])) if small.any() else None,
                         "small_batch_ms_p99": float(np.percentile(lat[small], 99)) if small.any() else None,
                         "queues": run.queues if run is not None else 0}
        k_, v_ = idx.export()
        finals[mode] = (k_.cpu(), v_.cpu())
        log("%s: %s" % (mode, results[mode]))
        del run
        idx.close()
        torch.cuda.empty_cache()
    results["_finals"] = finals
    return results


def mini_forms(torch, fx):
    """Short versions of the update-heavy and serving forms for the default line (the full forms are
    `--form update_heavy` and `--form served`): 16 uniform insert batches of 2^20 uint32 keys into an
    empty node-size-32 index with the full form's restructure policy, then 8 delete batches of a
    seeded half; and requests offered at 1e6
    ops/s (2000 requests of floor(2^U(0,12)) ops, 80/10/10 lookup/insert/delete over Zipf(0.9)) on
    2^24 preloaded uint64 keys (universe 2^25), through the server and through the plain path."""
    from paper_2604_16725_gb300.serve import Server, plain_serve
    out = {}
    ins, deletes = W.update_heavy("uniform", seed=3000, n_batches=16, batch=1 << 20, n_del_batches=8)
    idx = fx.Index(key_bits=32, node_size=32)
    st = torch.cuda.Stream()
    td = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()  # noqa: E731
    dev = [(td(k), td(v)) for k, v in ins]
    torch.cuda.synchronize()
    # the full form's restructure policy (nodes > 2 * buckets or a chain > 64) after every insert batch,
    # timed apart from the inserts as there
    t_ins = 0.0
    for k, v in dev:
        t0 = time.perf_counter()
        idx.insert(k, v, stream=st)
        st.synchronize()
        t_ins += time.perf_counter() - t0
        s_ = idx.stats(stream=st)
        if s_["nodes_used"] > 2 * s_["buckets"] or s_["max_chain"] > 64:
            idx.restructure(stream=st)
            st.synchronize()
    stored, _ = idx.export(stream=st)
    dels = [td(d) for d in deletes(stored.cpu().numpy().view(np.uint32))]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for d in dels:
        idx.delete(d, stream=st)
    st.synchronize()
    t_del = time.perf_counter() - t0
    out["update_heavy_uniform"] = {"insert_mops": round(16 * (1 << 20) / t_ins / 1e6, 1),
                                   "delete_mops": round(sum(int(d.numel()) for d in dels) / t_del / 1e6, 1),
                                   "live_keys": idx.stats(stream=st)["live_keys"]}
    idx.close()
    del dev, dels, stored
    ubits, pbits, seed = 25, 24, 5000
    pk = W.universe(64, seed, 0, 1 << pbits)
    pv = W.values_for(64, pk)
    idx = fx.Index(key_bits=64, node_size=64)
    idx.bulk_load(torch.from_numpy(pk.view(np.int64)).cuda(), torch.from_numpy(pv.view(np.int64)).cuda())
    srv = Server(idx, max_batch=1 << 18, depth=2, min_log=8, free_nodes_min=1 << 20)
    req = W.serving_requests(seed=seed + 6, universe_bits=ubits, preload_bits=pbits, offered_ops_per_s=1e6,
                             n_requests=2000)
    sv = srv.serve(req["arrival_s"], req["req_off"], req["ops"], req["keys"], req["aux"])
    lat = sv["latency_s"] * 1e3
    req = W.serving_requests(seed=seed + 7, universe_bits=ubits, preload_bits=pbits, offered_ops_per_s=1e6,
                             n_requests=300)
    pl = plain_serve(idx, req["arrival_s"], req["req_off"], req["ops"], req["keys"], req["aux"])
    plat = pl["latency_s"] * 1e3
    out["served_1e6"] = {"served": {"p50_ms": round(float(np.percentile(lat, 50)), 3),
                                    "p99_ms": round(float(np.percentile(lat, 99)), 3),
                                    "sustained_mops": round(sv["ops"] / sv["wall_s"] / 1e6, 3), "requests": 2000},
                         "plain_per_request": {"p50_ms": round(float(np.percentile(plat, 50)), 3),
                                               "p99_ms": round(float(np.percentile(plat, 99)), 3), "requests": 300}}
    del srv
    idx.close()
    torch.cuda.empty_cache()
    return out


def bench_batched(args):
    """Config 4's stream: a 2^27-key uint64 index and --batches (default 10,000) uneven mixed batches,
    sizes log-uniform 2^8..2^22 (about 4.3e9 ops), 60/15/5/10/10 lookup/successor/range/insert/
    delete, generated on the GPU (workload.device: gen.mixed_stream's recipe and key universe).
    Three paths over the same batches: plain per-batch flix_apply; the batched form with a CUDA
    graph per size class; and the batched form with the persistent kernel taking each batch of at
    most 2048 ops as it comes (queue depth 1; larger batches take the graphs).  Node size, sort variant and
    bucket threads come from the autotuner on a held-out seed.  Per batch: latency from submission
    to completion (CUDA events); throughput = all ops / wall time."""
    import torch
    import paper_2604_16725_gb300 as fx
    from paper_2604_16725_gb300.batched import BatchedRunner
    from paper_2604_16725_gb300.tune import autotune
    from workload import device as WD
    torch.cuda.set_device(0)
    log = lambda m: print(m, file=sys.stderr, flush=True)  # noqa: E731
    held = WD.mixed_stream_device(seed=4999, n_preload=1 << 22, n_batches=24, lo_exp=8, hi_exp=20)
    hb = list(held["batches"]())
    tune = autotune(64, held["preload_keys"], held["preload_vals"], hb, range_per_op=64, log=log)
    NS, sv, bt = tune["node_size"], tune["sort_variant"], tune.get("bucket_threads", 0)
    log("autotune: NS=%d sort_variant=%d bucket_threads=%d" % (NS, sv, bt))
    del hb, held
    n_pre = 1 << args.log_load if args.log_load != LOG_LOAD else 1 << 27
    n_stream = args.batches or 10000
    s = WD.mixed_stream_device(seed=4000, n_preload=n_pre, n_batches=n_stream)
    batches = list(s["batches"]())
    torch.cuda.synchronize()
    n_ops = sum(int(k.numel()) for _, k, _ in batches)
    sizes = np.array([int(k.numel()) for _, k, _ in batches])
    max_b = int(sizes.max())
    log("stream: %d batches, %d ops" % (len(batches), n_ops))
    results = run_stream(torch, fx, BatchedRunner, batches, s["preload_keys"], s["preload_vals"], NS, sv, bt, log,
                         queue_depth=1)
    finals = results.pop("_finals")
    # a stream of small batches only (2^4..2^11 ops: every batch fits the persistent kernel's queue)
    ss = WD.mixed_stream_device(seed=4100, n_preload=n_pre, n_batches=min(n_stream, 3000), lo_exp=4, hi_exp=11)
    sbatches = list(ss["batches"]())
    small_res = run_stream(torch, fx, BatchedRunner, sbatches, ss["preload_keys"], ss["preload_vals"], NS, sv, bt, log,
                           queue_depth=1)
    small_finals = small_res.pop("_finals")
    for dq in (2, 16):
        deep = run_stream(torch, fx, BatchedRunner, sbatches, ss["preload_keys"], ss["preload_vals"], NS, sv, bt, log,
                          queue_depth=dq, modes=("persistent",))
        deep_finals = deep.pop("_finals")
        small_res["persistent_queue%d" % dq] = deep["persistent"]
        small_finals["persistent_queue%d" % dq] = deep_finals["persistent"]
    small_same = all(bool(torch.equal(small_finals["plain"][0], small_finals[m][0]) and
                          torch.equal(small_finals["plain"][1], small_finals[m][1]))
                     for m in ("graph", "persistent", "persistent_queue2", "persistent_queue16"))
    sizes = np.array([int(k.numel()) for _, k, _ in batches])
    small = sizes <= fx.QUEUE_BATCH_MAX
    same_state = all(bool(torch.equal(finals["plain"][0], finals[m][0]) and torch.equal(finals["plain"][1], finals[m][1]))
                     for m in ("graph", "persistent"))
    best = max(("graph", "persistent"), key=lambda m: results[m]["mops"])
    line = {"form": "batched", "metric": METRIC, "value": results[best]["mops"], "unit": "Mops/s",
            "n_gpus": 1, "higher_is_better": True, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "batched: %d uint64 keys preloaded; %d mixed batches, sizes log-uniform "
                                   "2^8..2^22, 60/15/5/10/10 lookup/successor/range(1-1000)/insert/delete, "
                                   "generated on the GPU" % (n_pre, len(batches)),
                       "node_size": NS, "sort_variant": sv, "bucket_threads": bt, "ops": n_ops,
                       "small_batches": int(small.sum())},
            "plain": results["plain"], "graph": results["graph"], "persistent": results["persistent"],
            "best_batched_path": best, "speedup_vs_plain": results[best]["mops"] / results["plain"]["mops"],
            "final_state_equal": same_state,
            "small_batch_stream": {"workload": "%d batches of log-uniform 2^4..2^11 ops, same mix, same index size; "
                                               "persistent queue depth 1 (and 2, 16); a queued batch completes "
                                               "when its queue's launch has run" % len(sbatches),
                                   "ops": sum(int(k.numel()) for _, k, _ in sbatches),
                                   "plain": small_res["plain"], "graph": small_res["graph"],
                                   "persistent": small_res["persistent"],
                                   "persistent_queue2": small_res["persistent_queue2"],
                                   "persistent_queue16": small_res["persistent_queue16"],
                                   "final_state_equal": small_same},
            "autotune": tune["table"]}
    print(json.dumps(line))
    return 0


def bench_served(args):
    """Continuous batching of Poisson-arriving requests (1..4096 ops, 80/10/10 lookup/insert/delete
    over Zipf(0.9) keys) on a 2^28-key uint64 index (universe 2^29): p50/p99 latency and sustained
    Mops/s per offered load, and the plain per-request path at the lowest load."""
    import torch
    import paper_2604_16725_gb300 as fx
    from paper_2604_16725_gb300.serve import Server, plain_serve
    torch.cuda.set_device(0)
    log = lambda m: print(m, file=sys.stderr, flush=True)  # noqa: E731
    ubits = 29
    pbits = 28 if args.log_load == LOG_LOAD else args.log_load
    seed = 5000
    pk = W.universe(64, seed, 0, 1 << pbits)
    pv = W.values_for(64, pk)
    idx = fx.Index(key_bits=64, node_size=64)
    idx.bulk_load(torch.from_numpy(pk.view(np.int64)).cuda(), torch.from_numpy(pv.view(np.int64)).cuda())
    del pk, pv
    srv = Server(idx, max_batch=1 << 22, depth=2, min_log=8, free_nodes_min=1 << 22)
    loads = []
    for rate in (1e6, 1e7, 1e8, 1e9):
        mean_ops = 585.0
        n_req = int(min(max(rate * 2.0 / mean_ops, 2000), 80000))
        req = W.serving_requests(seed=seed + int(np.log10(rate)), universe_bits=ubits, preload_bits=pbits,
                                 offered_ops_per_s=rate, n_requests=n_req)
        out = srv.serve(req["arrival_s"], req["req_off"], req["ops"], req["keys"], req["aux"])
        lat = out["latency_s"] * 1e3
        loads.append({"offered_mops": rate / 1e6, "requests": n_req, "ops": out["ops"],
                      "sustained_mops": out["ops"] / out["wall_s"] / 1e6, "p50_ms": float(np.percentile(lat, 50)),
                      "p99_ms": float(np.percentile(lat, 99)), "batches": out["batches"],
                      "mean_batch_ops": out["ops"] / max(out["batches"], 1)})
        log("offered %.0e: %s" % (rate, loads[-1]))
    # the same server with every batch through the size-class graphs (no persistent kernel), at the
    # lowest offered load
    del srv
    srv_g = Server(idx, max_batch=1 << 22, depth=2, min_log=8, free_nodes_min=1 << 22, queue_depth=0)
    req = W.serving_requests(seed=seed + 6, universe_bits=ubits, preload_bits=pbits, offered_ops_per_s=1e6,
                             n_requests=2000)
    og = srv_g.serve(req["arrival_s"], req["req_off"], req["ops"], req["keys"], req["aux"])
    lat = og["latency_s"] * 1e3
    graphs_only = {"offered_mops": 1.0, "requests": 2000, "sustained_mops": og["ops"] / og["wall_s"] / 1e6,
                   "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99))}
    log("graphs only, offered 1e+06: %s" % graphs_only)
    del srv_g
    # plain per-request path at the lowest offered load (bounded number of requests)
    req = W.serving_requests(seed=seed + 6, universe_bits=ubits, preload_bits=pbits, offered_ops_per_s=1e6,
                             n_requests=600)
    pl = plain_serve(idx, req["arrival_s"], req["req_off"], req["ops"], req["keys"], req["aux"])
    lat = pl["latency_s"] * 1e3
    plain = {"offered_mops": 1.0, "requests": 600, "sustained_mops": pl["ops"] / pl["wall_s"] / 1e6,
             "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99))}
    line = {"form": "served", "metric": METRIC, "value": max(x["sustained_mops"] for x in loads), "unit": "Mops/s",
            "n_gpus": 1, "higher_is_better": True, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "served: 2^%d uint64 keys preloaded (universe 2^%d); Poisson requests of "
                                   "floor(2^U(0,12)) ops, 80/10/10 lookup/insert/delete over Zipf(0.9)" % (pbits, ubits),
                       "node_size": 64, "depth": 2,
                       "small_batches": "batches of at most 2048 ops through the persistent kernel, one per launch"},
            "loads": loads, "graphs_only_1e6": graphs_only, "plain_per_request": plain}
    print(json.dumps(line))
    return 0


def bench_update_heavy(args):
    """uint32 keys, node size 32, start empty: 64 insert batches of 2^20 keys per distribution
    (uniform, Zipf(0.99) over 2^30 scrambled and dense, sorted-sequential) with the restructure policy
    (nodes > 2 * buckets or a chain > 64), then 32 delete batches removing a random 50%, then a final
    restructure.  Reports throughput, restructures, bytes per key after each phase and the share of
    nodes the final restructure recovers (the quantity of the paper's Tab. 4)."""
    import torch
    import paper_2604_16725_gb300 as fx
    torch.cuda.set_device(0)
    log = lambda m: print(m, file=sys.stderr, flush=True)  # noqa: E731
    out = {}
    n_batches = args.batches or 64
    for dist in ("uniform", "zipf", "zipf_dense", "sequential"):
        ins, deletes = W.update_heavy(dist, seed=3000, n_batches=n_batches, batch=1 << 20)
        idx = fx.Index(key_bits=32, node_size=32)
        st = torch.cuda.Stream()
        dev = [(torch.from_numpy(k.view(np.int32)).cuda(), torch.from_numpy(v.view(np.int32)).cuda()) for k, v in ins]
        torch.cuda.synchronize()
        t_ins = t_res = 0.0
        n_res = 0
        for k, v in dev:
            t0 = time.perf_counter()
            idx.insert(k, v, stream=st)
            st.synchronize()
            t_ins += time.perf_counter() - t0
            s_ = idx.stats(stream=st)
            if s_["nodes_used"] > 2 * s_["buckets"] or s_["max_chain"] > 64:
                t0 = time.perf_counter()
                idx.restructure(stream=st)
                st.synchronize()
                t_res += time.perf_counter() - t0
                n_res += 1
        s_ins = idx.stats(stream=st)
        stored, _ = idx.export(stream=st)
        dels = [torch.from_numpy(d.view(np.int32)).cuda() for d in deletes(stored.cpu().numpy().view(np.uint32))]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for d in dels:
            idx.delete(d, stream=st)
        st.synchronize()
        t_del = time.perf_counter() - t0
        s_del = idx.stats(stream=st)
        t0 = time.perf_counter()
        idx.restructure(stream=st)
        st.synchronize()
        t_fin = time.perf_counter() - t0
        s_fin = idx.stats(stream=st)
        bpk = lambda s: s["used_bytes"] / max(s["live_keys"], 1)  # noqa: E731
        n_ins_ops = sum(int(k.numel()) for k, _ in dev)
        n_del_ops = sum(int(d.numel()) for d in dels)
        out[dist] = {"insert_mops": n_ins_ops / t_ins / 1e6, "restructures": n_res, "restructure_ms_total": t_res * 1e3,
                     "delete_mops": n_del_ops / t_del / 1e6, "final_restructure_ms": t_fin * 1e3,
                     "keys_after_inserts": s_ins["live_keys"], "bytes_per_key_after_inserts": bpk(s_ins),
                     "bytes_per_key_after_deletes": bpk(s_del), "bytes_per_key_after_restructure": bpk(s_fin),
                     "nodes_after_deletes": s_del["nodes_used"], "nodes_after_restructure": s_fin["nodes_used"],
                     "nodes_recovered_pct": 100.0 * (s_del["nodes_used"] - s_fin["nodes_used"]) / max(s_del["nodes_used"], 1)}
        log("%s: %s" % (dist, out[dist]))
        idx.close()
        del dev, dels
        torch.cuda.empty_cache()
    line = {"form": "update_heavy", "metric": METRIC, "value": out["uniform"]["insert_mops"], "unit": "Mops/s",
            "n_gpus": 1, "higher_is_better": True, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "update heavy: uint32, node size 32, start empty; %d insert batches of 2^20 per "
                                   "distribution, then 32 delete batches removing 50%%, final restructure" % n_batches},
            "distributions": out}
    print(json.dumps(line))
    return 0


def bench_light(args):
    """Light insert rounds (Sec. 5.3.6 setup): uint32 keys, build 2^25 uniform keys, 4 rounds of 2^23
    fresh uniform inserts (100% growth, about 2 keys per bucket per round at node size 16, 4 at node
    size 32), each round timed with CUDA events, inputs resident; once with the one-thread path for
    light one-node buckets (bucket_threads 0) and once with a warp for every bucket (32)."""
    import torch
    import paper_2604_16725_gb300 as fx
    torch.cuda.set_device(0)
    td = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()  # noqa: E731
    st = torch.cuda.Stream()
    build, per_round, rounds = 1 << 25, 1 << 23, 4
    keys = W.universe(32, 7000, 0, build + rounds * per_round)
    bk, ins = keys[:build], [keys[build + r * per_round: build + (r + 1) * per_round] for r in range(rounds)]
    out = {}
    for NS in (16, 32):
        for bt in (0, 32):
            idx = fx.Index(key_bits=32, node_size=NS, bucket_threads=bt)
            idx.bulk_load(td(bk), td(W.values_for(32, bk)), stream=st)
            nb = idx.stats(stream=st)["buckets"]
            ms = []
            for r in range(rounds):
                kd, vd = td(ins[r]), td(W.values_for(32, ins[r], salt=r))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(st)
                idx.insert(kd, vd, stream=st)
                b.record(st)
                b.synchronize()
                ms.append(a.elapsed_time(b))
            out["NS%d_%s" % (NS, "one_thread_light" if bt == 0 else "warp_every_bucket")] = {
                "buckets": nb, "keys_per_bucket_per_round": round(per_round / nb, 2),
                "insert_mops_per_round": [round(per_round / (t * 1e-3) / 1e6, 1) for t in ms],
                "ms_per_round": [round(t, 3) for t in ms]}
            print(json.dumps({k: out[k] for k in list(out)[-1:]}), file=sys.stderr, flush=True)
            idx.close()
            torch.cuda.empty_cache()
    tot = {k: rounds * per_round / (sum(v["ms_per_round"]) * 1e-3) / 1e6 for k, v in out.items()}
    line = {"form": "light", "metric": METRIC, "value": max(tot.values()), "unit": "Mops/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "light insert rounds: uint32, build 2^25 uniform, 4 rounds of 2^23 fresh "
                                   "uniform inserts (100% growth); value = the best variant's inserts / time"},
            "insert_mops": tot, "rounds": out}
    print(json.dumps(line))
    return 0


def bench_xy(args):
    """Dense-range (X/Y) update rounds, uint64 keys, node size 32 (Sec. 5.2.1 workloads).

    Rounds: build 2^24 uniform keys; 8 insert rounds of 3 * 2^21 keys (300% growth), Y = 90% of each
    round inside a hot interval covering X of the key range, X from 90% (uniform) down to 2%; after
    every insert round a batch of 2^25 lookups of stored keys (the skew experiment of Sec. 6.3); then
    8 delete rounds removing the inserted keys.  Restructure accounting (Sec. 6.6, Tab. 4): each
    printed row (builds of 1M, 33M and 100M keys, 8 insert rounds to the printed final size at
    X25Y90 and X90Y90), 8 delete rounds removing the share of the inserted keys that the row
    implies, then one restructure: nodes before and after, the share recovered, and the row's own
    figures beside them.  Every call is timed with
    CUDA events on its stream, inputs resident on the device."""
    import torch
    import paper_2604_16725_gb300 as fx
    torch.cuda.set_device(0)
    log = lambda m: print(m, file=sys.stderr, flush=True)  # noqa: E731
    td = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()  # noqa: E731
    st = torch.cuda.Stream()

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        fn()
        b.record(st)
        b.synchronize()
        return a.elapsed_time(b)

    rounds_out = {}
    tot_ops, tot_ms = 0, 0.0
    build = 1 << 24
    variants = (("plain", 0, False), ("elastic", 4, True))
    for X, (vname, split, merge) in [(X, v) for X in (0.9, 0.5, 0.25, 0.12, 0.03, 0.02) for v in variants]:
        if vname == "plain":
            w = W.xy_rounds(X, 0.9, build, 3 * build, 8, seed=6000, kw=64)
        idx = fx.Index(key_bits=64, node_size=32, split_chains_over=split, merge_underfull=merge)
        idx.bulk_load(td(w["build_keys"]), td(w["build_vals"]), stream=st)
        present = [w["build_keys"]]
        ins_ms, q_ms, del_ms, chains = [], [], [], []
        outv = torch.empty(1 << 25, dtype=torch.int64, device="cuda")
        for r, (k, v) in enumerate(w["insert"]):
            kd, vd = td(k), td(v)
            ins_ms.append(timed(lambda: idx.insert(kd, vd, stream=st)))
            present.append(k)
            allk = np.concatenate(present)
            q = td(allk[(W.uniform01(6000 + r, 6, 1 << 25) * allk.size).astype(np.int64)])   # hits, repeats allowed
            idx.lookup(q, stream=st, out=outv, found=False)           # warm (first touch of new nodes)
            q_ms.append(timed(lambda: idx.lookup(q, stream=st, out=outv, found=False)))
            chains.append(idx.stats(stream=st)["max_chain"])
        for k in w["delete"]:
            kd = td(k)
            del_ms.append(timed(lambda: idx.delete(kd, stream=st)))
        n_ins = sum(k.size for k, _ in w["insert"])
        n_del = sum(k.size for k in w["delete"])
        if vname == "plain":
            tot_ops += n_ins + n_del
            tot_ms += sum(ins_ms) + sum(del_ms)
        s_end = idx.stats(stream=st)
        name = "X%dY90%s" % (round(100 * X), "" if vname == "plain" else "_split4_merge")
        rounds_out[name] = {
            "insert_mops_per_round": [round(k.size / (t * 1e-3) / 1e6, 1) for (k, _), t in zip(w["insert"], ins_ms)],
            "lookup_2e25_ms_per_round": [round(t, 3) for t in q_ms],
            "delete_mops_per_round": [round(k.size / (t * 1e-3) / 1e6, 1) for k, t in zip(w["delete"], del_ms)],
            "max_chain_per_round": chains,
            "insert_mops": n_ins / (sum(ins_ms) * 1e-3) / 1e6, "delete_mops": n_del / (sum(del_ms) * 1e-3) / 1e6,
            "buckets_end": s_end["buckets"], "nodes_end": s_end["nodes_used"]}
        log("%s: %s" % (name, rounds_out[name]))
        idx.close()
        torch.cuda.empty_cache()

    table = []
    for name, b, final, p_rec, p_pct in W.TAB4:
        if b > args.xy_max_build:
            continue
        imp = W.tab4_implied((name, b, final, p_rec, p_pct))
        X = 0.25 if name.startswith("X25") else 0.9
        w = W.xy_rounds(X, 0.9, b, final - b, 8, seed=6100, kw=64, delete_share=imp["delete_share"])
        idx = fx.Index(key_bits=64, node_size=32)
        idx.bulk_load(td(w["build_keys"]), td(w["build_vals"]), stream=st)
        t_ins = t_del = 0.0
        for k, v in w["insert"]:
            kd, vd = td(k), td(v)
            t_ins += timed(lambda: idx.insert(kd, vd, stream=st))
            del kd, vd
        s_ins = idx.stats(stream=st)
        for k in w["delete"]:
            kd = td(k)
            t_del += timed(lambda: idx.delete(kd, stream=st))
            del kd
        s_del = idx.stats(stream=st)
        t_res = timed(lambda: idx.restructure(stream=st))
        s_res = idx.stats(stream=st)
        n_del = sum(k.size for k in w["delete"])
        row = {"workload": name, "build": b, "final": s_ins["live_keys"], "delete_share": round(imp["delete_share"], 4),
               "live_at_restructure": s_del["live_keys"],
               "nodes_after_inserts": s_ins["nodes_used"], "max_chain": s_ins["max_chain"],
               "nodes_before_restructure": s_del["nodes_used"], "nodes_after_restructure": s_res["nodes_used"],
               "nodes_recovered": s_del["nodes_used"] - s_res["nodes_used"],
               "recovered_pct": 100.0 * (s_del["nodes_used"] - s_res["nodes_used"]) / max(s_del["nodes_used"], 1),
               "paper": {"nodes_recovered": p_rec, "recovered_pct": p_pct,
                         "implied_nodes_before": round(imp["before"]), "implied_nodes_after": round(imp["after"])},
               "restructure_ms": t_res, "insert_mops": (final - b) / (t_ins * 1e-3) / 1e6,
               "delete_mops": n_del / (t_del * 1e-3) / 1e6}
        log("restructure accounting: %s" % row)
        table.append(row)
        idx.close()
        del w
        torch.cuda.empty_cache()

    line = {"form": "xy", "metric": METRIC, "value": tot_ops / (tot_ms * 1e-3) / 1e6, "unit": "Mops/s",
            "n_gpus": 1, "higher_is_better": True, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "dense-range updates: uint64, node size 32, build 2^24 uniform, 8 insert rounds "
                                   "of 3*2^21 keys with 90% in a hot interval of X of the key range, 8 delete "
                                   "rounds of the same keys; value = all insert and delete ops / their time "
                                   "(default structure; the _split4_merge rounds split chains past 4 nodes and "
                                   "merge underfull neighbours after every batch)"},
            "rounds": rounds_out, "restructure_accounting": table}
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
