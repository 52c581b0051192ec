#!/usr/bin/env python
"""PHOBIC construction + query benchmark on B300.

Workload: 1e8 distinct uniform uint64 keys, lambda = 7, alpha = 0.99 (Elias-Fano
remap of slots >= n), partition size 2500, interleaved dictionary encoding
(IC-D); then 1e8 uniform positive queries and 1e8 Zipf(s = 1) positive
queries.  One step = one build of the resident keys plus both query batches.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

`value` is build throughput (Mkeys/s, device-resident inputs, CUDA events on
the build stream); the query rates, bits/key, per-phase times, roofline,
end-to-end (host buffers) numbers and the CPU oracle baseline ride along on the
same JSON line.  Under torchrun each rank builds its own key set (independent
problems: weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import collections
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "build Mkeys/s & query Mkeys/s at 1e8 keys; bits/key; serve p50/p99 latency"
WORKLOAD = ("1e8 distinct uniform uint64 keys, lambda=7, alpha=0.99 with Elias-Fano free-slot remap, partition "
            "size 2500, interleaved dictionary (IC-D) pilot encoding; 1e8 uniform + 1e8 Zipf(s=1) positive queries")
SMALL = ("1e6 distinct uniform uint64 keys, lambda=7, alpha=1, partition size 2500, IC-C; 1e7 uniform positive "
         "queries")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--small", action="store_true", help="the 1e6-key configuration instead")
    ap.add_argument("--strings", action="store_true",
                    help="the 2e8-string configuration (random strings of 10-50 chars, lambda 7.5)")
    ap.add_argument("--n", type=float, default=None)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-target-s", type=float, default=12.0)
    ap.add_argument("--candidate-width", type=int, default=0, help="search window width (32/64; 0 = default)")
    ap.add_argument("--encoder", choices=["ic-c", "ic-d", "ic-r", "ic-ef"], default=None,
                    help="pilot encoder instead of the workload's own")
    ap.add_argument("--lam", type=float, default=None, help="average bucket size instead of the workload's own")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-build section")
    ap.add_argument("--no-xor", action="store_true", help="skip the XOR-pilot section")
    ap.add_argument("--batch-steps", type=int, default=3)
    ap.add_argument("--no-serve", action="store_true", help="skip the serving section")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--no-other-configs", action="store_true",
                    help="skip the 1e6-key and 2e8-string configurations measured after the default one")
    ap.add_argument("--sharded", action="store_true",
                    help="one MPHF over the keys of all ranks, built partition-sharded (all-to-all of master "
                         "hashes by partition owner; each rank holds --n keys)")
    ap.add_argument("--only", choices=["batch", "serve", "lambda", "ablation", "encoders", "table1"], default=None,
                    help="run one extra section alone (lambda: the large-lambda sweep; ablation: the bucket "
                         "functions of Fig. 3a)")
    return ap.parse_args()


STRINGS = ("2e8 random strings, lengths uniform in [10, 50] over [A-Za-z0-9], XXH64 master hashes on device, "
           "lambda=7.5, alpha=0.99 with Elias-Fano remap, partition size 2500, IC-D; every key queried once")


BATCH = ("batched build: 4096 independent sets of distinct uniform uint64 keys, sizes log-uniform in [1e3, 1e7] "
         "(seed 2024; about 4.45e9 keys in total), lambda=7, alpha=0.99, IC-D, each its own MPHF; partition size "
         "per size class, warps per partition and candidate width autotuned; compared with one phobic_build_ex per "
         "set (P 2500, default knobs)")
SERVE = ("serving: open-loop Poisson requests for {secs:g} s: builds (uint64 key sets, sizes log-uniform in "
         "[1e4, 5e7], lambda=7, alpha=0.99, IC-D) at {brate:g}/s and query batches (sizes log-uniform in [1e3, 1e6], "
         "90% members of a random resident MPHF, 10% random non-member keys) at {qrate:g}/s; 120 GB HBM budget; the "
         "oldest MPHF is released beyond {cap} resident; continuous batching compared with the same trace served "
         "one request at a time")


def workload(a):
    if a.strings:
        n = int(a.n or 2e8)
        return dict(name=STRINGS, n=n, lam=7.5, alpha=0.99, P=2500, encoder=1, q_uniform=n, q_zipf=0, strings=True)
    if a.small:
        n = int(a.n or 1e6)
        return dict(name=SMALL, n=n, lam=7.0, alpha=1.0, P=2500, encoder=0, q_uniform=10 * n, q_zipf=0)
    n = int(a.n or 1e8)
    w = dict(name=WORKLOAD, n=n, lam=7.0, alpha=0.99, P=2500, encoder=1, q_uniform=n, q_zipf=n)
    if a.encoder or a.lam:
        enc = {"ic-c": 0, "ic-d": 1, "ic-r": 2, "ic-ef": 3}[a.encoder] if a.encoder else w["encoder"]
        w.update(encoder=enc, lam=a.lam or w["lam"])
        w["name"] = (f"{n:.0e} distinct uniform uint64 keys, lambda={w['lam']:g}, alpha=0.99 with Elias-Fano remap, "
                     f"partition size 2500, {['IC-C', 'IC-D', 'IC-R', 'IC-EF'][enc]} pilot encoding; {n:.0e} uniform + "
                     f"{n:.0e} Zipf(s=1) positive queries (variant of the default workload)")
    return w


# Per-key counters from ncu captures (the 3e7-key case of
# this workload), valid only for the kernel sources they were taken on: each
# entry names the source files and the sha256 (first 16 hex digits) of their
# concatenation.  When a source changes, the counters are reported as null.
NCU_CAPTURES = {
    "k_search": {"files": ["paper_2404_18497_b300/csrc/k_search.cu", "paper_2404_18497_b300/csrc/phobic_dev.cuh"],
                 "sha": "ae6c0e449f2684ca", "n": 3e7, "warp_inst": 1927954660, "dram_bytes": 555685632 + 323745792},
    "k_query": {"files": ["paper_2404_18497_b300/csrc/k_query.cu", "paper_2404_18497_b300/csrc/phobic_dev.cuh"],
                "sha": "10e6fa277985462a", "n": 3e7, "dram_bytes": 249930240 + 198135296},
    "k_sort": {"files": ["paper_2404_18497_b300/csrc/k_sort.cu", "paper_2404_18497_b300/csrc/phobic_dev.cuh"],
               "sha": "5ad006ea5cf8bbe5", "n": 3e7,
               "dram_bytes": (240013824 + 186941952) + (240104192 + 196000512) + (240187392 + 195732736)},
    "k_hash": {"files": ["paper_2404_18497_b300/csrc/k_sort.cu", "paper_2404_18497_b300/csrc/phobic_dev.cuh"],
               "sha": "5ad006ea5cf8bbe5", "n": 3e7, "dram_bytes": 240025856 + 192203008},
}
ISSUE_SLOTS_PER_CLOCK = 148 * 4  # B300: 148 SMs x 4 warp schedulers, one warp instruction per clock each
SM_MAX_MHZ = 2032.0


def capture(name):
    import hashlib

    c = NCU_CAPTURES[name]
    h = hashlib.sha256()
    for f in c["files"]:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return c if h.hexdigest()[:16] == c["sha"] else None


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


class Clocks:
    """nvidia-smi samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            c = [x.strip() for x in line.split(",")]
            if len(c) < 9:
                continue
            try:
                sm.append(float(c[1]))
                mx.append(float(c[2]))
                power.append(float(c[3]))
            except ValueError:
                continue
            for nm, v in zip(names, c[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


# --------------------------------------------------------------- CPU oracle ---
def oracle_sample_rate(keys: np.ndarray, w: dict, target_s: float):
    """The oracle as it stands, on a bounded prefix of the same keys, all host
    cores.  Grows the sample until one build takes about target_s / 3."""
    from oracle import oracle as o

    o.lib()
    cores = os.cpu_count() or 1
    n_s = min(keys.size, 250_000)
    while True:
        t = time.perf_counter()
        h = o.Oracle(keys[:n_s], lam=w["lam"], alpha=w["alpha"], P=w["P"], encoder=w["encoder"], threads=cores)
        dt = time.perf_counter() - t
        if dt > target_s / 3 or n_s >= keys.size or n_s >= 20_000_000:
            break
        n_s = int(min(keys.size, n_s * max(2.0, (target_s / 3) / max(dt, 1e-3))))
    builds = [dt]
    while sum(builds) < target_s * 2 / 3 and len(builds) < 5:
        t = time.perf_counter()
        h = o.Oracle(keys[:n_s], lam=w["lam"], alpha=w["alpha"], P=w["P"], encoder=w["encoder"], threads=cores)
        builds.append(time.perf_counter() - t)
    qn = min(n_s, 1_000_000)
    t = time.perf_counter()
    h.query(keys[:qn])
    qdt = time.perf_counter() - t
    return {"value": n_s / min(builds) / 1e6, "unit": "Mkeys/s", "cores": cores, "kind": "oracle",
            "sample": f"oracle build of the first {n_s} keys of the workload (same lambda, alpha, P, encoder), "
                      f"best of {len(builds)}, OpenMP over partitions on {cores} threads; query of {qn} keys "
                      f"single-threaded",
            "query_value": qn / qdt / 1e6, "build_s": min(builds)}


def run_reference(a):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2404_18497_b300 import workloads

    w = workload(a)
    keys = workloads.distinct_u64(min(w["n"], 20_000_000), 2)
    from oracle import oracle as o

    o.lib()
    cores = os.cpu_count() or 1
    n_s = min(keys.size, 1_000_000 if not a.small else keys.size)
    times = []
    for i in range(a.warmup + a.steps):
        t = time.perf_counter()
        h = o.Oracle(keys[:n_s], lam=w["lam"], alpha=w["alpha"], P=w["P"], encoder=w["encoder"], threads=cores)
        dt = time.perf_counter() - t
        del h
        if i >= a.warmup:
            times.append(dt)
    ms = statistics.mean(times) * 1e3
    v = n_s / (ms / 1e3) / 1e6
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mkeys/s", "n_gpus": a.gpus, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "u64", "data": "synthetic",
           "config": {"workload": w["name"], "n": w["n"], "lambda": w["lam"], "alpha": w["alpha"], "P": w["P"],
                      "encoder": ["IC-C", "IC-D", "IC-R", "IC-EF"][w["encoder"]]},
           "cpu_baseline": {"value": v, "unit": "Mkeys/s", "cores": cores, "kind": "oracle",
                            "sample": f"each step: oracle build of the first {n_s} keys of the workload on {cores} "
                                      f"threads"},
           "e2e": {"value": v, "unit": "Mkeys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ------------------------------------------------------------------ ours -----
def run_ours(a):
    import torch

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2404_18497_b300 import build as libbuild

    libbuild.build()
    from paper_2404_18497_b300 import phobic, workloads

    w = workload(a)
    n = w["n"]
    keys = workloads.distinct_u64(n, 2 + 1000 * rank)
    qu = workloads.uniform_queries(keys, w["q_uniform"], 3 + 1000 * rank)
    qz = workloads.zipf_queries(keys, w["q_zipf"], 4 + 1000 * rank) if w["q_zipf"] else None
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    dqu = torch.from_numpy(qu.view(np.int64)).cuda()
    dqz = torch.from_numpy(qz.view(np.int64)).cuda() if qz is not None else None
    out = torch.empty(max(dqu.numel(), dqz.numel() if dqz is not None else 0), dtype=torch.int64, device="cuda")
    prm = phobic.make_params(w["lam"], w["alpha"], w["P"], seed=0, encoder=w["encoder"], record_timings=True,
                             candidate_width=a.candidate_width)
    stream = torch.cuda.current_stream()

    def step():
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record(stream)
        h = phobic.phobic_build_ex(dk, prm, stream)
        e[1].record(stream)
        phobic.phobic_query(h, dqu, out[: dqu.numel()], stream)
        e[2].record(stream)
        if dqz is not None:
            phobic.phobic_query(h, dqz, out[: dqz.numel()], stream)
        e[3].record(stream)
        return h, e

    for _ in range(a.warmup):
        h, _ = step()
        h.free()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    clk = Clocks(local)
    clk.start()
    l0 = phobic.phobic_kernel_launches()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    recs = []
    t0.record(stream)
    for _ in range(a.steps):
        h, e = step()
        recs.append((h, e))
    t1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    clocks = clk.stop()
    launches = phobic.phobic_kernel_launches() - l0
    total_ms = t0.elapsed_time(t1)
    build_ms = [e[0].elapsed_time(e[1]) for _, e in recs]
    qu_ms = [e[1].elapsed_time(e[2]) for _, e in recs]
    qz_ms = [e[2].elapsed_time(e[3]) for _, e in recs] if dqz is not None else [0.0]
    phases = [phobic.phobic_get_timings(h) for h, _ in recs]
    bpk = recs[-1][0].bits_per_key()
    info = recs[-1][0].info()
    # check the result on device: the query outputs are a permutation of [0, n)
    res = recs[-1][0].query(dk)
    perm_ok = bool(torch.equal(torch.sort(res).values, torch.arange(n, device="cuda")))
    ref_u = recs[-1][0].query(dqu).cpu().numpy()
    del res
    for h, _ in recs:
        h.free()

    ms_step = reduce_max(total_ms / a.steps, world)
    b_ms = reduce_max(statistics.mean(build_ms), world)
    u_ms = reduce_max(statistics.mean(qu_ms), world)
    z_ms = reduce_max(statistics.mean(qz_ms), world)
    ph = {k: statistics.mean(p[k] for p in phases) for k in phases[0]}

    # ---- roofline of the dominant kernel (CUDA events on the launching stream)
    hbm, src = peaks()
    kern = {
        "k_search (bucketing + pilot search)": ph["search_ms"],
        "k_sort_hist + 2 x k_sort_pass (hash + onesweep partition sort)": ph["sort_ms"],
        "k_query (uniform batch)": statistics.mean(qu_ms),
        "k_query (Zipf batch)": statistics.mean(qz_ms),
        "encode (offsets + IC-D)": ph["encode_ms"],
        "remap (Elias-Fano)": ph["remap_ms"],
    }
    dom = max(kern, key=kern.get)
    sm_mhz = (clocks.get("sm_mhz") or SM_MAX_MHZ) if isinstance(clocks, dict) else SM_MAX_MHZ
    # k_search: integer ALU + shared memory, no dense contraction; its ceiling is
    # the issue rate (warp instructions per second) at the SM clock
    cs = capture("k_search")
    peak_issue = ISSUE_SLOTS_PER_CLOCK * SM_MAX_MHZ * 1e6 / 1e9  # G warp-inst/s at the maximum clock
    if cs:
        inst = cs["warp_inst"] / cs["n"] * n
        achieved = inst / (ph["search_ms"] / 1e3) / 1e9
        traffic = cs["dram_bytes"] / cs["n"] * n
    else:
        inst = achieved = traffic = None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_issue, "unit": "G warp-inst/s",
                "frac": (achieved / peak_issue) if achieved else None, "traffic": traffic,
                "kernel": "k_search", "launch_ms": ph["search_ms"], "warp_inst_per_launch": inst,
                "peak_source": "148 SMs x 4 schedulers x 1 warp-inst/clock x 2032 MHz (unit counts and max clock)",
                "sm_mhz_measured": sm_mhz,
                "counters": f"ncu capture at {cs['n']:.0e} keys, scaled per key" if cs else
                            "stale: kernel source changed since the ncu capture",
                "dominant_kernel_by_time": dom, "per_kernel_ms": kern}
    cq = capture("k_query")
    q_bytes = 16.0 * w["q_uniform"]
    roofline["query"] = {"bound": "hbm", "achieved": q_bytes / (statistics.mean(qu_ms) / 1e3) / 1e9, "peak": hbm,
                         "unit": "GB/s", "kernel": "k_query (uniform batch)", "algorithmic_bytes_per_launch": q_bytes,
                         "traffic": (cq["dram_bytes"] / cq["n"] * w["q_uniform"]) if cq else None,
                         "peak_source": f"{src} hbm_gbs"}
    roofline["query"]["frac"] = roofline["query"]["achieved"] / hbm
    cso = capture("k_sort")
    # the method's bytes: histogram read 8 B + two passes x (8 B read + 8 B write) per key; the design moves
    # 8 B more (the histogram pass writes the hashes, so no pass hashes again), which the traffic shows
    sort_bytes = 40.0 * n
    roofline["sort"] = {"bound": "hbm", "achieved": sort_bytes / (ph["sort_ms"] / 1e3) / 1e9, "peak": hbm,
                        "unit": "GB/s", "kernel": "hash + onesweep partition sort",
                        "algorithmic_bytes_per_launch": sort_bytes,
                        "traffic": (cso["dram_bytes"] / cso["n"] * n) if cso else None}
    roofline["sort"]["frac"] = roofline["sort"]["achieved"] / hbm
    # the standalone hash stage (phobic_hash_u64: master hashes of the keys into a
    # second array, 16 B per key); the build fuses this hash into the sort
    hout = torch.empty_like(dk)
    for _ in range(3):
        phobic.phobic_hash_u64(dk, 0, hout, stream)
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h0.record(stream)
    for _ in range(5):
        phobic.phobic_hash_u64(dk, 0, hout, stream)
    h1.record(stream)
    torch.cuda.synchronize()
    hash_ms = h0.elapsed_time(h1) / 5
    del hout
    roofline["hash"] = {"bound": "hbm", "achieved": 16.0 * n / (hash_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                        "kernel": "k_hash_copy (phobic_hash_u64, 16-byte loads and stores)", "launch_ms": hash_ms,
                        "algorithmic_bytes_per_launch": 16.0 * n}
    roofline["hash"]["frac"] = roofline["hash"]["achieved"] / hbm
    chh = capture("k_hash")
    roofline["hash"]["traffic"] = (chh["dram_bytes"] / chh["n"] * n) if chh else None
    build_bytes = 8.3 * n
    roofline["build"] = {"bound": "hbm", "achieved": build_bytes / (b_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                         "kernel": "whole build", "algorithmic_bytes_per_launch": build_bytes}
    roofline["build"]["frac"] = roofline["build"]["achieved"] / hbm

    # ---- end to end through the host-buffer entry points
    e2e = None
    if not a.no_e2e:
        hk_pin = torch.from_numpy(keys.view(np.int64)).pin_memory()
        hq_pin = torch.from_numpy(qu.view(np.int64)).pin_memory()
        ho_pin = torch.empty_like(hq_pin).pin_memory()
        hkn, hqn, hon = hk_pin.numpy(), hq_pin.numpy(), ho_pin.numpy()
        prm2 = phobic.make_params(w["lam"], w["alpha"], w["P"], seed=0, encoder=w["encoder"])
        bt, qt = [], []
        for i in range(2 + min(a.steps, 5)):
            torch.cuda.synchronize()
            t = time.perf_counter()
            h = phobic.phobic_build_host(hkn, prm2, stream)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            phobic.phobic_query_host(h, hqn, hon.view(np.uint64), stream)
            t3 = time.perf_counter()
            if i >= 2:
                bt.append(t2 - t)
                qt.append(t3 - t2)
            h.free()
        ok = bool(np.array_equal(hon, ref_u))
        e2e = {"value": world * n / reduce_max(statistics.mean(bt), world) / 1e6, "unit": "Mkeys/s",
               "h2d_bytes_per_step": 8 * n + 8 * w["q_uniform"], "d2h_bytes_per_step": 8 * w["q_uniform"],
               "query_value": world * w["q_uniform"] / reduce_max(statistics.mean(qt), world) / 1e6,
               "note": "phobic_build_host (pinned keys, H2D inside) + phobic_query_host (H2D keys, D2H results)",
               "check": ok}

    xor = None
    if not a.no_xor and a.impl == "ours":
        xor = run_xor(a, phobic, torch, dk, dqu, out, w, n, world)

    batch = serve = None
    if world == 1 and not (a.no_batch and a.no_serve):
        dk = dqu = dqz = out = None
        torch.cuda.empty_cache()
        phobic.phobic_trim(0)
        if not a.no_batch:
            batch = run_batch(a, phobic, workloads, torch)
        if not a.no_serve:
            serve = run_serve(a, phobic, workloads, torch)

    others = None
    if world == 1 and not a.no_other_configs and a.impl == "ours" and n == int(1e8):
        dk = dqu = dqz = out = None
        torch.cuda.empty_cache()
        others = run_other_configs(a, phobic, workloads, torch)

    if rank != 0:
        return
    cpu = None
    if world == 1 and not a.no_cpu_baseline:
        cpu = oracle_sample_rate(keys, w, a.cpu_target_s)
    gpu_name = torch.cuda.get_device_name(local)
    res_line = {
        "metric": METRIC,
        "value": world * n / (b_ms / 1e3) / 1e6,
        "unit": "Mkeys/s",
        "n_gpus": world,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": w["name"], "n": n, "lambda": w["lam"], "alpha": w["alpha"], "P": w["P"],
                   "encoder": ["IC-C", "IC-D", "IC-R", "IC-EF"][w["encoder"]], "queries_uniform": w["q_uniform"],
                   "queries_zipf": w["q_zipf"], "parallelism": f"independent key set per GPU x{world}",
                   "l2": "inputs larger than L2 (8e8-byte key and query arrays vs 126 MB L2)", "gpu": gpu_name},
        "build_ms": b_ms,
        "build_mkeys_s": world * n / (b_ms / 1e3) / 1e6,
        "query_mkeys_s": world * w["q_uniform"] / (u_ms / 1e3) / 1e6,
        "query_zipf_mkeys_s": (world * w["q_zipf"] / (z_ms / 1e3) / 1e6) if w["q_zipf"] else None,
        "bits_per_key": bpk,
        "phase_ms": ph,
        "structure": {k: info[k] for k in ("M", "num_partitions", "num_buckets", "max_partition", "bits_pilots",
                                           "bits_offsets", "bits_remap", "device_bytes")},
        "result_is_permutation": perm_ok,
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": launches,
        "gpu_launches_per_step": launches / a.steps,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "xor_mode": xor,
        "batch": batch,
        "serve": serve,
        "other_configs": others,
    }
    print(json.dumps(res_line))


def _time_build_query(phobic, torch, build, query, steps, warmup):
    """Mean device ms of build() and of query(h) over `steps` after `warmup`,
    CUDA events on the current stream; returns (build ms, query ms, last handle)."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        h = build()
        query(h)
        h.free()
    bms, qms = [], []
    for i in range(steps):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        h = build()
        e[1].record(stream)
        query(h)
        e[2].record(stream)
        torch.cuda.synchronize()
        bms.append(e[0].elapsed_time(e[1]))
        qms.append(e[1].elapsed_time(e[2]))
        if i + 1 < steps:
            h.free()
    return statistics.mean(bms), statistics.mean(qms), h


def run_other_configs(a, phobic, workloads, torch):
    """The two other single-GPU configurations on the same run, after the timed
    region of the default one: C1 (1e6 u64 keys, lambda 7, alpha 1, IC-C, 1e7
    uniform queries) and C3 (2e8 random strings of 10-50 characters, lambda
    7.5, alpha 0.99, IC-D, every string queried once)."""
    hbm, _ = peaks()
    res = {}
    keys = workloads.distinct_u64(1_000_000, 1)
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    dq = torch.from_numpy(workloads.uniform_queries(keys, 10_000_000, 3).view(np.int64)).cuda()
    out = torch.empty_like(dq)
    prm = phobic.make_params(7.0, 1.0, 2500, seed=0, encoder="IC-C")
    b, q, h = _time_build_query(phobic, torch, lambda: phobic.phobic_build_ex(dk, prm),
                                lambda hh: phobic.phobic_query(hh, dq, out), 10, 3)
    res["C1"] = {"workload": SMALL, "build_ms": b, "build_mkeys_s": 1e6 / (b / 1e3) / 1e6, "query_ms": q,
                 "query_mkeys_s": 1e7 / (q / 1e3) / 1e6, "query_hbm_frac": 16.0 * 1e7 / (q / 1e3) / 1e9 / hbm,
                 "bits_per_key": h.bits_per_key(),
                 "result_is_permutation": bool(torch.equal(torch.sort(h.query(dk)).values,
                                                           torch.arange(1_000_000, device="cuda")))}
    h.free()
    del dk, dq, out
    n = 200_000_000
    data, off = workloads.random_strings_torch(n, 3, "cuda")
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    prm = phobic.make_params(7.5, 0.99, 2500, seed=0, encoder="IC-D")

    def build_s():
        while True:
            try:
                return phobic.phobic_build_strings(data, off, prm)
            except phobic.PhobicError as e:  # two strings share a 64-bit hash: take another seed
                if e.status != "DUP_HASH":
                    raise
                prm.seed += 1

    b, q, h = _time_build_query(phobic, torch, build_s, lambda hh: phobic.phobic_query_strings(hh, data, off, out),
                                5, 2)
    str_bytes = float(off[-1].item()) + 8.0 * (n + 1)
    res["C3"] = {"workload": STRINGS + " (strings drawn on the device with torch's generator)", "build_ms": b,
                 "build_mkeys_s": n / (b / 1e3) / 1e6, "query_ms": q, "query_mkeys_s": n / (q / 1e3) / 1e6,
                 "query_hbm_frac": (str_bytes + 8.0 * n) / (q / 1e3) / 1e9 / hbm, "bits_per_key": h.bits_per_key(),
                 "seed": int(prm.seed),
                 "result_is_permutation": bool(torch.equal(torch.sort(out).values,
                                                           torch.arange(n, device="cuda")))}
    h.free()
    del data, off, out
    torch.cuda.empty_cache()
    return res

# ------------------------------------------------------ partition-sharded ---
SHARDED = ("one MPHF over {total:.0e} distinct uint64 keys ({n:.0e} resident per GPU, counter-based stream), "
           "lambda=7, alpha=0.99 with Elias-Fano remap, partition size 2500, IC-D, built partition-sharded over "
           "{world} GPU(s); {n:.0e} uniform positive queries per GPU against the replicated structure")


def run_sharded(a):
    """The build of ONE MPHF whose keys are spread over all ranks (Section 4:
    partitions are independent): each rank hashes and groups its own keys, one
    all-to-all sends every partition's hashes to its owner, each rank searches
    its partitions, and one all-reduce merges pilots and occupancy; every rank
    then encodes the same structure.  Weak scaling: each rank holds n keys."""
    import hashlib
    import socket

    import torch
    import torch.distributed as dist

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        with socket.socket() as so:
            so.bind(("127.0.0.1", 0))
            port = so.getsockname()[1]
        dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1,
                                device_id=torch.device("cuda", local))
    from paper_2404_18497_b300 import build as libbuild

    libbuild.build()
    from paper_2404_18497_b300 import phobic, shard, workloads

    n = int(a.n or 1e8)
    keys = workloads.stream_keys_torch(rank * n, n, 2, "cuda")
    g = torch.Generator(device="cuda")
    g.manual_seed(3 + 1000 * rank)
    dq = keys[torch.randint(0, n, (n,), device="cuda", generator=g)]
    out = torch.empty_like(dq)
    prm = phobic.make_params(7.0, 0.99, 2500, seed=0, encoder="IC-D")
    comm = shard.TorchComm(device=torch.device("cuda", local))
    stream = torch.cuda.current_stream()

    def step():
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        h = shard.sharded_build(keys, prm, comm)
        e[1].record(stream)
        phobic.phobic_query(h, dq, out, stream)
        e[2].record(stream)
        return h, e

    for _ in range(a.warmup):
        h, _ = step()
        h.free()
    torch.cuda.synchronize()
    barrier(world)
    clk = Clocks(local)
    clk.start()
    l0 = phobic.phobic_kernel_launches()
    t0 = time.perf_counter()
    recs = []
    for _ in range(a.steps):
        recs.append(step())
    torch.cuda.synchronize()
    barrier(world)
    wall_ms = (time.perf_counter() - t0) * 1e3
    clocks = clk.stop()
    launches = phobic.phobic_kernel_launches() - l0
    b_ms = reduce_max(statistics.mean(e[0].elapsed_time(e[1]) for _, e in recs), world)
    q_ms = reduce_max(statistics.mean(e[1].elapsed_time(e[2]) for _, e in recs), world)
    ms_step = reduce_max(wall_ms / a.steps, world)
    h = recs[-1][0]
    digest = int(hashlib.sha256(h.export()).hexdigest()[:15], 16)
    same_everywhere = len(set(comm.all_gather_int(digest))) == 1
    srt = torch.sort(h.query(keys)).values  # this rank's keys get distinct positions below world * n
    distinct = int((srt[1:] != srt[:-1]).sum().item()) + 1
    ok_perm = distinct == n and int(srt[-1].item()) < world * n and int(srt[0].item()) >= 0
    ok_perm = min(comm.all_gather_int(int(ok_perm))) == 1
    del srt
    bpk = h.bits_per_key()
    single_equal = None
    if world == 1:
        ref = phobic.phobic_build_ex(keys, prm)
        single_equal = ref.export() == h.export()
        ref.free()
    for hh, _ in recs:
        hh.free()

    e2e = None
    if not a.no_e2e:
        pin = keys.cpu().pin_memory()
        dk2 = torch.empty_like(keys)
        ts = []
        for i in range(2 + min(a.steps, 3)):
            torch.cuda.synchronize()
            barrier(world)
            t = time.perf_counter()
            dk2.copy_(pin, non_blocking=True)
            hh = shard.sharded_build(dk2, prm, comm)
            torch.cuda.synchronize()
            if i >= 2:
                ts.append(time.perf_counter() - t)
            hh.free()
        e2e = {"value": world * n / reduce_max(statistics.mean(ts), world) / 1e6, "unit": "Mkeys/s",
               "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 0,
               "note": "each rank's keys copied from pinned host memory inside the timed region, then the sharded build"}
    if rank != 0:
        dist.destroy_process_group()
        return
    hbm, src = peaks()
    build_bytes = 8.3 * n
    line = {
        "metric": METRIC, "value": world * n / (b_ms / 1e3) / 1e6, "unit": "Mkeys/s", "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": SHARDED.format(total=world * n, n=n, world=world), "n_total": world * n,
                   "n_per_gpu": n, "lambda": 7.0, "alpha": 0.99, "P": 2500, "encoder": "IC-D",
                   "parallelism": f"partition-sharded x{world} (NCCL all-to-all + all-reduce)",
                   "l2": "inputs larger than L2 (8e8-byte key and query arrays vs 126 MB L2)",
                   "gpu": torch.cuda.get_device_name(local)},
        "build_ms": b_ms, "query_mkeys_s": world * n / (q_ms / 1e3) / 1e6, "bits_per_key": bpk,
        "structure_identical_on_all_ranks": same_everywhere, "equals_single_build": single_equal,
        "positions_distinct_per_rank": ok_perm, "clocks": clocks, "e2e": e2e, "gpu_launches": launches,
        "roofline": {"bound": "hbm", "achieved": build_bytes / (b_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                     "frac": build_bytes / (b_ms / 1e3) / 1e9 / hbm, "traffic": None,
                     "kernel": "whole sharded build (8.3 B/key algorithmic)", "peak_source": f"{src} hbm_gbs"},
        "cpu_baseline": None,
    }
    print(json.dumps(line))
    dist.destroy_process_group()


# ------------------------------------------------------------- XOR pilots ---
def run_xor(a, phobic, torch, dk, dqu, out, w, n, world):
    """The same workload with PTHash's pilot form, position h(x XOR h(p)) mod m
    and p = 0, 1, 2, ... (the form without displacement): one warm-up build, two
    timed builds and one timed uniform query batch, CUDA events on the stream."""
    stream = torch.cuda.current_stream()
    prm = phobic.make_params(w["lam"], w["alpha"], w["P"], seed=0, encoder=w["encoder"], mode="xor",
                             record_timings=True)
    h = phobic.phobic_build_ex(dk, prm, stream)
    h.free()
    bms, sms = [], []
    for _ in range(2):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        h = phobic.phobic_build_ex(dk, prm, stream)
        e1.record(stream)
        phobic.phobic_query(h, dqu, out[: dqu.numel()], stream)
        e2.record(stream)
        torch.cuda.synchronize()
        bms.append(e0.elapsed_time(e1))
        sms.append(phobic.phobic_get_timings(h)["search_ms"])
        qms = e1.elapsed_time(e2)
        if _ == 0:
            h.free()
    res = h.query(dk)
    perm_ok = bool(torch.equal(torch.sort(res).values, torch.arange(n, device="cuda")))
    bpk = h.bits_per_key()
    del res
    h.free()
    b_ms = reduce_max(statistics.mean(bms), world)
    return {"pilot_form": "h(x XOR h(p)) mod m, p = 0, 1, 2, ... (same keys, lambda, alpha, P and encoder)",
            "build_ms": b_ms, "build_mkeys_s": world * n / (b_ms / 1e3) / 1e6,
            "search_ms": statistics.mean(sms), "query_mkeys_s": world * w["q_uniform"] / (qms / 1e3) / 1e6,
            "bits_per_key": bpk, "result_is_permutation": perm_ok}


# ------------------------------------------------------- batched build (C4) ---
def run_batch(a, phobic, workloads, torch):
    """4096 sets built by one batched launch sequence (autotuned) against one
    build per set; device-resident keys, CUDA events on the build stream."""
    stream = torch.cuda.current_stream()
    off = workloads.batch_sets(4096, 1e3, 1e7, 2024)
    sizes = np.diff(off).astype(np.int64)
    total = int(off[-1])
    prm = phobic.make_params(7.0, 0.99, 2500, encoder=1)
    t = time.perf_counter()
    Ps, tuned, tinfo = phobic.phobic_tune_batch(off, prm, stream)
    tune_s = time.perf_counter() - t
    t = time.perf_counter()
    _, _, tinfo2 = phobic.phobic_tune_batch(off, prm, stream)
    tune_cached_s = time.perf_counter() - t
    keys = workloads.stream_keys_torch(0, total, 11, "cuda")
    torch.cuda.synchronize()

    def batched():
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        hs = phobic.phobic_build_batch(keys, off, tuned, partition_sizes=Ps, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        return hs, e0.elapsed_time(e1)

    hs, _ = batched()  # warm-up
    bits = sum(h.bits_per_key() * int(n) for h, n in zip(hs, sizes)) / total
    for h in hs:
        h.free()
    l0 = phobic.phobic_kernel_launches()
    ms = []
    for _ in range(a.batch_steps):
        hs, dt = batched()
        ms.append(dt)
        for h in hs:
            h.free()
    launches = (phobic.phobic_kernel_launches() - l0) / a.batch_steps
    # the plain path: one phobic_build_ex per set, P 2500, default knobs
    seq = phobic.make_params(7.0, 0.99, 2500, encoder=1)
    for s in range(16):
        phobic.phobic_build_ex(keys[int(off[s]):int(off[s + 1])], seq, stream).free()
    torch.cuda.synchronize()
    l0 = phobic.phobic_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    seq_bits = 0.0
    for s in range(sizes.size):
        h = phobic.phobic_build_ex(keys[int(off[s]):int(off[s + 1])], seq, stream)
        seq_bits += h.bits_per_key() * int(sizes[s])
        h.free()
    e1.record(stream)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1)
    seq_launches = phobic.phobic_kernel_launches() - l0
    del keys
    torch.cuda.empty_cache()
    phobic.phobic_trim(0)
    b_ms = statistics.mean(ms)
    return {
        "workload": BATCH, "sets": int(sizes.size), "keys": total, "steps": a.batch_steps,
        "batched_ms": b_ms, "batched_ms_all": ms, "batched_mkeys_s": total / (b_ms / 1e3) / 1e6,
        "batched_launches": launches, "bits_per_key": bits,
        "sequential_ms": seq_ms, "sequential_mkeys_s": total / (seq_ms / 1e3) / 1e6,
        "sequential_launches": seq_launches, "sequential_bits_per_key": seq_bits / total,
        "speedup_vs_sequential": seq_ms / b_ms,
        "tuned": {"partition_size_by_decade": {f"1e{c}": ci["partition_size"] for c, ci in tinfo["classes"].items()},
                  "sets_by_decade": {f"1e{c}": ci["sets"] for c, ci in tinfo["classes"].items()},
                  "ns_per_key_by_decade": {f"1e{c}": ci["ns_per_key"] for c, ci in tinfo["classes"].items()},
                  "warps_per_partition": tinfo["warps_per_partition"], "candidate_width": tinfo["candidate_width"],
                  "launch_ns_per_key": tinfo["launch_ns_per_key"], "total_partitions": tinfo["total_partitions"],
                  "search_schedule": {1: "one CTA per partition", 2: "persistent CTAs over the work queue"}.get(
                      tinfo["search_schedule"], tinfo["search_schedule"]),
                  "schedule_ns_per_key": tinfo["schedule_ns_per_key"],
                  "tune_s": tune_s, "tune_cached_s": tune_cached_s,
                  "cached_second_call": bool(tinfo2["cached_launch"])},
        "l2": "inputs larger than L2 (35.6 GB of keys vs 126 MB L2)",
    }


# ------------------------------------------------------ large-lambda sweep ---
# the paper's PHOBIC-GPU rows (RTX 3090 through Vulkan, 1e8 strings, IC-R, alpha 1), context only
PAPER_GPU_NS_PER_KEY = {9: 27.0, 13: 560.0, 14: 1470.0}


def run_lambda_sweep(a, phobic, workloads, torch):
    """Build and query across lambda = 7 .. 14 (IC-R, alpha 1, P 2500): the
    regime where the pilot search dominates (about e^lambda slot tests per
    key, Section 3).  1e8 keys up to lambda 10, 1e7 above (bounded time)."""
    stream = torch.cuda.current_stream()
    out = []
    for lam in (7.0, 8.0, 9.0, 10.0, 11.0, 12.0, 13.0, 14.0):
        n = 100_000_000 if lam <= 10 else 10_000_000
        keys = workloads.stream_keys_torch(0, n, 29, "cuda")
        res = torch.empty_like(keys)
        prm = phobic.make_params(lam, 1.0, 2500, encoder=2, record_timings=True)
        steps = 3 if lam <= 12 else 2
        bms, qms, tm = [], [], None
        h = phobic.phobic_build_ex(keys, prm, stream)  # warm-up
        h.free()
        for _ in range(steps):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
            h = phobic.phobic_build_ex(keys, prm, stream)
            e[1].record(stream)
            phobic.phobic_query(h, keys, res, stream)
            e[2].record(stream)
            torch.cuda.synchronize()
            bms.append(e[0].elapsed_time(e[1]))
            qms.append(e[1].elapsed_time(e[2]))
            tm = phobic.phobic_get_timings(h)
            bpk = h.bits_per_key()
            h.free()
        ok = bool(torch.equal(torch.sort(res).values, torch.arange(n, device="cuda")))
        b = statistics.mean(bms)
        out.append({"lambda": lam, "n": n, "build_ms": b, "ns_per_key": b * 1e6 / n, "build_mkeys_s": n / b / 1e3,
                    "search_ms": tm["search_ms"], "s_tries_per_key": tm["search_s_tries"] / n,
                    "bits_per_key": bpk, "query_mkeys_s": n / statistics.mean(qms) / 1e3, "permutation": ok,
                    "paper_gpu_ns_per_key": PAPER_GPU_NS_PER_KEY.get(int(lam))})
        del keys, res
    torch.cuda.empty_cache()
    phobic.phobic_trim(0)
    return {"workload": "large-lambda sweep: distinct uniform uint64 keys (counter-based stream), alpha=1, "
                        "partition size 2500, IC-R; 1e8 keys for lambda <= 10, 1e7 above; every key queried",
            "rows": out,
            "paper_context": "PHOBIC-GPU ns/key from the paper's Table 1 (RTX 3090, Vulkan, 1e8 strings, incl. "
                             "its CPU share); not the same machine or input"}


# ---------------------------------------------------------------- Table 1 ----
# the paper's PHOBIC-GPU rows: (lambda, encoder, ns/key, bits/key), RTX 3090 through Vulkan
PAPER_TABLE1 = [(9.0, 0, 28.0, 2.17), (9.0, 2, 27.0, 1.76), (13.0, 2, 560.0, 1.68), (14.0, 2, 1470.0, 1.67)]


def run_table1(a, phobic, workloads, torch):
    """The paper's own GPU workload (Table 1): 1e8 random strings, alpha = 1,
    partition size 2500, at its lambda and encoder pairs.  Reports the build
    with the strings resident on the device, the upload of the strings and
    offsets from pinned host memory (the paper's times include the transfer), and
    the space."""
    stream = torch.cuda.current_stream()
    n = 100_000_000
    data, off = workloads.random_strings(n, 17)
    hd = torch.from_numpy(data).pin_memory()
    ho = torch.from_numpy(off.view(np.int64)).pin_memory()
    dd = torch.empty_like(hd, device="cuda")
    do = torch.empty_like(ho, device="cuda")
    up = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dd.copy_(hd, non_blocking=True)
        do.copy_(ho, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        up.append(e0.elapsed_time(e1))
    up_ms = statistics.median(up)
    del data
    rows = []
    for lam, enc, paper_ns, paper_bits in PAPER_TABLE1:
        prm = phobic.make_params(lam, 1.0, 2500, seed=0, encoder=enc, record_timings=True)
        seed, bms = 0, []
        for it in range(2):
            while True:
                try:
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    h = phobic.phobic_build_strings(dd, do, prm, stream)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    break
                except phobic.PhobicError as e:  # a 64-bit collision of two strings: take another seed
                    if e.status != "DUP_HASH":
                        raise
                    seed += 1
                    prm.seed = seed
            bms.append(e0.elapsed_time(e1))
            bpk = h.bits_per_key()
            if it == 0:
                h.free()
        out = torch.empty(n, dtype=torch.int64, device="cuda")
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        phobic.phobic_query_strings(h, dd, do, out, stream)
        q1.record(stream)
        torch.cuda.synchronize()
        perm = bool(torch.equal(torch.sort(out).values, torch.arange(n, device="cuda")))
        h.free()
        del out
        b_ms = bms[-1]
        rows.append({"lambda": lam, "encoder": ["IC-C", "IC-D", "IC-R"][enc], "build_ms": b_ms,
                     "build_ns_per_key": b_ms * 1e6 / n, "with_upload_ns_per_key": (b_ms + up_ms) * 1e6 / n,
                     "bits_per_key": bpk, "query_ns_per_key": q0.elapsed_time(q1) * 1e6 / n,
                     "permutation": perm, "paper_gpu_ns_per_key": paper_ns, "paper_bits_per_key": paper_bits,
                     "speedup_vs_paper_incl_upload": paper_ns / ((b_ms + up_ms) * 1e6 / n)})
    del dd, do
    torch.cuda.empty_cache()
    phobic.phobic_trim(0)
    return {"workload": "the paper's Table 1 GPU workload: 1e8 random strings (lengths uniform in [10, 50] over "
                        "[A-Za-z0-9], XXH64 on the device), alpha = 1, partition size 2500",
            "upload_ms": up_ms, "upload_bytes": int(off[-1]) + 8 * (n + 1), "rows": rows,
            "paper_context": "PHOBIC-GPU on an RTX 3090 through Vulkan with 8 CPU threads (Table 1); its times "
                             "include the transfer of the input"}


# ---------------------------------------------------------------- encoders ---
def run_encoders(a, phobic, workloads, torch):
    """Figure 3b's comparison on this GPU: space and query rate of every pilot
    encoder, interleaved and mono (all pilots in one encoder), and of Compact/Rice
    mixtures with c leading Compact columns (lambda 8, alpha 1, P 2500, 1e8 keys,
    every key queried in random order)."""
    stream = torch.cuda.current_stream()
    n = 100_000_000
    keys = workloads.stream_keys_torch(0, n, 37, "cuda")
    perm = torch.randperm(n, device="cuda", generator=torch.Generator(device="cuda").manual_seed(3))
    qkeys = keys[perm]
    del perm
    out = torch.empty_like(qkeys)
    rows = []
    configs = [("IC-C", 0, 0), ("IC-D", 1, 0), ("IC-EF", 3, 0), ("IC-R", 2, 0)] + [
        (f"IC-CR c={c}", 4, c) for c in (8, 32, 80, 160)] + [
        ("mono-C", 5, 0), ("mono-D", 6, 0), ("mono-EF", 8, 0), ("mono-R", 7, 0)]
    for name, enc, c in configs:
        prm = phobic.make_params(8.0, 1.0, 2500, encoder=enc, compact_columns=c, record_timings=True)
        h = phobic.phobic_build_ex(keys, prm, stream)
        for _ in range(3):
            phobic.phobic_query(h, qkeys, out, stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(5):
            phobic.phobic_query(h, qkeys, out, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        q_ms = e0.elapsed_time(e1) / 5
        rows.append({"encoder": name, "bits_per_key": h.bits_per_key(), "query_ns_per_key": q_ms * 1e6 / n,
                     "query_mkeys_s": n / q_ms / 1e3, "encode_ms": phobic.phobic_get_timings(h)["encode_ms"]})
        h.free()
    del keys, qkeys, out
    torch.cuda.empty_cache()
    phobic.phobic_trim(0)
    return {"workload": "pilot encoders (Fig. 3b): 1e8 distinct uniform uint64 keys (counter-based stream), lambda=8, "
                        "alpha=1, partition size 2500; every key queried once in a random order",
            "rows": rows,
            "paper_context": "Fig. 3b (CPU queries, 1e8 strings): IC-C 2.208 b/k, IC-D 2.599, IC-EF 1.824, IC-R 1.775; "
                             "mono-C 3.012, mono-D 2.163, mono-EF 1.909, mono-R 1.862"}


# ------------------------------------------------------- bucket functions ---
def run_ablation(a, phobic, workloads, torch):
    """Figure 3a's comparison on this GPU: construction time and space of each
    bucket assignment function (the optimised beta_eps, beta_* without eps,
    PTHash's skewed split, CHD's uniform one) across lambda.  1e7 keys, IC-R,
    alpha 1, P 2500; device-resident keys, CUDA events."""
    stream = torch.cuda.current_stream()
    n = 10_000_000
    keys = workloads.stream_keys_torch(0, n, 31, "cuda")
    names = {0: "optimized (beta_eps)", 1: "beta_* (eps = 0)", 2: "skewed (PTHash)", 3: "uniform (CHD)"}
    rows = []
    for fn in (0, 1, 2, 3):
        for lam in (4.0, 5.0, 6.0, 7.0, 8.0):
            prm = phobic.make_params(lam, 1.0, 2500, encoder=2, bucket_function=fn, record_timings=True)
            try:
                phobic.phobic_build_ex(keys, prm, stream).free()
                ms, sms = [], []
                for _ in range(3):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    h = phobic.phobic_build_ex(keys, prm, stream)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ms.append(e0.elapsed_time(e1))
                    t = phobic.phobic_get_timings(h)
                    sms.append(t["search_ms"])
                    bpk = h.bits_per_key()
                    tries = t["search_s_tries"]
                    h.free()
                rows.append({"bucket_function": names[fn], "lambda": lam, "build_ms": statistics.mean(ms),
                             "ns_per_key": statistics.mean(ms) * 1e6 / n, "search_ms": statistics.mean(sms),
                             "s_tries_per_key": tries / n, "bits_per_key": bpk})
            except phobic.PhobicError as e:
                rows.append({"bucket_function": names[fn], "lambda": lam, "error": e.status})
    del keys
    torch.cuda.empty_cache()
    phobic.phobic_trim(0)
    return {"workload": "bucket assignment functions (Fig. 3a): 1e7 distinct uniform uint64 keys (counter-based "
                        "stream), IC-R, alpha=1, partition size 2500, lambda 4..8", "rows": rows}


# ------------------------------------------------------------ serving (C5) ---
def _percentiles(x):
    if len(x) == 0:
        return {"p50_ms": None, "p99_ms": None, "mean_ms": None, "max_ms": None}
    x = np.asarray(x, dtype=np.float64) / 1e6
    return {"p50_ms": float(np.percentile(x, 50)), "p99_ms": float(np.percentile(x, 99)),
            "mean_ms": float(x.mean()), "max_ms": float(x.max())}


def serve_trace(secs, brate, qrate, seed, build_sizes=(1e4, 5e7), query_sizes=(1e3, 1e6)):
    """Seeded open-loop trace: (arrival s, kind, size) sorted by arrival."""
    rng = np.random.default_rng(seed)
    ev = []
    for kind, rate, (lo, hi) in ((0, brate, build_sizes), (1, qrate, query_sizes)):
        t = 0.0
        while True:
            t += rng.exponential(1.0 / rate)
            if t >= secs:
                break
            ev.append((t, kind, int(np.exp(rng.uniform(np.log(lo), np.log(hi))))))
    ev.sort()
    return ev


def _serve_warmup(srv, keys_pool, prm):
    """One build per build slot, a query against each, then their release, all
    waited for: the worker threads, the memory pool and the query path are warm
    before the clock starts (a long-running server is)."""
    n = 1_000_000
    ids = []
    for k in range(2):
        ids.append(srv.submit_build(keys_pool[k * n:(k + 1) * n], prm))
    srv.drain(600)
    hids = [int(c["handle_id"]) for c in srv.poll() if int(c["kind"]) == 0 and int(c["status"]) == 0]
    import torch
    out = torch.empty(10_000, dtype=torch.int64, device=keys_pool.device)
    for h in hids:
        srv.submit_query(h, keys_pool[:10_000], out)
        srv.drain(600)
        srv.submit_release(h)
    srv.drain(600)
    srv.poll()


def run_serve_mode(phobic, torch, trace, serial, keys_pool, cap, seed, check_every=100, budget=120 * 10**9):
    """Replays the trace against a server.  Latency is measured from each
    request's scheduled arrival (open loop: a late submission counts against
    it) to its completion, on the steady clock the library also uses.

    Every key set is a window [ps, ps + n) of a pool of distinct keys.  A query
    batch of m keys is one slice of the pool that covers 90% of it inside the
    set's window and 10% just outside it (keys of the pool that are not in the
    set: random non-members), so no request needs a copy of its input.

    The client keeps its per-request records in arrays indexed by request id
    and takes completions in vectorised batches, so that its own bookkeeping
    does not limit the offered load."""
    P = keys_pool.numel()
    margin = 1 << 20
    rng = np.random.default_rng(seed)
    prm = phobic.make_params(7.0, 0.99, 2500, encoder=1)
    srv = phobic.Server(hbm_budget_bytes=budget, build_slots=2, serial=serial)
    ring = 1 << 27
    qout = torch.empty(ring, dtype=torch.int64, device="cuda")
    _serve_warmup(srv, keys_pool, prm)
    cap_ids = 2 * len(trace) + 4096
    arrival = np.zeros(cap_ids, dtype=np.int64)
    pending = np.zeros(cap_ids, dtype=bool)
    is_sample = np.zeros(cap_ids, dtype=bool)
    qregion = {}    # sampled query id -> (ring start, keys)
    binfo = {}      # build id -> (pool start, keys)
    pend_q = collections.deque()  # (request id, ring start, keys) of submitted queries, oldest first
    resident = []   # (handle id, pool start, n), oldest first
    keep = set()    # handles kept for the final checks
    samples = []    # (handle id, pool start, m, request id)
    outs = {}
    parts = []      # per poll: (kind, latency from arrival, latency from submission, batch requests, keys)
    checked_builds = []
    tt = np.array([e[0] for e in trace], dtype=np.float64)
    tk = np.array([e[1] for e in trace], dtype=np.int64)
    ts = np.array([e[2] for e in trace], dtype=np.int64)
    head = 0
    torch.cuda.synchronize()

    def handle_completions():
        comp = srv.poll()
        if comp.size == 0:
            return 0
        rid = comp["request_id"].astype(np.int64)
        kind = comp["kind"].astype(np.int64)
        tdone = comp["t_done_ns"].astype(np.int64)
        pending[rid] = False
        parts.append((kind, tdone - arrival[rid], tdone - comp["t_submit_ns"].astype(np.int64),
                      comp["batch_requests"].astype(np.int64), comp["keys"].astype(np.int64)))
        for i in np.flatnonzero(kind == 0):  # builds: few
            if int(comp["status"][i]) != 0:
                continue
            ps, n = binfo.pop(int(rid[i]))
            hid = int(comp["handle_id"][i])
            resident.append((hid, ps, n))
            if len(checked_builds) < 3 and n < 3_000_000:
                checked_builds.append((hid, ps, n))
                keep.add(hid)
        for i in np.flatnonzero(is_sample[rid]):  # sampled queries: their answers, for the final check
            st0, m0 = qregion[int(rid[i])]
            outs[int(rid[i])] = qout[st0:st0 + m0].clone()
        return comp.size

    t0 = time.monotonic_ns()
    i = 0
    since_poll = 0
    while i < len(trace):
        now = time.monotonic_ns()
        arr = t0 + int(tt[i] * 1e9)
        if arr > now:
            if handle_completions() == 0:
                time.sleep(min(2e-4, (arr - now) / 1e9))
            since_poll = 0
            continue
        kind, size = int(tk[i]), int(ts[i])
        i += 1
        if kind == 0:
            n = size
            ps = int(rng.integers(margin, P - n - margin))
            rid = srv.submit_build(keys_pool[ps:ps + n], prm)
            arrival[rid] = arr
            pending[rid] = True
            binfo[rid] = (ps, n)
        else:
            if not resident:
                continue
            hid, ps, n = resident[int(rng.integers(0, len(resident)))]
            m = size
            mp = min(n, (m * 9) // 10)
            mn = m - mp
            # members at the head or the tail of the set's window, non-members beside them
            q0 = ps - mn if rng.integers(0, 2) else ps + n - mp
            if head + m > ring:
                head = 0
            # the output region must be free: wait while the oldest pending query's
            # region overlaps it (regions are handed out in ring order, so when the
            # oldest one does not overlap, no newer one does)
            while pend_q:
                r0, st0, m0 = pend_q[0]
                if not pending[r0]:
                    pend_q.popleft()
                elif st0 < head + m and head < st0 + m0:
                    handle_completions()
                else:
                    break
            rid = srv.submit_query(hid, keys_pool[q0:q0 + m], qout[head:head + m])
            arrival[rid] = arr
            pending[rid] = True
            pend_q.append((rid, head, m))
            if len(samples) < 400 and rid % check_every == 0:
                samples.append((hid, q0, m, rid))
                is_sample[rid] = True
                qregion[rid] = (head, m)
                keep.add(hid)
            head += m
        if len(resident) > cap:
            for j, (hid, ps0, n0) in enumerate(resident):
                if hid not in keep:
                    resident.pop(j)
                    rid = srv.submit_release(hid)
                    arrival[rid] = time.monotonic_ns()
                    pending[rid] = True
                    break
        since_poll += 1
        if since_poll >= 256:  # keep completion batches small while the client runs flat out
            handle_completions()
            since_poll = 0
    submit_s = (time.monotonic_ns() - t0) / 1e9
    srv.drain(600)
    handle_completions()
    wall = (time.monotonic_ns() - t0) / 1e9
    st = srv.stats()
    kind = np.concatenate([p[0] for p in parts]) if parts else np.zeros(0, dtype=np.int64)
    lat = np.concatenate([p[1] for p in parts]) if parts else np.zeros(0, dtype=np.int64)
    lat_srv = np.concatenate([p[2] for p in parts]) if parts else np.zeros(0, dtype=np.int64)
    batch = np.concatenate([p[3] for p in parts]) if parts else np.zeros(0, dtype=np.int64)
    keys = np.concatenate([p[4] for p in parts]) if parts else np.zeros(0, dtype=np.int64)
    q, b = kind == 1, kind == 0
    # results in the mix equal the results alone (answered now, nothing else running)
    ok_q, n_q = True, 0
    for hid, q0, m, rid in samples:
        if outs.get(rid) is None:
            continue
        n_q += 1
        ok_q = ok_q and bool(torch.equal(srv.handle(hid).query(keys_pool[q0:q0 + m]), outs[rid]))
    ok_b, n_b = True, 0
    for hid, ps, n in checked_builds:
        h = phobic.phobic_build_ex(keys_pool[ps:ps + n], prm)
        ok_b = ok_b and (h.export() == srv.handle(hid).export())
        h.free()
        n_b += 1
    srv.close()
    del qout
    return {
        "requests": {"builds": int(b.sum()), "queries": int(q.sum()), "releases": int((kind == 2).sum())},
        "query_latency": _percentiles(lat[q]), "build_latency": _percentiles(lat[b]),
        "query_latency_from_submit": _percentiles(lat_srv[q]), "build_latency_from_submit": _percentiles(lat_srv[b]),
        "query_mkeys_s": float(keys[q].sum()) / wall / 1e6, "build_mkeys_s": float(keys[b].sum()) / wall / 1e6,
        "wall_s": wall, "submit_s": submit_s,
        "query_launches": st["query_launches"],
        "mean_requests_per_launch": float(batch[q].mean()) if q.any() else None,
        "max_requests_per_launch": st["max_batch_requests_seen"],
        "peak_accounted_gb": st["peak_accounted_bytes"] / 1e9,
        "builds_waited_for_memory": st["builds_waited_for_memory"],
        "check": {"queries_compared": n_q, "queries_equal_alone": ok_q, "builds_compared": n_b,
                  "builds_equal_alone": ok_b},
    }


def run_serve(a, phobic, workloads, torch):
    secs, brate, qrate, cap = a.serve_seconds, 40.0, 4000.0, 200
    trace = serve_trace(secs, brate, qrate, 77)
    keys_pool = workloads.stream_keys_torch(40_000_000_000, 1 << 28, 13, "cuda")
    torch.cuda.synchronize()
    cont = run_serve_mode(phobic, torch, trace, False, keys_pool, cap, 5)
    phobic.phobic_trim(0)
    ser = run_serve_mode(phobic, torch, trace, True, keys_pool, cap, 5)
    del keys_pool
    torch.cuda.empty_cache()
    phobic.phobic_trim(0)
    sweep = run_serve_sweep(phobic, torch, workloads, cap)
    return {"workload": SERVE.format(secs=secs, brate=brate, qrate=qrate, cap=cap),
            "offered": {"seconds": secs, "build_per_s": brate, "query_per_s": qrate,
                        "builds": sum(1 for e in trace if e[1] == 0), "queries": sum(1 for e in trace if e[1] == 1)},
            "continuous": cont, "serial": ser,
            "query_p99_speedup": (ser["query_latency"]["p99_ms"] / cont["query_latency"]["p99_ms"])
            if cont["query_latency"]["p99_ms"] else None,
            **sweep}


SERVE_SWEEP = ("offered-load sweep: {secs:g} s per point, builds (sizes log-uniform in [1e4, 5e6]) at 20/s and small "
               "query batches (sizes log-uniform in [1e3, 3e4], 90% members) at each offered rate, continuous "
               "batching against one request at a time; budget point: builds of 1e7-5e7 keys at 100/s under a "
               "4 GB HBM budget, so admission waits for memory")


def _point(r):
    return {"query_p50_ms": r["query_latency"]["p50_ms"], "query_p99_ms": r["query_latency"]["p99_ms"],
            "build_p50_ms": r["build_latency"]["p50_ms"], "build_p99_ms": r["build_latency"]["p99_ms"],
            "query_req_per_s": r["requests"]["queries"] / r["wall_s"], "query_mkeys_s": r["query_mkeys_s"],
            "build_mkeys_s": r["build_mkeys_s"], "mean_requests_per_launch": r["mean_requests_per_launch"],
            "submit_lag_s": r["submit_s"] - r["offered_s"], "builds_waited_for_memory": r["builds_waited_for_memory"],
            "peak_accounted_gb": r["peak_accounted_gb"],
            "equal_alone": r["check"]["queries_equal_alone"] and r["check"]["builds_equal_alone"]}


def run_serve_sweep(phobic, torch, workloads, cap, secs=6.0, rates=(2000, 8000, 32000, 64000, 128000)):
    """Throughput and p50/p99 per request type against offered query load, up
    to the rate the submitting thread sustains, continuous against serial; and
    one point where the HBM budget binds."""
    keys_pool = workloads.stream_keys_torch(80_000_000_000, 1 << 28, 14, "cuda")
    torch.cuda.synchronize()
    points = []
    for qr in rates:
        trace = serve_trace(secs, 20.0, qr, 100 + qr, build_sizes=(1e4, 5e6), query_sizes=(1e3, 3e4))
        pt = {"offered_query_per_s": qr}
        for mode, serial in (("continuous", False), ("serial", True)):
            r = run_serve_mode(phobic, torch, trace, serial, keys_pool, cap, 7, check_every=500)
            r["offered_s"] = secs
            pt[mode] = _point(r)
        points.append(pt)
    trace = serve_trace(secs, 100.0, 500.0, 9, build_sizes=(1e7, 5e7), query_sizes=(1e3, 1e5))
    budget = {"hbm_budget_gb": 4.0}
    for mode, serial in (("continuous", False), ("serial", True)):
        r = run_serve_mode(phobic, torch, trace, serial, keys_pool, cap, 8, check_every=50, budget=4 * 10**9)
        r["offered_s"] = secs
        budget[mode] = _point(r)
    del keys_pool
    phobic.phobic_trim(0)
    torch.cuda.empty_cache()
    return {"sweep_workload": SERVE_SWEEP.format(secs=secs), "sweep": points, "budget_point": budget}


def run_strings(a):
    """String-key configuration: build and query throughput of 2e8 strings."""
    import torch

    torch.cuda.set_device(0)
    from paper_2404_18497_b300 import build as libbuild

    libbuild.build()
    from paper_2404_18497_b300 import phobic, workloads

    w = workload(a)
    n = w["n"]
    data, off = workloads.random_strings(n, 3)
    dd = torch.from_numpy(data).cuda()
    do = torch.from_numpy(off.view(np.int64)).cuda()
    del data
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    prm = phobic.make_params(w["lam"], w["alpha"], w["P"], seed=0, encoder=w["encoder"], record_timings=True)
    stream = torch.cuda.current_stream()
    seed = 0
    for _ in range(a.warmup):
        while True:
            try:
                h = phobic.phobic_build_strings(dd, do, prm, stream)
                break
            except phobic.PhobicError as e:  # a 64-bit collision of two strings: take another seed
                if e.status != "DUP_HASH":
                    raise
                seed += 1
                prm.seed = seed
        phobic.phobic_query_strings(h, dd, do, out, stream)
        h.free()
    torch.cuda.synchronize()
    clk = Clocks(0)
    clk.start()
    l0 = phobic.phobic_kernel_launches()
    bms, qms, phases = [], [], []
    for _ in range(a.steps):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        h = phobic.phobic_build_strings(dd, do, prm, stream)
        e[1].record(stream)
        phobic.phobic_query_strings(h, dd, do, out, stream)
        e[2].record(stream)
        torch.cuda.synchronize()
        bms.append(e[0].elapsed_time(e[1]))
        qms.append(e[1].elapsed_time(e[2]))
        phases.append(phobic.phobic_get_timings(h))
        bpk = h.bits_per_key()
        h.free()
    clocks = clk.stop()
    launches = phobic.phobic_kernel_launches() - l0
    perm_ok = bool(torch.equal(torch.sort(out).values, torch.arange(n, device="cuda")))
    b_ms, q_ms = statistics.mean(bms), statistics.mean(qms)
    ph = {k: statistics.mean(p[k] for p in phases) for k in phases[0]}
    hbm, src = peaks()
    str_bytes = float(off[-1]) + 8.0 * (n + 1)
    print(json.dumps({
        "metric": METRIC, "value": n / (b_ms / 1e3) / 1e6, "unit": "Mkeys/s", "n_gpus": 1, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": b_ms + q_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8 strings -> u64", "data": "synthetic",
        "config": {"workload": w["name"], "n": n, "lambda": w["lam"], "alpha": w["alpha"], "P": w["P"],
                   "encoder": "IC-D", "bytes": int(off[-1]), "seed": seed,
                   "l2": "inputs larger than L2 (about 7.6e9 bytes of strings and offsets vs 126 MB L2)"},
        "build_ms": b_ms, "query_ms": q_ms, "query_mkeys_s": n / (q_ms / 1e3) / 1e6, "bits_per_key": bpk,
        "phase_ms": ph, "result_is_permutation": perm_ok, "clocks": clocks,
        "roofline": {"bound": "hbm", "kernel": "k_query_strings", "unit": "GB/s", "peak": hbm,
                     "achieved": (str_bytes + 8.0 * n) / (q_ms / 1e3) / 1e9,
                     "frac": (str_bytes + 8.0 * n) / (q_ms / 1e3) / 1e9 / hbm,
                     "algorithmic_bytes_per_launch": str_bytes + 8.0 * n, "peak_source": f"{src} hbm_gbs"},
        "e2e": None, "gpu_launches": launches, "gpu_launches_per_step": launches / a.steps, "cpu_baseline": None}))


def run_only(a):
    import torch

    torch.cuda.set_device(0)
    from paper_2404_18497_b300 import build as libbuild

    libbuild.build()
    from paper_2404_18497_b300 import phobic, workloads

    if a.only == "batch":
        print(json.dumps({"batch": run_batch(a, phobic, workloads, torch)}))
    elif a.only == "lambda":
        print(json.dumps({"lambda_sweep": run_lambda_sweep(a, phobic, workloads, torch)}))
    elif a.only == "ablation":
        print(json.dumps({"ablation": run_ablation(a, phobic, workloads, torch)}))
    elif a.only == "encoders":
        print(json.dumps({"encoders": run_encoders(a, phobic, workloads, torch)}))
    elif a.only == "table1":
        print(json.dumps({"table1": run_table1(a, phobic, workloads, torch)}))
    else:
        print(json.dumps({"serve": run_serve(a, phobic, workloads, torch)}))


def main():
    a = parse()
    if a.only and a.impl != "reference":
        return run_only(a)
    if a.strings and a.impl != "reference":
        return run_strings(a)
    if a.sharded and a.impl != "reference":
        return run_sharded(a)
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
