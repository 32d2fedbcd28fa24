#!/usr/bin/env python3
"""Benchmark: all-pairs minimax-path (APPD) matrix on GB300.

Default workload: one solve of a dense complete graph with n = 65536 vertices,
W = FP32 Euclidean distances of 16-D points from a 32-component Gaussian
mixture (means N(0, 25 I), sigma 1), seeded; W (17.2 GB) is generated on the
device and stays resident; each step writes the 17.2 GB matrix M.

Metric: APPD entries per second (n^2 / seconds per solve), whole job.
Prints one JSON line (rank 0).  Roofline bytes per solve: the fill writes
4 n^2; the round-1 minima read the upper triangle of W, 2 n (n - 1); the
level-0 contraction reads it again and writes and re-reads P, 16 c1^2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload big|n16384|n16384u32|n1000]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "big": dict(n=65536, kind="gmm16", desc="single solve n=65536, FP32 Euclidean distances of "
                                             "16-D points, 32-component Gaussian mixture"),
    "n16384": dict(n=16384, kind="uniform2", desc="single solve n=16384, FP32 Euclidean "
                                                   "distances of 2-D uniform points"),
    "n16384u32": dict(n=16384, kind="u32", desc="single solve n=16384, uint32 weights uniform "
                                                 "in [0, 2^16), heavy ties"),
    "n1000": dict(n=1000, kind="gmm2", desc="single solve n=1000, FP32 Euclidean distances of "
                                             "2-D points, 5-component Gaussian mixture"),
    "gmm16_16k": dict(n=16384, kind="gmm16", desc="single solve n=16384, FP32 Euclidean distances "
                                                   "of 16-D points, 32-component Gaussian mixture"),
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="big", choices=sorted(WORKLOADS))
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-batched", action="store_true")
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--no-insert", action="store_true")
    p.add_argument("--no-configs", action="store_true")
    p.add_argument("--no-points", action="store_true")
    p.add_argument("--no-wide", action="store_true")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def points_for(kind: str, n: int, seed_shift: int = 0):
    import synth
    if kind == "gmm16":
        return synth.gmm_points(n, 16, 32, sigma=1.0, seed=4 + seed_shift, mean_std=5.0)
    if kind == "uniform2":
        return synth.uniform_points(n, 2, seed=2 + seed_shift)
    if kind == "gmm2":
        return synth.gmm_points(n, 2, 5, sigma=0.5, seed=1 + seed_shift, mean_box=10.0)
    return None


def host_matrix(kind: str, n: int):
    import synth
    if kind == "u32":
        return synth.hash_u32(n, seed=3)
    return synth.euclid(points_for(kind, n))


# ------------------------------------------------------------ measurement
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [x.strip() for x in l.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def ncu_traffic(kernel: str):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, or
    None if there is none or the kernel's source changed since it was taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        ent = d[kernel]
        h = hashlib.sha256()
        for rel in ent["sources"]:
            h.update(open(os.path.join(ROOT, rel), "rb").read())
        h = h.hexdigest()[:16]
        if h != ent["source_sha256_16"]:
            return None
        return ent["bytes_per_launch_full"]
    except Exception:
        return None


def device_matrix(kind: str, n: int, dev, stream):
    """The workload's W generated on the device (same bytes as host_matrix)."""
    import torch

    import synth
    if kind == "u32":
        W = torch.empty((n, n), dtype=torch.int32, device=dev)
        synth.device_hash_u32(3, n, W.data_ptr(), stream.cuda_stream)
    else:
        pts = torch.from_numpy(points_for(kind, n)).to(dev)
        W = torch.empty((n, n), dtype=torch.float32, device=dev)
        synth.device_euclid(pts.data_ptr(), n, pts.shape[1], W.data_ptr(), stream.cuda_stream)
        del pts
    return W


def bench_configs(dev, peak: float, reps: int = 10):
    """The smaller single-solve configurations (n = 1000 GMM, n = 16384
    uniform FP32, n = 16384 uint32 ties): median device time of a solve over
    reps launches, entries/s, and the solve's W-read-plus-M-write bytes over
    that time as a fraction of the HBM peak.  At n = 16384 the Algorithm 4
    form (appd_solve_alg4: the paper's per-edge cross-block fill) is timed
    beside the tiled fill, phase by phase."""
    import torch

    from paper_2407_07058_gb300 import appd
    st = torch.cuda.current_stream()
    out = {}
    for name in ("n1000", "n16384", "n16384u32"):
        wl = WORKLOADS[name]
        n = wl["n"]
        W = device_matrix(wl["kind"], n, dev, st)
        M = torch.empty_like(W)
        for _ in range(3):
            appd.solve(W, out=M)
        torch.cuda.synchronize()
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            appd.solve(W, out=M)
            e1.record(st)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = statistics.median(times)
        ent = {"workload": wl["desc"], "ms": ms, "entries_per_s": n * n / (ms / 1e3),
               "hbm_frac_w_plus_m": 8.0 * n * n / (ms / 1e3) / 1e9 / peak,
               "l2": "W and M fit in L2" if 8 * n * n < 120e6 else "W and M larger than L2"}
        if name == "n16384":
            ph = {}
            for alg4 in (False, True):
                for _ in range(2):
                    appd.solve(W, out=M, alg4=alg4)
                torch.cuda.synchronize()
                appd.profile_begin()
                for _ in range(reps):
                    appd.solve(W, out=M, alg4=alg4)
                prof = appd.profile_end()
                ph["alg4" if alg4 else "tiled"] = {k: prof[k] / reps for k in appd.PHASES[:6]}
            ent["fill_ms_tiled"] = ph["tiled"]["fill"]
            ent["fill_ms_alg4_form"] = ph["alg4"]["fill"]
            ent["solve_ms_alg4_form"] = sum(ph["alg4"].values())
            ent["fill_gbs_tiled"] = 4.0 * n * n / (ph["tiled"]["fill"] / 1e3) / 1e9
            ent["fill_gbs_alg4_form"] = 4.0 * n * n / (ph["alg4"]["fill"] / 1e3) / 1e9
        if appd.last_device_status() != 0:
            raise RuntimeError(f"device status error in {name}")
        out[name] = ent
        del W, M
        torch.cuda.empty_cache()
    return out


def alu_peak_ops(dev) -> float:
    """FP32 lane operations per second at the maximum SM clock: SMs x 128
    FP32 lanes x clock (one add or one fused multiply-add per lane per cycle)."""
    import torch
    props = torch.cuda.get_device_properties(dev)
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f)["sm_max_mhz"])
    except Exception:
        mhz = 2070.0
    return props.multi_processor_count * 128 * mhz * 1e6


def bench_points(dev, peak: float, reps: int = 10):
    """The point-set solve (appd_solve_points: W computed where it is used,
    never stored): median device time per solve, phase times, the M write as
    a fraction of the HBM peak, and the two distance passes (round-1 minima
    and level-0 contraction, 2 d FP32 operations per pair and pass over the
    upper triangle) as a fraction of the FP32 ALU peak."""
    import torch

    import synth
    from paper_2407_07058_gb300 import appd
    st = torch.cuda.current_stream()
    alu = alu_peak_ops(dev)
    cases = [("gmm16_n65536", synth.cfg3_points(65536),
              "n=65536 16-D points, 32-component mixture (the n=65536 workload's points)"),
             ("uniform2_n65536", synth.uniform_points(65536, 2, seed=2),
              "n=65536 2-D points uniform in [0,1]^2"),
             ("uniform2_n16384", synth.cfg2a_points(),
              "n=16384 2-D points uniform in [0,1]^2 (the n=16384 workload's points)")]
    out = {}
    for name, X, desc in cases:
        n, d = X.shape
        T = torch.from_numpy(X).to(dev)
        M = torch.empty((n, n), dtype=torch.float32, device=dev)
        for _ in range(3):
            appd.solve_points(T, out=M)
        torch.cuda.synchronize()
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            appd.solve_points(T, out=M)
            e1.record(st)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        appd.profile_begin()
        for _ in range(reps):
            appd.solve_points(T, out=M)
        prof = appd.profile_end()
        if appd.last_device_status() != 0:
            raise RuntimeError(f"device status error in points {name}")
        ms = statistics.median(times)
        ph = {k: prof[k] / reps for k in appd.PHASES[:6]}
        pairs = n * (n - 1) / 2.0
        ops = 2.0 * d * pairs
        out[name] = {"workload": desc, "ms": ms, "entries_per_s": n * n / (ms / 1e3),
                     "phases_ms": ph,
                     "hbm_frac_m_write": (4.0 * n * n + 4.0 * n * d) / (ms / 1e3) / 1e9 / peak,
                     "rowmin_alu_frac": ops / (ph["rowmin"] / 1e3) / alu if ph["rowmin"] > 0 else None,
                     "contract0_alu_frac": ops / (ph["contract_w"] / 1e3) / alu if ph["contract_w"] > 0 else None,
                     "alu_peak_lane_ops_per_s": alu}
        del T, M
        torch.cuda.empty_cache()
    return out


def bench_wide(dev, peak: float, reps: int = 5, n: int = 92680):
    """A solve above 65536 vertices, near the largest the packed edges allow
    (92682; 92680 keeps rows 16-byte aligned): FP32 distances of 16-D
    mixture points, W and M 34.4 GB each; median device time per solve,
    phases, W-read-plus-M-write fraction."""
    import torch

    import synth
    from paper_2407_07058_gb300 import appd
    st = torch.cuda.current_stream()
    pts = torch.from_numpy(synth.gmm_points(n, 16, 32, sigma=1.0, seed=4, mean_std=5.0)).to(dev)
    W = torch.empty((n, n), dtype=torch.float32, device=dev)
    synth.device_euclid(pts.data_ptr(), n, 16, W.data_ptr(), st.cuda_stream)
    del pts
    M = torch.empty_like(W)
    for _ in range(2):
        appd.solve(W, out=M)
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        appd.solve(W, out=M)
        e1.record(st)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    appd.profile_begin()
    for _ in range(reps):
        appd.solve(W, out=M)
    prof = appd.profile_end()
    if appd.last_device_status() != 0:
        raise RuntimeError(f"device status error in the n={n} solve")
    ms = statistics.median(times)
    out = {"workload": f"single solve n={n}, FP32 Euclidean distances of 16-D points, "
                       "32-component Gaussian mixture (W and M 34.4 GB each)",
           "n": n, "ms": ms, "entries_per_s": n * n / (ms / 1e3),
           "hbm_frac_w_plus_m": 8.0 * n * n / (ms / 1e3) / 1e9 / peak,
           "phases_ms": {k: prof[k] / reps for k in appd.PHASES[:6]}, "c1": prof["c1"]}
    del W, M
    torch.cuda.empty_cache()
    return out


def cpu_baseline(kind: str, n_full: int, budget_s: float = 12.0):
    """The oracle (Prim + Algorithm 4, single thread) on a bounded sample of the
    same workload: a smaller graph from the same distribution."""
    import oracle
    import synth
    n = min(n_full, 16384 if kind != "u32" else 16384)
    if kind == "u32":
        W = synth.hash_u32(n, seed=3)
    else:
        W = synth.euclid(points_for(kind, n))
    runs, total = 0, 0.0
    while runs < 3 and (total < budget_s or runs == 0):
        t0 = time.perf_counter()
        oracle.appd(W)
        total += time.perf_counter() - t0
        runs += 1
    return {"value": runs * n * n / total, "unit": "entries/s", "cores": 1, "kind": "oracle",
            "sample": f"n={n} graph from the same distribution, {runs} run(s), "
                      f"{total:.1f} s total, Prim + Algorithm 4, one thread"}


def bench_batched(steps: int, warmup: int, dev, rank: int = 0, world: int = 1):
    """4096 graphs, n = floor(32 * 64^u) clipped to [32, 2048], FP32 uniform(0,1)
    weights seeded per graph: one batched call vs one plain solve per graph.
    With N ranks each solves its shard of the graphs (weak scaling by graphs)."""
    import torch

    import synth
    from paper_2407_07058_gb300 import appd, replicas
    all_sizes = [int(x) for x in synth.cfg4_sizes(4096)]
    mine = replicas.rank_graphs(all_sizes, rank, world)
    sizes = [all_sizes[g] for g in mine]
    offs = np.cumsum([0] + [n * n for n in sizes])[:-1].astype(np.int64)
    total = int(offs[-1] + sizes[-1] ** 2)
    W = torch.empty(total, dtype=torch.float32, device=dev)
    M = torch.empty_like(W)
    st = torch.cuda.current_stream()
    for k, g in enumerate(mine):
        synth.device_uniform01(synth.cfg4_seed(g), sizes[k], W.data_ptr() + 4 * int(offs[k]),
                               st.cuda_stream)
    torch.cuda.synchronize()
    # parameters searched on this GPU (cached beside the built library)
    tuning = appd.batched_autotune(os.path.join(os.path.dirname(appd.__file__), "_build",
                                                "tuning.jsonl"))
    for _ in range(max(1, warmup)):
        appd.solve_batched(W, offs, sizes, out=M)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    replicas.barrier()
    appd.profile_begin()
    e0.record(st)
    for _ in range(steps):
        appd.solve_batched(W, offs, sizes, out=M)
    e1.record(st)
    torch.cuda.synchronize()
    prof = appd.profile_end()
    replicas.barrier()
    ms_b = replicas.max_over_ranks(e0.elapsed_time(e1) / steps, dev)
    # one by one: 4096 plain solves on the same stream
    views = [(W[o: o + n * n].view(n, n), M[o: o + n * n].view(n, n)) for o, n in zip(offs, sizes)]
    for w, m in views[:64]:
        appd.solve(w, out=m)
    torch.cuda.synchronize()
    e0.record(st)
    for w, m in views:
        appd.solve(w, out=m)
    e1.record(st)
    torch.cuda.synchronize()
    ms_1 = replicas.max_over_ranks(e0.elapsed_time(e1), dev)
    if appd.last_device_status() != 0:
        raise RuntimeError("device status error in the batched run")
    ent = float(sum(n * n for n in all_sizes))
    G = len(all_sizes)
    return {"workload": "4096 graphs, n log-uniform in [32, 2048], FP32 uniform(0,1) weights",
            "graphs": G, "graphs_per_rank": len(sizes), "ms_per_batch": ms_b,
            "graphs_per_s": G / (ms_b / 1e3), "entries_per_s": ent / (ms_b / 1e3),
            "one_by_one_ms": ms_1, "one_by_one_graphs_per_s": G / (ms_1 / 1e3),
            "speedup_vs_one_by_one": ms_1 / ms_b, "kernel_launches_per_batch": prof["launches"] / steps,
            "bytes_w_plus_m": 8.0 * ent, "tuning": tuning}


def serving_requests(count: int, seed: int = 5):
    """n = floor(64 * 128^u) (log-uniform in [64, 8192]), dtype Bernoulli(1/2)."""
    rng = np.random.default_rng(seed)
    u = rng.random(count)
    ns = np.clip(np.floor(64.0 * np.power(128.0, u)).astype(np.int64), 64, 8192)
    dts = (rng.random(count) < 0.5).astype(np.int64)   # 1 = uint32, 0 = FP32 mixture
    return ns, dts


class ServingInputs:
    """Inputs of the serving mix, staged on the device before any timing.

    Request k has n = ns[k] vertices; an FP32 request carries a 2-D point set
    (5-component mixture, means uniform in [0, 10]^2, sigma 0.5, seeded by
    seed * 1000003 + k) whose distances are computed in FP32 arithmetic when
    the request is generated; a uint32 request carries hashed weights in
    [0, 2^16) with that seed.  Generation writes W into the request's slot
    on the device (one launch per admission group)."""

    def __init__(self, ns, dts, dev, seed: int = 5):
        import torch

        import synth
        self.ns = np.asarray(ns, dtype=np.int64)
        self.dts = np.asarray(dts, dtype=np.int64)
        self.seeds = (seed * 1000003 + np.arange(len(ns))).astype(np.uint64)
        self.pts_host = {}
        off = np.zeros(len(ns), dtype=np.int64)
        chunks, acc = [], 0
        for k in np.nonzero(self.dts == 0)[0]:
            p = synth.gmm_points(int(self.ns[k]), 2, 5, sigma=0.5, seed=int(self.seeds[k]),
                                 mean_box=10.0)
            self.pts_host[int(k)] = p
            off[k] = acc
            chunks.append(p.reshape(-1))
            acc += p.size
        flat = np.concatenate(chunks) if chunks else np.zeros(2, np.float32)
        self.pts_dev = torch.from_numpy(flat).to(dev)
        base = self.pts_dev.data_ptr()
        self.pts_ptr = np.where(self.dts == 0, base + 4 * off, 0).astype(np.uint64)

    def descs(self, idx, slots):
        import synth
        idx = np.asarray(idx, dtype=np.int64)
        return synth.request_descs(slots, self.pts_ptr[idx], self.ns[idx], self.dts[idx],
                                   self.seeds[idx], d=2)

    def host_matrix(self, k: int) -> np.ndarray:
        """Request k's W on the host, from the host twin of the generator."""
        import synth
        if self.dts[k]:
            return synth.hash_u32(int(self.ns[k]), seed=int(self.seeds[k]))
        return synth.euclid32(self.pts_host[int(k)])


def _upload(desc, dev):
    import torch
    return torch.from_numpy(desc.view(np.uint8)).to(dev, non_blocking=True)


def run_serving(sv, inp, idx, arrivals, dev, on_done=None):
    """Drives the server with the requests idx (arrival times `arrivals`, s,
    relative, ascending): arrived requests are admitted in order as the
    budget allows (one submit call for every request that fits), their W
    generated into the slots by one device launch, and the group committed
    with one call (the solves wait for the generation on the device);
    completions are polled and released in groups.  on_done(k, M_ptr), if
    given, runs before request k is released.  Returns per-request latency
    (arrival -> completion seen), host time to enqueue each group's ingress
    per request, and the wall time."""
    import torch

    import synth
    from paper_2407_07058_gb300 import appd
    idx = np.asarray(idx, dtype=np.int64)
    N = len(idx)
    st = torch.cuda.current_stream()
    lat = np.zeros(N)
    ingress = []
    owner = {}
    keep = []          # descriptor uploads in flight (stream-ordered reuse)
    arrived = head = done = 0
    t0 = time.perf_counter()
    while done < N:
        now = time.perf_counter() - t0
        while arrived < N and arrivals[arrived] <= now:
            arrived += 1
        progressed = False
        if head < arrived:
            sel = idx[head:arrived]
            ids, slots = sv.submit_many(inp.ns[sel], inp.dts[sel], st)
            k = len(ids)
            if k:
                tg = time.perf_counter()
                desc, tiles = inp.descs(sel[:k], slots)
                d_dev = _upload(desc, dev)
                synth.device_requests(d_dev.data_ptr(), k, tiles, st.cuda_stream)
                keep.append(d_dev)
                sv.commit_many(ids, st)
                ingress.append((time.perf_counter() - tg) / k)
                owner.update(zip(ids.tolist(), range(head, head + k)))
                head += k
                progressed = True
                if len(keep) > 64:
                    keep = keep[-8:]
        ids, ptrs = sv.poll_arrays(4096)
        if len(ids):
            tdone = time.perf_counter() - t0
            for rid, ptr in zip(ids.tolist(), ptrs.tolist()):
                j = owner.pop(rid)
                lat[j] = tdone - arrivals[j]
                if on_done is not None:
                    on_done(int(idx[j]), ptr)
            sv.release_many(ids, st)
            done += len(ids)
            progressed = True
        if not progressed:
            time.sleep(0.00005)
    torch.cuda.synchronize()
    return lat, np.array(ingress), time.perf_counter() - t0


def one_by_one(inp, idx, dev):
    """The same requests one at a time: generate W, then one plain appd_solve,
    on one stream.  Returns (wall seconds, device seconds)."""
    import torch

    import synth
    from paper_2407_07058_gb300 import appd
    idx = np.asarray(idx, dtype=np.int64)
    nmax = int(inp.ns[idx].max())
    Wb = torch.empty(nmax * nmax, dtype=torch.float32, device=dev)
    Mb = torch.empty_like(Wb)
    desc, _ = inp.descs(idx, np.full(len(idx), Wb.data_ptr(), dtype=np.uint64))
    tiles = (inp.ns[idx] ** 2 + synth.REQ_TILE - 1) // synth.REQ_TILE
    desc["tile0"] = 0
    d_dev = _upload(desc, dev)
    st = torch.cuda.current_stream()

    def run(ks):
        for q in ks:
            n = int(inp.ns[idx[q]])
            synth.device_requests(d_dev.data_ptr() + desc.itemsize * q, 1, int(tiles[q]), st.cuda_stream)
            w = Wb[: n * n].view(n, n)
            m = Mb[: n * n].view(n, n)
            if inp.dts[idx[q]]:
                w, m = w.view(torch.int32), m.view(torch.int32)
            appd.solve(w, out=m)

    run(range(min(64, len(idx))))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(st)
    run(range(len(idx)))
    e1.record(st)
    torch.cuda.synchronize()
    return time.perf_counter() - t0, e0.elapsed_time(e1) / 1e3


def bench_serving(dev, count: int = 20000):
    """Continuous batching under a 40 GB budget, at two size cut-overs of the
    server's batched path: graphs up to 2048 vertices one per CTA and larger
    ones on the whole GPU (latency-oriented), or every graph of the mix one per
    CTA (capacity-oriented).  For each: capacity at saturation and Poisson
    arrivals at fractions of it (graphs/s, p50/p99 latency); the same
    requests one at a time with plain solves for comparison."""
    from paper_2407_07058_gb300 import appd
    budget = 40 << 30
    ns, dts = serving_requests(count)
    inp = ServingInputs(ns, dts, dev)
    m = min(count, 4000)
    wall1, dev1 = one_by_one(inp, np.arange(m), dev)
    base = appd.get_batched_tuning()
    out = {"workload": f"{count} requests, n log-uniform in [64, 8192), half FP32 2-D "
                       "mixture distances (FP32 arithmetic), half uint32 uniform [0, 2^16); "
                       "40 GB budget",
           "capacity_requests": m,
           "one_by_one_graphs_per_s": m / wall1,
           "one_by_one_device_graphs_per_s": m / dev1}
    rng = np.random.default_rng(55)
    try:
        for mode, n_split, fracs in (("latency_mode", 2048, (0.5, 0.8)), ("capacity_mode", 8192, (0.5,))):
            appd.batched_tuning(base["ctas_per_sm"], base["fill_rows"], n_split)
            sv = appd.Server(budget, 8192)
            try:
                # warm-up, then capacity: a saturating burst (all arrive at t = 0)
                run_serving(sv, inp, np.arange(300), np.zeros(300), dev)
                _, _, wall = run_serving(sv, inp, np.arange(m), np.zeros(m), dev)
                cap = m / wall
                res = {"n_split": n_split, "capacity_graphs_per_s": cap,
                       "served_vs_one_by_one": cap / (m / wall1), "rates": []}
                for frac in fracs:
                    lam = frac * cap
                    arr = np.cumsum(rng.exponential(1.0 / lam, size=count))
                    lat, ing, wall = run_serving(sv, inp, np.arange(count), arr, dev)
                    res["rates"].append({"rate_frac_of_capacity": frac, "rate_per_s": lam,
                                         "graphs_per_s": count / wall,
                                         "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                                         "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                                         "max_ms": 1e3 * float(lat.max()),
                                         "ingress_host_p50_ms": 1e3 * float(np.percentile(ing, 50))})
                out[mode] = res
            finally:
                sv.close()
    finally:
        appd.batched_tuning(base["ctas_per_sm"], base["fill_rows"], base["n_split"])
    return out


# ------------------------------------------------------------------ arms
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    wl = WORKLOADS[args.workload]
    import oracle
    import synth
    n = min(wl["n"], 8192)
    if wl["kind"] == "u32":
        W = synth.hash_u32(n, seed=3)
    else:
        W = synth.euclid(points_for(wl["kind"], n))
    for _ in range(args.warmup):
        oracle.appd(W)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.appd(W)
    dt = time.perf_counter() - t0
    value = args.steps * n * n / dt
    line = {
        "impl": "reference", "metric": "APPD entries/s", "value": value, "unit": "entries/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32 order keys" + (" (FP32 input)" if wl["kind"] != "u32" else ""),
        "data": "synthetic",
        "config": {"workload": wl["desc"], "n": wl["n"], "sample_n": n},
        "cpu_baseline": {"value": value, "unit": "entries/s", "cores": 1, "kind": "oracle",
                         "sample": f"each step: the oracle on an n={n} graph from the same "
                                   "distribution (Prim + Algorithm 4, one thread)"},
        "e2e": {"value": value, "unit": "entries/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, rank, world, local):
    import torch
    import torch.distributed as dist

    import synth
    from paper_2407_07058_gb300 import appd, replicas

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl", device_id=dev)

    barrier = replicas.barrier

    wl = WORKLOADS[args.workload]
    n, kind = wl["n"], wl["kind"]
    stream = torch.cuda.current_stream()
    # ---- inputs resident on the device
    W = device_matrix(kind, n, dev, stream)
    M = torch.empty_like(W)
    torch.cuda.synchronize()

    for _ in range(args.warmup):
        appd.solve(W, out=M)
    torch.cuda.synchronize()
    if appd.last_device_status() != 0:
        raise RuntimeError("device status error during warm-up")

    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        appd.profile_begin()
        ev0.record(stream)
        for _ in range(args.steps):
            appd.solve(W, out=M)
        ev1.record(stream)
        torch.cuda.synchronize()
        prof = appd.profile_end()
    barrier()
    ms = ev0.elapsed_time(ev1)
    if appd.last_device_status() != 0:
        raise RuntimeError("device status error in the timed region")
    ms = replicas.max_over_ranks(ms, dev)
    ms_step = ms / args.steps
    value = world * args.steps * n * n / (ms / 1e3)

    # ---- roofline of the dominant kernel (algorithmic bytes per launch)
    peak, peak_src = measured_peaks()
    c1 = prof["c1"]
    # algorithmic bytes per launch: the round-1 minima and the level-0
    # contraction read the upper triangle of W (2 n (n-1) bytes), the latter
    # writes P (8 c1^2) whose column minima are read back (8 c1^2); the fill
    # writes M (4 n^2)
    tri = 2.0 * n * (n - 1)
    cand = {
        "k_fill": (prof["fill"], 4.0 * n * n),
        "k_contract_tma+k_colmin_p": (prof["contract_w"], tri + 16.0 * c1 * c1),
        "k_rowmin_sym": (prof["rowmin"], tri),
    }
    dom = max(cand, key=lambda k: cand[k][0])
    dom_ms = cand[dom][0] / args.steps
    achieved = cand[dom][1] / (dom_ms / 1e3) / 1e9 if dom_ms > 0 else None
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                "peak_source": peak_src, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None,
                # the stored counters are scaled to one launch of the n = 65536
                # mixture solve; other workloads have no capture of their own
                "traffic": ncu_traffic(dom) if (args.workload == "big") else None,
                "algorithmic_bytes_per_launch": cand[dom][1], "ms_per_launch": dom_ms}
    # solve-level fractions with fixed numerators: the design count (28/3) n^2
    # and the algorithmic minimum 4 n (n-1) / 2 + 4 n^2 (read each edge once,
    # write M); moving more bytes cannot raise either
    design_bytes = (28.0 / 3.0) * n * n
    min_bytes = 2.0 * n * (n - 1) + 4.0 * n * n
    solve_frac = design_bytes / (ms_step / 1e3) / 1e9 / peak
    min_frac = min_bytes / (ms_step / 1e3) / 1e9 / peak
    # the solve's own input and output: all of W read once, all of M written
    wm_frac = 8.0 * n * n / (ms_step / 1e3) / 1e9 / peak

    # ---- warm start: insert one vertex into the solved matrix (Section 6.1)
    insert = None
    if not args.no_insert:
        w_new = W[1].clone()                      # the new vertex's weights (a copy of vertex 1's row)
        Mo = torch.empty((n + 1, n + 1), dtype=W.dtype, device=dev)
        for _ in range(2):
            appd.insert_vertex(M, w_new, out=Mo)
        torch.cuda.synchronize()
        ki = 5
        ev0.record(stream)
        for _ in range(ki):
            appd.insert_vertex(M, w_new, out=Mo)
        ev1.record(stream)
        torch.cuda.synchronize()
        if appd.last_device_status() != 0:
            raise RuntimeError("device status error in the insertion run")
        ms_i = ev0.elapsed_time(ev1) / ki
        ib = 8.0 * n * n + 4.0 * (n + 1) * (n + 1)   # M read twice, M' written
        # the same insertion through the tree (appd_insert_vertex_tree): the
        # new tree from G's tree and the star of p, leaf order, one fill
        tree = appd.mst_edges(W)
        for _ in range(2):
            appd.insert_vertex_tree(tree, w_new, n, W.dtype, out=Mo, tree_out=False)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(ki):
            appd.insert_vertex_tree(tree, w_new, n, W.dtype, out=Mo, tree_out=False)
        ev1.record(stream)
        torch.cuda.synchronize()
        if appd.last_device_status() != 0:
            raise RuntimeError("device status error in the tree insertion run")
        ms_t = ev0.elapsed_time(ev1) / ki
        tb = 4.0 * (n + 1) * (n + 1)   # M' written; the tree work is O(n log n)
        insert = {"workload": f"insert one vertex into the solved n={n} graph",
                  "tree_update": {"api": "appd_insert_vertex_tree (G's tree + p's edges -> "
                                         "new tree, leaf order, one fill)",
                                  "ms": ms_t, "entries_per_s": (n + 1) * (n + 1) / (ms_t / 1e3),
                                  "algorithmic_bytes": tb, "achieved_gbs": tb / (ms_t / 1e3) / 1e9,
                                  "frac_of_peak": tb / (ms_t / 1e3) / 1e9 / peak},
                  "from_matrix": {"api": "appd_insert_vertex (two passes over M, M' written)",
                                  "ms": ms_i, "entries_per_s": (n + 1) * (n + 1) / (ms_i / 1e3),
                                  "algorithmic_bytes": ib, "achieved_gbs": ib / (ms_i / 1e3) / 1e9,
                                  "frac_of_peak": ib / (ms_i / 1e3) / 1e9 / peak},
                  "solve_from_scratch_ms": ms_step}
        del Mo, w_new, tree
        torch.cuda.empty_cache()

    # ---- end to end through the host entry point (pinned buffers)
    e2e = None
    if not args.no_e2e:
        Wh = torch.empty((n, n), dtype=W.dtype, pin_memory=True)
        Wh.copy_(W)
        Mh = torch.empty((n, n), dtype=W.dtype, pin_memory=True)
        dt_code = appd.F32 if W.dtype == torch.float32 else appd.U32
        # results alternate between two pinned buffers, so that consecutive
        # pipelined calls never write the same host memory
        Mh2 = torch.empty((n, n), dtype=W.dtype, pin_memory=True)
        appd.solve_host_async_ptr(Wh.data_ptr(), n, dt_code, Mh.data_ptr())   # warm staging
        appd.solve_host_async_ptr(Wh.data_ptr(), n, dt_code, Mh2.data_ptr())
        appd.solve_host_wait()
        torch.cuda.synchronize()
        barrier()
        ke = max(2, min(args.steps, 10))
        t0 = time.perf_counter()
        for k in range(ke):
            appd.solve_host_async_ptr(Wh.data_ptr(), n, dt_code, (Mh if k % 2 == 0 else Mh2).data_ptr())
        appd.solve_host_wait()
        torch.cuda.current_stream().synchronize()
        te = replicas.max_over_ranks(time.perf_counter() - t0, dev)
        barrier()
        if appd.last_device_status() != 0:
            raise RuntimeError("device status error in the end-to-end run")
        e2e = {"value": world * ke * n * n / te, "unit": "entries/s",
               "h2d_bytes_per_step": 4 * n * n, "d2h_bytes_per_step": 4 * n * n,
               "steps": ke, "ms_per_step": 1e3 * te / ke,
               "api": "appd_solve_host_async (pinned host buffers, calls pipelined)"}
        del Wh, Mh, Mh2

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(kind, n)
    configs = None
    if not args.no_configs:
        del W, M
        torch.cuda.empty_cache()
        configs = bench_configs(dev, peak)
    points = None
    if not args.no_points:
        W = M = None
        torch.cuda.empty_cache()
        points = bench_points(dev, peak)
    wide = None
    if not args.no_wide:
        W = M = None
        torch.cuda.empty_cache()
        wide = bench_wide(dev, peak)
    batched = None
    if not args.no_batched:
        W = M = None
        torch.cuda.empty_cache()
        batched = bench_batched(max(3, min(args.steps, 10)), args.warmup, dev, rank, world)
    serving = None
    if not args.no_serving:
        torch.cuda.empty_cache()
        serving = bench_serving(dev)

    if rank == 0:
        line = {
            "metric": "APPD entries/s", "value": value, "unit": "entries/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32 order keys" + (" (FP32 input)" if kind != "u32" else ""),
            "data": "synthetic",
            "config": {"workload": wl["desc"], "n": n, "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (W and M 4n^2 bytes each)"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": prof["launches"],
            "clocks": clk.summary(),
            "phases_ms_per_step": {k: prof[k] / args.steps for k in appd.PHASES},
            "c1": c1,
            "hbm_frac_solve_design_bytes": solve_frac,
            "hbm_frac_solve_min_bytes": min_frac, "hbm_frac_solve_w_plus_m": wm_frac,
            "insert": insert,
            "configs": configs,
            "points": points,
            "wide": wide,
            "batched": batched,
            "serving": serving,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
