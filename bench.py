"""K-truss benchmark: Medges/s at fixed K on one GB300 (JSON line on stdout).

Workload (default): R-MAT scale 23, edge factor 16, (a,b,c,d) = (.57,.19,.19,.05),
symmetrised, de-duplicated, with 64 planted cliques of 20..200 vertices,
upper-triangular int32 CSR with original vertex ids, seed 0; K = 3.  A step is
one whole K-truss computation (every peel round: support, prune, compaction,
convergence test, final outputs) of that graph.

  value     = edges / device time of ktruss_run, graph resident in HBM
  e2e       = the same metric through the public C ABI with host buffers:
              ktruss_load_csr from pinned host memory + ktruss_run with pinned
              host outputs + ktruss_free, all inside the timed region
  roofline  = the support kernel (dominant) against measured HBM bandwidth.
              achieved = the bytes the kernel's design moves per launch
              (counted on the host from the CSR: probe reads, staged-row
              reads, credits, segment records) / its CUDA-event time; the
              merge accounting 4*W + 8*m + 16*T + 8*(n+1) (W = sum over live
              edges of tail + row-kappa lengths) is reported beside it.
              `bound` names what the committed ncu capture of the kernel says
              limits it (DRAM, L2 or SM instruction issue)
  cpu_baseline = the CPU oracle, single thread, on a bounded sample

Between timed steps L2 is flushed by writing a buffer larger than L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload rmat23c|rmat20|rmat20r|er2000] [--K 3]
                  [--kernel auto|balanced|edge|coarse]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "K-truss Medges/s at fixed K on 1 GB300"
UNIT = "Medges/s"
WORKLOAD_DESC = {
    "rmat20": "RMAT scale 20, edge factor 16, a=.57 b=.19 c=.19 d=.05, original ids, seed 0",
    "rmat20r": "RMAT scale 20, edge factor 16, degree-ascending relabel, seed 0",
    "rmat23c": "RMAT scale 23, edge factor 16, 64 planted cliques 20..200, seed 0",
    "er2000": "Erdos-Renyi G(n=2000, m=16000), seed 0",
}
CPU_SAMPLE_SCALE = 17  # oracle sample: R-MAT scale 17, same recipe, full K-truss run
L2_FLUSH_BYTES = 512 << 20
UPDATE_MODES = {"never": 0, "always": 1, "auto": 2}  # KTRUSS_UPDATE_*


_T0 = time.perf_counter()


def progress(msg):
    """One line per phase on stderr (the JSON line alone goes to stdout)."""
    print(f"[bench {time.perf_counter() - _T0:8.1f}s] {msg}", file=sys.stderr, flush=True)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None
        self.first = threading.Event()
        self.t_start = 0.0
        self.t_end = float("inf")

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # nvidia-smi takes a moment to start: let its first sample arrive
            # before the timed region begins, so that the region is sampled
            self.first.wait(timeout=2.0)
        except OSError:
            self.proc = None
        self.t_start = time.perf_counter()
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))
            self.first.set()

    def __exit__(self, *a):
        self.t_end = time.perf_counter()
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        """Median SM clock, maximum clock and throttle reasons of the samples
        taken inside the timed region (the last earlier sample when the region
        was too short to hold one)."""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        inside = [ln for t, ln in self.lines if self.t_start <= t <= self.t_end]
        if not inside:
            inside = [ln for t, ln in self.lines if t < self.t_start][-1:]
        for ln in inside:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, device=None) -> float:
    """Maximum of x over all ranks of the default process group (x itself
    without one).  Each rank runs an independent replica of the whole
    K-truss computation, so this is the only collective: timing."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def algorithmic_bytes(n, live, merge, tris):
    """The merge accounting of a support step: both lists of every task read
    once (4*W), S zeroed and the owner written (8 per live edge), two credit
    RMWs per triangle, row_ptr."""
    return 4 * merge + 8 * live + 16 * tris + 8 * (n + 1)


def support_work(row_ptr, col, light=64):
    """Work of the first support step of a CSR, counted on the host.

    For the task of edge e = (i, kappa) at slot e: t = tail length of row i
    after e, d = length of row kappa.  W = sum of (t + d) over all edges (the
    merge work the library reports as merge_work).  Tasks with t + d <= light
    are merged by one thread; every other task with min(t, d) > 0 is a segment
    that stages the longer list (row kappa if t < d, else row i) and probes it
    with min(t, d) items.  Returns W, probes (items), staged (total length of
    the distinct staged rows), segments and active_rows (distinct staged
    rows)."""
    import numpy as np
    rp = np.asarray(row_ptr, dtype=np.int64)
    c = np.asarray(col, dtype=np.int64)
    n, m = rp.shape[0] - 1, c.shape[0]
    deg = np.diff(rp)
    row = np.repeat(np.arange(n, dtype=np.int64), deg)
    t = rp[row + 1] - np.arange(m, dtype=np.int64) - 1
    d = deg[c]
    W = int(t.sum() + d.sum())
    short = np.minimum(t, d)
    heavy = (t + d > light) & (short > 0)
    staged = np.zeros(max(n, 1), dtype=bool)
    staged[np.where(t < d, c, row)[heavy]] = True
    return {"W": W, "probes": int(short[heavy].sum()), "staged": int(deg[staged[:n]].sum()),
            "segments": int(heavy.sum()), "active_rows": int(staged.sum())}


def design_bytes(work, tris):
    """Bytes the support kernel's design moves in one launch: 4 per probe
    read, 12 per staged column (read once, plus the read-modify-write that
    flushes its credits), 8 per triangle (the credit RMW at the probe
    position), 28 per segment (its records: owner, probe start, active-row
    rank, item prefix, and the owner's credit RMW), 16 per active staged row
    (row pointers, active-row tables)."""
    return (4 * work["probes"] + 12 * work["staged"] + 8 * tris + 28 * work["segments"]
            + 16 * work["active_rows"])


KERNEL_SOURCES = ("support_balanced.cu", "support_shape.cuh")


def kernel_source_sha256(root=None) -> str:
    """SHA-256 over the support kernel's source files (in a fixed order)."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        p = os.path.join(root or ROOT, "paper_2009_07929_gb300", "csrc", name)
        with open(p, "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()


def traffic_record(workload, K):
    """The committed ncu record of the support kernel for this workload and K
    (profiles/support_traffic.json: a list of captures).  Returns (record,
    fresh): fresh is False when the kernel source changed since the capture,
    in which case its counters no longer describe the kernel and are not
    reported."""
    p = os.path.join(ROOT, "profiles", "support_traffic.json")
    try:
        with open(p) as f:
            recs = json.load(f)
    except (OSError, ValueError):
        return None, False
    if isinstance(recs, dict):
        recs = [recs]
    h = kernel_source_sha256()
    for rec in recs:
        if rec.get("workload") == f"{workload} K={K} round 1":
            return rec, rec.get("source_sha256") == h
    return None, False


def host_cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the record
    beside the oracle's timing."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=5).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine() or "unknown"


def cpu_baseline(seconds_cap=30.0, scale=CPU_SAMPLE_SCALE):
    import graphgen as gg
    import oracle
    g = gg.rmat(scale, 16, 0)
    runs, t0 = 0, time.perf_counter()
    while True:
        oracle.ktruss(g.row_ptr, g.col, 3)
        runs += 1
        el = time.perf_counter() - t0
        if el > seconds_cap / 3 or runs >= 3:
            break
    return {"value": round(g.m * runs / el / 1e6, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
            "cpu_model": host_cpu_model(), "host_cores": os.cpu_count(),
            "sample": f"full K=3 run of the single-thread C oracle on R-MAT scale {scale}, "
                      f"edge factor 16 (same recipe, {g.m} edges), {runs} run(s), "
                      f"{el:.1f} s on {os.cpu_count()} host cores (1 used)"}


def cpu_f_baseline(K=3, name="rmat20"):
    """The paper's fine-grained CPU design (oracle/cpu_f.c: per-edge tasks,
    atomic supports, zero-terminated rows; OpenMP) timed once on all host
    cores on the R-MAT-20 workload, next to the GPU's number for the same
    graph."""
    import graphgen as gg
    import oracle
    try:
        oracle.build_cpu_f()
    except Exception as e:  # no OpenMP compiler on this host
        return {"unavailable": f"cpu_f.c did not build: {str(e)[:160]}"}
    g = gg.cached_workload(name, 0)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    r = oracle.cpu_f_ktruss(g.row_ptr, g.col, K, cores)
    el = time.perf_counter() - t0
    return {"value": round(g.m / el / 1e6, 4), "unit": UNIT, "cores": cores,
            "kind": "cpu_f (the paper's fine-grained CPU design, OpenMP)",
            "cpu_model": host_cpu_model(),
            "sample": f"one full K={K} run ({r.rounds} rounds) on {WORKLOAD_DESC[name]} "
                      f"({g.m} edges), {el:.1f} s on {cores} threads"}


def measure_workload(kt, gg, name, K, steps, flush):
    """Medges/s of ktruss_run (K, graph resident in HBM, L2 flushed between
    steps, CUDA events) and the time of its K_max sweep (ktruss_decompose) on
    another workload, for comparison with the headline one."""
    import torch
    progress(f"extra workload {name}")
    g = gg.cached_workload(name, 0)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    h = kt.load(torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col).to(dev))
    mask = torch.empty(g.m, dtype=torch.uint8, device=dev)
    sup = torch.empty(g.m, dtype=torch.int32, device=dev)
    for _ in range(3):
        flush.fill_(1)
        h.run(K, out=(mask, sup))
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    sup1 = 0.0
    for i in range(steps):
        flush.fill_(i)
        ev[i][0].record(stream)
        h.run(K, out=(mask, sup))
        ev[i][1].record(stream)
        sup1 += h.stats().ms_support_per_round[0]
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    h.decompose()
    torch.cuda.synchronize()
    d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.fill_(7)
    d0.record(stream)
    _, kmax = h.decompose()
    d1.record(stream)
    torch.cuda.synchronize()
    st = h.stats()
    h.close()
    return {"workload": WORKLOAD_DESC[name] + f", K={K}", "n": g.n, "m": g.m,
            "value": round(g.m * steps / (ms / 1e3) / 1e6, 2), "unit": UNIT,
            "ms_per_step": round(ms / steps, 4), "support_ms_round1": round(sup1 / steps, 4),
            "kmax_sweep": {"kmax": kmax, "ms": round(d0.elapsed_time(d1), 3),
                           "rounds": st.rounds, "support_steps": st.support_launches}}


def measure_batched(kt, gg, count, m_hi, seed=0, autotune=True):
    """Batched graphs/s against the plain path on the batching workload
    (graphgen.batch_config: sizes log-uniform in [1e3, m_hi] edges, half G(n,m)
    with degree 8..64, half R-MAT scale 10..17, K uniform in 3..12).  Plain:
    every graph preloaded into its own handle, then one ktruss_run per graph.
    Batched: the block-diagonal batch preloaded into one handle, then one
    ktruss_run_batch.  Both timed with CUDA events, graphs resident in HBM.
    The plain arm runs with the library's defaults (what a caller running one
    graph at a time gets); with autotune, ktruss_autotune picks the batch
    arm's settings on the batch first (settings tuned for one batch of 4096
    graphs are not the best ones for each graph alone: a per-edge/balanced
    threshold tuned on the batch slowed the plain arm by a third)."""
    import torch
    progress(f"batched: generating {count} graphs, m up to {m_hi:g}")
    batch = gg.batch_config(count, seed=seed, m_lo=1e3, m_hi=m_hi)
    graphs = [b[0] for b in batch]
    Ks = [b[1] for b in batch]
    edges = sum(g.m for g in graphs)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    vo, rp, col, eo = kt.concat_graphs(graphs)
    tune = None
    if autotune:
        # the library's autotuner picks the support kernel's CTA shape, the
        # merge/probe threshold, the per-edge/balanced threshold and the
        # update rule on the batch, for the batch arm
        progress("batched: autotuning on the batch")
        hb = kt.load_batch(vertex_offsets=vo, row_ptr=torch.from_numpy(rp).to(dev),
                           col=torch.from_numpy(col).to(dev))
        tune = hb.autotune(Ks, reps=1)
        hb.close()

    def apply(h):
        if tune is not None:
            h.set_support_shape(tune["support_shape"])
            h.set_option(kt.OPT_LIGHT_MERGE, tune["light_merge"])
            h.set_option(kt.OPT_SMALL_EDGES, tune["small_edges"])
            h.set_update(tune["update_mode"])
        return h

    progress(f"batched: {edges} edges generated; loading plain handles")
    # plain
    handles = [kt.load(torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col).to(dev))
               for g in graphs]
    outs = [(torch.empty(max(g.m, 1), dtype=torch.uint8, device=dev)[:g.m],
             torch.empty(max(g.m, 1), dtype=torch.int32, device=dev)[:g.m]) for g in graphs]
    progress("batched: plain warm-up")
    for h, K, o in zip(handles, Ks, outs):
        h.run(K, out=o)
    torch.cuda.synchronize()
    progress("batched: plain timed")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for h, K, o in zip(handles, Ks, outs):
        h.run(K, out=o)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1)
    for h in handles:
        h.close()
    progress(f"batched: plain {plain_ms:.1f} ms; loading the batch")
    # batched
    hb = apply(kt.load_batch(vertex_offsets=vo, row_ptr=torch.from_numpy(rp).to(dev),
                             col=torch.from_numpy(col).to(dev)))
    mb = torch.empty(max(int(eo[-1]), 1), dtype=torch.uint8, device=dev)[:int(eo[-1])]
    sb = torch.empty(max(int(eo[-1]), 1), dtype=torch.int32, device=dev)[:int(eo[-1])]
    hb.run_batch(Ks, out=(mb, sb))
    torch.cuda.synchronize()
    progress("batched: batch timed")
    e0.record(stream)
    _, _, rounds = hb.run_batch(Ks, out=(mb, sb))
    e1.record(stream)
    torch.cuda.synchronize()
    batch_ms = e0.elapsed_time(e1)
    brounds = hb.stats().rounds
    hb.close()
    return {"graphs": count, "edges": int(edges), "m_range": [1000, int(m_hi)],
            "graphs_per_s": round(count / (batch_ms / 1e3), 1),
            "plain_graphs_per_s": round(count / (plain_ms / 1e3), 1),
            "speedup": round(plain_ms / batch_ms, 2), "batch_ms": round(batch_ms, 3),
            "plain_ms": round(plain_ms, 3), "batch_rounds": int(brounds),
            "max_graph_rounds": int(max(rounds)) if len(rounds) else 0,
            "plain_settings": "library defaults",
            "autotuned": ({k: tune[k] for k in ("support_shape", "light_merge", "small_edges",
                                                  "update_mode", "trials")}
                          if tune is not None else None)}


def measure_serving(kt, gg, count, m_hi, seed=0):
    """Serving workload (graphgen.serve_config: R-MAT or G(n,m) with p = 1/2,
    sizes log-uniform in [1e4, m_hi] edges, K uniform in 3..16) through the
    request server: first all requests at once (saturated graphs/s), then
    Poisson arrivals at 70% of that rate (p50/p99 latency, graphs/s).  For
    comparison the same requests one after another through the plain path,
    host arrays in and out as the server's are: load, run, free per request.
    Every arm writes into the same caller-owned host output arrays, touched
    once before any timing."""
    progress(f"serving: generating {count} requests, m up to {m_hi:g}")
    reqs = gg.serve_config(count, seed=seed, m_lo=1e4, m_hi=m_hi)
    edges = sum(g.m for g, _ in reqs)
    progress(f"serving: {edges} edges; warm-up")
    mv = sum(g.n for g, _ in reqs) + 1
    me = min(edges + 1, (1 << 31) - 1)

    def server():
        return kt.Server(max_vertices=mv, max_edges=me, max_requests=max(8, count))

    # one set of caller-owned host output buffers per request, written once
    # before any timing, shared by every arm (so that no arm pays the first
    # touch of fresh host pages inside its timed region)
    import numpy as np
    outs = [(np.ones(max(g.m, 1), np.uint8), np.ones(max(g.m, 1), np.int32)) for g, _ in reqs]
    warm = server()
    kt.serve_poisson(warm, reqs[: min(4, count)], rate=None, outputs=outs)
    warm.close()
    srv = server()
    progress("serving: saturated")
    steps = []
    _, sat_s, _ = kt.serve_poisson(srv, reqs, rate=None, outputs=outs, step_times=steps)
    srv.close()
    sat = count / sat_s
    progress(f"serving: saturated {sat:.2f} graphs/s; Poisson arrivals")
    srv = server()
    lat, mk, _ = kt.serve_poisson(srv, reqs, rate=0.7 * sat, seed=seed + 1, outputs=outs)
    srv.close()
    progress("serving: plain path, one request after another")
    t0 = time.perf_counter()
    for (g, K), (mo, so) in zip(reqs, outs):
        h = kt.load(g.row_ptr, g.col)
        h.run_host(K, mask_out=mo, support_out=so)
        h.close()
    plain = count / (time.perf_counter() - t0)
    return {"requests": count, "edges": int(edges), "m_range": [10000, int(m_hi)],
            "saturated_graphs_per_s": round(sat, 2),
            "plain_graphs_per_s": round(plain, 2), "saturated_vs_plain": round(sat / plain, 2),
            "arrival_rate": round(0.7 * sat, 2),
            "graphs_per_s": round(count / mk, 2),
            "p50_latency_ms": round(float(np.percentile(lat, 50)) * 1e3, 3),
            "p99_latency_ms": round(float(np.percentile(lat, 99)) * 1e3, 3),
            "saturated_steps": len(steps),
            "step_host_ms": {"mean": round(1e3 * float(np.mean(steps)), 3),
                             "p50": round(1e3 * float(np.percentile(steps, 50)), 3),
                             "p99": round(1e3 * float(np.percentile(steps, 99)), 3),
                             "sum": round(1e3 * float(np.sum(steps)), 1)},
            "what": "latency from arrival to results in host memory; step_host_ms = wall time "
                    "of each Server.step of the saturated run (admission, one batched peel "
                    "round of every active request on the device, output copies of finished "
                    "requests)"}


def run_reference(args, world, rank):
    """Reference arm: the CPU oracle as it stands, on a bounded sample."""
    if rank != 0:
        return
    import numpy as np
    import graphgen as gg
    import oracle
    oracle.build()
    g = gg.rmat(args.ref_scale, 16, 0)
    for _ in range(args.warmup):
        oracle.ktruss(g.row_ptr, g.col, args.K)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.ktruss(g.row_ptr, g.col, args.K)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = g.m * args.steps / tot / 1e6
    sample = (f"each step: full K={args.K} run of the single-thread C oracle on R-MAT scale "
              f"{args.ref_scale}, edge factor 16 (same recipe as the workload, {g.m} edges)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1000 * tot / args.steps, 3),
        "ms_per_step_median": round(1000 * float(np.median(times)), 3),
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC[args.workload] + f", K={args.K}",
                   "reference_sample": f"rmat{args.ref_scale}", "K": args.K},
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "cpu_model": host_cpu_model(), "host_cores": os.cpu_count(),
                         "sample": sample},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat23c", choices=sorted(WORKLOAD_DESC))
    ap.add_argument("--K", type=int, default=3)
    ap.add_argument("--kernel", default="auto", choices=["auto", "balanced", "edge", "coarse"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-kmax", action="store_true", help="skip the K_max sweep timing")
    ap.add_argument("--no-reorder", action="store_true",
                    help="run from the loaded vertex numbering instead of the degree-ordered "
                         "relabel the library makes at load (KTRUSS_OPT_REORDER)")
    ap.add_argument("--no-rmat20", action="store_true",
                    help="skip the extra R-MAT-20 measurement (value and K_max sweep)")
    ap.add_argument("--batch-graphs", type=int, default=4096,
                    help="graphs of the batched-vs-plain measurement (0 = skip)")
    ap.add_argument("--update", choices=sorted(UPDATE_MODES), default="auto",
                    help="supports after the first round: decremental update (auto/always) or "
                         "recomputed every round (never, Alg. 1 as written)")
    ap.add_argument("--serve-requests", type=int, default=256,
                    help="requests of the serving measurement (0 = skip)")
    ap.add_argument("--serve-mmax", type=float, default=5e7,
                    help="largest request size (edges) of the serving measurement (the "
                         "serving workload: 5e7)")
    ap.add_argument("--batch-mmax", type=float, default=2e6,
                    help="largest graph size (edges) of that batch (the batching workload: "
                         "2e6)")
    ap.add_argument("--ref-scale", type=int, default=CPU_SAMPLE_SCALE,
                    help="R-MAT scale of the oracle sample timed by --impl reference")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_setup()

    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import numpy as np
    import torch

    import graphgen as gg
    import paper_2009_07929_gb300 as kt

    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    lib = kt.lib()
    progress(f"loading workload {args.workload}")
    g = gg.cached_workload(args.workload, 0)
    progress(f"workload n={g.n} m={g.m}; timed steps")
    n, m = g.n, g.m
    dev = torch.device("cuda", local)
    rp_d = torch.from_numpy(g.row_ptr).to(dev)
    col_d = torch.from_numpy(g.col).to(dev)
    # the library runs from the degree-ordered relabel it makes at load
    # (KTRUSS_OPT_REORDER, default on): count the support step's work on the
    # same CSR, which the generators' relabel of the same edges reproduces
    if args.no_reorder:
        progress("counting the support step's work on the host")
        work = support_work(g.row_ptr, g.col)
    else:
        progress("relabelling by degree on the host and counting the support step's work")
        gr = gg.from_edges(g.n, g.edges(), relabel=True)
        work = support_work(gr.row_ptr, gr.col)
        del gr
    h = kt.load(rp_d, col_d)
    h.set_kernel({"balanced": kt.KERNEL_BALANCED, "edge": kt.KERNEL_EDGE,
                  "coarse": kt.KERNEL_COARSE, "auto": kt.KERNEL_AUTO}[args.kernel])
    h.set_update(UPDATE_MODES[args.update])
    h.set_reorder(not args.no_reorder)
    mask = torch.empty(m, dtype=torch.uint8, device=dev)
    sup = torch.empty(m, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        h.run(args.K, out=(mask, sup))

    for _ in range(args.warmup):
        flush.fill_(1)
        step()
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    sup_ms, launches, st = 0.0, 0, None
    with ClockSampler(local) as clk:
        wall0 = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(i)
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
            st = h.stats()
            launches += st.kernel_launches
            # the round-1 support kernel (events around its launch only)
            sup_ms += st.ms_support_per_round[0] if st.ms_support_per_round else 0.0
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_ms = max_over_ranks(sum(step_ms), dev)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    value = world * m * args.steps / (tot_ms / 1000.0) / 1e6

    # ---- the same run with S recomputed every round (Alg. 1 as written), for
    # comparison with the decremental update (identical outputs)
    recompute = None
    if args.update != "never":
        h.set_update(kt.UPDATE_NEVER)
        step()
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.fill_(i)
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        rms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), dev)
        rst = h.stats()
        recompute = {"value": round(world * m * args.steps / (rms / 1000.0) / 1e6, 2),
                     "unit": UNIT, "ms_per_step": round(rms / args.steps, 4),
                     "support_steps": rst.support_launches, "rounds": rst.rounds}
        h.set_update(UPDATE_MODES[args.update])

    progress(f"value {value:.1f} Medges/s; e2e")
    # ---- e2e through the C ABI with pinned host buffers
    rp_h = torch.from_numpy(g.row_ptr).pin_memory()
    col_h = torch.from_numpy(g.col).pin_memory()
    mask_h = torch.empty(m, dtype=torch.uint8).pin_memory()
    sup_h = torch.empty(m, dtype=torch.int32).pin_memory()
    st_ptr = kt._stream_ptr()

    def e2e_step():
        hh = ctypes_load(lib, rp_h, col_h, n, m, st_ptr)
        if args.no_reorder:
            rc = lib.ktruss_set_option(hh, kt.OPT_REORDER, 0)
            if rc != 0:
                raise kt.KtrussError(rc, "ktruss_set_option")
        rc = lib.ktruss_run(hh, args.K, mask_h.data_ptr(), sup_h.data_ptr(), kt.HOST, st_ptr)
        if rc != 0:
            raise kt.KtrussError(rc, "ktruss_run")
        lib.ktruss_free(hh)

    for _ in range(2):
        e2e_step()
    e2e_times = []
    for i in range(max(3, min(args.steps, 5))):
        flush.fill_(i)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step()
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(sum(e2e_times) / len(e2e_times), dev)
    e2e_value = world * m / e2e_s / 1e6

    # ---- K_max sweep (truss decomposition) of the same graph, for context
    kmax, dec_ms = None, None
    if not args.no_kmax:
        h.decompose()
        torch.cuda.synchronize()
        d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(7)
        d0.record(stream)
        _, kmax = h.decompose()
        d1.record(stream)
        torch.cuda.synchronize()
        dec_ms = d0.elapsed_time(d1)
        dec_steps = h.stats().support_launches
        dec_rounds = h.stats().rounds

    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return

    peak, peak_kind = peaks()
    sup_avg_ms = sup_ms / args.steps
    # merge accounting (W counted on the host) and the design's own bytes,
    # both for the support step of round 1, the only one of a K = 3 run with
    # the decremental update (later support steps run on smaller graphs)
    tri1 = st.triangles_per_round[0] if st.triangles_per_round else 0
    survey_b = algorithmic_bytes(n, m, work["W"], tri1)
    design_b = design_bytes(work, tri1)
    achieved = design_b / (sup_avg_ms / 1000.0) / 1e9 if sup_avg_ms > 0 else None
    rec, fresh = traffic_record(args.workload + ("" if args.no_reorder else " reordered"), args.K)
    roofline = {
        "bound": None, "roof": "hbm",
        "achieved": round(achieved, 1) if achieved else None, "peak": peak,
        "unit": "GB/s", "frac": round(achieved / peak, 4) if achieved else None,
        "traffic": None,
        "peak_kind": f"{peak_kind} (HBM copy)",
        "kernel": "support_kernel (support step, Alg. 3)",
        "support_ms_per_launch": round(sup_avg_ms, 4),
        "design_bytes_per_launch": int(design_b),
        "work": work,
        "accounting": "design bytes: 4 per probe + 12 per staged column + 8 per triangle + 28 per "
                      "segment + 16 per active staged row (counted on the host from the CSR; "
                      "triangles from the run)",
        "survey_bytes_per_launch": int(survey_b),
        "frac_survey_accounting": round(survey_b / (sup_avg_ms / 1e3) / 1e9 / peak, 4)
        if sup_avg_ms > 0 else None,
        "survey_accounting": "4*W + 8*m + 16*T + 8*(n+1): a full merge of both lists of every "
                             "task; the kernel probes only the shorter list, so this exceeds the "
                             "bytes it moves",
    }
    if rec is not None and fresh:
        dram = rec["dram_bytes_per_launch"]
        roofline["traffic"] = int(dram)
        roofline["dram_frac"] = round(dram / (sup_avg_ms / 1e3) / 1e9 / peak, 4)
        roofline["l2_frac"] = rec.get("l2_throughput")
        roofline["sm_issue_active"] = rec.get("sm_issue_active")
        for key in ("l2_hit_rate", "warp_exec_efficiency", "warps_active", "traffic_note"):
            if key in rec:
                roofline[key] = rec[key]
        # what limits the kernel: the busiest of DRAM, L2 and SM issue among
        # the counters the record holds
        cand = {"hbm": roofline["dram_frac"], "l2": roofline["l2_frac"],
                "sm_issue": roofline["sm_issue_active"]}
        cand = {k: v for k, v in cand.items() if v is not None}
        roofline["bound"] = max(cand, key=cand.get)
        missing = [k for k in ("l2_frac", "sm_issue_active") if roofline.get(k) is None]
        if missing:
            roofline["bound_note"] = "not in the ncu record of this workload: " + ", ".join(missing)
        roofline["ncu_command"] = rec.get("command")
    else:
        roofline["traffic_record"] = ("stale: the kernel changed since the committed ncu capture"
                                      if rec is not None else "none for this workload")
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(tot_ms / args.steps, 4),
        "ms_per_step_median": round(float(np.median(step_ms)), 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC[args.workload] + f", K={args.K}", "K": args.K,
                   "reorder": not args.no_reorder,
                   "n": n, "m": m, "rounds": st.rounds, "kernel": args.kernel,
                   "update": args.update, "support_steps": st.support_launches,
                   "parallelism": f"replicas{world}", "l2": "flushed between steps (512 MiB write)"},
        "e2e": {"value": round(e2e_value, 2), "unit": UNIT,
                "h2d_bytes_per_step": 4 * (n + 1) + 4 * m, "d2h_bytes_per_step": 5 * m},
        "gpu_launches": launches,
        "recompute_every_round": recompute,
        "roofline": roofline,
        "clocks": clk.summary(),
        "wall_s_timed": round(wall, 3),
    }
    if kmax is not None:
        out["kmax_sweep"] = {"kmax": kmax, "ms": round(dec_ms, 3), "support_steps": dec_steps,
                             "rounds": dec_rounds,
                             "Medges_per_s": round(m / (dec_ms / 1e3) / 1e6, 2),
                             "what": "ktruss_decompose: K = 3 .. K_max, each K from the previous truss"}
    if not args.no_rmat20 and args.workload != "rmat20":
        out["rmat20"] = measure_workload(kt, gg, "rmat20", args.K, args.steps, flush)
    if args.batch_graphs > 0:
        out["batched"] = measure_batched(kt, gg, args.batch_graphs, args.batch_mmax)
    if args.serve_requests > 0:
        out["serving"] = measure_serving(kt, gg, args.serve_requests, args.serve_mmax)
    if not args.no_cpu_baseline:
        progress("cpu baseline (oracle)")
        out["cpu_baseline"] = cpu_baseline()
        progress("cpu baseline (paper's fine-grained CPU design, all cores)")
        out["cpu_f"] = cpu_f_baseline(args.K)
    print(json.dumps(out), flush=True)
    if pg:
        pg.destroy_process_group()


def ctypes_load(lib, rp_h, col_h, n, m, stream_ptr):
    import ctypes
    hh = ctypes.c_void_p(0)
    rc = lib.ktruss_load_csr(ctypes.byref(hh), n, m, rp_h.data_ptr(), col_h.data_ptr(), 0,
                             stream_ptr)
    if rc != 0:
        import paper_2009_07929_gb300 as kt
        raise kt.KtrussError(rc, "ktruss_load_csr")
    return hh


if __name__ == "__main__":
    main()
