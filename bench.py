"""Benchmark: walk steps/s of the GPU walk engine, with its HBM roofline, an
end-to-end number through the C ABI with host buffers, and the CPU oracle's
throughput on a bounded sample beside it.

Default workload: node2vec p=1, q=2 (fast mode, FP32 weights) on the R-MAT
scale-25 graph (edge factor 16, symmetrised, 1.07e9 CSR entries, int64 row
offsets, int32 columns), walks of length 80, one query per vertex; one bench
step = one launch over a batch of 2^21 of those queries (vertices
v = k mod 16 for step k).  The graph (8.9 GB) is far larger than L2, so no L2
flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line on rank 0.
"""

from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (scale, algo, p, q, mode, L, types)
    "rmat25_node2vec": dict(scale=25, algo="node2vec", p=1.0, q=2.0, mode="fast", L=80, types=None,
                            batch_log2=21, slices=16),
    "rmat22_node2vec": dict(scale=22, algo="node2vec", p=1.0, q=2.0, mode="fast", L=80, types=None,
                            batch_log2=20, slices=4),
    "rmat20_node2vec": dict(scale=20, algo="node2vec", p=2.0, q=0.5, mode="fast", L=80, types=None,
                            batch_log2=20, slices=1),
    "rmat20_node2vec_exact": dict(scale=20, algo="node2vec", p=2.0, q=0.5, mode="exact", L=80, types=None,
                                  batch_log2=20, slices=1),
    "rmat22_weighted": dict(scale=22, algo="weighted", p=1.0, q=1.0, mode="fast", L=80, types=None,
                            batch_log2=22, slices=1),
    "rmat25_weighted": dict(scale=25, algo="weighted", p=1.0, q=1.0, mode="fast", L=80, types=None,
                            batch_log2=22, slices=8),
    # extra distributions: log-normal weights (Appendix C.1, sigma = 3) and
    # the paper's PPR workload, every query from the max-degree vertex
    "rmat22_weighted_lognormal3": dict(scale=22, algo="weighted", p=1.0, q=1.0, mode="fast", L=80, types=None,
                                       batch_log2=20, slices=4, weights="lognormal3"),
    "rmat22_ppr_maxdeg": dict(scale=22, algo="ppr", p=1.0, q=1.0, mode="fast", L=100, types=None,
                              batch_log2=20, slices=1, starts="maxdeg"),
    # small case of the headline kernel for ncu captures with DRAM counters
    # (graph 4.3 GB, 2^18 queries per launch)
    "rmat24_node2vec": dict(scale=24, algo="node2vec", p=1.0, q=2.0, mode="fast", L=80, types=None,
                            batch_log2=18, slices=64),
}

NOMINAL_HBM_GBS = 8000.0  # the HBM figure the hot-path target is stated against


def describe(w):
    wt = w.get("weights", "grid14")
    wdesc = "weights [1,5) on a 2^-14 grid" if wt == "grid14" else f"log-normal weights sigma={wt[len('lognormal'):]}"
    sdesc = ("every query from the max-degree vertex" if w.get("starts") == "maxdeg"
             else f"1/{w['slices']} of one query per vertex")
    algo = "PPR stop 0.2" if w["algo"] == "ppr" else f"{w['algo']} p={w['p']:g} q={w['q']:g}"
    return (f"{algo}, {w['mode']} mode, R-MAT scale {w['scale']} "
            f"(a,b,c=.57,.19,.19, ef 16, symmetrised, {wdesc}), L={w['L']}, "
            f"{2 ** w['batch_log2']} queries per step ({sdesc})")


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # raw samples: FW_CLOCKS_DIR if set, else the temp directory (the
        # bench line carries their summary)
        import tempfile
        self.path = os.path.join(os.environ.get("FW_CLOCKS_DIR", tempfile.gettempdir()), f"clocks_gpu{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
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
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


KERNEL_SOURCES = ("paper_2404_08364_gb300/csrc/fw_walk.cu", "paper_2404_08364_gb300/csrc/fw_internal.cuh")


def _code_tokens(text):
    """The source with its comments and whitespace runs removed: what the
    compiler sees.  String literals are kept whole (a "//" inside one is not a
    comment)."""
    import re
    tok = re.compile(r'"(?:\\.|[^"\\])*"|//[^\n]*|/\*.*?\*/|\s+', re.S)
    return tok.sub(lambda m: m.group(0) if m.group(0).startswith('"') else " ", text).split()


def kernel_sources_hash():
    """Hash of the walk kernel's sources, comments and layout excluded, so
    that a profile stays tied to the code it was captured on and not to the
    wording of its comments."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
            h.update(" ".join(_code_tokens(fh.read())).encode())
        h.update(b"\0")
    return h.hexdigest()[:16]


def profiled_traffic_ratio(workload):
    """DRAM bytes per algorithmic byte of the walk kernel on `workload`, from
    an ncu capture summarised under profiles/, if that capture was taken of
    the kernel as it is now; else None."""
    import glob
    import re
    pat = re.compile(r"^traffic-per-algorithmic-byte: ([0-9.]+) \(workload (\S+), sources ([0-9a-f]+)"
                     r"(?:, stands for (\S+))?\)")
    cur = kernel_sources_hash()
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(path) as f:
            for line in f:
                m = pat.match(line.strip())
                if m and workload in (m.group(2), m.group(4)) and m.group(3) == cur:
                    return float(m.group(1)), os.path.relpath(path, ROOT), m.group(2)
    return None


def make_graph(w, device):
    import fw_inputs as fi
    t0 = time.time()
    g = fi.rmat(w["scale"], types_seed=w["types"], weights=w.get("weights", "grid14"), device=device)
    return g, time.time() - t0


def slice_starts(n, k, slices, batch, device, w=None, g=None):
    import torch
    if w is not None and w.get("starts") == "maxdeg":
        deg = g.row_ptr[1:] - g.row_ptr[:-1]
        return torch.full((batch,), int(torch.argmax(deg)), dtype=torch.int32, device=device)
    s = torch.arange(k % slices, n, slices, dtype=torch.int32, device=device)
    return s[:batch]


def cpu_oracle_sample(g_host, w, seconds=15.0, threads=None, seed=42):
    """The CPU oracle (as it stands: the exact-mode C walker) on a bounded
    sample of the workload's queries, on `threads` host threads over disjoint
    query ranges.  The sample's starts are drawn uniformly over the whole
    vertex range by hash, so the oracle sees the same mix of hub and leaf
    starts as one query per vertex.  Returns (steps/s, threads, description)."""
    import numpy as np

    import fw_inputs as fi
    import oracle
    oracle.build()
    csr = oracle.CSR(g_host)
    prm = oracle.Params(p=w["p"], q=w["q"], scale=2)
    threads = threads or os.cpu_count() or 1
    n = g_host.n
    per_call = 8
    total_steps = 0
    calls = 0
    t0 = time.time()
    pool = fi.random_starts(n, 1 << 20, 4243 + seed).numpy()

    hub = None
    if w.get("starts") == "maxdeg":
        hub = int(np.argmax(np.diff(g_host.row_ptr.numpy())))

    def run(ci):
        if hub is not None:
            st = np.full(per_call, hub, dtype=np.int32)
        else:
            st = pool[(ci * per_call) % pool.size:][:per_call]
        _, plen = oracle.walk_exact(csr, w["algo"], prm, st, w["L"], seed, q0=ci * per_call)
        return int((plen - 1).sum())

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        futs = []
        ci = 0
        while time.time() - t0 < seconds:
            while len(futs) < 2 * threads:
                futs.append(ex.submit(run, ci))
                ci += 1
            done, _ = cf.wait(futs, return_when=cf.FIRST_COMPLETED)
            for f in done:
                total_steps += f.result()
                calls += 1
                futs.remove(f)
        for f in futs:
            total_steps += f.result()
            calls += 1
    dt = time.time() - t0
    where = ("every start at the max-degree vertex" if hub is not None
             else "starts uniform over the whole vertex range by hash")
    desc = (f"oracle (exact-mode C walker, integer weights) on {calls * per_call} queries of the same graph, "
            f"algorithm and length ({where}), {threads} threads, {dt:.1f} s; the GPU line walks in "
            f"{w['mode']} mode")
    return total_steps / dt, threads, desc


def run_reference(args, w):
    """--impl reference: the CPU oracle as the reference arm."""
    rank, _, world = _dist_env()
    if rank != 0:
        return
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    g, _ = make_graph(w, dev)
    g = g.to("cpu")
    if dev == "cuda":
        torch.cuda.empty_cache()
    per_step = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    vals = []
    for i in range(args.warmup + args.steps):
        v, cores, desc = cpu_oracle_sample(g, w, seconds=per_step, seed=42 + i)
        if i >= args.warmup:
            vals.append(v)
    value = sum(vals) / len(vals)
    line = {
        "impl": "reference", "metric": "walk steps/s", "value": value, "unit": "steps/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": per_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32 (exact-mode integer weights)", "data": "synthetic",
        "config": {"workload": describe(w)},
        "cpu_baseline": {"value": value, "unit": "steps/s", "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _dist_env():
    from paper_2404_08364_gb300.shard import env_rank
    return env_rank()[0], env_rank()[1], env_rank()[2]


def serve_block(args):
    """Served form (config 5): Poisson arrivals at swept offered loads on a
    resident R-MAT graph; per load the served steps/s, p50/p99 latency
    (submission to results in the caller's host buffers) and the clocks seen,
    beside the plain batch of the same request mix."""
    import numpy as np
    import torch

    import fw_inputs as fi
    from paper_2404_08364_gb300.build import build
    build()
    from paper_2404_08364_gb300 import DeviceGraph, Server

    torch.cuda.set_device(0)
    scale = args.serve_scale
    g = fi.rmat(scale, device="cuda")
    dg = DeviceGraph.from_tensors(g.row_ptr, g.col, g.w_f32, None, None, borrow=True)
    rng = np.random.default_rng(7)
    n_req = args.serve_requests
    algos = ["weighted", "node2vec", "ppr"]
    reqs = []
    for i in range(n_req):
        n_q = int(min(65536, max(1, round(2 ** rng.uniform(0, 16)))))
        a = algos[int(rng.integers(0, 3))]
        L = 100 if a == "ppr" else int(rng.integers(10, 81))
        reqs.append(dict(algo=a, starts=fi.random_starts(g.n, n_q, 1000 + i), max_len=L, seed=(i * 2654435761) & 0xFFFFFFFF,
                         p=2.0, q=0.5, ppr_stop=0.2))
    total_q = sum(r["starts"].numel() for r in reqs)

    # plain batch of the same mix: all requests of one algorithm merged into
    # one launch, the three launches back to back (an upper bound for any
    # batch server: no request boundaries, no admission, no copies out)
    def batch_once():
        outs = []
        for a in algos:
            rs = [r for r in reqs if r["algo"] == a]
            if not rs:
                continue
            st = torch.cat([r["starts"] for r in rs]).cuda()
            L = max(r["max_len"] for r in rs)
            ln = torch.cat([torch.full((r["starts"].numel(),), r["max_len"], dtype=torch.int32) for r in rs]).cuda()
            outs.append(dg.walk(a, st, L, 7, mode="fast", p=2.0, q=0.5, lengths=ln))
        torch.cuda.synchronize()
        return sum(int((pl - 1).sum()) for _, pl in outs)
    batch_once()
    clocks = ClockSampler(0)
    clocks.start()
    t0 = time.perf_counter()
    steps_b = batch_once()
    tb = time.perf_counter() - t0
    batch_clk = clocks.stop()
    batch_rate = steps_b / tb
    req_rate_cap = n_req / tb
    lines = []
    for frac in args.serve_rates:
        srv = Server(dg, mode="fast", mem_budget=args.serve_mem_mb << 20, idle_ms=5.0)
        lam = frac * req_rate_cap
        gaps = rng.exponential(1.0 / lam, size=n_req)
        clocks = ClockSampler(0)
        clocks.start()
        t_start = time.perf_counter()
        at = t_start
        tickets = []
        for r, gap in zip(reqs, gaps):
            at += gap
            while time.perf_counter() < at:
                pass
            tickets.append(srv.submit(r["algo"], r["starts"], r["max_len"], r["seed"], p=2.0, q=0.5))
        lat = []
        steps = 0
        for t in tickets:
            paths, plen, l = srv.result(t)
            lat.append(l)
            steps += int((plen - 1).sum())
        t_end = time.perf_counter()
        clk = clocks.stop()
        st = srv.stats()
        srv.close()
        lat = np.array(lat)
        lines.append({"offered_load": frac, "served_steps_per_s": steps / (t_end - t_start),
                      "served_over_batch": steps / (t_end - t_start) / batch_rate,
                      "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                      "engine_launches": st["launches"], "clocks": clk})
    best = max(lines, key=lambda d: d["served_steps_per_s"])
    dg.free()
    del g
    torch.cuda.empty_cache()
    return {
        "metric": "served walk steps/s", "value": best["served_steps_per_s"], "unit": "steps/s",
        "workload": f"served mix on R-MAT scale {scale}: {n_req} requests, sizes log-uniform [1, 65536] "
                    f"({total_q} queries), algo uniform {{weighted, node2vec p=2 q=0.5, PPR 0.2}}, "
                    f"length uniform [10, 80] (PPR cap 100), Poisson arrivals, fast mode, host outputs",
        "arena_mb": args.serve_mem_mb,
        "plain_batch_steps_per_s": batch_rate, "plain_batch_clocks": batch_clk,
        "plain_batch": "the same requests merged per algorithm into 3 device launches back to back "
                       "(device outputs): an upper bound for a batch server",
        "served_over_batch": best["served_steps_per_s"] / batch_rate,
        "best_offered_load": best["offered_load"],
        "sweep": lines,
    }


def served_child(args, limit_s=600.0):
    """The served block in a child process with a time limit, so that a
    served run that stops making progress ends the child (and its CUDA
    context) instead of the benchmark."""
    cmd = [sys.executable, os.path.abspath(__file__), "--serve", "--serve-scale", str(args.serve_scale),
           "--serve-requests", str(args.serve_requests), "--serve-mem-mb", str(args.serve_mem_mb),
           "--serve-rates", *[str(r) for r in args.serve_rates]]
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=limit_s)
    except subprocess.TimeoutExpired:
        return {"error": f"served run exceeded {limit_s:.0f} s and was stopped"}
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    if r.returncode != 0 or not lines:
        return {"error": f"served run failed (rc {r.returncode}): {r.stderr.strip().splitlines()[-1:] }"}
    return json.loads(lines[-1])


def run_serve(args):
    out = serve_block(args)
    out.update({"n_gpus": 1, "higher_is_better": True, "data": "synthetic", "dtype": "f32"})
    print(json.dumps(out), flush=True)


def run_sweep(args):
    """Scalability (Appendix C.5): throughput in scanned CSR
    entries (edges) per second on an R-MAT graph, (a) against the number of
    queries 10^2..10^7 at length 80, (b) against the length 10..80 at 10^6
    queries; random starts; one warm-up launch, then one timed launch per
    point (CUDA events on the launching stream)."""
    import torch

    import fw_inputs as fi
    from paper_2404_08364_gb300.build import build
    build()
    from paper_2404_08364_gb300 import DeviceGraph

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    scale = args.sweep_scale
    g = fi.rmat(scale, device=dev)
    dg = DeviceGraph.from_tensors(g.row_ptr, g.col, g.w_f32, None, None, borrow=True, device=dev)
    algo, p, q = {"node2vec": ("node2vec", 1.0, 2.0), "weighted": ("weighted", 1.0, 1.0)}[args.sweep_algo]
    stream = torch.cuda.current_stream(dev)
    points = [(10 ** e, 80) for e in range(2, 8)] + [(10 ** 6, L) for L in (10, 20, 40)]
    rows = []
    clocks = ClockSampler(0)
    clocks.start()
    for nq, L in points:
        starts = fi.random_starts(g.n, nq, 4242).to(dev)
        paths = torch.empty((nq, L + 1), dtype=torch.int32, device=dev)
        plen = torch.empty(nq, dtype=torch.int32, device=dev)
        dg.walk(algo, starts, L, 7, mode="fast", p=p, q=q, paths=paths, path_len=plen, stream=stream)
        torch.cuda.synchronize(dev)
        dg.stats_reset(stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dg.walk(algo, starts, L, 8, mode="fast", p=p, q=q, q_id0=nq, paths=paths, path_len=plen, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        s = e0.elapsed_time(e1) / 1e3
        st = dg.stats()
        rows.append({"queries": nq, "length": L, "edges_per_s": st["rows_scanned"] / s,
                     "steps_per_s": st["steps"] / s, "ms": s * 1e3})
        del paths, plen
    clk = clocks.stop()
    out = {"metric": "edges/s (scanned CSR entries per second)", "unit": "edges/s", "higher_is_better": True,
           "clocks": clk,
           "n_gpus": 1, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"{algo} p={p:g} q={q:g}, fast mode, R-MAT scale {scale} "
                                  f"(a,b,c=.57,.19,.19, ef 16, symmetrised), random starts",
                      "tuning": dg.get_tuning()},
           "sweep": rows}
    print(json.dumps(out), flush=True)
    dg.free()


def run_batched(args):
    """Out-of-memory batches (Section 5.2, Eq. 3): node2vec p=1 q=2 on R-MAT
    with host inputs and outputs through fw_walk_batched, the byte budget set
    so the queries take `--batches` batches, against one device-resident
    launch of the same queries followed by the copy of its paths to the host."""
    import torch

    import fw_inputs as fi
    from paper_2404_08364_gb300.build import build
    build()
    from paper_2404_08364_gb300 import DeviceGraph

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    scale, L = args.sweep_scale, 80
    g = fi.rmat(scale, device=dev)
    dg = DeviceGraph.from_tensors(g.row_ptr, g.col, g.w_f32, None, None, borrow=True, device=dev)
    nq = 1 << 22
    starts = fi.random_starts(g.n, nq, 99)
    per_query = (L + 3) * 4
    budget = 2 * per_query * ((nq + args.batches - 1) // args.batches)
    hp = torch.empty((nq, L + 1), dtype=torch.int32).pin_memory()
    hl = torch.empty(nq, dtype=torch.int32).pin_memory()
    kw = dict(mode="fast", p=1.0, q=2.0)
    dg.walk_batched("node2vec", starts[:4096], L, 1, budget_bytes=budget, **kw)  # warm-up
    dg.stats_reset()
    clocks = ClockSampler(0)
    clocks.start()
    t0 = time.perf_counter()
    _, _, bq = dg.walk_batched("node2vec", starts, L, 2, budget_bytes=budget, paths=hp, path_len=hl, **kw)
    t_b = time.perf_counter() - t0
    steps_b = dg.stats()["steps"]
    ds = starts.to(dev)
    dp = torch.empty((nq, L + 1), dtype=torch.int32, device=dev)
    dl = torch.empty(nq, dtype=torch.int32, device=dev)
    torch.cuda.synchronize(dev)
    dg.stats_reset()
    t0 = time.perf_counter()
    dg.walk("node2vec", ds, L, 2, paths=dp, path_len=dl, **kw)
    hp.copy_(dp)
    hl.copy_(dl)
    torch.cuda.synchronize(dev)
    t_1 = time.perf_counter() - t0
    clk = clocks.stop()
    steps_1 = dg.stats()["steps"]
    out = {"metric": "walk steps/s, host outputs", "unit": "steps/s", "higher_is_better": True, "n_gpus": 1,
           "dtype": "f32", "data": "synthetic", "clocks": clk,
           "config": {"workload": f"node2vec p=1 q=2, fast mode, R-MAT scale {scale}, L={L}, {nq} random starts, "
                                  f"host (pinned) outputs of {nq * (L + 1) * 4 / 1e9:.2f} GB",
                      "budget_bytes": budget, "queries_per_batch": bq, "batches": (nq + bq - 1) // bq},
           "batched_steps_per_s": steps_b / t_b, "batched_s": t_b,
           "one_launch_then_copy_steps_per_s": steps_1 / t_1, "one_launch_then_copy_s": t_1,
           "batched_over_one_launch": (steps_b / t_b) / (steps_1 / t_1)}
    print(json.dumps(out), flush=True)
    dg.free()


def run_samplers(args):
    """Section 4's samplers side by side (fw_sampler_run): DPRS (Alg. 3), ZPRS
    (Alg. 4) and the engine's exponential-jump reservoir, at warp and CTA
    width, over sampling sizes 2^0..2^20 (Section 6.3's sampling-size sweep).
    Weights [1, 5) on the 2^-14 grid; enough independent draws per launch to
    fill the GPU; the array stays in L2, so this times the samplers' own
    work, not DRAM."""
    import torch

    from paper_2404_08364_gb300.build import build
    build()
    from paper_2404_08364_gb300 import sample

    torch.cuda.set_device(0)
    rows = []
    clocks = ClockSampler(0)
    clocks.start()
    for e in range(0, 21):
        n = 1 << e
        k = torch.arange(n, dtype=torch.int64)
        w = (1.0 + ((k * 2654435761) % 65536).double() / 16384.0).float().cuda()
        for width in (32, 256):
            reps = max(152 * (64 if width == 32 else 8), min(1 << 22, (1 << 27) // n))
            out = torch.empty(reps, dtype=torch.int32, device="cuda")
            res = {}
            for m in ("expj", "dprs", "zprs"):
                sample(m, w, min(reps, 4096), seed=1, width=width, out=out[:min(reps, 4096)])  # warm-up
                _, ms = sample(m, w, reps, seed=2, width=width, out=out)
                res[m] = {"draws_per_s": reps / (ms / 1e3), "elements_per_s": reps * n / (ms / 1e3), "ms": ms}
            best = max(res, key=lambda m: res[m]["draws_per_s"])
            rows.append({"n": n, "width": width, "reps": reps, "best": best, **{m: res[m] for m in res}})
    clk = clocks.stop()
    out = {"metric": "weighted draws per second", "unit": "draws/s", "higher_is_better": True, "n_gpus": 1,
           "dtype": "f32", "data": "synthetic", "clocks": clk,
           "config": {"workload": "one weight array of n entries ([1,5) on a 2^-14 grid), independent draws, "
                                  "samplers: expj (engine), dprs (Alg. 3), zprs (Alg. 4)"},
           "sweep": rows}
    print(json.dumps(out), flush=True)


def full_config_block(dg, g, w, dev, stream, peak):
    """The configuration as stated, in one launch: every query of the
    workload (one per vertex) walked by a single engine launch, timed with
    CUDA events on the launching stream, with its own clock samples."""
    import torch
    n_q = g.n
    L = w["L"]
    starts = torch.arange(n_q, dtype=torch.int32, device=dev)
    paths = torch.empty((n_q, L + 1), dtype=torch.int32, device=dev)
    plen = torch.empty(n_q, dtype=torch.int32, device=dev)
    kw = dict(mode=w["mode"], p=w["p"], q=w["q"], scale=2)
    torch.cuda.synchronize(dev)
    dg.stats_reset(stream)
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    dg.walk(w["algo"], starts, L, 42, paths=paths, path_len=plen, stream=stream, **kw)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    st = dg.stats()
    achieved = st["algo_bytes"] / (ms / 1e3) / 1e9
    out = {"queries": n_q, "launches": 1, "ms": ms, "steps": st["steps"],
           "steps_per_s": st["steps"] / (ms / 1e3), "walks": st["walks"],
           "output_bytes": paths.numel() * 4 + plen.numel() * 4,
           "roofline": {"achieved": achieved, "peak": peak, "frac": achieved / peak,
                        "frac_vs_8tbs": achieved / NOMINAL_HBM_GBS, "algo_bytes": st["algo_bytes"]},
           "clocks": clk}
    del paths, plen, starts
    torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat25_node2vec", choices=sorted(WORKLOADS))
    ap.add_argument("--batch-log2", type=int, default=None)
    ap.add_argument("--algo", default=None, choices=["weighted", "node2vec", "metapath", "ppr"],
                    help="walk rule instead of the workload's (same graph and queries)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5, help="launches timed end to end (host buffers)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-full", action="store_true", help="skip the one-launch run of every query of the workload")
    ap.add_argument("--no-served", action="store_true", help="skip the served-form block")
    ap.add_argument("--threads", type=int, default=0, help="CTA size (0 = library default)")
    ap.add_argument("--slots", type=int, default=0, help="walk slots per CTA (0 = default)")
    ap.add_argument("--d-t", type=int, default=0, help="hub threshold d_t (0 = default)")
    ap.add_argument("--serve", action="store_true", help="served-form benchmark (config 5) instead")
    ap.add_argument("--sweep", action="store_true", help="scalability sweep (edges/s vs queries and length)")
    ap.add_argument("--sweep-scale", type=int, default=22)
    ap.add_argument("--sweep-algo", default="node2vec", choices=["node2vec", "weighted"])
    ap.add_argument("--batched", action="store_true", help="out-of-memory batches on two streams (Eq. 3)")
    ap.add_argument("--samplers", action="store_true", help="DPRS / ZPRS / engine reservoir, sampling-size sweep")
    ap.add_argument("--batches", type=int, default=8)
    ap.add_argument("--serve-scale", type=int, default=24)
    ap.add_argument("--serve-requests", type=int, default=400)
    ap.add_argument("--serve-mem-mb", type=int, default=2048)
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[0.25, 0.5, 0.75, 0.9, 1.0, 1.2])
    args = ap.parse_args()
    w = dict(WORKLOADS[args.workload])
    if args.batch_log2 is not None:
        w["batch_log2"] = args.batch_log2
    if args.algo is not None:
        w["algo"] = args.algo
        if args.algo == "metapath" and w["types"] is None:
            w["types"] = 2
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args, w)
    if args.serve:
        return run_serve(args)
    if args.sweep:
        return run_sweep(args)
    if args.batched:
        return run_batched(args)
    if args.samplers:
        return run_samplers(args)

    import torch
    import torch.distributed as dist

    from paper_2404_08364_gb300.build import build
    from paper_2404_08364_gb300.shard import reduce_scalar, shard_range

    rank, local, world = _dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build()
    from paper_2404_08364_gb300 import DeviceGraph

    g, gen_s = make_graph(w, dev)
    g_host = g.to("cpu") if (rank == 0 and world == 1 and not args.no_cpu) else None
    # fast mode needs only FP32 weights on the device
    keep_u32 = w["mode"] == "exact"
    dg = DeviceGraph.from_tensors(g.row_ptr, g.col, g.w_f32, g.w_u32 if keep_u32 else None, g.etype,
                                  borrow=True, device=dev)
    if args.threads or args.slots or args.d_t:
        dg.set_tuning(block_threads=args.threads, slots=args.slots, d_warp=args.d_t)
    graph_bytes = sum(t.numel() * t.element_size() for t in (g.row_ptr, g.col, g.w_f32))
    batch = 2 ** w["batch_log2"]
    # weak scaling: every rank runs `batch` queries per step, from its own shard
    # of the query space (slices of one query per vertex)
    stream = torch.cuda.current_stream(dev)
    steps_total = args.warmup + args.steps
    starts = []
    for k in range(steps_total):
        s = slice_starts(g.n, k, w["slices"], batch * world, dev, w, g)
        b, e = shard_range(s.numel(), rank, world)
        starts.append((s[b:e].contiguous(), (k % w["slices"]) * (g.n // w["slices"]) + b))
    paths = torch.empty((batch, w["L"] + 1), dtype=torch.int32, device=dev)
    plen = torch.empty(batch, dtype=torch.int32, device=dev)
    kw = dict(mode=w["mode"], p=w["p"], q=w["q"], scale=2)

    def step(k):
        s, qid0 = starts[k]
        dg.walk(w["algo"], s, w["L"], 42, q_id0=qid0, paths=paths[:s.numel()], path_len=plen[:s.numel()],
                stream=stream, **kw)

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    dg.stats_reset(stream)
    clocks = ClockSampler(local)
    clocks.start()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    evs[0].record(stream)
    for i in range(args.steps):
        step(args.warmup + i)
        evs[i + 1].record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms_each = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    ms_total = sum(ms_each)
    st = dg.stats()
    steps_local = st["steps"]
    ms_max = reduce_scalar(ms_total, "max", dev)
    steps_all = reduce_scalar(steps_local, "sum", dev)
    value = steps_all / (ms_max / 1e3)

    # end to end through the C ABI with pinned host buffers (rank-local)
    e2e = None
    if not args.no_e2e:
        hs = [s.cpu().pin_memory() for s, _ in starts]
        hp = torch.empty((batch, w["L"] + 1), dtype=torch.int32).pin_memory()
        hl = torch.empty(batch, dtype=torch.int32).pin_memory()
        dg.stats_reset(stream)
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        e2e_k = max(1, min(args.steps, args.e2e_steps))
        t0 = time.perf_counter()
        h2d = d2h = 0
        for i in range(e2e_k):
            k = args.warmup + i
            n_q = hs[k].numel()
            dg.walk(w["algo"], hs[k], w["L"], 42, q_id0=starts[k][1], paths=hp[:n_q], path_len=hl[:n_q],
                    stream=stream, **kw)
            h2d += n_q * 4
            d2h += n_q * (w["L"] + 1) * 4 + n_q * 4
        t1 = time.perf_counter()
        e2e_steps = reduce_scalar(dg.stats()["steps"], "sum", dev)
        e2e_s = reduce_scalar(t1 - t0, "max", dev)
        e2e = {"value": e2e_steps / e2e_s, "unit": "steps/s", "h2d_bytes_per_step": h2d // e2e_k,
               "d2h_bytes_per_step": d2h // e2e_k, "launches": e2e_k,
               "how": "fw_walk_ex with pinned host starts, paths and path_len (the library stages them); "
                      "wall clock around the launches, copies included"}

    peak, peak_kind = load_peaks()
    algo_bytes_per_launch = st["algo_bytes"] / args.steps
    prof = profiled_traffic_ratio(args.workload) if w["algo"] == WORKLOADS[args.workload]["algo"] else None
    achieved = algo_bytes_per_launch / (ms_total / args.steps / 1e3) / 1e9
    line = {
        "metric": "walk steps/s", "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if w["mode"] == "fast" else "u32",
        "data": "synthetic",
        "config": {"workload": describe(w), "graph": g.name, "n": g.n, "m": g.m,
                   "graph_bytes_on_device": graph_bytes, "l2": "inputs larger than L2 (no flush)",
                   "parallelism": f"query shards x{world} (graph replicas)",
                   "graph_gen_s": round(gen_s, 1), "tuning": dg.get_tuning()},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "frac_vs_8tbs": achieved / NOMINAL_HBM_GBS,
                     "traffic": prof[0] * algo_bytes_per_launch if prof else None,
                     "traffic_source": (f"{prof[1]}: ncu dram__bytes_read.sum + dram__bytes_write.sum of one "
                                        f"launch of {prof[2]} per algorithmic byte ({prof[0]}), times this run's "
                                        f"algorithmic bytes per launch") if prof else
                                       "no ncu capture of the kernel as built now",
                     "peak_kind": f"{peak_kind} (copy bandwidth)",
                     "algo_bytes_per_launch": algo_bytes_per_launch,
                     "kernel": "walk_kernel (persistent engine)"},
        "gpu_launches": args.steps,
        "clocks": clk,
        "e2e": e2e,
        "counters": {k: st[k] for k in ("steps", "rows_scanned", "warp_steps", "block_steps", "n2v_tests")},
    }
    del paths, plen
    if not args.no_full and world == 1 and w.get("starts") != "maxdeg":
        line["full_config"] = full_config_block(dg, g, w, dev, stream, peak)
    if g_host is not None:
        del g
        torch.cuda.empty_cache()
        v, cores, desc = cpu_oracle_sample(g_host, w, seconds=args.cpu_seconds)
        line["cpu_baseline"] = {"value": v, "unit": "steps/s", "cores": cores, "kind": "oracle", "sample": desc}
    dg.free()
    if not args.no_served and world == 1:
        del g_host
        torch.cuda.empty_cache()
        line["served"] = served_child(args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
