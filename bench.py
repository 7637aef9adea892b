"""Benchmark: KADABRA samples/s and time-to-stop on one GB300 per rank.

One step = one complete KADABRA query (calibration, adaptive sampling until the
stop rule holds, b~ = c/tau) on the resident R-MAT scale-20 graph (edge factor
16, a,b,c = .57,.19,.19, undirected, largest component; eps = .01, delta = .1,
seed 1) through the C ABI (kad_run_device).  The graph's inputs are in HBM
before the timed region; L2 (129 MB) is flushed by writing a 512 MB buffer
between timed steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload rmat20]

N > 1 runs under torch.distributed.run: every rank answers its own replica of
the query stream (the sampling path has no data exchange between GPUs), the
timed region is bracketed by barriers, the max over ranks is taken, and the
value is the sum of samples over ranks divided by that time.

--impl reference times the oracle (the plain CPU statement of the method) on
the host cores on a bounded sample of the same workload.
"""
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

METRIC = "KADABRA samples/s and time-to-stop at fixed eps,delta; batched query p50/p99 vs plain"
UNIT = "samples/s"

# Algorithmic bytes per unit of the adaptive-phase work counters: 8 B row-offset
# pair per expanded frontier vertex; 4 B column + 4 B neighbour state per scanned
# arc; 12 B state + sigma per labelled vertex; 8 B sigma per arc into the next
# level (or meeting set); 4 B per path increment.  The trace-back's reads are not
# counted: they depend on how the predecessors are found, not on the sample.
BYTES_PER = dict(expanded=8, scanned=8, labelled=12, pred_arcs=8, trace_arcs=0, increments=4)

# DRAM traffic of the sampling kernel measured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum), bytes per computed sample, with the SHA-256 prefix of
# the kernel source it was measured on (source_hash).  A workload without an entry, or
# whose kernel source has changed since, reports traffic null.  Each figure is a
# query's first sampling launch, which under ncu computes every sample its ring
# admits: rmat20 2.727 GB over 31,000 samples; rmat20d (directed) 2.212 GB over
# 36,000; rmat18 0.757 GB over 31,000; hyp4m 28.79 GB over 142,000; grid2048
# 715.3 GB over 56,000 (profiles/k_sample_rmat20_dram.md,
# profiles/k_sample_rmat20d_dram.md, profiles/k_sample_hyp4m_grid2048_dram.md;
# rmat18 from the same command with --workload rmat18).
NCU_TRAFFIC_PER_SAMPLE = {
    ("k_sample", "rmat20"): (87_975, "9232d11af77f9ede"),
    ("k_sample", "rmat20d"): (61_436, "9232d11af77f9ede"),
    ("k_sample", "rmat18"): (24_431, "9232d11af77f9ede"),
    ("k_sample", "hyp4m"): (202_770, "9232d11af77f9ede"),
    ("k_sample", "grid2048"): (12_772_322, "9232d11af77f9ede"),
}
# a kernel's source file and the headers it includes (launch arguments, defaults)
KERNEL_SOURCE = {"k_sample": ("kad_sample.cu", "kad_internal.cuh", "kad_device.cuh"),
                 "k_wsample": ("kad_wsample.cu", "kad_internal.cuh", "kad_device.cuh")}


def source_hash(kernel):
    """SHA-256 prefix of the kernel's source file and its headers, in that order."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCE[kernel]:
        with open(os.path.join(ROOT, "paper_1903_09422_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic_per_sample(kernel, workload):
    """(bytes per computed sample, note): None when unmeasured or stale."""
    ent = NCU_TRAFFIC_PER_SAMPLE.get((kernel, workload))
    if ent is None:
        return None, "no ncu capture of this kernel on this workload"
    if ent[1] != source_hash(kernel):
        return None, "stale: the kernel source changed since its ncu capture"
    return ent[0], "ncu dram__bytes_read.sum + dram__bytes_write.sum per computed sample x samples computed"


def alg_bytes(counters):
    return sum(BYTES_PER[k] * int(v) for k, v in counters.items())


def phase_total(results):
    tot = {}
    for r in results:
        for k, v in r.get("phase_cycles", {}).items():
            tot[k] = tot.get(k, 0) + v
    return tot


def phase_share(results):
    """Share of the sampling blocks' cycles per stage of a sample (adaptive phase)."""
    tot = {}
    for r in results:
        for k, v in r.get("phase_cycles", {}).items():
            tot[k] = tot.get(k, 0) + v
    s = sum(tot.values()) or 1
    return {k: round(v / s, 4) for k, v in tot.items()}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms while running."""

    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        rows = []
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 10:
                continue
            if self.uuid and p[1] != self.uuid:
                continue
            rows.append(p)
        if not rows:
            return None
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup(n_gpus):
    if n_gpus <= 1 or "RANK" not in os.environ:
        return 0, 1, None
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    world = int(os.environ["WORLD_SIZE"])
    backend = "nccl"
    dist.init_process_group(backend=backend)
    return rank, world, dist


def reduce_ranks(dist, total_ms, samples, computed, device):
    """Whole-job figures of the replicas: the slowest rank's time, the samples of
    all ranks.  Without a process group the rank's own figures."""
    if not dist:
        return total_ms, samples, computed
    import torch
    t = torch.tensor([total_ms, float(samples), float(computed)], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return mx[0].item(), t[1].item(), t[2].item()


def graph_for(workload):
    from paper_1903_09422_gb300 import gen
    w = gen.WORKLOADS[workload]
    return gen.workload_graph(workload), w


def cpu_oracle_sample(g, w, budget_s=20.0):
    """Time the oracle on a bounded prefix of the same query: calibration plus the
    first k adaptive epochs, k grown until the run takes at least a few seconds."""
    import oracle
    k, best = 1, None
    while True:
        t0 = time.perf_counter()
        r = oracle.kadabra(g, w["eps"], w["delta"], w["seed"], max_epochs=k)
        dt = time.perf_counter() - t0
        best = (k, r, dt)
        if dt > budget_s / 4 or r["tau"] >= r["omega"] or k >= 64:
            break
        k *= 2
    k, r, dt = best
    samples = r["calib_samples"] + r["tau"]
    return {"value": samples / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"calibration ({r['calib_samples']} samples) + first {r['epochs']} adaptive epochs "
                      f"({r['tau']} samples) of the same query, single-threaded C, {dt:.2f} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_1903_09422_gb300 import gen
    g, w = graph_for(args.workload)
    import oracle
    oracle.build()
    # each step: calibration + one adaptive epoch of the query (the bounded sample)
    for _ in range(args.warmup):
        oracle.kadabra(g, w["eps"], w["delta"], w["seed"], max_epochs=1)
    tot, samples = 0.0, 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.kadabra(g, w["eps"], w["delta"], w["seed"], max_epochs=1)
        tot += time.perf_counter() - t0
        samples += r["calib_samples"] + r["tau"]
    v = samples / tot
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {gen.describe(args.workload)}; n={g.n} arcs={g.m}"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "per step: calibration + first adaptive epoch of the query, "
                                       "single-threaded C oracle"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _serve_graph(spec):
    from paper_1903_09422_gb300 import gen
    i, kind, n_t = spec
    if kind == 0:
        return gen.rmat(max(4, int(round(np.log2(n_t)))), 16, seed=i + 1)
    if kind == 1:
        return gen.grid(max(8, int(round(np.sqrt(n_t)))), seed=i + 1)
    return gen.hyperbolic(n_t, seed=i + 1)


def serve_graphs(count, seed=20261203, workers=8):
    """count graphs: generator = idx mod 3 (R-MAT, grid + shortcuts, hyperbolic),
    target size n = round(10^(4 + 2u)), u uniform in [0, 1) (log-uniform 1e4..1e6).
    Each graph depends only on its index; they are generated by a pool of spawned
    processes (no CUDA state is inherited)."""
    import multiprocessing as mpx
    rng = np.random.default_rng(seed)
    specs = [(i, i % 3, int(round(10 ** (4 + 2 * rng.random())))) for i in range(count)]
    if workers <= 1:
        return [_serve_graph(s) for s in specs]
    with mpx.get_context("spawn").Pool(workers) as pool:
        return pool.map(_serve_graph, specs, chunksize=1)


def open_loop(kad, graphs, workers, qg, qe, qseed, arrivals, policy=0):
    """Submit query q at arrivals[q] seconds (Poisson process) to a server with
    `workers` workers; return (makespan s, latencies ms incl. queueing, samples)."""
    import threading
    Q = len(arrivals)
    with kad.Server(workers=workers, policy=policy) as S:
        gids = [S.add_graph(g, trusted=True) for g in graphs]
        for q in range(min(5, Q)):  # warm-up
            S.wait(S.submit(gids[qg[q]], qe[q], 0.1, int(qseed[q]), want_bc=False))
        tickets = [None] * Q

        def submitter():
            start = time.perf_counter()
            for q in range(Q):
                dt = arrivals[q] - (time.perf_counter() - start)
                if dt > 0:
                    time.sleep(dt)
                tickets[q] = S.submit(gids[qg[q]], qe[q], 0.1, int(qseed[q]), want_bc=False)

        t_start = time.perf_counter()
        th = threading.Thread(target=submitter)
        th.start()
        lat, samples = [], 0
        for q in range(Q):
            while tickets[q] is None:
                time.sleep(0.0002)
            r = S.wait(tickets[q])
            lat.append(r["latency_ms"])
            samples += r["tau"] + r["calib_samples"]
        makespan = time.perf_counter() - t_start
        th.join()
    return makespan, lat, samples


def run_serve(args):
    """Serving stream: resident graphs, Poisson arrivals at several loads.  Each
    load runs the same arrival sequence twice: 'plain' (one query at a time with
    every sampling slot of the GPU, first come first served) and 'served' (the
    query server with several workers: queries overlap on the device, and the
    next query is the one with the highest response ratio)."""
    import torch
    from paper_1903_09422_gb300 import build, kad
    torch.cuda.set_device(0)
    build.build()
    t0 = time.perf_counter()
    graphs = serve_graphs(args.serve_graphs)
    gen_s = time.perf_counter() - t0
    rng = np.random.default_rng(7)
    Q = args.serve_queries
    qg = rng.integers(0, len(graphs), Q)
    qe = np.array([0.05, 0.02, 0.01])[rng.integers(0, 3, Q)]
    qseed = np.arange(1, Q + 1)

    # capacity of plain: back-to-back queries, one at a time
    plain_n = min(Q, args.serve_plain)
    with kad.Server(workers=1, policy=1) as P:
        gids = [P.add_graph(g, trusted=True) for g in graphs]
        for q in range(min(5, Q)):  # warm-up
            P.wait(P.submit(gids[qg[q]], qe[q], 0.1, int(qseed[q]), want_bc=False))
        t0 = time.perf_counter()
        for q in range(plain_n):
            P.wait(P.submit(gids[qg[q]], qe[q], 0.1, int(qseed[q]), want_bc=False))
        plain_s = time.perf_counter() - t0
    plain_qps = plain_n / plain_s

    def summary(makespan, lat, samples):
        return {"queries_per_s": Q / makespan, "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "samples_per_s": samples / makespan}

    sweep = []
    for load in [float(x) for x in args.serve_load.split(",")]:
        lam = load * plain_qps
        arrivals = np.cumsum(np.random.default_rng(11).exponential(1.0 / lam, Q))
        row = {"load": load, "arrival_qps": lam}
        row["plain"] = summary(*open_loop(kad, graphs, 1, qg, qe, qseed, arrivals, policy=1))
        row["served"] = summary(*open_loop(kad, graphs, args.serve_workers, qg, qe, qseed, arrivals, policy=0))
        print(json.dumps({"load": load, "plain": row["plain"], "served": row["served"]}), file=sys.stderr, flush=True)
        sweep.append(row)
    top = sweep[-1]
    line = {
        "metric": METRIC, "value": top["served"]["queries_per_s"], "unit": "queries/s", "n_gpus": 1, "steps": Q,
        "warmup": 5, "ms_per_step": 1000.0 / top["served"]["queries_per_s"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"serving stream: {len(graphs)} resident graphs (R-MAT / grid+shortcuts / hyperbolic, "
                               f"n log-uniform 1e4..1e6), {Q} queries per arm and load, Poisson arrivals at "
                               f"{args.serve_load} x the plain back-to-back throughput, eps in {{.05,.02,.01}}, "
                               f"delta .1, seed = query index + 1",
                   "workers": args.serve_workers, "served_policy": "highest response ratio next",
                   "plain_policy": "arrival order",
                   "value": "served queries/s at the highest load"},
        "plain_capacity_qps": plain_qps,
        "sweep": sweep,
        "graph_generation_s": gen_s,
    }
    print(json.dumps(line), flush=True)
    return 0


def serve_specs(count, seed=20261203):
    rng = np.random.default_rng(seed)
    return [(i, i % 3, int(round(10 ** (4 + 2 * rng.random())))) for i in range(count)]


# The other configured workloads (C1, C3, C4), measured in the default run like
# the main line: inputs resident in HBM, L2 flushed between queries, CUDA events
# on the launching stream, clocks sampled during the timed queries.
OTHER_WORKLOADS = ("rmat12", "grid2048", "hyp4m")


def _workload_graph(name):
    from paper_1903_09422_gb300 import gen
    return name, gen.workload_graph(name)


def workloads_record(kad, graphs, flush, uuid, steps=5, warmup=3):
    import torch
    from paper_1903_09422_gb300 import gen
    peak, peak_kind = load_peaks()
    stream = torch.cuda.current_stream()
    out = {}
    for name, g in graphs:
        w = gen.WORKLOADS[name]
        d_rp = torch.from_numpy(g.row_ptr).cuda()
        d_col = torch.from_numpy(g.col).cuda()
        d_bc = torch.empty(g.n, dtype=torch.float64, device="cuda")
        G = kad.Graph.from_device(d_rp, d_col, directed=g.directed)
        try:
            for _ in range(warmup):
                G.run_device(w["eps"], w["delta"], w["seed"], d_bc=d_bc, timing=True)
            torch.cuda.synchronize()
            clocks = ClockSampler(uuid)
            clocks.start()
            time.sleep(0.4)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            res = []
            for i in range(steps):
                flush.fill_(i & 0xff)
                ev[i][0].record(stream)
                res.append(G.run_device(w["eps"], w["delta"], w["seed"], d_bc=d_bc, timing=True))
                ev[i][1].record(stream)
            torch.cuda.synchronize()
            clk = clocks.stop()
        finally:
            G.close()
        ms = [a.elapsed_time(b) for a, b in ev]
        used = sum(r["tau"] + r["calib_samples"] for r in res)
        ab = sum(alg_bytes(r["counters"]) for r in res)
        kt = sum(r["t_ads_kernel_ms"] for r in res)
        r0 = res[-1]
        out[name] = {"workload": f"{name}: {gen.describe(name)}; n={g.n} arcs={g.m}",
                     "value": used / (sum(ms) / 1000.0), "unit": UNIT, "time_to_stop_ms": statistics.median(ms),
                     "step_ms": [round(x, 3) for x in ms], "tau": r0["tau"], "epochs": r0["epochs"],
                     "vd_bound": r0["vd_bound"], "samples_computed": int(statistics.median(r["samples_computed"] for r in res)),
                     "roofline_frac": (ab / (kt / 1000.0) / 1e9) / peak, "peak_kind": peak_kind,
                     "kernel_variant": f"{r0['block_threads_used']} threads x {r0['blocks_per_sm_used']} blocks/SM",
                     "clocks": clk}
        del d_rp, d_col, d_bc
        torch.cuda.empty_cache()
    return out


def serving_record(kad, graphs, queries=300, plain_n=150, load=4.0, workers=4):
    """A bounded sample of the serving stream for the default bench line: the
    plain arm's back-to-back capacity (one query at a time with every sampling
    slot) and its device-busy fraction (the sum of the queries' CUDA-event device
    time over the wall time: overlapping queries can raise throughput by at most
    1 / busy), then the same Poisson arrivals at `load` x that capacity, plain
    (arrival order) against served (several workers, highest response ratio)."""
    rng = np.random.default_rng(7)
    qg = rng.integers(0, len(graphs), queries)
    qe = np.array([0.05, 0.02, 0.01])[rng.integers(0, 3, queries)]
    qseed = np.arange(1, queries + 1)
    with kad.Server(workers=1, policy=1) as P:
        gids = [P.add_graph(g, trusted=True) for g in graphs]
        for q in range(min(5, queries)):
            P.wait(P.submit(gids[qg[q]], qe[q], 0.1, int(qseed[q]), want_bc=False))
        dev_ms = 0.0
        t0 = time.perf_counter()
        for q in range(plain_n):
            r = P.wait(P.submit(gids[qg[q]], qe[q], 0.1, int(qseed[q]), want_bc=False))
            dev_ms += r["t_total_ms"]
        plain_s = time.perf_counter() - t0
    cap_qps = plain_n / plain_s
    busy = dev_ms / (1000.0 * plain_s)
    arrivals = np.cumsum(np.random.default_rng(11).exponential(1.0 / (load * cap_qps), queries))

    def summary(makespan, lat, samples):
        return {"queries_per_s": queries / makespan, "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "samples_per_s": samples / makespan}

    plain = summary(*open_loop(kad, graphs, 1, qg, qe, qseed, arrivals, policy=1))
    served = summary(*open_loop(kad, graphs, workers, qg, qe, qseed, arrivals, policy=0))
    return {"workload": f"{len(graphs)} resident graphs (R-MAT / grid+shortcuts / hyperbolic, n log-uniform "
                        f"1e4..1e6), {queries} queries per arm, Poisson arrivals at {load} x plain capacity, "
                        f"eps in {{.05,.02,.01}}, delta .1 (a bounded sample of the 10,000-query stream)",
            "plain_capacity_qps": cap_qps, "plain_device_busy": busy,
            "overlap_bound": (1.0 / busy) if busy > 0 else None,
            "plain": plain, "served": served, "served_over_plain": served["queries_per_s"] / plain["queries_per_s"],
            "workers": workers}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="rmat20")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tight-vd", action="store_true", help="the double-sweep vertex-diameter bound (undirected)")
    ap.add_argument("--no-completion-order", action="store_true", help="skip the completion-order comparison")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--block-threads", type=int, default=0)
    ap.add_argument("--slots", type=int, default=0)
    ap.add_argument("--blocks-per-sm", type=int, default=0)
    ap.add_argument("--samples-per-block", type=int, default=0, help="> 0: the warp-per-sample kernel")
    ap.add_argument("--flush-mb", type=int, default=512, help="L2 flush buffer written between timed steps")
    ap.add_argument("--eps", type=float, default=None, help="override the workload's eps (experiments)")
    ap.add_argument("--serve-graphs", type=int, default=64)
    ap.add_argument("--serve-queries", type=int, default=1000, help="queries per arm and load")
    ap.add_argument("--serve-plain", type=int, default=400, help="queries timed for the one-at-a-time baseline")
    ap.add_argument("--serve-load", default="0.5,1,2,4", help="arrival rates, as multiples of plain queries/s")
    ap.add_argument("--serve-workers", type=int, default=4)
    ap.add_argument("--no-serving", action="store_true", help="skip the serving record of the default line")
    ap.add_argument("--no-other-workloads", action="store_true",
                    help="skip the record of the other configured workloads (C1, C3, C4) in the default line")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serve":
        return run_serve(args)

    # the serving record's graphs are generated by spawned processes while this
    # process builds the library and its own graph (single GPU only)
    serve_pool = serve_async = None
    if not args.no_serving and args.gpus == 1 and int(os.environ.get("WORLD_SIZE", "1")) == 1:
        import multiprocessing as mpx
        serve_pool = mpx.get_context("spawn").Pool(8)
        serve_async = serve_pool.map_async(_serve_graph, serve_specs(args.serve_graphs), chunksize=1)
    others_pool = others_async = None
    if (not args.no_other_workloads and args.workload == "rmat20" and args.gpus == 1 and
            int(os.environ.get("WORLD_SIZE", "1")) == 1):
        import multiprocessing as mpx
        others_pool = mpx.get_context("spawn").Pool(len(OTHER_WORKLOADS))
        others_async = others_pool.map_async(_workload_graph, OTHER_WORKLOADS, chunksize=1)

    import torch
    rank, world, dist = dist_setup(args.gpus)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1903_09422_gb300 import build, kad
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    kad.load()

    from paper_1903_09422_gb300 import gen
    g, w = graph_for(args.workload)
    eps, delta, seed = w["eps"], w["delta"], w["seed"]
    if args.eps:
        eps = args.eps
    opts = dict(block_threads=args.block_threads or None, slots=args.slots or None,
                blocks_per_sm=args.blocks_per_sm or None, samples_per_block=args.samples_per_block or None)
    stream = torch.cuda.current_stream()

    # the graph generators of the serving and other-workload records run on the
    # host's cores: let them finish first, so that no timed leg (the host's L
    # table inside a query, the end-to-end leg's host work) shares the host
    for pending in (serve_async, others_async):
        if pending is not None:
            pending.wait(timeout=900)

    # inputs resident in HBM before timing
    d_rp = torch.from_numpy(g.row_ptr).to(dev)
    d_col = torch.from_numpy(g.col).to(dev)
    t0 = time.perf_counter()
    G = kad.Graph.from_device(d_rp, d_col, directed=g.directed, tight_vd=args.tight_vd)
    torch.cuda.synchronize()
    setup_ms = 1000 * (time.perf_counter() - t0)
    d_bc = torch.empty(g.n, dtype=torch.float64, device=dev)
    flush = torch.empty(max(args.flush_mb, 1) << 20, dtype=torch.uint8, device=dev)

    for _ in range(args.warmup):
        G.run_device(eps, delta, seed, d_bc=d_bc, timing=True, **opts)
    torch.cuda.synchronize()

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    clocks.start()
    time.sleep(0.4)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    results = []
    for i in range(args.steps):
        flush.fill_(i & 0xff)
        ev[i][0].record(stream)
        r = G.run_device(eps, delta, seed, d_bc=d_bc, timing=True, **opts)
        ev[i][1].record(stream)
        results.append(r)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    samples = sum(r["tau"] + r["calib_samples"] for r in results)
    computed = sum(r["samples_computed"] for r in results)  # calibration + adaptive
    total_ms_all, samples_all, computed_all = reduce_ranks(dist, total_ms, samples, computed, dev)

    # ---- the same query in completion order (the non-deterministic epochs of
    # the local-/shared-frame algorithms): what determinism costs
    co = None
    if not args.no_completion_order:
        for _ in range(2):
            G.run_device(eps, delta, seed, d_bc=d_bc, flags=kad.KAD_RUN_COMPLETION_ORDER, **opts)
        co_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        co_res = []
        for i in range(args.steps):
            flush.fill_(i & 0xff)
            co_ev[i][0].record(stream)
            co_res.append(G.run_device(eps, delta, seed, d_bc=d_bc, flags=kad.KAD_RUN_COMPLETION_ORDER, **opts))
            co_ev[i][1].record(stream)
        torch.cuda.synchronize()
        co_ms = [a.elapsed_time(b) for a, b in co_ev]
        co_used = sum(r["tau"] + r["calib_samples"] for r in co_res)
        co = {"value": co_used / (sum(co_ms) / 1000.0), "unit": UNIT, "time_to_stop_ms": statistics.median(co_ms),
              "tau": [r["tau"] for r in co_res], "samples_computed": statistics.median(r["samples_computed"] for r in co_res),
              "mode": "KAD_RUN_COMPLETION_ORDER: epoch k = the (kN+1)-th..(k+1)N-th samples to complete "
                      "(non-deterministic; the headline value above is the deterministic mode)"}

    # ---- end to end through the C ABI with host buffers: pinned CSR -> graph
    # create (copy + set-up) -> run -> b~ back to pinned host memory
    h_rp = torch.from_numpy(g.row_ptr).pin_memory()
    h_col = torch.from_numpy(g.col).pin_memory()
    h_bc = torch.empty(g.n, dtype=torch.float64).pin_memory()
    lib = kad.load()
    import ctypes
    e2e_times, e2e_samples = [], 0
    for i in range(args.e2e_steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = ctypes.c_void_p()
        gflags = (kad.KAD_GRAPH_DIRECTED if g.directed else 0) | (kad.KAD_GRAPH_TIGHT_VD if args.tight_vd else 0)
        st = lib.kad_graph_create(g.n, h_rp.data_ptr(), h_col.data_ptr(), gflags, stream.cuda_stream, ctypes.byref(h))
        if st != 0:
            raise kad.KadError(st, "kad_graph_create")
        res = kad.Result()
        res.bc = h_bc.data_ptr()
        o = kad.options(**opts)
        st = lib.kad_run(h, eps, delta, seed, stream.cuda_stream, ctypes.byref(o), ctypes.byref(res))
        lib.kad_graph_free(h)
        if st != 0:
            raise kad.KadError(st, "kad_run")
        dt = time.perf_counter() - t0
        if i > 0:  # first call warms the allocator
            e2e_times.append(dt)
            e2e_samples += res.tau + res.calib_samples
    e2e_value = e2e_samples / sum(e2e_times)
    if dist:
        t = torch.tensor([e2e_value], dtype=torch.float64, device=dev)
        dist.all_reduce(t)
        e2e_value = t.item()

    # ---- roofline of the dominant kernel (adaptive-phase sampling launch)
    peak, peak_kind = load_peaks()
    ab = [alg_bytes(r["counters"]) for r in results]
    kt = [r["t_ads_kernel_ms"] for r in results]
    achieved = sum(ab) / (sum(kt) / 1000.0) / 1e9
    per_sample = sum(ab) / max(1, sum(r["samples_computed"] for r in results))
    traffic = None
    tps, traffic_note = ncu_traffic_per_sample("k_wsample" if args.samples_per_block else "k_sample", args.workload)
    if tps is not None:
        traffic = tps * statistics.mean(r["samples_computed"] for r in results)
    # DRAM bytes actually moved per second, from the ncu traffic (a separate
    # figure: the headline fraction is the algorithmic bytes' rate)
    dram_gbs = traffic / (statistics.mean(kt) / 1000.0) / 1e9 if traffic is not None else None
    r0 = results[-1]
    scanned = sum(r["counters"]["scanned"] for r in results)

    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            try:
                cpu = cpu_oracle_sample(g, w)
            except Exception as ex:  # the baseline must not sink the bench line
                cpu = {"error": str(ex)}
        line = {
            "metric": METRIC, "value": samples_all / (total_ms_all / 1000.0), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms_all / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {gen.describe(args.workload)}; n={g.n} arcs={g.m}",
                       "step": "one full KADABRA query (calibration + adaptive sampling to stop + b~)",
                       "l2": f"flushed between steps ({args.flush_mb} MB write)", "parallelism": f"replicas x{world}",
                       "vd_bound": "double sweep (KAD_GRAPH_TIGHT_VD)" if args.tight_vd else "2 ecc(v0) + 1"},
            "time_to_stop_ms": statistics.median(step_ms),
            "step_ms": [round(x, 3) for x in step_ms],
            "time_to_stop_ads_ms": statistics.median(r["t_ads_ms"] for r in results),
            "samples_computed_per_s": computed_all / (total_ms_all / 1000.0),
            "samples_computed": int(statistics.median(r["samples_computed"] for r in results)),
            "tau": r0["tau"], "calib_samples": r0["calib_samples"], "epochs": r0["epochs"], "omega": r0["omega"],
            "vd_bound": r0["vd_bound"], "stopped_by_omega": r0["stopped_by_omega"],
            "algorithmic_teps": scanned / (sum(kt) / 1000.0),
            "graph_setup_ms": setup_ms,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "traffic_note": traffic_note,
                         "dram_gbs": dram_gbs, "dram_frac": (dram_gbs / peak) if dram_gbs is not None else None,
                         "kernel": ("k_wsample" if r0.get("samples_per_block_used") else "k_sample") +
                                   " (calibration + adaptive phase, one persistent launch)",
                         "alg_bytes_per_sample": per_sample, "peak_kind": f"{peak_kind} (hbm_gbs burst)",
                         "kernel_ms": statistics.median(kt)},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(4 * (g.n + 1) + 4 * g.m),
                    "d2h_bytes_per_step": int(8 * g.n), "steps": args.e2e_steps,
                    "ms_per_step": 1000 * statistics.mean(e2e_times),
                    "step_ms": [round(1000 * t, 3) for t in e2e_times]},
            "phase_share": phase_share(results),
            "phase_cycles_per_sample": {k: round(v / max(1, sum(r["samples_computed"] for r in results)))
                                        for k, v in phase_total(results).items()},
            "kernel_variant": (f"warp per sample: {r0['samples_per_block_used']} samples per block of 1024 threads, "
                               f"{r0['slots_used']} slots") if r0.get("samples_per_block_used") else
                              (f"{r0['block_threads_used']} threads x {r0['blocks_per_sm_used']} blocks/SM, "
                               f"{r0['slots_used']} slots"),
            "gpu_launches": int(sum(r["kernel_launches"] for r in results)),
            "clocks": clk,
            "completion_order": co,
            "cpu_baseline": cpu,
        }
        if others_async is not None:
            try:
                line["other_workloads"] = workloads_record(kad, others_async.get(timeout=900), flush, uuid)
            except Exception as ex:  # the record must not sink the bench line
                line["other_workloads"] = {"error": str(ex)}
            finally:
                others_pool.close()
        if serve_async is not None:
            try:
                graphs = serve_async.get(timeout=900)
                line["serving"] = serving_record(kad, graphs, workers=args.serve_workers)
            except Exception as ex:  # the record must not sink the bench line
                line["serving"] = {"error": str(ex)}
            finally:
                serve_pool.close()
        print(json.dumps(line), flush=True)
    G.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
