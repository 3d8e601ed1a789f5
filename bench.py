#!/usr/bin/env python3
"""Skipper maximal matching benchmark on GB300.

Workload (default): plain Skipper on an R-MAT graph of scale 27, edge factor
16 (a = 0.57, b = c = 0.19, d = 0.05), vertex ids permuted, symmetrised and
de-duplicated, stored as a uint32 CSR with int64 offsets -- a seeded
synthetic stand-in for the paper's large power-law graphs (Section VI-A,
Table I).  One step is one full Skipper pass through the C ABI: state
initialisation + merge-path partition, then the single sweep over all
entries (Algorithm 1).  The metric is GEdges/s with edges counted as stored
CSR entries (Table I's |E| counts the symmetrised graph's entries).

Launch: ``python bench.py [--gpus N --steps K --warmup W]``; for N > 1 under
torchrun every rank runs an independent replica on its own GPU (one graph's
pass does not shard, and batches of independent graphs would shard without
any exchange), and the job value is all ranks' entries over the slowest
rank's time.  ``--impl reference`` times the oracle (single-thread
sequential greedy MM in C) on a bounded sample of the same graph on the host
cores instead.  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GEdges/s Skipper MM at RMAT-27 (% HBM roofline); batched p50/p99 vs plain"
UNIT = "GEdges/s"


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def parse():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--scale", type=int, default=27)
    ap.add_argument("--graph", choices=["rmat", "uniform", "skew"], default="rmat",
                    help="the timed graph: R-MAT (.57/.19/.19/.05, the headline), uniform random pairs, "
                         "or high-skew R-MAT (.7/.1/.1/.1); edge-factor x 2^scale draws each")
    ap.add_argument("--edge-factor", type=int, default=16)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--bits", type=int, default=8, choices=[2, 8, 32])
    ap.add_argument("--grain", type=int, default=8192)
    ap.add_argument("--block", type=int, default=512)
    ap.add_argument("--blocks-per-sm", type=int, default=0,
                    help="mm_options.blocks_per_sm of the timed sweep (0 = the layout's default)")
    ap.add_argument("--stage-windows", action="store_true",
                    help="mm_options.stage_windows = 1 for the timed sweep (opt-in TMA window tiles)")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--e2e-grain", type=int, default=0,
                    help="grain of the end-to-end runs; 0 = the library's choice for the handle "
                         "(larger units for a CSR read in place over the host link)")
    ap.add_argument("--e2e-pieces", type=int, default=0,
                    help="launches whose finished mate prefixes are copied back while the pass runs "
                         "(mm_skipper_to_host); 0 = one launch, then one copy")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="approximate host seconds for the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-edge-list", action="store_true")
    ap.add_argument("--no-side-graphs", action="store_true",
                    help="skip the uniform and high-skew graphs of the headline's size")
    ap.add_argument("--side-steps", type=int, default=10)
    ap.add_argument("--layout-steps", type=int, default=20,
                    help="steps for the headline graph in the 2- and 32-bit layouts (0 = skip)")
    ap.add_argument("--served-in-place-max-nnz", type=int, default=1 << 20)
    ap.add_argument("--symmetric-steps", type=int, default=50)
    ap.add_argument("--edge-list-steps", type=int, default=20)
    ap.add_argument("--edge-list-bits", type=int, default=2)
    ap.add_argument("--batch-graphs", type=int, default=4096)
    ap.add_argument("--batch-reps", type=int, default=20)
    ap.add_argument("--batched-only", action="store_true",
                    help="run the batched workload alone, without its one-call-per-graph arm, and print "
                         "its object (for profiling the batch sweep)")
    ap.add_argument("--batch-opts", default="",
                    help="grain,status_bits,blocks_per_sm,unit_order,warps_per_graph for the batch "
                         "instead of the autotuner's pick")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--served-rate", type=float, default=2000.0, help="Poisson arrivals per second")
    ap.add_argument("--served-seconds", type=float, default=4.0)
    ap.add_argument("--served-pool", type=int, default=16)
    ap.add_argument("--served-min-edges", type=float, default=1e4)
    ap.add_argument("--served-max-edges", type=float, default=2e8)
    return ap.parse_args()


# ----------------------------------------------------------------------------
# helpers
# ----------------------------------------------------------------------------
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, dist=None) -> float:
    """Largest value of x over all ranks (x itself without a process group);
    CUDA tensors under NCCL, host tensors under gloo."""
    if dist is None or not dist.is_initialized():
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gedges(world: int, entries_per_rank: int, seconds: float) -> float:
    """Whole-job GEdges/s: every rank's entries over the slowest rank's time."""
    return world * entries_per_rank / seconds / 1e9


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash(files=("state.cuh", "walk.cuh", "sweep.cu")) -> str:
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2507_04420_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


COO_SOURCES = ("state.cuh", "walk.cuh", "coo.cu")


def ncu_traffic(workload: str, bits: int, prefix: str = "sweep", files=None):
    """DRAM bytes per sweep launch from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", f"{prefix}_u{bits}_{workload}.md")
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    src = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    val = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    want = kernel_source_hash(files) if files else kernel_source_hash()
    if not src or not val or src.group(1) != want:
        return None
    return float(val.group(1))


class Clocks:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "50"]
            if self.uuid:
                cmd += ["-i", self.uuid]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception as e:  # no nvidia-smi: report what we know
            log("clock sampling unavailable:", e)
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9], parts[4]))
            except ValueError:
                continue
        os.remove(self.path)
        if not rows:
            return out
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        out.update(sm_mhz=statistics.median(r[0] for r in rows), sm_max_mhz=max(r[1] for r in rows),
                   reasons=reasons, samples=len(rows))
        return out


def make_graph(args, device):
    import graphgen as gg
    import torch
    # source-range chunks bound the CSR build's temporaries (same output for any count)
    chunks = (16 << max(0, args.scale - 27)) if args.scale >= 26 else 1
    t = time.time()
    if args.graph == "uniform":
        g = gg.uniform(1 << args.scale, args.edge_factor << args.scale, seed=args.seed, device=device,
                       chunks=chunks)
    else:
        a, b, c = (0.7, 0.1, 0.1) if args.graph == "skew" else (0.57, 0.19, 0.19)
        g = gg.rmat(args.scale, args.edge_factor, a, b, c, seed=args.seed, device=device, chunks=chunks)
    if device != "cpu":
        torch.cuda.synchronize()
    log(f"{args.graph}{args.scale}: n={g.n} nnz={g.nnz} generated in {time.time() - t:.1f}s")
    if device != "cpu":
        torch.cuda.empty_cache()  # hand the generator's temporaries back
    return g


def workload_config(args, g):
    if args.graph == "uniform":
        name = f"uniform{args.scale}_ef{args.edge_factor}"
        desc = (f"{args.edge_factor} x 2^{args.scale} uniform random pairs on 2^{args.scale} vertices, loops "
                "and repeats dropped, symmetrised; uint32 ids, int64 offsets")
    else:
        skew = args.graph == "skew"
        name = f"rmat{args.scale}_ef{args.edge_factor}" + ("_skew" if skew else "")
        desc = (f"R-MAT scale {args.scale}, edge factor {args.edge_factor}, a/b/c/d="
                + (".7/.1/.1/.1" if skew else ".57/.19/.19/.05")
                + ", ids permuted, symmetrised, deduplicated; uint32 ids, int64 offsets")
    return {
        "workload": name, "graph": desc,
        "n": g.n, "nnz": g.nnz, "m_undirected": g.nnz // 2, "seed": args.seed,
        "edges_counted": "stored CSR entries (both directions)",
    }


def cpu_sample(off_np, nb_np, seconds):
    """Time the oracle on rows [0, R) of the graph, R sized to about `seconds`."""
    import oracle
    n = off_np.size - 1
    # calibration on a small prefix
    r = int(min(n, max(1024, n // 512)))
    _, sec, ent = oracle.sgmm_rows_timed(off_np, nb_np, r)
    rate = ent / max(sec, 1e-6)
    target_entries = rate * seconds
    import numpy as np
    R = int(min(n, np.searchsorted(off_np, target_entries)))
    R = max(R, r)
    _, sec, ent = oracle.sgmm_rows_timed(off_np, nb_np, R)
    return {"rows": R, "entries": ent, "seconds": sec, "gedges_s": ent / sec / 1e9}


# ----------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# ----------------------------------------------------------------------------
def skipper_cpu_sample(off_np, nb_np, threads, row_skip, seconds):
    """Algorithm 1 on host threads over rows [0, R), R sized to about `seconds`,
    with SGMM timed over the same rows."""
    import numpy as np
    import oracle
    n = off_np.size - 1
    r = int(min(n, max(4096, n // 256)))
    _, sec, _ = oracle.cpu_skipper(off_np, nb_np, threads, row_skip, rows=(0, r))
    rate = int(off_np[r]) / max(sec, 1e-6)
    R = int(min(n, max(r, np.searchsorted(off_np, rate * seconds))))
    _, sec, cnf = oracle.cpu_skipper(off_np, nb_np, threads, row_skip, rows=(0, R))
    _, sgmm_sec, ent = oracle.sgmm_rows_timed(off_np, nb_np, R)
    return {"threads": threads, "row_skip": bool(row_skip), "rows": R, "entries": ent,
            "seconds": sec, "gedges_s": ent / sec / 1e9, "failed_cas": cnf,
            "sgmm_seconds_same_rows": sgmm_sec}


def run_reference(args):
    import numpy as np
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import torch
    device = "cuda" if torch.cuda.is_available() else "cpu"
    g = make_graph(args, device)
    off = g.offsets.cpu().numpy()
    nb = g.nbrs.cpu().numpy()
    cfg = workload_config(args, g)
    del g
    per_step = max(0.05, min(10.0, 150.0 / max(1, args.steps + args.warmup)))
    import oracle
    cal = cpu_sample(off, nb, per_step)
    R = cal["rows"]
    times = []
    ent = cal["entries"]
    for i in range(args.warmup + args.steps):
        _, sec, ent = oracle.sgmm_rows_timed(off, nb, R)
        if i >= args.warmup:
            times.append(sec)
    med = statistics.median(times)
    value = ent / med / 1e9
    sample = (f"single-thread SGMM over rows [0, {R}) of the same graph: {ent} of {nb.size} entries "
              f"({100.0 * ent / max(nb.size, 1):.1f}%), median of {len(times)} runs")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": med * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
# batched: many independent graphs in one launch vs one launch per graph
# ----------------------------------------------------------------------------
def pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, int(round(q / 100.0 * (len(xs) - 1))))]


def batch_profile_name(G: int, o) -> str:
    """Workload part of the committed ncu summary for a batch launch configuration."""
    order = {1: "ascending", 2: "dispersed"}.get(o.unit_order, "auto")
    return f"c4batch{G}_g{o.grain}_b{o.blocks_per_sm}_{order}_w{o.warps_per_graph}"


def run_batched(args, skp, plain=True):
    import graphgen as gg
    import torch
    t = time.time()
    packed, kinds = gg.batch_packed(args.batch_graphs, 1e3, 1e6, seed=args.seed + 100, device="cuda",
                                    chunks=4)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    G = args.batch_graphs
    csr = packed.csr
    log(f"batch: {G} graphs, n={csr.n} nnz={csr.nnz} generated in {time.time() - t:.1f}s")
    out = {"workload": f"{G} graphs, undirected edges log-uniform in [1e3, 1e6], ER / R-MAT "
                       "(ef 8-32) / 2-D grid in turn, packed block-diagonally with global ids",
           "graphs": G, "n": csr.n, "nnz": csr.nnz}
    mate = torch.empty(csr.n, dtype=torch.int32, device="cuda")
    peak, peak_kind = measured_peaks()
    sweep_bytes = 8 * (csr.n + 1) + 4 * csr.nnz
    with skp.Graph(csr.offsets, csr.nbrs) as h:
        t0 = time.perf_counter()
        if args.batch_opts:
            gr, bi, bp, uo, wp = (int(x) for x in args.batch_opts.split(","))
            tuned = skp.options(grain=gr, status_bits=bi, block_threads=512, blocks_per_sm=bp,
                                unit_order=uo, warps_per_graph=wp)
        else:
            tuned = h.autotune_batched(packed.vbase, packed.ebase)
        tune_s = time.perf_counter() - t0
        tuned.use_graph = 1
        out["tuned"] = {"grain": tuned.grain, "status_bits": tuned.status_bits,
                        "block_threads": tuned.block_threads, "blocks_per_sm": tuned.blocks_per_sm,
                        "unit_order": {1: "ascending", 2: "dispersed"}.get(tuned.unit_order, "auto"),
                        "warps_per_graph": tuned.warps_per_graph, "autotune_seconds": tune_s,
                        "searched": "grain {1024,2048,4096,8192} x status_bits {2,8,32} x blocks per SM "
                                    "{40-register instance, 32-register instance} (512 threads) x unit order "
                                    "{ascending, dispersed} x warps_per_graph {0 (no cap),4,16}; every new "
                                    "best checked"}
        for _ in range(3):
            h.batched(packed.vbase, packed.ebase, mate=mate, opts=tuned)
        lat = []
        for _ in range(args.batch_reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h.batched(packed.vbase, packed.ebase, mate=mate, opts=tuned)   # waits for its status
            lat.append((time.perf_counter() - t0) * 1e3)
        v = h.validate(mate)
        if v.flags != 0:
            raise SystemExit(f"invalid batched matching: {v.as_dict()}")
        # kernel times of the same launches outside the graph (CUDA events per kernel)
        o_t = skp.options(status_bits=tuned.status_bits, grain=tuned.grain, block_threads=tuned.block_threads,
                          blocks_per_sm=tuned.blocks_per_sm, warps_per_graph=tuned.warps_per_graph,
                          unit_order=tuned.unit_order, timing=1, nosync=1)
        for _ in range(3):
            h.batched(packed.vbase, packed.ebase, mate=mate, opts=o_t)
        h.sync()
        h.timing_history()
        for _ in range(10):
            h.batched(packed.vbase, packed.ebase, mate=mate, opts=o_t)
        h.sync()
        hist = h.timing_history(256)
        sweep_ms = statistics.mean(t["sweep_ms"] for t in hist)
        init_ms = statistics.mean(t["init_ms"] for t in hist)
        achieved = sweep_bytes / (sweep_ms * 1e-3) / 1e9
        out.update(p50_ms=pct(lat, 50), p99_ms=pct(lat, 99),
                   gedges_s=csr.nnz / (pct(lat, 50) * 1e-3) / 1e9, launches_per_batch=3 if tuned.warps_per_graph else 2,
                   kernel_ms={"init": init_ms, "sweep": sweep_ms},
                   roofline={"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak,
                             "traffic": ncu_traffic(batch_profile_name(G, tuned), tuned.status_bits),
                             "bytes_per_launch": sweep_bytes,
                             "kernel": "sweep over the packed batch", "peak_kind": f"{peak_kind} hbm_gbs (burst copy)",
                             "step_frac": sweep_bytes / (pct(lat, 50) * 1e-3) / 1e9 / peak},
                   how="mm_skipper_batched, CUDA graph replay, host wall time per batch incl. status read")
        if args.batch_opts:
            out["tuned"]["searched"] = "fixed by --batch-opts"
    if not plain:
        return out
    # one mm_skipper launch sequence per graph, same data (local ids)
    parts = [gg.unpack(packed, g) for g in range(G)]
    mates = [torch.empty(p.n, dtype=torch.int32, device="cuda") for p in parts]
    handles = [skp.Graph(p.offsets, p.nbrs, check=False) for p in parts]
    def plain_replay(opts):
        """The 4096 calls captured once into a CUDA graph and replayed: one launch
        sequence per graph with no host work between them (median of 3, ms)."""
        for hg, m in zip(handles, mates):
            hg.skipper(mate=m, opts=opts)
        torch.cuda.synchronize()
        cg = torch.cuda.CUDAGraph()
        s_cap = torch.cuda.Stream()
        s_cap.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s_cap):
            with torch.cuda.graph(cg, stream=s_cap):
                for hg, m in zip(handles, mates):
                    hg.skipper(mate=m, opts=opts)
        torch.cuda.synchronize()
        cg.replay()
        torch.cuda.synchronize()
        rt = []
        for _ in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            cg.replay()
            e1.record()
            torch.cuda.synchronize()
            rt.append(e0.elapsed_time(e1))
        del cg
        return statistics.median(rt)

    # the plain arm gets its own settings: the grain and state layout that make
    # one call per graph fastest (a batch-sized grain leaves a small graph to a
    # few warps)
    search = {}
    for grain in (128, 512, 2048, 8192):
        for bits in (2, 8):
            o_try = skp.options(status_bits=bits, grain=grain, block_threads=512, nosync=1)
            try:
                search[f"grain{grain}_u{bits}"] = plain_replay(o_try)
            except Exception as e:   # capture refused: no replay figures
                log("plain arm graph capture failed:", e)
                torch.cuda.synchronize()
                break
    best_key = min(search, key=search.get) if search else None
    if best_key:
        gbest, bbest = int(best_key[5:best_key.index("_")]), int(best_key[best_key.index("_u") + 2:])
    else:
        gbest, bbest = 512, tuned.status_bits
    o = skp.options(status_bits=bbest, grain=gbest, block_threads=512, nosync=1)
    replay = search.get(best_key) if best_key else None
    for hg, m in zip(handles, mates):
        hg.skipper(mate=m, opts=o)
    torch.cuda.synchronize()
    lat, span = [], []
    for _ in range(max(3, args.batch_reps // 4)):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record()
        for hg, m in zip(handles, mates):
            hg.skipper(mate=m, opts=o)
        e1.record()
        for hg in handles:
            hg.sync()
        lat.append((time.perf_counter() - t0) * 1e3)
        torch.cuda.synchronize()
        span.append(e0.elapsed_time(e1))
    bad = sum(handles[g].validate(mates[g]).flags != 0 for g in range(0, G, max(1, G // 64)))
    if bad:
        raise SystemExit("invalid per-graph matching")
    for hg in handles:
        hg.close()
    out.update(plain_p50_ms=pct(lat, 50), plain_p99_ms=pct(lat, 99),
               plain_gedges_s=csr.nnz / (pct(lat, 50) * 1e-3) / 1e9,
               plain_device_span_ms=statistics.median(span),
               plain_graph_replay_ms=replay,
               plain_settings={"grain": gbest, "status_bits": bbest, "block_threads": 512,
                               "replay_ms_by_setting": search},
               plain_how="one mm_skipper call per graph (nosync; init + sweep launches and a 4-byte "
                         "status copy each, grids sized to the graph), then one status read per graph, "
                         "with the grain and layout that make the replayed loop fastest; wall = host "
                         "time of the loop; device span = CUDA events around the launches; graph replay "
                         "= the same calls captured once into a CUDA graph (no host work between "
                         "launches)",
               speedup_vs_plain=pct(lat, 50) / out["p50_ms"],
               speedup_vs_plain_device_span=statistics.median(span) / out["p50_ms"],
               speedup_vs_plain_graph_replay=(replay / out["p50_ms"]) if replay else None)
    return out


# ----------------------------------------------------------------------------
# the other scale-27 graphs: uniform and high-skew R-MAT, every state layout
# ----------------------------------------------------------------------------
def time_sweep(h, mate, opts, steps, warmup):
    """Device time per call and mean init / sweep kernel times of `steps`
    back-to-back calls (CUDA events on the launching stream)."""
    import torch
    for _ in range(max(3, warmup)):
        h.skipper(mate=mate, opts=opts)
    h.sync()
    h.timing_history()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        h.skipper(mate=mate, opts=opts)
    e1.record()
    torch.cuda.synchronize()
    h.sync()
    hist = h.timing_history(256)
    return (e0.elapsed_time(e1) / steps, statistics.mean(t["sweep_ms"] for t in hist),
            statistics.mean(t["init_ms"] for t in hist))


def run_side_graphs(args, skp, m_headline):
    """Config C3's companions of the headline graph: a uniform random graph with
    the same n and edge draws, and a high-skew R-MAT (a = .7, b = c = d = .1),
    each timed in the byte, 2-bit and 32-bit state layouts (and the 2-bit
    layout with symmetric = 1), with the same roofline arithmetic as the
    headline line."""
    import graphgen as gg
    import torch
    scale, ef = args.scale, args.edge_factor
    n = 1 << scale
    chunks = (16 << max(0, scale - 27)) if scale >= 26 else 1
    peak, peak_kind = measured_peaks()
    gens = {
        f"uniform{scale}": (lambda: gg.uniform(n, m_headline, seed=args.seed, device="cuda", chunks=chunks),
                            f"{m_headline} uniform random pairs on 2^{scale} vertices (the headline R-MAT's n "
                            "and undirected m), loops and repeats dropped, symmetrised"),
        f"rmat{scale}_skew": (lambda: gg.rmat(scale, ef, 0.7, 0.1, 0.1, seed=args.seed, device="cuda",
                                              chunks=chunks),
                              f"R-MAT scale {scale}, edge factor {ef}, a/b/c/d=.7/.1/.1/.1, ids permuted, "
                              "symmetrised, deduplicated"),
    }
    out = {}
    for name, (gen, desc) in gens.items():
        t = time.time()
        g = gen()
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        log(f"{name}: n={g.n} nnz={g.nnz} generated in {time.time() - t:.1f}s")
        sweep_bytes = 8 * (g.n + 1) + 4 * g.nnz
        res = {"workload": desc, "n": g.n, "nnz": g.nnz, "grain": args.grain, "block_threads": args.block,
               "l2": "inputs larger than L2 (CSR %.1f GB); no flush" % (sweep_bytes / 1e9), "layouts": {}}
        mate = torch.empty(g.n, dtype=torch.int32, device="cuda")
        with skp.Graph(g.offsets, g.nbrs, check=True) as h:
            for bits, sym, order in ((8, 0, 0), (2, 0, 0), (32, 0, 0), (2, 1, 0), (8, 0, 2)):
                o = skp.options(status_bits=bits, grain=args.grain, block_threads=args.block, nosync=1,
                                timing=1, symmetric=sym, unit_order=order)
                ms, sweep_ms, init_ms = time_sweep(h, mate, o, args.side_steps, args.warmup)
                v = h.validate(mate)
                if v.flags != 0:
                    raise SystemExit(f"invalid matching on {name} (bits {bits}): {v.as_dict()}")
                s = {2: 0.25, 8: 1.0, 32: 4.0}[bits]
                step_bytes = int(8 * (g.n + 1) + 4 * g.nnz + s * g.n + (4 * g.n if bits != 32 else 0))
                achieved = sweep_bytes / (sweep_ms * 1e-3) / 1e9
                res["layouts"][f"u{bits}" + ("_symmetric" if sym else "") + ("_dispersed" if order == 2 else "")] = {
                    "ms_per_step": ms, "sweep_ms": sweep_ms, "init_ms": init_ms,
                    "value": g.nnz / (ms * 1e-3) / 1e9, "unit": UNIT,
                    "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                                 "frac": achieved / peak,
                                 "traffic": None if (sym or order) else ncu_traffic(name, bits),
                                 "bytes_per_launch": sweep_bytes,
                                 "kernel": f"sweep_kernel<{ {2: 'TwoBit', 8: 'Byte', 32: 'Word'}[bits]}State>",
                                 "peak_kind": f"{peak_kind} hbm_gbs (burst copy)",
                                 "step_bytes_alg": step_bytes,
                                 "step_frac": step_bytes / (ms * 1e-3) / 1e9 / peak},
                    "verdict": {"flags": v.flags, "n_pairs": v.n_pairs}}
            # the library's single-graph autotuner on this graph, then the same timing
            t0 = time.time()
            o_at = h.autotune()
            at_s = time.time() - t0
            o_at.nosync, o_at.timing = 1, 1
            ms, sweep_ms, init_ms = time_sweep(h, mate, o_at, args.side_steps, args.warmup)
            v = h.validate(mate)
            if v.flags != 0:
                raise SystemExit(f"invalid matching on {name} (autotuned): {v.as_dict()}")
            achieved = sweep_bytes / (sweep_ms * 1e-3) / 1e9
            res["layouts"]["autotuned"] = {
                "ms_per_step": ms, "sweep_ms": sweep_ms, "init_ms": init_ms,
                "value": g.nnz / (ms * 1e-3) / 1e9, "unit": UNIT,
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": None, "bytes_per_launch": sweep_bytes,
                             "peak_kind": f"{peak_kind} hbm_gbs (burst copy)"},
                "verdict": {"flags": v.flags, "n_pairs": v.n_pairs},
                "settings": {"status_bits": o_at.status_bits, "grain": o_at.grain,
                             "blocks_per_sm": o_at.blocks_per_sm,
                             "unit_order": {1: "ascending", 2: "dispersed"}.get(o_at.unit_order, "auto"),
                             "autotune_seconds": at_s}}
            h.skipper(mate=mate, status_bits=8, grain=args.grain, block_threads=args.block, stats=1)
            st = h.stats()
            res["stats_u8"] = {k: st[k] for k in ("entries_read", "windows", "chunks", "attempts", "matches",
                                                   "conflicts", "id_loads", "id_loads_open")}
            res["stats_u8"]["ids_read_frac"] = st["entries_read"] / max(1, g.nnz)
        best = max(res["layouts"].items(), key=lambda kv: kv[1]["value"])
        res["best_layout"] = best[0]
        out[name] = res
        del g, mate
        torch.cuda.empty_cache()
    return out


# ----------------------------------------------------------------------------
# served: Poisson request stream through the continuous-batching server
# ----------------------------------------------------------------------------
# ----------------------------------------------------------------------------
# edge-list input (Section V-C): the raw R-MAT draws as a coordinate list
# ----------------------------------------------------------------------------
def run_edge_list(args, skp):
    import torch
    import graphgen as gg
    n = 1 << args.scale
    src, dst = gg.rmat_edges(args.scale, args.edge_factor << args.scale, .57, .19, .19, args.seed, "cuda")
    m = src.numel()
    bits = args.edge_list_bits
    mate = torch.empty(n, dtype=torch.int32, device="cuda")
    out = {"workload": f"rmat{args.scale}_ef{args.edge_factor} raw generator draws as an edge list "
                       f"(each draw once, repeats and loops kept, no symmetrisation)",
           "n": n, "m": m, "status_bits": bits, "grain": args.grain, "block_threads": args.block}
    with skp.EdgeList(n, src, dst, check=True) as h:
        h.skipper(mate=mate, status_bits=bits, grain=args.grain, block_threads=args.block)
        v = h.validate(mate)
        if v.flags != 0:
            raise SystemExit(f"invalid edge-list matching: {v.as_dict()}")
        o = skp.options(status_bits=bits, grain=args.grain, block_threads=args.block, nosync=1, timing=1)
        for _ in range(max(3, args.warmup)):
            h.skipper(mate=mate, opts=o)
        h.sync()
        h.timing_history()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(args.edge_list_steps):
            h.skipper(mate=mate, opts=o)
        ev1.record()
        torch.cuda.synchronize()
        h.sync()
        ms = ev0.elapsed_time(ev1) / args.edge_list_steps
        hist = h.timing_history(256)
        sweep_ms = statistics.mean(t["sweep_ms"] for t in hist)
        v = h.validate(mate)
        if v.flags != 0:
            raise SystemExit(f"invalid edge-list matching after timing: {v.as_dict()}")
        h.skipper(mate=mate, status_bits=bits, grain=args.grain, block_threads=args.block, stats=1)
        st = h.stats()
    peak, peak_kind = measured_peaks()
    sweep_bytes = 8 * m                     # every listed edge read once
    achieved = sweep_bytes / (sweep_ms * 1e-3) / 1e9
    out.update({
        "ms_per_step": ms, "sweep_ms": sweep_ms, "gedges_s": m / (ms * 1e-3) / 1e9,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": ncu_traffic(f"rmat{args.scale}_raw", bits, "coo_sweep", COO_SOURCES),
                     "bytes_per_launch": sweep_bytes,
                     "kernel": f"coo_sweep_kernel<{ {2: 'TwoBit', 8: 'Byte', 32: 'Word'}[bits]}State>",
                     "peak_kind": f"{peak_kind} hbm_gbs (burst copy)",
                     "note": "bound in practice by L2 requests for the random line-10 state reads"},
        "verdict": {"flags": v.flags, "n_pairs": v.n_pairs},
        "stats": {k: st[k] for k in ("attempts", "matches", "conflicts", "conflicted_entries", "max_conflicts")},
        "l2": "inputs larger than L2 (%.1f GB listed edges); no flush" % (sweep_bytes / 1e9),
    })
    del src, dst, mate
    torch.cuda.empty_cache()
    return out


def run_served(args, skp, min_edges=None, max_edges=None, seconds=None, rate=None, serial=True):
    import math
    import numpy as np
    import torch
    import graphgen as gg
    from paper_2507_04420_gb300.server import Server
    t = time.time()
    P = args.served_pool
    min_edges = args.served_min_edges if min_edges is None else min_edges
    max_edges = args.served_max_edges if max_edges is None else max_edges
    seconds = args.served_seconds if seconds is None else seconds
    rate = args.served_rate if rate is None else rate
    lo, hi = math.log(min_edges), math.log(max_edges)
    pool = []
    for i in range(P):   # stratified log-uniform sizes, R-MAT and uniform graphs in turn
        m = int(math.exp(lo + (i + 0.5) / P * (hi - lo)))
        if i % 2 == 0:
            scale = max(4, int(round(math.log2(max(m / 16, 16)))))
            g = gg.rmat(scale, max(1, m >> scale), seed=args.seed + 300 + i, device="cuda")
        else:
            g = gg.uniform(max(16, m // 8), m, seed=args.seed + 300 + i, device="cuda")
        pool.append((g.offsets.cpu().pin_memory(), g.nbrs.cpu().pin_memory(), g.n, g.nnz))
        del g
    torch.cuda.empty_cache()
    rng = np.random.default_rng(args.seed + 400)
    gaps = rng.exponential(1.0 / rate, size=int(rate * seconds * 2) + 16)
    times = np.cumsum(gaps)
    times = times[times < seconds]
    picks = rng.integers(0, P, size=times.size)
    entries = int(sum(pool[p][3] for p in picks))
    log(f"served: pool of {P} graphs ({sum(x[3] for x in pool)} entries) in {time.time() - t:.1f}s; "
        f"{times.size} requests over {seconds}s")
    out = {"workload": f"Poisson arrivals {rate:g}/s for {seconds:g}s; each request "
                       f"one of {P} pre-generated graphs (R-MAT / uniform in turn, undirected edges "
                       f"log-uniform in [{min_edges:g}, {max_edges:g}]) held in "
                       "pinned host memory", "requests": int(times.size), "entries": entries}

    def run_trace(submit, finish):
        t0 = time.perf_counter()
        for tt, p in zip(times, picks):
            now = time.perf_counter() - t0
            if tt > now:
                time.sleep(tt - now)
            submit(p, t0 + tt)
        return t0, finish()

    srv = Server(status_bits=args.bits, grain=2048, in_place_max_nnz=args.served_in_place_max_nnz)
    outs = [torch.empty(x[2], dtype=torch.int32, pin_memory=True) for x in pool]  # result buffers, reused
    reqs = []      # (request, scheduled arrival): latency counts from the schedule, as in the serial run
    t0, _ = run_trace(lambda p, at: reqs.append((srv.submit(pool[p][0], pool[p][1], outs[p]), at)),
                      lambda: [r.wait(600) for r, _ in reqs])
    srv.close()   # raises the worker's error, if any
    if any(r.done_t is None for r, _ in reqs):
        raise SystemExit("served: requests did not complete")
    bad = sum(1 for r, _ in reqs if r.error is not None or r.verdict is None or r.verdict.flags != 0)
    lat = [(r.done_t - at) * 1e3 for r, at in reqs]
    reqs = [r for r, _ in reqs]
    end = max(r.done_t for r in reqs)
    out["served"] = {"p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99),
                     "gedges_s": entries / (end - t0) / 1e9, "launches": srv.ticks,
                     "mean_graphs_per_launch": statistics.mean(srv.tick_sizes), "invalid": bad,
                     "how": "server.Server over the native mm_server: admission by device-memory "
                            "budget; requests up to 1M entries read in place from pinned host memory, "
                            "larger ones copied on a copy stream; one mm_skipper_multi launch per tick "
                            "on two alternating compute streams, mm_validate_multi before completion, "
                            "D2H on a second copy stream into a result buffer per pool graph (reused, "
                            "as the serial run does)"}
    # the trace's copy ceiling: each pool graph's CSR copied host -> device
    # (pinned, one stream, no kernel), timed, and summed over the requests
    big = max(x[3] for x in pool)
    d_off = torch.empty(max(x[2] for x in pool) + 1, dtype=torch.int64, device="cuda")
    d_nb = torch.empty(max(big, 4), dtype=torch.int32, device="cuda")
    t_copy = []
    for off, nb, n, nnz in pool:
        ts = []
        for _ in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            d_off[: n + 1].copy_(off, non_blocking=True)
            d_nb[:nnz].copy_(nb, non_blocking=True)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e-3)
        t_copy.append(statistics.median(ts))
    del d_off, d_nb
    ceil_s = float(sum(t_copy[p] for p in picks))
    ceil_bytes = int(sum(8 * (pool[p][2] + 1) + 4 * pool[p][3] for p in picks))
    out["copy_ceiling"] = {"gedges_s": entries / ceil_s / 1e9, "seconds": ceil_s,
                           "link_gbs": ceil_bytes / ceil_s / 1e9, "bytes": ceil_bytes,
                           "served_frac": out["served"]["gedges_s"] / (entries / ceil_s / 1e9),
                           "how": "every pool graph's CSR copied host -> device from pinned memory on one "
                                  "stream with no kernel (median of 3, CUDA events), summed over the "
                                  "trace's requests: the rate at which the link alone could deliver them"}
    if not serial:
        return out
    # serial plain: one request at a time through the plain API, in arrival order
    sess = skp.HostSession(max(x[2] for x in pool), max(x[3] for x in pool))
    lat2 = []
    bad2 = 0
    mates = {}

    def serial_submit(p, at):
        nonlocal bad2
        off, nb, n, _ = pool[p]
        if p not in mates:
            mates[p] = torch.empty(n, dtype=torch.int32, pin_memory=True)
        sess.run(off, nb, mates[p], check=True, status_bits=args.bits, grain=2048)
        bad2 += sess.last_verdict.flags != 0
        lat2.append((time.perf_counter() - at) * 1e3)

    t0, _ = run_trace(serial_submit, lambda: None)
    end2 = time.perf_counter()
    sess.close()
    out["serial_plain"] = {"p50_ms": pct(lat2, 50), "p99_ms": pct(lat2, 99),
                           "gedges_s": entries / (end2 - t0) / 1e9, "invalid": bad2,
                           "how": "HostSession.run per request: H2D, mm_skipper (library handles "
                                  "kept per graph size), mm_validate, D2H, synchronous"}
    out["throughput_vs_serial"] = out["served"]["gedges_s"] / out["serial_plain"]["gedges_s"]
    return out


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch
    world, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU for the GB300 arm")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2507_04420_gb300 as skp

    if args.batched_only:
        print(json.dumps({"batched": run_batched(args, skp, plain=False)}), flush=True)
        return 0
    g = make_graph(args, "cuda")
    n, nnz = g.n, g.nnz
    cfg = workload_config(args, g)
    stage = 1 if args.stage_windows else 0
    opts = skp.options(status_bits=args.bits, grain=args.grain, block_threads=args.block,
                       blocks_per_sm=args.blocks_per_sm, nosync=1, timing=1, stage_windows=stage)
    mate = torch.empty(n, dtype=torch.int32, device="cuda")
    h = skp.Graph(g.offsets, g.nbrs, check=True)

    # one checked run before timing: the device checker must accept it
    h.skipper(mate=mate, status_bits=args.bits, grain=args.grain, block_threads=args.block,
              blocks_per_sm=args.blocks_per_sm, stage_windows=stage)
    verdict = h.validate(mate)
    if verdict.flags != 0:
        raise SystemExit(f"invalid matching: {verdict.as_dict()}")

    for _ in range(args.warmup):
        h.skipper(mate=mate, opts=opts)
    h.sync()
    h.timing_history()

    props = torch.cuda.get_device_properties(local)
    uuid = getattr(props, "uuid", None)
    clocks = Clocks(("GPU-" + str(uuid)) if uuid is not None else None)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        h.skipper(mate=mate, opts=opts)
    ev1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    h.sync()
    if dist:
        dist.barrier()
    ms_step = ev0.elapsed_time(ev1) / args.steps
    hist = h.timing_history(256)
    sweep_ms = statistics.mean(t["sweep_ms"] for t in hist)
    init_ms = statistics.mean(t["init_ms"] for t in hist)
    v_end = h.validate(mate)
    if v_end.flags != 0:
        raise SystemExit(f"invalid matching after timing: {v_end.as_dict()}")
    ms_step = max_over_ranks(ms_step, dist)
    value = job_gedges(world, nnz, ms_step * 1e-3)

    # roofline of the dominant kernel (the sweep): algorithmic bytes = CSR once
    peak, peak_kind = measured_peaks()
    sweep_bytes = 8 * (n + 1) + 4 * nnz
    achieved = sweep_bytes / (sweep_ms * 1e-3) / 1e9
    s = {2: 0.25, 8: 1.0, 32: 4.0}[args.bits]   # state bytes per vertex
    step_bytes = int(8 * (n + 1) + 4 * nnz + s * n + (4 * n if args.bits != 32 else 0))
    # the committed counters are the default instance's
    traffic = None if (args.stage_windows or args.blocks_per_sm) else ncu_traffic(cfg["workload"], args.bits)
    if args.stage_windows:
        cfg["stage_windows"] = 1

    # the same graph with mm_options.symmetric = 1 (the CSR is symmetric by
    # construction): each edge tested once, from its lower endpoint's row
    symmetric = None
    if args.symmetric_steps > 0:
        o_sym = skp.options(status_bits=args.bits, grain=args.grain, block_threads=args.block,
                            nosync=1, timing=1, symmetric=1)
        for _ in range(max(3, args.warmup)):
            h.skipper(mate=mate, opts=o_sym)
        h.sync()
        h.timing_history()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.symmetric_steps):
            h.skipper(mate=mate, opts=o_sym)
        e1.record()
        torch.cuda.synchronize()
        h.sync()
        ms_sym = max_over_ranks(e0.elapsed_time(e1) / args.symmetric_steps, dist)
        hist_sym = h.timing_history(256)
        sweep_sym = statistics.mean(t["sweep_ms"] for t in hist_sym)
        v_sym = h.validate(mate)
        if v_sym.flags != 0:
            raise SystemExit(f"invalid matching with symmetric=1: {v_sym.as_dict()}")
        ach_sym = sweep_bytes / (sweep_sym * 1e-3) / 1e9
        symmetric = {"value": job_gedges(world, nnz, ms_sym * 1e-3), "unit": UNIT, "ms_per_step": ms_sym,
                     "sweep_ms": sweep_sym, "roofline_frac": ach_sym / peak, "achieved": ach_sym,
                     "verdict": {"flags": v_sym.flags, "n_pairs": v_sym.n_pairs},
                     "how": "mm_options.symmetric = 1: the caller asserts the CSR is symmetric; the "
                            "sweep tests each edge once, from its lower endpoint's row; same graph, "
                            "same launch, edges counted as stored entries like the headline"}

    # the same graph in the other state layouts (and the byte layout with the
    # 32-register instance), timed the same way: the library's choices beside
    # the paper's one byte per vertex
    layouts = {}
    if args.layout_steps > 0:
        for name, kw in (("u2", dict(status_bits=2)), ("u32", dict(status_bits=32)),
                         ("u8_64warps", dict(status_bits=8, blocks_per_sm=4)),
                         ("u8_dispersed", dict(status_bits=8, unit_order=2))):
            o_l = skp.options(grain=args.grain, block_threads=args.block, nosync=1, timing=1, **kw)
            ms_l, sw_l, _ = time_sweep(h, mate, o_l, args.layout_steps, args.warmup)
            v_l = h.validate(mate)
            if v_l.flags != 0:
                raise SystemExit(f"invalid matching ({name}): {v_l.as_dict()}")
            a_l = sweep_bytes / (sw_l * 1e-3) / 1e9
            s_l = {"u2": 0.25, "u32": 4.0, "u8_64warps": 1.0, "u8_dispersed": 1.0}[name]
            sb_l = int(8 * (n + 1) + 4 * nnz + s_l * n + (4 * n if name != "u32" else 0))
            layouts[name] = {"value": job_gedges(world, nnz, max_over_ranks(ms_l, dist) * 1e-3), "unit": UNIT,
                             "ms_per_step": ms_l, "sweep_ms": sw_l, "roofline_frac": a_l / peak,
                             "step_frac": sb_l / (ms_l * 1e-3) / 1e9 / peak,
                             "verdict": {"flags": v_l.flags, "n_pairs": v_l.n_pairs},
                             "options": {k: int(v) for k, v in kw.items()}}

    # end to end through the public API with host buffers: the host session
    # reads the pinned host CSR in place (MM_HOST_MAPPED, over NVLink-C2C), and,
    # beside it, the copy path (whole CSR host -> device, then the same call)
    e2e = None
    if not args.no_e2e and args.e2e_steps > 0:
        h_off = torch.empty(n + 1, dtype=torch.int64, pin_memory=True)
        h_nb = torch.empty(nnz, dtype=torch.int32, pin_memory=True)
        h_off.copy_(g.offsets)
        h_nb.copy_(g.nbrs)
        h_mate = torch.empty(n, dtype=torch.int32, pin_memory=True)

        def time_session(zero_copy):
            sess = skp.HostSession(n, nnz, zero_copy=zero_copy, pieces=args.e2e_pieces)
            sess.run(h_off, h_nb, h_mate, status_bits=args.bits, grain=args.e2e_grain)  # warm
            mode = sess.last_mode + (f", {sess.last_pieces} pieces" if sess.last_pieces else "")
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(args.e2e_steps):
                sess.run(h_off, h_nb, h_mate, status_bits=args.bits, grain=args.e2e_grain)
            sec = max_over_ranks((time.perf_counter() - t0) / args.e2e_steps, dist)
            sess.close()
            return sec, mode

        zc_s, zc_mode = time_session(True)
        cp_s, cp_mode = time_session(False)
        # bytes the in-place reads move: every row end (the windows read all of
        # them) and the 16-byte id quads the selective walk loads (the
        # statistics counter of the same decision in an eager run)
        with skp.Graph(h_off, h_nb, check=False, host_mapped=True) as hm:
            hm.skipper(status_bits=args.bits, grain=args.e2e_grain, stats=1)
            quads = hm.stats()["id_loads_open"]
        read_bytes = 8 * (n + 1) + 16 * quads
        e2e = {"value": job_gedges(world, nnz, zc_s), "unit": UNIT, "ms_per_step": zc_s * 1e3,
               "h2d_bytes_per_step": read_bytes, "d2h_bytes_per_step": 4 * n, "mode": zc_mode,
               "how": "HostSession.run on pinned host tensors: the kernels read the CSR in place "
                      "(MM_HOST_MAPPED, selective id loads) -- h2d bytes = all row ends + the id "
                      "quads loaded (stats counter); grain by the library (larger units over the "
                      "host link); mm_skipper, then the mate -> pinned host in one copy (with "
                      "--e2e-pieces K: mm_skipper_to_host, K ascending launches, each finished "
                      "prefix of the mate copied back while the next ones run); sync",
               "copy_path": {"value": job_gedges(world, nnz, cp_s), "unit": UNIT, "ms_per_step": cp_s * 1e3,
                             "h2d_bytes_per_step": 8 * (n + 1) + 4 * nnz, "d2h_bytes_per_step": 4 * n,
                             "mode": cp_mode,
                             "how": "HostSession(zero_copy=False).run: whole CSR host -> device, "
                                    "mm_skipper, mate -> pinned host, sync"}}
    else:
        h_off = h_nb = None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        off_np = (h_off if h_off is not None else g.offsets.cpu()).numpy()
        nb_np = (h_nb if h_nb is not None else g.nbrs.cpu()).numpy()
        cs = cpu_sample(off_np, nb_np, args.cpu_seconds)
        cpu = {"value": cs["gedges_s"], "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(),
               "kind": "oracle",
               "sample": f"single-thread SGMM (oracle) over rows [0, {cs['rows']}) of the same graph: "
                         f"{cs['entries']} entries ({100.0 * cs['entries'] / nnz:.1f}% of nnz) "
                         f"in {cs['seconds']:.2f}s"}

    cpu_skipper = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the paper's own setting on this host (Section VI-D): Algorithm 1 on all
        # host cores (as printed, and with the row skip) and on one core, each
        # against SGMM over the same rows
        T = os.cpu_count() or 1
        par = skipper_cpu_sample(off_np, nb_np, T, False, args.cpu_seconds / 4)
        par_rs = skipper_cpu_sample(off_np, nb_np, T, True, args.cpu_seconds / 4)
        one = skipper_cpu_sample(off_np, nb_np, 1, False, args.cpu_seconds / 8)
        one_rs = skipper_cpu_sample(off_np, nb_np, 1, True, args.cpu_seconds / 8)
        cpu_skipper = {
            "kind": "Algorithm 1 on host threads (oracle/skipper_cpu.c), not the oracle",
            "host_cores": T,
            "parallel": par, "parallel_row_skip": par_rs, "one_thread": one, "one_thread_row_skip": one_rs,
            "parallelization_gain": par["sgmm_seconds_same_rows"] / par["seconds"],
            "parallelization_gain_row_skip": par_rs["sgmm_seconds_same_rows"] / par_rs["seconds"],
            "serial_slowdown": one["seconds"] / one["sgmm_seconds_same_rows"],
            "serial_slowdown_row_skip": one_rs["seconds"] / one_rs["sgmm_seconds_same_rows"],
            "gpu_vs_host_skipper": value / max(par["gedges_s"], par_rs["gedges_s"]),
            "how": "parallelization gain = t_SGMM / t_Skipper(T threads), serial slowdown = "
                   "t_Skipper(1 thread) / t_SGMM (Section VI-D, Figs. 10-11), each pair on the "
                   "same rows [0, R) of this graph, R sized by a short calibration",
        }

    serial_mode = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # one GPU thread walking the CSR in SGMM order (serial mode) against SGMM
        # on one host core, on the ER graph of n = 100,000, m = 1,000,000
        import oracle
        import graphgen as gg
        er = gg.erdos_renyi(100_000, 1_000_000, seed=args.seed)
        er_d = er.to("cuda")
        with skp.Graph(er_d.offsets, er_d.nbrs) as he:
            he.skipper(serial=1, status_bits=8)
            ts = []
            for _ in range(3):
                he.skipper(serial=1, status_bits=8, timing=1)
                ts.append(he.timing()["total_ms"])
        _, sgmm_s = oracle.sgmm_timed(er.offsets.numpy(), er.nbrs.numpy())
        serial_mode = {"workload": "erdos_renyi n=100000 m=1000000 (nnz 2000000)",
                       "gpu_one_thread_ms": statistics.median(ts), "sgmm_one_core_ms": sgmm_s * 1e3,
                       "ratio": statistics.median(ts) / (sgmm_s * 1e3),
                       "how": "mm_skipper serial=1 (one GPU thread, CUDA events) vs the oracle's SGMM "
                              "(one host core); a GPU thread is not a CPU core: this is the cost of the "
                              "debug mode, not a kernel-quality figure"}

    batched = None
    h.close()
    del g, h_off, h_nb
    torch.cuda.empty_cache()
    side = None
    if not args.no_side_graphs:
        side = run_side_graphs(args, skp, nnz // 2)
    edge_list = None
    if not args.no_edge_list:
        edge_list = run_edge_list(args, skp)
    if not args.no_batched:
        batched = run_batched(args, skp)

    served = None
    if not args.no_served:
        torch.cuda.empty_cache()
        served = run_served(args, skp)
        torch.cuda.empty_cache()
        served["small_graphs"] = run_served(args, skp, 1e3, 1e5, 1.0, 20000.0)
        # the same pool at five times the rate: what the server sustains (the
        # serial loop's rate does not depend on the offered load: the line above)
        torch.cuda.empty_cache()
        sat = run_served(args, skp, 1e3, 1e5, 0.5, 100000.0, serial=False)
        sat["throughput_vs_serial"] = (sat["served"]["gedges_s"] /
                                       served["small_graphs"]["serial_plain"]["gedges_s"])
        served["small_graphs_100k_per_s"] = sat

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {2: "u2", 8: "u8", 32: "u32"}[args.bits], "data": "synthetic",
        "config": dict(cfg, status_bits=args.bits, grain=args.grain, block_threads=args.block,
                       blocks_per_sm=args.blocks_per_sm or "layout default",
                       parallelism=f"replicas x{world}" if world > 1 else "1 GPU",
                       l2="inputs larger than L2 (CSR %.1f GB vs 129 MB L2); no flush" % (sweep_bytes / 1e9)),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": f"sweep_kernel<{ {2: 'TwoBit', 8: 'Byte', 32: 'Word'}[args.bits]}State>",
                     "bytes_per_launch": sweep_bytes, "sweep_ms": sweep_ms,
                     "peak_kind": f"{peak_kind} hbm_gbs (burst copy)",
                     "step_bytes_alg": step_bytes,
                     "step_frac": step_bytes / (ms_step * 1e-3) / 1e9 / peak},
        "kernel_ms": {"init": init_ms, "sweep": sweep_ms},
        "verdict": {"flags": v_end.flags, "n_pairs": v_end.n_pairs},
        "symmetric_option": symmetric,
        "layouts": layouts,
        "side_graphs": side,
        "edge_list": edge_list,
        "batched": batched,
        "served": served,
        "cpu_baseline": cpu,
        "cpu_skipper": cpu_skipper,
        "serial_mode": serial_mode,
        "e2e": e2e,
        "gpu_launches": 2 * args.steps,
        "clocks": clk,
    }
    h.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
