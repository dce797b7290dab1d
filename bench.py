#!/usr/bin/env python3
"""Benchmark: ray-bounce queries/s of the batched ray-propagation path.

Workload: the procedural open-air theatre (436,796 triangles, 20,459
surfaces, 6 materials, ISO 9613-1 air at 20 C / 50 % RH), one source 1.6 m
above the stage, 16 receiver spheres of radius 2 m on the tiers, 1,000,000
Fibonacci rays x up to 30 bounces.  One step is the whole path on one batch:
the tree build from the resident mesh + rt_trace (rays, bounces, records,
image sources) + rt_rir (8-band histograms, 2 s at 48 kHz).  The builder
is chosen per workload before the warm-up: three steps each with the plain
LBVH (rt_build_tree) and the LBVH with SAH top levels (rt_build_tree_sah),
the faster median step kept ("tree" and "tree_selection_ms_per_step" in
config).

value      nearest-element queries resolved (hits + escapes) per second, over
           all ranks, inputs resident in HBM, timed with CUDA events on the
           launching stream, L2 flushed (256 MB write) before every step.
e2e        the same metric through the C ABI from pinned host buffers: mesh
           H2D, trace, histograms and their D2H copy inside the timed region.
roofline   the bounce kernel's algorithmic L2-path bytes over its live
           duration, against the L2 read bandwidth measured in the same run
           (MEASURED_PEAKS.json has no L2 figure); HBM fraction beside it.
           Bytes per query: 64 B per tree node visited (a binary node's
           two child boxes) and 48 B per triangle tested, counted by an
           instrumented pass; the kernel's own 4-wide nodes read 112 B per
           visit, reported beside it as "achieved_wide".
surrogate  the metric's second half: RIRs/s of the surrogate-tail pipeline
           (model trained in this run) against plain 1M-ray full tracing on
           64 held-out rooms, with T30 / EDT errors and fallbacks.
config2    the same measurement on the closed L-room (102,400 triangles,
           1M rays x 50 bounces, 4 receivers): every ray lives to its last
           bounce, so it measures full-length traversal.
extras     three short measurements: one iteration of the paper's scaling
           workload at N = M = 2^20 (tree build apart), a moved listener on the
           theatre (recorded paths replayed for 17 new receivers, against a
           full trace; the two must agree), and the surrogate network's
           first-layer GEMM at batch 65,536 against the BF16 peak.
ms_step_spread  median, min and max of the timed steps (Python's garbage
           collector is off during them).
phases_ms  medians over the timed steps (CUDA events): tree build, ray
           generation, bounce loop, image sources (dedup + FP64
           reconstruction), the rest of rt_trace (uploads, queue set-up,
           result sizes), RIR binning.
cpu_baseline  the FP64 oracle (oracle/, C + numpy) on a bounded sample of the
           same workload on this host's cores; beside it the oracle's trace
           on one thread and the paper's single-core rate (Table 2).
parity     that sample's rays traced on the GPU (the headline's
           configuration) against the oracle: shares of identical triangle and
           surface sequences.

--impl reference runs that oracle as the reference arm.
Under torchrun each rank traces its own ray shard of a world_size x 1M-ray
job (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import gc
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import scenes  # noqa: E402

METRIC = "ray-bounce hits/s at 436k tris, 1M rays"   # the second half (surrogate RIRs/s) is its own object
UNIT = "queries/s"
DURATION = 2.0          # seconds of impulse response
N_RAYS = 1_000_000
N_BOUNCES = 30


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--tail-rays", type=int, default=None, help="override the autotuned tail threshold")
    ap.add_argument("--tree", choices=["auto", "lbvh", "sah_top"], default="auto",
                    help="tree builder of the theatre and L-room steps (auto: the faster over three steps each)")
    ap.add_argument("--cpu-sample-rays", type=int, default=200_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-config2", action="store_true", help="skip the closed L-room object of the default line")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the surrogate-tail object of the default line")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the tetra 2^20, moved-listener and GEMM objects of the default line")
    ap.add_argument("--clock-log", default=None, help="keep the nvidia-smi samples of the timed region here")
    ap.add_argument("--workload", choices=["theatre", "lroom", "batched", "tetra", "trees", "gemm"], default="theatre",
                    help="theatre: the headline line; lroom: the closed L-room alone (102,400 tris, 1M rays x 50 "
                         "bounces); batched: 64 rooms x 16 pairs x 262,144 rays x 30 bounces "
                         "in batched launches; tetra: the N = M scaling sweep of one iteration on the refined "
                         "tetrahedron; trees: the LBVH against the paper's median-split tree and the SAH top "
                         "(each its own line, one GPU)")
    ap.add_argument("--batch-chunk", type=int, default=262_144,
                    help="rays per pair per batched trace (default: all of them, one trace per step)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def shard(rank: int, world: int, n_per_rank: int = N_RAYS):
    """Weak scaling: rank r traces rays [r n, (r+1) n) of a world x n-ray job."""
    return dict(ray_begin=rank * n_per_rank, ray_count=n_per_rank), n_per_rank * world


def reduce_over_ranks(dist, torch, device, seconds, e2e_seconds, queries, e2e_queries):
    """Max of the timed regions and sum of the work over ranks (all-reduce)."""
    t = torch.tensor([seconds, e2e_seconds], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    q = torch.tensor([float(queries), float(e2e_queries)], device=device, dtype=torch.float64)
    dist.all_reduce(q, op=dist.ReduceOp.SUM)
    return float(t[0]), float(t[1]), float(q[0]), float(q[1])


def workload(world: int):
    sc = scenes.theatre(n_rays=N_RAYS * world, n_bounces=N_BOUNCES)
    return sc


def workload_name(world):
    return (f"open-air theatre 436,796 tris / 20,459 surfaces, {N_RAYS * world:,} rays x {N_BOUNCES} bounces, "
            f"16 receivers r=2 m, air 20C/50%RH, RIR 8 bands x {DURATION:g} s at 48 kHz")


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, path=None):
        self.gpu = gpu_index
        self.proc = None
        if path is None:
            fd, path = tempfile.mkstemp(prefix=f"clocks_gpu{gpu_index}_", suffix=".csv")
            os.close(fd)
        self.path = path

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def wait_first_sample(self, timeout=3.0):
        """Block until nvidia-smi has written its first sample (its start-up
        calls into the NVIDIA driver then happen before, not inside, a timed
        region)."""
        t_end = time.time() + timeout
        while self.proc is not None and time.time() < t_end:
            self.f.flush()
            if os.path.getsize(self.path) > 0:
                return True
            time.sleep(0.01)
        return False

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for k, n in enumerate(names):
                if p[5 + k].lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------
# oracle (CPU) runs
# ----------------------------------------------------------------------------
def oracle_sample(sc, n_rays, seed=0, keep=False):
    """Trace a seeded subset of the workload's rays with the FP64 oracle
    (median-split tree), build image sources and histograms; returns
    (queries, seconds, threads), and with keep the trace and the ray ids."""
    import oracle
    rng = np.random.default_rng(seed)
    t0 = time.perf_counter()
    osc = oracle.OracleScene(sc, tree=True)
    ids = np.sort(rng.choice(sc.n_rays, min(n_rays, sc.n_rays), replace=False))
    tr = oracle.trace(osc, ray_ids=ids)
    isrc = oracle.image_sources(sc, tr)
    oracle.rir(isrc, len(sc.rcv_center), sc.fs, DURATION)
    dt = time.perf_counter() - t0
    if keep:
        return tr.queries, dt, oracle.default_threads(), tr, ids
    return tr.queries, dt, oracle.default_threads()


def parity_object(rt, torch, stream, sc, kw, tree, chosen, tr, ids):
    """The GPU trace of the workload (the headline's configuration) against
    the oracle's free-running trace of the sampled rays: shares of rays with
    the same triangle sequence and the same surface sequence, overall and
    among the rays the oracle finds unambiguous (no path within its edge
    band).  Float32 and FP64 trajectories drift apart by ulps per bounce, so
    the triangle inside one surface may differ late in a long path; the
    tests hold the tolerances, this line reports the figures."""
    cfg = dict(tail_rays=chosen["tail_rays"] if chosen["tail_rays"] > 0 else -1, block_size=chosen["block_size"],
               compaction_period=chosen["compaction_period"], stack_entries=chosen["stack_entries"])
    with torch.cuda.stream(stream):
        isrc = rt.rt_trace(tree, stream=stream, **cfg, **kw)
        g = isrc.hist[:, torch.as_tensor(ids, device=isrc.hist.device)].cpu().numpy().T
    stream.synchronize()
    o = np.asarray(tr.hist)
    surf = np.append(np.asarray(sc.surface_id), -1)
    same_tri = np.all(g == o, axis=1)
    same_surf = np.all(surf[g] == surf[o], axis=1)
    unamb = np.asarray(tr.first_amb) == tr.B
    return {"rays": int(len(ids)), "identical_triangle_sequences": float(same_tri.mean()),
            "identical_surface_sequences": float(same_surf.mean()), "unambiguous_rays": float(unamb.mean()),
            "identical_triangles_among_unambiguous": float(same_tri[unamb].mean()) if unamb.any() else None,
            "oracle": "FP64, median-split tree, free-running (oracle/rt_oracle.c)"}


def oracle_single_thread(sc, n_rays, seed=1):
    """The oracle's trace alone (tree built beforehand) on one host thread,
    for a seeded subset of the workload's rays: queries per second."""
    import oracle
    try:
        rng = np.random.default_rng(seed)
        osc = oracle.OracleScene(sc, tree=True)
        ids = np.sort(rng.choice(sc.n_rays, min(n_rays, sc.n_rays), replace=False))
        t0 = time.perf_counter()
        tr = oracle.trace(osc, ray_ids=ids, threads=1)
        dt = time.perf_counter() - t0
    except Exception as e:  # a context figure only: never costs the benchmark line
        return {"value": None, "unit": UNIT, "error": f"{type(e).__name__}: {e}"}
    return {"value": tr.queries / dt, "unit": UNIT, "sample": f"{len(ids):,} seeded rays, trace only, 1 thread"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    sc = workload(1)
    n = args.cpu_sample_rays
    for _ in range(args.warmup):
        oracle_sample(sc, max(1000, n // 20))
    q_tot, t_tot = 0, 0.0
    for k in range(args.steps):
        q, dt, threads = oracle_sample(sc, n, seed=k)
        q_tot += q
        t_tot += dt
    v = q_tot / t_tot
    sample = f"{n:,} seeded rays of the workload per step (of {sc.n_rays:,}), oracle tree + image sources + RIR"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": workload_name(1)},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


# ----------------------------------------------------------------------------
# native GPU runs
# ----------------------------------------------------------------------------
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json)"
    return 6800.0, "fallback"


def kernel_source_sha():
    """First 16 hex digits of the SHA-256 of the bounce kernel's sources
    (rt_trace.cu followed by rt_traverse.cuh)."""
    import hashlib
    h = hashlib.sha256()
    for f in ("rt_trace.cu", "rt_traverse.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1811_05784_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def tree_source_sha():
    """First 16 hex digits of the SHA-256 of the tree builder's sources
    (rt_build.cu followed by rt_sah_top.cuh): a capture on the SAH-top tree
    holds for this builder only."""
    import hashlib
    h = hashlib.sha256()
    for f in ("rt_build.cu", "rt_sah_top.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1811_05784_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(name, tail, tree="lbvh"):
    """DRAM bytes per trace of the bounce kernel from a committed ncu
    summary under profiles/, if one of its captures matches the current
    kernel source, the configuration and the tree (else None).  A capture is
    a block of traffic_* lines starting with traffic_bytes_per_trace; one
    without a traffic_tree line was taken on the plain LBVH, and a capture on
    the SAH-top tree holds only for the builder source it names
    (traffic_tree_source_sha256_16)."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    blocks = []
    for line in open(path):
        if ":" in line and line.split(":")[0].startswith("traffic_"):
            k, v = (x.strip() for x in line.split(":", 1))
            if k == "traffic_bytes_per_trace":
                blocks.append({})
            if blocks:
                blocks[-1][k] = v
    for kv in blocks:
        tree_sha = kv.get("traffic_tree_source_sha256_16")
        if (kv.get("traffic_source_sha256_16") == kernel_source_sha() and kv.get("traffic_config") == f"tail_rays={tail}"
                and kv.get("traffic_tree", "lbvh") == tree
                and (tree == "lbvh" or tree_sha == tree_source_sha())):
            return float(kv["traffic_bytes_per_trace"])
    return None


def host_cpu():
    """Architecture and model name of the host cores (for the oracle timing)."""
    import platform
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return f"{platform.machine()} {model} x{os.cpu_count()}".strip()


def l2_roofline(rt, torch, tree, sc, kw, chosen, bounce_ms, stream, dev, l2_peak, hbm, traffic):
    """Roofline object of the bounce kernel for one trace: node visits and
    triangle tests counted by an instrumented pass of the same
    configuration, over the bounce loop's CUDA-event time."""
    B, n = sc.n_bounces, kw.get("ray_count") or sc.n_rays
    cost = torch.zeros((B, n, 2), dtype=torch.int32, device=dev)
    fixed_tail = chosen["tail_rays"] if chosen["tail_rays"] > 0 else -1
    isrc = rt.rt_trace(tree, tail_rays=fixed_tail, block_size=chosen["block_size"], stream=stream,
                       compaction_period=chosen["compaction_period"], stack_entries=chosen["stack_entries"],
                       debug_cost=cost, **kw)
    torch.cuda.synchronize()
    c = cost.double().sum((0, 1)).cpu().numpy()
    del cost
    n_q = isrc.queries
    l2_bytes = 64.0 * c[0] + 48.0 * c[1]                 # a node visited, a triangle tested
    wide_bytes = 112.0 * c[0] + 48.0 * c[1]              # the 4-wide node's six box float4 and its refs
    hbm_bytes = n_q * 4.0 + n * (80.0 + 44.0) + isrc.n_records * 24.0   # hist, state in / out, records
    sec = bounce_ms / 1e3
    hbm_peak, hbm_src = hbm
    return {"bound": "l2", "kernel": "k_bounce (all launches of one trace)",
            "achieved": l2_bytes / sec / 1e9, "peak": l2_peak, "unit": "GB/s",
            "frac": l2_bytes / sec / 1e9 / l2_peak,
            "peak_source": "measured in this run: rt_measure_l2_bandwidth (32 MiB L2-resident, ld.global.cg)",
            "traffic": traffic, "algorithmic_bytes": l2_bytes,
            "bytes_per_query": "64 B per node visited + 48 B per triangle tested",
            "achieved_wide": {"value": wide_bytes / sec / 1e9, "frac": wide_bytes / sec / 1e9 / l2_peak,
                              "bytes_per_query": "112 B per 4-wide node visited + 48 B per triangle tested"},
            "hbm": {"achieved": hbm_bytes / sec / 1e9, "peak": hbm_peak, "unit": "GB/s",
                    "frac": hbm_bytes / sec / 1e9 / hbm_peak, "peak_source": hbm_src},
            "ms_per_launch_set": bounce_ms, "nodes_per_query": c[0] / n_q, "tris_per_query": c[1] / n_q}


TREES = ("lbvh", "sah_top")


def timed_trace_steps(rt, torch, sc, kw, stream, tail, warmup, steps, flush, dev, duration, tree_kind="auto"):
    """Tree build + trace + RIR per step on device-resident inputs: the
    autotuner's trials first; then, with tree_kind "auto", three steps with
    each builder (rt_build_tree, rt_build_tree_sah), the faster median kept;
    then `warmup` steps, then `steps` timed steps (CUDA events on the
    launching stream, L2 flushed before each)."""
    V, T, Mt, St = (torch.as_tensor(x, device=dev) for x in (sc.vertices, sc.tris, sc.material_id, sc.surface_id))
    ws_trace = rt.Workspace()
    kind = ["lbvh" if tree_kind == "auto" else tree_kind]
    selection = {}

    def step(ev=None):
        tree = rt.rt_build_tree(V, T, Mt, St, stream=stream, sah=kind[0] == "sah_top")
        if ev is not None:
            ev[0].record(stream)
        isrc = rt.rt_trace(tree, tail_rays=tail, stream=stream, workspace=ws_trace, **kw)
        if ev is not None:
            ev[1].record(stream)
        resp = rt.rt_rir(isrc, sc.fs, duration=duration, stream=stream)
        return tree, isrc, resp

    with torch.cuda.stream(stream):
        # the autotuner tries one configuration per call until it has timed
        # each candidate twice; finish that before the warm-up steps, so that
        # the timed steps run the chosen configuration whatever W is
        if tail == rt.RT_TAIL_AUTOTUNE:
            prev = None
            for _ in range(40):
                _, isrc_t, _ = step()
                cur = (isrc_t.block_size, int(isrc_t.tail_rays), isrc_t.compaction_period, isrc_t.stack_entries)
                if cur == prev:
                    break
                prev = cur
        if tree_kind == "auto":  # the builder whose whole step is faster
            for k in TREES:
                kind[0] = k
                t = []
                for _ in range(3):
                    flush.zero_()
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    step()
                    b.record(stream)
                    b.synchronize()
                    t.append(a.elapsed_time(b))
                selection[k] = statistics.median(t)
            kind[0] = min(TREES, key=lambda k: selection[k])
        for _ in range(max(warmup, 1)):
            _, isrc_w, _ = step()
        torch.cuda.synchronize()
        chosen = {"block_size": isrc_w.block_size, "tail_rays": int(isrc_w.tail_rays),
                  "compaction_period": isrc_w.compaction_period, "stack_entries": isrc_w.stack_entries}
        torch.cuda.synchronize()
        launches0 = rt.rt_launch_count()
        ms, queries = [], []
        phases = {k: [] for k in ("build", "rays", "bounces", "image_sources", "trace_other", "rir")}
        # no Python garbage collection inside the timed steps: a collection
        # pause stalls the host while the GPU waits for the next launch
        gc.collect()
        gc.disable()
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            a.record(stream)
            tree, isrc, resp = step(ev)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
            queries.append(isrc.queries)
            t_trace = ev[0].elapsed_time(ev[1])
            phases["build"].append(a.elapsed_time(ev[0]))
            phases["rays"].append(isrc.ms_rays)
            phases["bounces"].append(isrc.ms_bounces)
            phases["image_sources"].append(isrc.ms_image_sources)
            phases["trace_other"].append(t_trace - isrc.ms_rays - isrc.ms_bounces - isrc.ms_image_sources)
            phases["rir"].append(ev[1].elapsed_time(b))
        torch.cuda.synchronize()
        gc.enable()
        launches = rt.rt_launch_count() - launches0
    return dict(ms=ms, queries=queries, phases=phases, chosen=chosen, launches=launches, tree=tree,
                graph=ws_trace.graph_launches > 0, ws=ws_trace, mesh=(V, T, Mt, St), tree_kind=kind[0],
                tree_selection_ms_per_step=selection)


def lroom_object(rt, torch, stream, tail, args, flush, dev, l2_peak, hbm, rng_kw):
    """The closed L-room (102,400 triangles, 1M rays x 50 bounces, every ray
    alive to its last bounce): queries/s per step of tree build + trace + RIR,
    and the bounce kernel's roofline."""
    sc2 = scenes.lroom(n_rays=N_RAYS, n_bounces=50)
    kw2 = rt.scene_args(sc2)
    kw2.update(rng_kw)
    run2 = timed_trace_steps(rt, torch, sc2, kw2, stream, tail, args.warmup, args.steps, flush, dev, 1.0, args.tree)
    with torch.cuda.stream(stream):
        roof2 = l2_roofline(rt, torch, run2["tree"], sc2, kw2, run2["chosen"],
                            statistics.median(run2["phases"]["bounces"]), stream, dev, l2_peak, hbm,
                            profiled_traffic("k_bounce_lroom.md", run2["chosen"]["tail_rays"], run2["tree_kind"]))
    t2 = sum(run2["ms"]) / 1e3
    return {"workload": f"closed L-room 102,400 tris / 8 surfaces, {N_RAYS:,} rays x 50 bounces, 4 receivers "
                        f"r=0.5 m, RIR 8 bands x 1 s at 48 kHz",
            "value": sum(run2["queries"]) / t2, "unit": UNIT, "ms_per_step": 1e3 * t2 / args.steps,
            "queries_per_step": int(statistics.median(run2["queries"])), "bounce_kernel": run2["chosen"],
            "tree": run2["tree_kind"], "tree_selection_ms_per_step": run2["tree_selection_ms_per_step"],
            "phases_ms": {k: statistics.median(v) for k, v in run2["phases"].items()},
            "roofline": roof2, "gpu_launches": int(run2["launches"])}


def run_lroom(args):
    import torch
    from paper_1811_05784_gb300 import rt
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    tail = rt.RT_TAIL_AUTOTUNE if args.tail_rays is None else args.tail_rays
    l2_peak = rt.rt_measure_l2_bandwidth(stream=stream)
    with ClockSampler(0, args.clock_log) as clk:
        o = lroom_object(rt, torch, stream, tail, args, flush, dev, l2_peak, measured_peaks(), {})
    o.update({"metric": "ray-bounce hits/s, closed L-room", "n_gpus": 1, "steps": args.steps,
              "warmup": args.warmup, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
              "clocks": clk.summary()})
    print(json.dumps(o))


SUR_TRAIN_ROOMS, SUR_TEST_ROOMS, SUR_TEST_SEED0 = 2048, 64, 1_000_000


def surrogate_object(rt, torch, stream, args):
    """Second half of the metric: RIRs/s of the surrogate-tail pipeline
    against plain 1M-ray full tracing on the same GPU, over 64 held-out rooms
    (seeds 1,000,000+), with per-band T30 / EDT errors of the surrogate
    responses against those full traces and the fallback count.  The model
    is trained in this run: 2,048 seeded rooms (targets: 65,536-ray full
    traces), two networks, 600 AdamW steps.  Each pipeline builds its trees;
    both run once untimed over the same rooms first."""
    import scenes as SC
    from paper_1811_05784_gb300 import surrogate as S
    from paper_1811_05784_gb300.train_surrogate import errors
    ws = rt.Workspace()
    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        parts = {}
        for k in range(0, SUR_TRAIN_ROOMS, 128):
            rooms = [SC.surrogate_room(s) for s in range(k, min(k + 128, SUR_TRAIN_ROOMS))]
            d = S.inputs(rooms, stream=stream, workspace=ws)
            _, d["tail_db"] = S.reference(rooms, d["trees"], full_rays=65_536, stream=stream, workspace=ws)
            for key in ("desc", "early", "probe", "prior_db", "base_db", "X", "tail_db"):
                parts.setdefault(key, []).append(d[key])
        data = {k: torch.cat(v).contiguous() for k, v in parts.items()}
        t1 = time.perf_counter()
        model = S.train(data, n_nets=2, steps=600, batch=512, seed=0, stream=stream)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        del data, parts
        rooms = [SC.surrogate_room(s) for s in range(SUR_TEST_SEED0, SUR_TEST_SEED0 + SUR_TEST_ROOMS)]
        sur_fn = lambda: S.respond(rooms, model, full_rays=N_RAYS, stream=stream, workspace=ws)
        plain_fn = lambda: S.reference(rooms, full_rays=N_RAYS, stream=stream, workspace=ws)
        sur_fn(), plain_fn()
        (env, fb), dt_s = S.timed(sur_fn)
        (ref, _), dt_p = S.timed(plain_fn)
        err = errors(S.decay_times(env, stream), S.decay_times(ref, stream))
        info = model.info()
    out = {"metric": "RIRs/s, surrogate tail vs plain full tracing", "unit": "RIRs/s",
           "value": SUR_TEST_ROOMS / dt_s, "plain": SUR_TEST_ROOMS / dt_p, "speedup": dt_p / dt_s,
           "rooms": SUR_TEST_ROOMS, "fallback_rooms": int(fb.sum()),
           "config": {"rooms": "seeded shoeboxes and L-rooms 50-20,000 m3, r = 0.5 m (scenes.surrogate_room)",
                      "surrogate": "rt_rir_surrogate: 64k-ray 0-50 ms trace + 16k-ray 2 s probe + 2 networks, "
                                   "full 1M-ray trace for rooms failing the gate (charged)",
                      "plain": "1M-ray full traces to 2 s (rt_surrogate_reference)",
                      "training": f"{SUR_TRAIN_ROOMS} rooms in this run: tracing {t1 - t0:.1f} s, "
                                  f"networks {t2 - t1:.1f} s", "gate_db": [info["join_db"], info["probe_db"]]},
           "targets": {"speedup_min": 4.0, "max_rel_error": 0.05}}
    for name, e in err.items():
        out[name] = {"mean_rel_error": float(np.nanmean(e)),
                     "worst_band_mean": float(np.nanmax(np.nanmean(e, axis=0))),
                     "estimate_undefined": int(np.sum(e == 1.0)), "reference_undefined": int(np.isnan(e).sum())}
    out["meets_targets"] = bool(out["speedup"] >= 4.0 and out["T30"]["worst_band_mean"] <= 0.05
                                and out["EDT"]["worst_band_mean"] <= 0.05)
    return out


def run_native(args):
    import torch
    import torch.distributed as dist
    from paper_1811_05784_gb300 import rt

    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream()
    sc = workload(ws)
    kw = rt.scene_args(sc)
    rng_kw, _ = shard(rank, ws)
    kw.update(rng_kw)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    tail = rt.RT_TAIL_AUTOTUNE if args.tail_rays is None else args.tail_rays
    l2_peak = rt.rt_measure_l2_bandwidth(stream=stream)
    hbm = measured_peaks()

    # clocks sampled from the first warm-up step through the timed steps
    clk = ClockSampler(torch.cuda.current_device(), args.clock_log)
    clk.__enter__()
    clk.wait_first_sample()
    if ws > 1:
        dist.barrier()
    run = timed_trace_steps(rt, torch, sc, kw, stream, tail, args.warmup, args.steps, flush, dev, DURATION,
                            args.tree)
    clk.__exit__(None, None, None)
    if ws > 1:
        dist.barrier()
    ms, queries, chosen = run["ms"], run["queries"], run["chosen"]
    t_total = sum(ms) / 1e3
    q_total = sum(queries)

    with torch.cuda.stream(stream):
        # -- end to end through host buffers ----------------------------------
        host = [torch.as_tensor(x).pin_memory() for x in (sc.vertices, sc.tris, sc.material_id, sc.surface_id)]
        h2d = sum(x.numel() * x.element_size() for x in host)
        h2d += sc.sources.nbytes + sc.rcv_center.nbytes + sc.rcv_radius.nbytes + sc.rcv_source.nbytes
        h2d += sc.alpha.nbytes + sc.beta.nbytes
        out = torch.empty((len(sc.rcv_center), 8, int(math.ceil(DURATION * sc.fs))), dtype=torch.float32).pin_memory()
        d2h = out.numel() * 4
        e2e_ms, e2e_q = [], 0
        for k in range(args.warmup + args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            tree = rt.rt_build_tree(*host, stream=stream, sah=run["tree_kind"] == "sah_top")
            isrc = rt.rt_trace(tree, tail_rays=tail, stream=stream, workspace=run["ws"], **kw)
            resp = rt.rt_rir(isrc, sc.fs, duration=DURATION, stream=stream)
            resp.download(out, stream=stream)
            dt = time.perf_counter() - t0
            if k >= args.warmup:
                e2e_ms.append(dt * 1e3)
                e2e_q += isrc.queries
        roof = l2_roofline(rt, torch, run["tree"], sc, kw, chosen, statistics.median(run["phases"]["bounces"]),
                           stream, dev, l2_peak, hbm,
                           profiled_traffic("k_bounce_theatre.md", chosen["tail_rays"], run["tree_kind"]))

    # -- the closed L-room (config 2): full-length traversal -------------------
    cfg2 = None if args.no_config2 else lroom_object(rt, torch, stream, tail, args, flush, dev, l2_peak, hbm, rng_kw)

    # max over ranks
    t_max = t_total
    if ws > 1:
        t_max, e2e_t, q_all, e2e_q_all = reduce_over_ranks(dist, torch, dev, t_total, sum(e2e_ms) / 1e3,
                                                           q_total, e2e_q)
    else:
        e2e_t, q_all, e2e_q_all = sum(e2e_ms) / 1e3, q_total, e2e_q
    value = q_all / t_max
    clocks = clk.summary()
    clocks["window"] = "nvidia-smi every 200 ms from the first warm-up step to the last timed step"
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(ws), "rays_per_gpu": N_RAYS, "n_bounces": N_BOUNCES,
                   "queries_per_step_per_gpu": int(statistics.median(queries)),
                   "bounce_kernel": chosen, "cuda_graph": run["graph"], "tree": run["tree_kind"],
                   "tree_selection_ms_per_step": run["tree_selection_ms_per_step"],
                   "l2": "flushed (256 MB write) before every timed step", "parallelism": f"ray shards x{ws}"},
        "e2e": {"value": e2e_q_all / e2e_t, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "roofline": roof,
        "phases_ms": {k: statistics.median(v) for k, v in run["phases"].items()},
        "ms_step_spread": {"median": statistics.median(ms), "min": min(ms), "max": max(ms)},
        "gpu_launches": int(run["launches"]),
        "clocks": clocks,
    }
    if cfg2 is not None:
        result["config2"] = cfg2
    if ws == 1 and not args.no_surrogate:
        try:
            result["surrogate"] = surrogate_object(rt, torch, stream, args)
        except Exception as e:  # reported, never costs the benchmark line
            result["surrogate"] = {"error": f"{type(e).__name__}: {e}"}
    if ws == 1 and not args.no_extras:
        try:
            result["extras"] = extras_object(rt, torch, stream, sc, kw, run["tree"], chosen, args.steps, dev)
        except Exception as e:  # reported, never costs the benchmark line
            result["extras"] = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        q, dt, threads, tr_o, ids_o = oracle_sample(sc, args.cpu_sample_rays, keep=True)
        try:
            result["parity"] = parity_object(rt, torch, stream, sc, kw, run["tree"], chosen, tr_o, ids_o)
        except Exception as e:  # reported, never costs the benchmark line
            result["parity"] = {"error": f"{type(e).__name__}: {e}"}
        del tr_o
        result["cpu_baseline"] = {"value": q / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
                                  "single_thread": oracle_single_thread(sc, 20_000),
                                  "paper_single_core": {"value": 2 ** 20 / 13.78, "unit": UNIT,
                                                        "source": "Table 2: 2^20 rays and faces, one "
                                                                  "iteration with the tree in 13.78 s"},
                                  "sample": f"{args.cpu_sample_rays:,} seeded rays of the workload "
                                            f"(oracle median-split tree, image sources, RIR): {q:,} queries",
                                  "cpu": host_cpu()}
    if rank == 0:
        print(json.dumps(result))
    if ws > 1:
        dist.destroy_process_group()


def extras_object(rt, torch, stream, sc, kw, tree, chosen, steps, dev):
    """Three short measurements beside the headline, so that the line itself
    carries them: the paper's scaling workload at N = M = 2^20 (one
    iteration, tree build apart), a moved listener on the theatre (the
    recorded paths replayed for new receivers, against a full trace with
    them) and the surrogate network's first-layer GEMM at batch 65,536.
    Device times from CUDA events on the launching stream, medians of
    `steps` after two untimed calls; the traces run in the bounce-kernel
    configuration the headline chose."""
    import copy
    out = {}
    n_meas = max(steps, 3)
    with torch.cuda.stream(stream):
        # -- tetrahedron N = M = 2^20, one bounce -----------------------------
        tsc = scenes.tetra(9)
        tkw = rt.scene_args(tsc)
        mesh = tuple(torch.as_tensor(x, device=dev) for x in (tsc.vertices, tsc.tris, tsc.material_id,
                                                              tsc.surface_id))
        b_ms, t_ms = [], []
        for k in range(n_meas + 2):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
            ttree = rt.rt_build_tree(*mesh, stream=stream)
            e[1].record(stream)
            isrc = rt.rt_trace(ttree, stream=stream, **tkw)
            e[2].record(stream)
            e[2].synchronize()
            if k >= 2:
                b_ms.append(e[0].elapsed_time(e[1]))
                t_ms.append(e[1].elapsed_time(e[2]))
        out["tetra_2p20"] = {"faces": len(tsc.tris), "rays": tsc.n_rays, "queries": int(isrc.queries),
                             "tree_ms": statistics.median(b_ms), "iteration_ms": statistics.median(t_ms),
                             "paper_single_core_s": 13.78}
        del isrc, ttree
        # -- moved listener: replay against a full trace ----------------------
        cfg = dict(tail_rays=chosen["tail_rays"] if chosen["tail_rays"] > 0 else -1, block_size=chosen["block_size"],
                   compaction_period=chosen["compaction_period"], stack_entries=chosen["stack_entries"])
        first = rt.rt_trace(tree, stream=stream, **cfg, **kw)
        moved = copy.copy(sc)
        lo, hi = sc.vertices.min(0), sc.vertices.max(0)
        g = np.random.default_rng(3)
        n = len(sc.rcv_center) + 1
        moved.rcv_center = scenes.f32(g.uniform(lo + 0.25 * (hi - lo), hi - 0.25 * (hi - lo), (n, 3)))
        moved.rcv_radius = scenes.f32(g.uniform(0.3, 1.5, n))
        moved.rcv_source = np.zeros(n, np.int32)
        mkw = rt.scene_args(moved)
        times = {"full": [], "replay": []}
        for k in range(n_meas + 2):
            for name, extra in (("full", {}), ("replay", {"replay": first})):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                r = rt.rt_trace(tree, stream=stream, **cfg, **mkw, **extra)
                e1.record(stream)
                e1.synchronize()
                if k >= 2:
                    times[name].append(e0.elapsed_time(e1))
                if name == "replay":
                    same = bool(torch.equal(r.hist, full_hist)) and r.n == full_n
                else:
                    full_hist, full_n = r.hist.clone(), r.n
                del r
        out["moved_listener"] = {"receivers": n, "full_trace_ms": statistics.median(times["full"]),
                                 "replay_ms": statistics.median(times["replay"]), "identical_to_full": same}
        del first
        # -- the surrogate network's GEMM -------------------------------------
        gen = torch.Generator(device="cuda").manual_seed(0)
        A = torch.randn(65536, 960, device=dev, generator=gen).to(torch.bfloat16)
        B = torch.randn(512, 960, device=dev, generator=gen).to(torch.bfloat16)
        C = torch.empty((65536, 512), dtype=torch.float32, device=dev)
        g_ms = []
        for k in range(n_meas + 2):
            _, ms = rt.rt_gemm_bf16(A, B, out=C, stream=stream, timed=True)
            if k >= 2:
                g_ms.append(ms)
        tf = 2.0 * 65536 * 512 * 960 / (statistics.median(g_ms) * 1e-3) / 1e12
        bf16 = None
        p = os.path.join(ROOT, "MEASURED_PEAKS.json")
        if os.path.exists(p):
            bf16 = float(json.load(open(p))["bf16_tflops"])
        out["gemm_65536x512x960"] = {"tflops": tf, "ms": statistics.median(g_ms),
                                     "frac_of_bf16_peak": tf / bf16 if bf16 else None,
                                     "kernel": "k_gemm_tma (TMA, tcgen05, TMEM)"}
        del A, B, C
    return out


def run_batched(args):
    """64 seeded rooms of 12 to 182,400 triangles, 16 source / receiver pairs
    each, 262,144 rays per pair, 30 bounces: every step builds the 64 trees
    (the builder chosen by one step with each, as for the theatre) and
    traces all 268M rays of all rooms in one batched trace (its bounce loop one
    CUDA graph of persistent launches, configuration autotuned), followed by
    the 8-band RIRs of all 1,024 receivers.  --batch-chunk splits the rays of
    each pair into several traces instead (the shards add up exactly)."""
    import torch
    from paper_1811_05784_gb300 import rt
    torch.cuda.set_device(0)
    rooms_sc = scenes.batched_rooms()
    n_rays, B = rooms_sc[0].n_rays, rooms_sc[0].n_bounces
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream()
    ws_trace = rt.Workspace()
    mesh = [tuple(torch.as_tensor(x, device=dev) for x in (r.vertices, r.tris, r.material_id, r.surface_id))
            for r in rooms_sc]
    chunk = min(args.batch_chunk, n_rays)
    kind = ["lbvh" if args.tree == "auto" else args.tree]
    selection = {}

    def step():
        trees = [rt.rt_build_tree(*m, stream=stream, sah=kind[0] == "sah_top") for m in mesh]
        rooms = [dict(tree=t, sources=r.sources, rcv_center=r.rcv_center, rcv_radius=r.rcv_radius,
                      rcv_source=r.rcv_source, band_absorption=r.alpha) for t, r in zip(trees, rooms_sc)]
        q, cfg = 0, None
        for begin in range(0, n_rays, chunk):
            isrc = rt.rt_trace_batch(rooms, n_rays, B, ray_begin=begin, ray_count=min(chunk, n_rays - begin),
                                     tail_rays=rt.RT_TAIL_AUTOTUNE, stream=stream, workspace=ws_trace)
            rt.rt_rir(isrc, 48_000.0, duration=1.0, stream=stream)
            q += isrc.queries
            cfg = {"block_size": isrc.block_size, "tail_rays": int(isrc.tail_rays),
                   "compaction_period": isrc.compaction_period, "stack_entries": isrc.stack_entries,
                   "ms_bounces": isrc.ms_bounces}
            del isrc
        return q, cfg

    with torch.cuda.stream(stream):
        # finish the autotuner's trials (one configuration per call) first,
        # as in the theatre workload
        trees = [rt.rt_build_tree(*m, stream=stream) for m in mesh]
        rooms = [dict(tree=t, sources=r.sources, rcv_center=r.rcv_center, rcv_radius=r.rcv_radius,
                      rcv_source=r.rcv_source, band_absorption=r.alpha) for t, r in zip(trees, rooms_sc)]
        prev = None
        for _ in range(40):
            isrc = rt.rt_trace_batch(rooms, n_rays, B, ray_begin=0, ray_count=chunk, tail_rays=rt.RT_TAIL_AUTOTUNE,
                                     stream=stream, workspace=ws_trace)
            cur = (isrc.block_size, int(isrc.tail_rays), isrc.compaction_period, isrc.stack_entries)
            del isrc
            if cur == prev:
                break
            prev = cur
        del trees, rooms
        if args.tree == "auto":  # the builder whose whole step is faster (one step each)
            for k in TREES:
                kind[0] = k
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                step()
                b.record(stream)
                b.synchronize()
                selection[k] = a.elapsed_time(b)
            kind[0] = min(TREES, key=lambda k: selection[k])
        for _ in range(max(args.warmup, 1)):
            step()
        torch.cuda.synchronize()
        launches0 = rt.rt_launch_count()
        ms, queries = [], []
        with ClockSampler(0, args.clock_log) as clk:
            for _ in range(args.steps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                q, cfg = step()
                queries.append(q)
                b.record(stream)
                b.synchronize()
                ms.append(a.elapsed_time(b))
        launches = rt.rt_launch_count() - launches0
    t = sum(ms) / 1e3
    tris = [len(r.tris) for r in rooms_sc]
    print(json.dumps({
        "metric": "ray-bounce hits/s, batched rooms", "value": sum(queries) / t, "unit": "queries/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{len(rooms_sc)} rooms ({min(tris)}-{max(tris)} tris, {sum(tris)} in total) x "
                               f"{len(rooms_sc[0].sources)} pairs x {n_rays} rays x {B} bounces, receivers r=0.5 m",
                   "rays_per_trace_per_pair": chunk, "traces_per_step": -(-n_rays // chunk),
                   "bounce_kernel": cfg, "queries_per_step": statistics.mean(queries),
                   "tree": kind[0], "tree_selection_ms_per_step": selection,
                   "step": "64 tree builds + batched traces + RIRs", "l2": "inputs larger than L2"},
        "gpu_launches": launches, "clocks": clk.summary()}))


# single-core times of one iteration on the refined tetrahedron (N = M) as the
# paper prints them (Sec. 2.2, Table 2): faces -> (without tree, with tree) seconds
PAPER_TABLE2 = {1024: (0.26, 0.2), 2048: (0.4, 0.2), 4096: (0.91, 0.25), 8192: (3.05, 0.3), 16384: (11.44, 0.33),
                32768: (46.02, 0.55), 65536: (181.61, 0.77), 131072: (725.17, 1.85), 262144: (2927.9, 2.76),
                524288: (None, 8.36), 1048576: (None, 13.78)}


def run_tetra(args):
    """One ray-tracing iteration (one nearest-face query per ray) with N = M
    rays and faces, source at the centre of the unit tetrahedron refined to
    M = 4 * 4^level faces (M = 2^10 ... 2^20): tree build and iteration on the
    GPU, and the FP64 oracle (its median-split tree) on the host cores."""
    import torch
    import oracle
    from paper_1811_05784_gb300 import rt
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream()
    rows = []
    for level in range(4, 10):
        sc = scenes.tetra(level)
        M = len(sc.tris)
        kw = rt.scene_args(sc)
        mesh = tuple(torch.as_tensor(x, device=dev) for x in (sc.vertices, sc.tris, sc.material_id, sc.surface_id))
        with torch.cuda.stream(stream):
            for _ in range(max(args.warmup, 1)):
                rt.rt_trace(rt.rt_build_tree(*mesh, stream=stream), stream=stream, **kw)
            torch.cuda.synchronize()
            b_ms, t_ms, q_ms = [], [], []
            for _ in range(args.steps):
                e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                e[0].record(stream)
                tree = rt.rt_build_tree(*mesh, stream=stream)
                e[1].record(stream)
                isrc = rt.rt_trace(tree, stream=stream, **kw)
                e[2].record(stream)
                e[2].synchronize()
                b_ms.append(e[0].elapsed_time(e[1]))
                t_ms.append(e[1].elapsed_time(e[2]))
                q_ms.append(isrc.ms_bounces)
        t0 = time.perf_counter()
        osc = oracle.OracleScene(sc, tree=True)
        t1 = time.perf_counter()
        tr = oracle.trace(osc)
        t2 = time.perf_counter()
        single = None
        if M <= 65_536:
            t3 = time.perf_counter()
            oracle.trace(osc, threads=1)
            single = time.perf_counter() - t3
        paper = PAPER_TABLE2.get(M, (None, None))
        rows.append({"faces": M, "rays": M, "queries": isrc.queries, "gpu_tree_ms": statistics.median(b_ms),
                     "gpu_iteration_ms": statistics.median(t_ms), "gpu_query_loop_ms": statistics.median(q_ms),
                     "oracle_tree_s": t1 - t0, "oracle_iteration_s": t2 - t1,
                     "oracle_threads": oracle.default_threads(), "oracle_iteration_1thread_s": single,
                     "oracle_queries": tr.queries, "paper_with_tree_s": paper[1], "paper_without_tree_s": paper[0]})
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    print(json.dumps({"metric": "time of one ray-tracing iteration, tetrahedron N = M", "unit": "s",
                      "higher_is_better": False, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "dtype": "f32", "data": "synthetic",
                      "config": {"workload": "unit tetrahedron refined to M = 4 * 4^level faces (level 4..9), "
                                             "N = M Fibonacci rays from the centre, 1 bounce",
                                 "gpu_iteration": "rt_trace: ray generation, one query per ray, measurement "
                                                  "sphere, image sources"},
                      "sweep": rows}))


def run_trees(args):
    """The LBVH against the paper's median-split tree and the LBVH with SAH
    top levels on the same meshes and rays: build time, node visits and
    triangle tests per query, bounce-loop time (the same 4-wide traversal
    kernel); and for the first bounce's
    queries the per-ray stack traversal against the paper's level-by-level
    distribution of rays through the tree (rt_nearest_hits): time, node
    visits, triangle tests and the bytes they read."""
    import torch
    from paper_1811_05784_gb300 import rt
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream()
    rows = []
    for name, make in (("theatre", lambda: scenes.theatre(n_rays=N_RAYS, n_bounces=N_BOUNCES)),
                       ("lroom", lambda: scenes.lroom(n_rays=N_RAYS, n_bounces=50)),
                       ("tetra 2^20, 1 bounce", lambda: scenes.tetra(9))):
        sc = make()
        kw = rt.scene_args(sc)
        mesh = tuple(torch.as_tensor(x, device=dev) for x in (sc.vertices, sc.tris, sc.material_id, sc.surface_id))
        for kind in ("lbvh", "median", "sah_top"):
            build = dict(median=kind == "median", sah=kind == "sah_top")
            with torch.cuda.stream(stream):
                for _ in range(max(args.warmup, 1)):
                    tree = rt.rt_build_tree(*mesh, stream=stream, **build)
                    rt.rt_trace(tree, tail_rays=N_RAYS, block_size=256, stream=stream, **kw)
                torch.cuda.synchronize()
                b_ms, q_ms = [], []
                for _ in range(args.steps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    tree = rt.rt_build_tree(*mesh, stream=stream, **build)
                    e1.record(stream)
                    isrc = rt.rt_trace(tree, tail_rays=N_RAYS, block_size=256, stream=stream, **kw)
                    torch.cuda.synchronize()
                    b_ms.append(e0.elapsed_time(e1))
                    q_ms.append(isrc.ms_bounces)
                cost = torch.zeros((sc.n_bounces, isrc.n_traced, 2), dtype=torch.int32, device=dev)
                isrc = rt.rt_trace(tree, tail_rays=N_RAYS, block_size=256, stream=stream, debug_cost=cost, **kw)
                torch.cuda.synchronize()
                c = cost.double().sum((0, 1)).cpu().numpy()
                del cost
            info = tree.info()
            row = {"mesh": name, "tris": len(sc.tris),
                   "tree": {"lbvh": "LBVH", "median": "median split", "sah_top": "LBVH + SAH top"}[kind],
                   "depth": info["depth"], "wide_nodes": info["n_nodes"], "build_ms": statistics.median(b_ms),
                   "bounce_ms": statistics.median(q_ms), "queries": isrc.queries,
                   "nodes_per_query": c[0] / isrc.queries, "tris_per_query": c[1] / isrc.queries}
            # the first bounce's queries by the per-ray stack and by the paper's
            # level-by-level distribution of rays through the tree
            n0 = isrc.n_traced
            ds = torch.empty((1, n0, 6), dtype=torch.float32, device=dev)
            kw1 = dict(kw, n_bounces=1)
            rt.rt_trace(tree, debug_state=ds, stream=stream, **kw1)
            torch.cuda.synchronize()
            o, d = ds[0, :, :3].contiguous(), ds[0, :, 3:].contiguous()
            for method, label in ((rt.RT_NEAREST_STACK, "stack"), (rt.RT_NEAREST_LEVELS, "levels")):
                with torch.cuda.stream(stream):
                    rt.rt_nearest_hits(tree, o, d, method=method, stream=stream)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    _, _, stt = rt.rt_nearest_hits(tree, o, d, method=method, stream=stream)
                    e1.record(stream)
                    e1.synchronize()
                row[f"first_bounce_{label}"] = {"ms": e0.elapsed_time(e1), "queries": n0,
                                                "nodes_per_query": stt[0] / n0, "tris_per_query": stt[1] / n0,
                                                "node_bytes_per_query": 112.0 * stt[0] / n0,
                                                "tri_bytes_per_query": 48.0 * stt[1] / n0}
            del ds
            rows.append(row)
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    print(json.dumps({"metric": "tree comparison: build time and traversal cost", "n_gpus": 1, "steps": args.steps,
                      "warmup": args.warmup, "data": "synthetic", "rows": rows}))


def run_gemm(args):
    """The surrogate network's BF16 GEMMs (rt_gemm_bf16) at batch 65,536: the
    forward products 960 -> 512, 512 -> 512, 512 -> 1568 and a weight
    gradient (K = batch, cut along K into a workspace), with the persistent
    TMA kernel and the register-staged one.  TFLOP/s from the device time of
    the product's kernels (CUDA events the library records on the stream;
    median of the timed calls), against the measured cuBLAS BF16 burst peak;
    each call also writes C (>= 64 MB), larger than half the L2, between
    timed launches."""
    import torch
    from paper_1811_05784_gb300 import rt
    torch.cuda.set_device(0)
    peak = None
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        peak = float(json.load(open(p))["bf16_tflops"])
    g = torch.Generator(device="cuda").manual_seed(0)
    ws = torch.empty(16 * 512 * 1568, dtype=torch.float32, device="cuda")
    rows = []
    for M, N, K in ((65536, 512, 960), (65536, 512, 512), (65536, 1568, 512), (512, 960, 65536)):
        A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
        B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
        C = torch.empty((M, N), dtype=torch.float32, device="cuda")
        row = {"M": M, "N": N, "K": K}
        for kernel, name in ((rt.RT_GEMM_TMA, "tma"), (rt.RT_GEMM_STAGED, "staged")):
            for _ in range(max(args.warmup, 3)):
                rt.rt_gemm_bf16(A, B, kernel=kernel, out=C, workspace=ws)
            ms, wall = [], []
            for _ in range(args.steps):
                t0 = time.perf_counter()
                _, t = rt.rt_gemm_bf16(A, B, kernel=kernel, out=C, workspace=ws, timed=True)
                wall.append((time.perf_counter() - t0) * 1e3)
                ms.append(t)
            t = statistics.median(ms)
            tf = 2.0 * M * N * K / (t * 1e-3) / 1e12
            row[name] = {"ms": t, "tflops": tf, "frac_of_bf16_peak": tf / peak if peak else None,
                         "call_ms": statistics.median(wall)}
        rows.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    print(json.dumps({"metric": "BF16 GEMM TFLOP/s of the surrogate network", "unit": "TFLOP/s", "n_gpus": 1,
                      "steps": args.steps, "warmup": args.warmup, "dtype": "bf16 x bf16 -> f32",
                      "peak": {"bf16_tflops": peak, "source": "MEASURED_PEAKS.json (cuBLAS, burst)"},
                      "note": "ms: device time of the product's kernels; call_ms: the whole call (tensor maps, "
                              "status read, synchronisation)",
                      "rows": rows}))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "lroom":
        run_lroom(args)
    elif args.workload == "gemm":
        run_gemm(args)
    elif args.workload == "tetra":
        run_tetra(args)
    elif args.workload == "trees":
        run_trees(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
