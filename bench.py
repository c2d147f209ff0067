"""Benchmark of the superpixel refinement hot path on GB300.

One step = one pass of the whole hot path over one image: level images (box sums),
seeding, every stage's refinement sweeps (with merges and prediction), as
``rapid_run`` runs it on the C ABI, starting from the image already in HBM.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle instead (the
method has no published implementation; the oracle is the reference arm), on a bounded
sample of the same workload.

Launch: ``python bench.py [--gpus N --steps K --warmup W]``; for N > 1 under
``torch.distributed.run`` (one process per GPU, independent replicas, no collective on the
data path).
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

METRIC = "Mpixel/s superpixel refinement (bit-exact) plain vs learned; % of HBM roofline"
UNIT = "Mpixel/s"
DEFAULT_WORKLOAD = "he4096_k4096_l3"
BATCH_WORKLOAD = "batch64_l3"   # the batched sub-object of the default line
DEFAULT_PRUNE = 0.05            # the learned sub-object: threshold, and the stages it prunes
DEFAULT_PRUNE_STAGES = "finest"  # (the finest stage alone: 0.37 points of boundary recall lost
                                 # at 0.05 on the 4096^2 tile, profiles/scorer_sweep_he4096_k4096_l3.md)
L2_FLUSH_BYTES = 256 << 20
SAMPLE_SIDE = 1024  # CPU legs: a 1024 x 1024 tile of the same generator and parameters


# builds of the stage kernel, by index: the queue schedule's evaluation-tile shape (blocks per
# tile), the threads per CTA, and the sweep schedule's bitmap walk (warp or CTA)
TILE_NAMES = ["32x16/cta", "32x8/warp", "64x16/cta", "32x16/512t/cta", "32x8/512t/warp", "64x16/512t/cta"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="rapid", choices=["rapid", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="full grid for every stage")
    ap.add_argument("--no-graph", action="store_true", help="launch stage by stage instead of a CUDA graph")
    ap.add_argument("--geometry", default=None,
                    help="pinned launch geometry instead of autotuning: 'grid,grid,...:shape,shape,...' per stage")
    ap.add_argument("--prune", type=float, default=None,
                    help="the learned path: train the block scorer (untimed) and prune at this threshold")
    ap.add_argument("--prune-stages", default="all", choices=["all", "finest"],
                    help="the stages the learned path prunes")
    ap.add_argument("--no-extra", action="store_true",
                    help="the plain line alone, without the learned and batched sub-objects")
    ap.add_argument("--classifier", action="store_true",
                    help="fit the linear classifier of Eq. predict on the superpixel features (untimed) and use it")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------- CPU sample (oracle legs)
def cpu_sample(workload: str):
    """A bounded sample of the workload for the CPU oracle: a tile of at most 1024 x 1024
    pixels of the same generator with the same superpixel size, region density and
    parameters (the whole image when it fits)."""
    from paper_1704_02083_gb300 import synth
    if workload in synth.SLIDES:
        sd = synth.SLIDES[workload]
        params = dict(sd["params"], K=max(1, SAMPLE_SIDE * SAMPLE_SIDE // sd["px_per_superpixel"]))
        img = synth.slide_image(SAMPLE_SIDE, SAMPLE_SIDE, sd["seed"])
        return img.rgb, params, (f"{SAMPLE_SIDE}x{SAMPLE_SIDE} slide of the same generator (seed {sd['seed']}) and "
                                 f"parameters (K={params['K']}), full schedule")
    if workload in synth.BATCHES:
        b = synth.BATCHES[workload]
        params = dict(b["params"])
        npx = SAMPLE_SIDE * SAMPLE_SIDE
        params["K"] = max(1, npx // b["px_per_superpixel"])
        cells = max(1, npx // b["px_per_cell"])
        seed = b["seed"]
        side_h = side_w = SAMPLE_SIDE
    else:
        w = synth.WORKLOADS[workload]
        side_h, side_w = min(SAMPLE_SIDE, w["H"]), min(SAMPLE_SIDE, w["W"])
        frac = (side_h * side_w) / float(w["H"] * w["W"])  # 1 when the image fits the sample: the workload itself
        params = dict(w["params"])
        params["K"] = max(1, int(round(params["K"] * frac)))
        cells = max(1, int(round(w["n_cells"] * frac)))
        seed = w["seed"]
    img = synth.he_image(side_h, side_w, cells, seed)
    desc = (f"{side_h}x{side_w} tile of the same generator (seed {seed}, {cells} regions) and parameters "
            f"(K={params['K']}, superpixel size and density as the workload), full schedule")
    return img.rgb, params, desc


def load_workload(name: str):
    """Images, per-image K and the common parameters of a workload (one image or a batch)."""
    from paper_1704_02083_gb300 import synth
    if name in synth.BATCHES:
        imgs, K = synth.batch_workload(name)
        return imgs, K, dict(synth.BATCHES[name]["params"])
    w = synth.WORKLOADS[name]
    params = dict(w["params"])
    return [synth.workload_image(name).rgb], [params.pop("K")], params


def host_cpu():
    """The host's CPU model and the cores this process may run on."""
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            key = line.split(":")[0].strip().lower()
            if key in ("model name", "cpu model", "hardware") and ":" in line:
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    if model is None:
        import platform
        model = platform.processor() or platform.machine()
    return {"cpu_model": model, "host_cores": len(os.sched_getaffinity(0)), "threads_used": 1}


def time_oracle(rgb, params, reps=1):
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle
    ts = []
    for _ in range(reps):
        o = oracle.Oracle(rgb, **params)
        t = time.perf_counter()
        o.run()
        ts.append(time.perf_counter() - t)
    return ts


def time_oracle_all_cores(rgb, params, reps=1):
    """The oracle's OpenMP build on every core this process may use: (seconds of the last
    run, threads)."""
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle
    threads = len(os.sched_getaffinity(0))
    t = None
    for _ in range(reps):
        o = oracle.Oracle(rgb, omp=True, threads=threads, **params)
        t0 = time.perf_counter()
        o.run()
        t = time.perf_counter() - t0
    return t, o.threads


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return

        def rd():
            for line in self.proc.stdout:
                self.rows.append([x.strip() for x in line.split(",")])

        self.thread = threading.Thread(target=rd, daemon=True)
        self.thread.start()

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) < 9:
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- algorithmic bytes
def stage_alg_bytes(H, W, stage_counters, level_factor, frontier=False):
    """Algorithmic bytes of one stage's refinement launch: one read of the block-resolution
    label map per sweep, one 4-byte write per move, and one read of the stage's colour
    source (3 bytes per pixel at full resolution, 3 int32 sums per coarse cell above it).
    The frontier schedule reads instead one queue bit per block per sweep and the label of
    each eligible block it pops."""
    s = stage_counters.block
    nb = -(-W // s) * -(-H // s)
    f = level_factor[stage_counters.level]
    src = 3 * H * W if f == 1 else 12 * (-(-W // f)) * (-(-H // f))
    if frontier:
        return nb * stage_counters.sweeps / 8 + 4 * stage_counters.eligible + 4 * stage_counters.moves + src
    return 4 * nb * stage_counters.sweeps + 4 * stage_counters.moves + src


def kernel_traffic(workload: str):
    """Per-launch DRAM bytes (ncu dram__bytes_read.sum + dram__bytes_write.sum) of the finest
    stage's launch on this workload from the committed ncu summary, when it was taken on the
    current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "stage_kernel_traffic.json")
    if not os.path.exists(path):
        return None, None
    d = json.load(open(path)).get(workload)
    if not d or d.get("kernel_source_sha256") != kernel_source_sha256():
        return None, d
    return d.get("dram_bytes_per_launch"), d


def kernel_source_sha256(csrc=None):
    """Hash of the code the stage kernel is compiled from: its sources with // comments,
    trailing blanks and empty lines removed, so that editing a comment keeps the counters."""
    csrc = csrc or os.path.join(ROOT, "paper_1704_02083_gb300", "csrc")
    h = hashlib.sha256()
    for name in ("stage_impl.cuh", "eval_tile.cuh", "eval_sweep.cuh", "rapid_dev.cuh", "k_stage_s0.cu",
                 "k_stage_s1.cu", "k_stage_s2.cu", "k_stage_s3.cu", "k_stage_s4.cu", "k_stage_s5.cu"):
        for line in open(os.path.join(csrc, name), encoding="utf-8"):
            code = line.split("//", 1)[0].rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()


# ---------------------------------------------------------------- replicas
def max_over_ranks(v: float, dist) -> float:
    """The largest value over all ranks (the slowest replica's time); v itself with one rank."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return v
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, steps: int, seconds_local: float, dist) -> float:
    """Units per second of the whole job: every rank's units over the slowest rank's time
    (replicas do the same work, so the job ends when the slowest one does)."""
    world = dist.get_world_size() if dist is not None and dist.is_initialized() else 1
    return world * units_per_rank * steps / max_over_ranks(seconds_local, dist)


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def golden_parity(workload: str, imgs, ctx, gpath=None):
    """The refined images' labels and statistics against the oracle's golden hashes
    (tests/golden/<workload>.json, written by make_golden.py from the oracle alone; a batch
    keeps one record per tile).  None when there is no record for this workload."""
    import numpy as np

    gpath = gpath or os.path.join(ROOT, "tests", "golden", f"{workload}.json")
    if not os.path.exists(gpath):
        return None
    g = json.load(open(gpath))
    records = g["tiles"] if "tiles" in g else [g]
    if len(records) != len(imgs):
        return None
    fields = ("n", "sum_r", "sum_g", "sum_b", "sum_x", "sum_y", "init_size")

    def sha(a):
        return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()

    def matches(i, rec):
        st_np = ctx.image_stats(i)
        stats7 = np.stack([st_np[f] for f in fields], 1).astype("<i8")
        return (sha(imgs[i]) == rec["image_sha256"] and sha(ctx.image_labels(i).astype("<i4")) == rec["labels_sha256"]
                and sha(stats7) == rec["stats_sha256"])

    ok = all(matches(i, rec) for i, rec in enumerate(records))
    what = "labels, S" if len(imgs) == 1 else f"labels, S of all {len(imgs)} tiles"
    return f"bit-exact vs the oracle's golden hashes ({what})" if ok else "MISMATCH vs the oracle's golden hashes"


# ---------------------------------------------------------------- arms
def run_reference(args, rank, world):
    """The reference arm: the oracle (the method has no published implementation) on every
    host core (its OpenMP build), each step one run of the workload itself; when W + K runs
    of it would take more than about four minutes, each step is the bounded 1024^2 sample
    instead (stated in `sample`)."""
    if rank != 0:
        return
    imgs, Ks, params = load_workload(args.workload)
    if len(imgs) == 1:
        rgb, params = imgs[0], dict(params, K=Ks[0])
        desc = f"the workload itself ({rgb.shape[0]}x{rgb.shape[1]}, K={params['K']}), one full run per step"
    else:
        rgb, params, desc = cpu_sample(args.workload)
    t_first, threads = time_oracle_all_cores(rgb, params)
    if t_first * (args.warmup + args.steps) > 240.0 and rgb.shape[0] * rgb.shape[1] > SAMPLE_SIDE ** 2:
        rgb, params, desc = cpu_sample(args.workload)
        t_first, threads = time_oracle_all_cores(rgb, params)
    npx = rgb.shape[0] * rgb.shape[1]
    ts = [t_first] + [time_oracle_all_cores(rgb, params)[0] for _ in range(args.warmup + args.steps - 1)]
    ts = ts[args.warmup:] if args.steps > 0 else ts
    total = sum(ts)
    value = npx * len(ts) / total / 1e6
    cpu = {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle (OpenMP build, every host core)",
           "sample": desc, **dict(host_cpu(), threads_used=threads)}
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": len(ts), "warmup": args.warmup, "ms_per_step": 1e3 * total / len(ts),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": args.workload, "sample": desc},
        "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_rapid(args, rank, world, local):
    import torch

    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    out = measure(args, rank, world, local, dist, args.workload, args.prune, args.classifier, args.geometry,
                  args.prune_stages)
    extras = (not args.no_extra and args.workload == DEFAULT_WORKLOAD and args.prune is None
              and not args.classifier and not args.geometry)
    if extras:  # plain vs learned vs batched, side by side in the same line
        learned = measure(args, rank, world, local, dist, args.workload, DEFAULT_PRUNE, False, None,
                          DEFAULT_PRUNE_STAGES)
        batched = measure(args, rank, world, local, dist, BATCH_WORKLOAD, None, False, None)
        if rank == 0:
            out["learned"] = sub_line(learned)
            out["batched"] = sub_line(batched)
    if rank == 0:
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baselines(args.workload)
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def sub_line(m):
    """The parts of a measurement that a side-by-side sub-object keeps."""
    keep = ("value", "unit", "ms_per_step", "ms_per_step_median", "roofline", "e2e", "gpu_launches", "clocks")
    out = {k: m[k] for k in keep if k in m}
    out["config"] = {k: m["config"].get(k) for k in ("workload", "images", "pixels", "K_total", "M_total", "path",
                                                       "scorer", "parity", "stage_grids", "stage_tiles",
                                                       "cuda_graph")}
    return out


def cpu_baselines(workload: str):
    """The oracle on the host cores: single-threaded and on every core (OpenMP over the
    blocks of a phase), each timing one run of the workload itself."""
    imgs, Ks, params = load_workload(workload)
    if len(imgs) != 1:
        rgb, params, desc = cpu_sample(workload)
    else:
        rgb, params = imgs[0], dict(params, K=Ks[0])
        desc = f"the workload itself ({rgb.shape[0]}x{rgb.shape[1]}, K={params['K']}), one full run"
    npx = rgb.shape[0] * rgb.shape[1]
    t1 = time_oracle(rgb, params, reps=1)[0]
    tn, threads = time_oracle_all_cores(rgb, params)
    return {"value": npx / t1 / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc, **host_cpu(),
            "all_cores": {"value": npx / tn / 1e6, "unit": UNIT, "cores": threads, "kind": "oracle (OpenMP build)",
                          "sample": desc, "speedup_over_one_core": t1 / tn}}


def stage_count(params) -> int:
    """Stages of the schedule: block sides halving from the initial block (at least the
    coarsest level's factor) to the final grain, each on the coarsest level whose factor
    divides it."""
    L, C = params["num_levels"], params.get("ratio_C", 4)
    f1 = C ** (L - 1)
    s, n = max(params["init_block"], f1), 0
    while s >= 1 and s >= params.get("final_grain", 1):
        if not any(C ** (L - l) <= s for l in range(1, L + 1)):
            break
        n += 1
        s //= 2
    return max(n, 1)


def measure(args, rank, world, local, dist, workload, prune, use_classifier, geometry, prune_stages="all"):
    """One workload's measurement (the JSON line without the CPU baseline)."""
    import numpy as np
    import torch

    import paper_1704_02083_gb300 as pkg

    imgs, Ks, params = load_workload(workload)
    n = len(imgs)
    scorer = None
    if prune is not None:  # the learned path: move logs of plain runs on other seeds, then training
        from paper_1704_02083_gb300 import scorer as sc
        w_scorer, train_info = sc.collect_and_train(*sc.training_tiles())
        scorer = dict(threshold=prune, stages=prune_stages, train=train_info)
    classifier = None
    if use_classifier:  # features and ground truth at the prediction point of other seeds, then the fit
        from paper_1704_02083_gb300 import roi
        theta, cls_info = roi.train()
        classifier = dict(train=cls_info)
    sizes = [(int(x.shape[0]), int(x.shape[1])) for x in imgs]
    npx = sum(h * w for h, w in sizes)
    stream = torch.cuda.Stream()  # a graph needs a non-default stream
    torch.cuda.set_stream(stream)
    dev_imgs = [torch.from_numpy(x).cuda() for x in imgs]
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    ctx = pkg.Context(stream=stream, **params)
    ctx.set_images(dev_imgs, Ks)
    stage_on = None
    if prune_stages == "finest":
        nst_p = stage_count(params)
        stage_on = [0] * (nst_p - 1) + [1]
    if scorer is not None:
        ctx.set_scorer(w_scorer, prune)
        if stage_on is not None:
            ctx.set_scorer_stages(stage_on)
    if classifier is not None:
        ctx.set_classifier(theta)
    if geometry:
        g_str, s_str = geometry.split(":")
        grids, shapes = [int(x) for x in g_str.split(",")], [int(x) for x in s_str.split(",")]
        ctx.set_stage_grids(grids)
        ctx.set_stage_shapes(shapes)
    else:
        grids, shapes = ctx.autotune() if not args.no_autotune else (None, None)
    ctx.set_profiling(True)
    ctx.set_graph(not args.no_graph)
    for _ in range(args.warmup):
        ctx.run()
    ctx.sync()
    c0 = ctx.counters(0)
    nst = None  # stages of the schedule, known after the first run
    L, C = params["num_levels"], params["ratio_C"]
    lf = {l: C ** (L - l) for l in range(1, L + 1)}

    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    step_ms, stage_ms, stage_bytes = [], [], []
    for _ in range(args.steps):
        flush.zero_()  # L2 flush between steps (outside the timed events)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.run()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        if nst is None:
            nst = ctx.counters(0).num_stages
            stage_ms, stage_bytes = [0.0] * nst, [0] * nst
        for i in range(n):
            c = ctx.counters(i)
            for s in range(nst):
                st = c.stage[s]
                if i == 0:
                    stage_ms[s] += st.kernel_ms  # the launch covers every image
                stage_bytes[s] += stage_alg_bytes(sizes[i][0], sizes[i][1], st, lf, params.get("schedule", 0) == 1)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    c1 = ctx.counters(0)
    launches_per_step = (c1.launches - c0.launches) / max(1, args.steps)

    total_ms = max_over_ranks(sum(step_ms), dist)
    value = whole_job_rate(npx, args.steps, total_ms / 1e3, dist) / 1e6

    # end to end through the C ABI from pinned host memory: H2D images, run, D2H labels + stats
    e2e = None
    if not args.no_e2e:
        pins = [torch.from_numpy(x).pin_memory() for x in imgs]
        labs = [torch.empty(hw, dtype=torch.int32).pin_memory() for hw in sizes]
        Ms = [ctx.image_info(i)["M"] for i in range(n)]
        stats_host = [np.zeros(m, pkg.SP_STATS_DTYPE) for m in Ms]
        e2e_ctx = pkg.Context(stream=stream, **params)
        if grids is not None:
            e2e_ctx.set_stage_grids(grids)
            e2e_ctx.set_stage_shapes(shapes)
        if scorer is not None:
            e2e_ctx.set_scorer(w_scorer, prune)
            if stage_on is not None:
                e2e_ctx.set_scorer_stages(stage_on)
        ptrs = [p.data_ptr() for p in pins]
        times = []
        for it in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            t = time.perf_counter()
            pkg.rapid_set_images(e2e_ctx.h, ptrs, [h for h, _ in sizes], [w for _, w in sizes],
                                 [3 * w for _, w in sizes], Ks, 0)
            pkg.rapid_run(e2e_ctx.h)
            for i in range(n):
                pkg.rapid_read_image_labels(e2e_ctx.h, i, labs[i].data_ptr(), 4 * sizes[i][1], 0)
                pkg.rapid_read_image_stats(e2e_ctx.h, i, stats_host[i].ctypes.data, Ms[i])
            if it >= args.warmup:
                times.append(time.perf_counter() - t)
        e2e_ctx.close()
        e2e = {"value": whole_job_rate(npx, len(times), sum(times), dist) / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": 3 * npx,
               "d2h_bytes_per_step": 4 * npx + sum(Ms) * pkg.SP_STATS_DTYPE.itemsize}

    # parity in the same run: the plain path's labels and statistics against the oracle's
    # golden hashes (written by tests/golden/make_golden.py from the oracle alone)
    parity = None
    if scorer is None and classifier is None:
        parity = golden_parity(workload, imgs, ctx)
    elif scorer is not None:
        parity = ("pruned sweeps bit-exact vs the oracle under the same keep masks (tests/test_gpu_keep_mask.py); "
                  "the masks here are the scorer's, judged by quality against the plain run")

    if scorer is not None:  # judged by the plain method: its labels, and the ground truth
        from paper_1704_02083_gb300 import quality, synth
        gts = [synth.workload_image(workload).regions] if n == 1 else None
        plain = pkg.Context(stream=stream, **params)
        plain.set_images(dev_imgs, Ks)
        plain.run()
        q = dict(disagreement=0.0, br_plain=0.0, br_pruned=0.0, ue_plain=0.0, ue_pruned=0.0)
        for i in range(n):
            a, b = plain.image_labels(i), ctx.image_labels(i)
            wgt = a.size / npx
            q["disagreement"] += wgt * quality.disagreement(a, b)
            if gts is not None:
                q["br_plain"] += wgt * quality.boundary_recall(a, gts[i])
                q["br_pruned"] += wgt * quality.boundary_recall(b, gts[i])
                q["ue_plain"] += wgt * quality.undersegmentation_error(a, gts[i])
                q["ue_pruned"] += wgt * quality.undersegmentation_error(b, gts[i])
        plain.close()
        scorer["quality"] = {k: round(v, 5) for k, v in q.items()}
        scorer["evaluated_blocks"] = int(sum(ctx.counters_array(i)[:, 4].sum() for i in range(n)))

    if classifier is not None and n == 1 and rank == 0:  # judged against the brightness stand-in (untimed)
        from paper_1704_02083_gb300 import roi, synth
        classifier["eval"] = roi.evaluate(theta, synth.workload_image(workload), Ks[0], dict(params),
                                          stream=stream)
        classifier["parity"] = "bit-exact vs the oracle in tests/test_gpu_classifier.py (features, y, runs)"

    sched_quality = None
    if params.get("schedule", 0) == 1 and n == 1 and rank == 0:  # judged by the sweep schedule (untimed)
        from paper_1704_02083_gb300 import quality, synth
        gt = synth.workload_image(workload).regions
        sw = pkg.Context(stream=stream, **dict(params, schedule=0))
        sw.set_images(dev_imgs, Ks)
        sw.run()
        a, b = sw.image_labels(0), ctx.image_labels(0)
        sched_quality = {"br_sweeps": quality.boundary_recall(a, gt), "br_frontier": quality.boundary_recall(b, gt),
                         "ue_sweeps": quality.undersegmentation_error(a, gt),
                         "ue_frontier": quality.undersegmentation_error(b, gt),
                         "disagreement": float(quality.disagreement(a, b)),
                         "evaluated_sweeps": int(sw.counters_array(0)[:, 4].sum()),
                         "evaluated_frontier": int(ctx.counters_array(0)[:, 4].sum())}
        sched_quality = {k: (round(v, 5) if isinstance(v, float) else v) for k, v in sched_quality.items()}
        sw.close()

    # roofline of the dominant launch: the stage launch with the largest device time (the
    # finest stage); its duration from CUDA events around each stage launch on ``stream``
    peak, peak_kind = measured_peak()
    dom = max(range(nst), key=lambda s: stage_ms[s])
    launch_ms = stage_ms[dom] / args.steps
    launch_bytes = stage_bytes[dom] / args.steps
    achieved = launch_bytes / (launch_ms / 1e3) / 1e9 if launch_ms > 0 else None
    all_ms, all_bytes = sum(stage_ms), sum(stage_bytes)
    all_achieved = all_bytes / (all_ms / 1e3) / 1e9 if all_ms > 0 else None
    traffic, _ = kernel_traffic(workload)
    st_dom = c1.stage[dom]
    out = None
    if rank == 0:
        cfg = {"workload": workload, "images": n, "pixels": npx, "K_total": int(sum(Ks)),
               "M_total": int(sum(ctx.image_info(i)["M"] for i in range(n))),
               "levels": params["num_levels"], "ratio_C": params["ratio_C"], "init_block": params["init_block"],
               "final_grain": params["final_grain"], "size_mode": params["size_mode"],
               "predict": params["predict"], "reuse": params["reuse"],
               "stage_grids": grids[:nst] if grids is not None else None,
               "stage_tiles": [TILE_NAMES[k] for k in shapes[:nst]] if shapes else None,
               "cuda_graph": not args.no_graph,
               "path": "plain" if scorer is None else "learned pruning", "scorer": scorer, "parity": parity,
               "schedule": "frontier queue" if params.get("schedule", 0) == 1 else "sweeps",
               "schedule_quality": sched_quality,
               "classifier": classifier,
               "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write, untimed)",
               "parallelism": f"replicas x{world}"}
        if n == 1:
            cfg.update({"H": sizes[0][0], "W": sizes[0][1]})
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "ms_per_step_median": statistics.median(step_ms), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg,
            "roofline": {"kernel": f"stage_kernel, stage {dom} (level {st_dom.level}, block side {st_dom.block})",
                         "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": (achieved / peak) if achieved else None, "peak_source": peak_kind,
                         "traffic": traffic, "alg_bytes_per_launch": launch_bytes, "launch_ms": launch_ms,
                         "kernel_source_sha256": kernel_source_sha256()[:16],
                         "share_of_step": launch_ms / (total_ms / args.steps),
                         "all_stage_launches": {"launches_per_step": nst,
                                                "ms_per_step": all_ms / args.steps,
                                                "stage_ms": [round(x / args.steps, 3) for x in stage_ms],
                                                "alg_bytes_per_step": all_bytes / args.steps,
                                                "achieved": all_achieved,
                                                "frac": (all_achieved / peak) if all_achieved else None}},
            "cpu_baseline": None,
            "e2e": e2e,
            "gpu_launches": int(round(launches_per_step * args.steps)),
            "clocks": clk,
        }
    ctx.close()
    return out


def slide_batches(H, W, max_tile, px_per_superpixel, max_batch=64, max_px=1 << 30) -> int:
    """How many batches rapid_refine_slide makes of a slide's tiles (up to max_batch tiles
    and max_px pixels each, at least one tile)."""
    from paper_1704_02083_gb300 import synth
    n, k, px = 0, 0, 0
    for (_, _, h, w, _) in synth.slide_tiles(H, W, max_tile, px_per_superpixel):
        if k == 0 or k == max_batch or px + h * w > max_px:
            n, k, px = n + 1, 0, 0
        k, px = k + 1, px + h * w
    return n


def slide_parity(workload: str, rgb, labels, stats):
    """The sampled tiles of a slide against the oracle's records (tests/golden/<workload>.json,
    written by make_golden.py from the host restatement of the generator and the oracle
    alone): the tile's pixels, its labels (slide-wide ids minus the tile's first id) and the
    statistics of its ids.  None when there is no record."""
    import numpy as np

    import paper_1704_02083_gb300 as pkg

    gpath = os.path.join(ROOT, "tests", "golden", f"{workload}.json")
    if not os.path.exists(gpath):
        return None
    g = json.load(open(gpath))
    fields = ("n", "sum_r", "sum_g", "sum_b", "sum_x", "sum_y", "init_size")
    st_all = stats.view(-1, pkg.SP_STATS_DTYPE.itemsize)

    def sha(a):
        return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()

    ok = []
    for rec in g["sampled"]:
        r0, c0, h, w, base, M = rec["row0"], rec["col0"], rec["H"], rec["W"], rec["id_base"], rec["M"]
        img = rgb[r0:r0 + h, c0:c0 + w].cpu().numpy()
        lab = (labels[r0:r0 + h, c0:c0 + w].cpu().numpy().astype(np.int64) - base).astype("<i4")
        st = st_all[base:base + M].cpu().numpy().copy().view(pkg.SP_STATS_DTYPE).reshape(-1)
        st7 = np.stack([st[f] for f in fields], 1).astype("<i8")
        ok.append(sha(img) == rec["image_sha256"] and sha(lab) == rec["labels_sha256"] and
                  sha(st7) == rec["stats_sha256"])
    tiles = ", ".join(str(r["tile"]) for r in g["sampled"])
    return (f"bit-exact vs the oracle's records of sampled tiles {tiles} (pixels, labels, S)" if all(ok)
            else f"MISMATCH vs the oracle's records (tiles {tiles}: {ok})")


def run_slide(args, rank, world, local):
    """A whole slide through rapid_refine_slide: tiles of at most max_tile px as views into the
    slide in HBM, refined in batches; one step = the whole slide."""
    import numpy as np
    import torch

    import __graft_entry__
    import paper_1704_02083_gb300 as pkg
    from paper_1704_02083_gb300 import synth

    __graft_entry__.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    sd = synth.SLIDES[args.workload]
    H, W, params = sd["H"], sd["W"], dict(sd["params"])
    npx = H * W
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    gen_s, img = None, None
    if sd.get("generator") == "counter":  # made on the device (the counter-based definition)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rgb = pkg.synth_slide_device(H, W, sd["seed"], px_per_cell=sd["px_per_cell"], white_frac=sd["white_frac"],
                                     fold_frac=sd["fold_frac"], stream=stream)
        torch.cuda.synchronize()
        gen_s = time.perf_counter() - t0
    else:
        img = synth.slide_image(H, W, sd["seed"])
        rgb = torch.from_numpy(img.rgb).cuda()
    labels = torch.empty((H, W), dtype=torch.int32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    ctx = pkg.Context(stream=stream, **params)
    ctx.set_profiling(True)
    geometry = args.geometry or sd.get("geometry")
    if geometry:  # a pinned launch geometry instead of tuning on the first batch
        g_str, s_str = geometry.split(":")
        ctx.set_stage_grids([int(x) for x in g_str.split(",")])
        ctx.set_stage_shapes([int(x) for x in s_str.split(",")])
    kw = dict(max_tile=sd["max_tile"], px_per_superpixel=sd["px_per_superpixel"], labels=labels)
    _, M, T = ctx.refine_slide(rgb, autotune=not args.no_autotune and not geometry, **kw)  # first warm-up run tunes
    stats = torch.empty(M * pkg.SP_STATS_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    kw["stats"] = stats  # the statistics of every slide-wide id, with the labels
    for _ in range(max(0, args.warmup - 1)):
        ctx.refine_slide(rgb, **kw)
    ctx.sync()
    c0 = ctx.counters(0)
    L, C = params["num_levels"], params["ratio_C"]
    lf = {l: C ** (L - l) for l in range(1, L + 1)}
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    step_ms, stage_ms, stage_bytes, nst, nimg = [], [], [], None, 0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.refine_slide(rgb, **kw)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        if nst is None:
            nst = ctx.counters(0).num_stages
            stage_ms, stage_bytes = [0.0] * nst, [0] * nst
        nimg = 0
        while True:  # the images of the slide's last batch (every tile when it fits in one)
            try:
                info = ctx.image_info(nimg)
            except pkg.RapidError:
                break
            c = ctx.counters(nimg)
            for st_i in range(nst):
                if nimg == 0:
                    stage_ms[st_i] += c.stage[st_i].kernel_ms
                stage_bytes[st_i] += stage_alg_bytes(info["H"], info["W"], c.stage[st_i], lf,
                                                     params.get("schedule", 0) == 1)
            nimg += 1
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    c1 = ctx.counters(0)
    total_ms = max_over_ranks(sum(step_ms), dist)
    value = whole_job_rate(npx, args.steps, total_ms / 1e3, dist) / 1e6

    e2e = None
    if not args.no_e2e:  # pinned host slide -> HBM, refine, labels -> pinned host
        if img is not None:
            pin = torch.from_numpy(img.rgb).pin_memory()
        else:
            pin = torch.empty((H, W, 3), dtype=torch.uint8).pin_memory()
            pin.copy_(rgb)
        lab_host = torch.empty((H, W), dtype=torch.int32).pin_memory()
        times = []
        for it in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            t = time.perf_counter()
            rgb.copy_(pin, non_blocking=True)
            ctx.refine_slide(rgb, **kw)
            lab_host.copy_(labels, non_blocking=True)
            torch.cuda.synchronize()
            if it >= args.warmup:
                times.append(time.perf_counter() - t)
        e2e = {"value": whole_job_rate(npx, len(times), sum(times), dist) / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": 3 * npx, "d2h_bytes_per_step": 4 * npx}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rgb_s, params_s, desc = cpu_sample(args.workload)
        ts = time_oracle(rgb_s, params_s, reps=1)
        cpu = {"value": rgb_s.shape[0] * rgb_s.shape[1] / ts[0] / 1e6, "unit": UNIT, "cores": 1,
               "kind": "oracle", "sample": desc, **host_cpu()}

    free_b, total_b = torch.cuda.mem_get_info()
    dev_used_gb = (total_b - free_b) / 1e9  # the slide, its labels and the context's buffers
    parity = slide_parity(args.workload, rgb, labels, stats) if rank == 0 else None
    peak, peak_kind = measured_peak()
    dom = max(range(nst), key=lambda i: stage_ms[i])
    launch_ms, launch_bytes = stage_ms[dom] / args.steps, stage_bytes[dom] / args.steps
    achieved = launch_bytes / (launch_ms / 1e3) / 1e9 if launch_ms > 0 else None
    st_dom = c1.stage[dom]
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "ms_per_step_median": statistics.median(step_ms), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "H": H, "W": W, "tiles": T, "max_tile": sd["max_tile"],
                       "M_total": M, "px_per_superpixel": sd["px_per_superpixel"],
                       "batches": slide_batches(H, W, sd["max_tile"], sd["px_per_superpixel"]),
                       "levels": L, "ratio_C": C,
                       "init_block": params["init_block"], "predict": params["predict"],
                       "schedule": "frontier queue" if params.get("schedule", 0) == 1 else "sweeps",
                       "generator": ("counter-based, on the device" if gen_s is not None else "host"),
                       "generation_s": gen_s, "parity": parity,
                       "device_memory_in_use_gb": dev_used_gb,
                       "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write, untimed)",
                       "parallelism": f"replicas x{world}"},
            "roofline": {"kernel": f"stage_kernel, stage {dom} (level {st_dom.level}, block side {st_dom.block}), "
                                   f"last batch ({nimg} tiles)",
                         "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": (achieved / peak) if achieved else None, "peak_source": peak_kind, "traffic": None,
                         "alg_bytes_per_launch": launch_bytes, "launch_ms": launch_ms},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(round((c1.launches - c0.launches))),
            "clocks": clk,
        }
        print(json.dumps(out), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    from paper_1704_02083_gb300 import synth
    if args.workload in synth.SLIDES:
        run_slide(args, rank, world, local)
        return
    run_rapid(args, rank, world, local)


if __name__ == "__main__":
    main()
