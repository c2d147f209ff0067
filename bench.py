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
L2_FLUSH_BYTES = 256 << 20
SAMPLE_SIDE = 1024  # CPU legs: a 1024 x 1024 tile of the same generator and parameters


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="rapid", choices=["rapid", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------- CPU sample (oracle legs)
def cpu_sample(workload: str):
    from paper_1704_02083_gb300 import synth
    w = synth.WORKLOADS[workload]
    frac = (SAMPLE_SIDE * SAMPLE_SIDE) / float(w["H"] * w["W"])
    side_h, side_w = min(SAMPLE_SIDE, w["H"]), min(SAMPLE_SIDE, w["W"])
    params = dict(w["params"])
    params["K"] = max(1, int(round(params["K"] * frac)))
    cells = max(1, int(round(w["n_cells"] * frac)))
    img = synth.he_image(side_h, side_w, cells, w["seed"])
    desc = (f"{side_w}x{side_h} tile of the same generator (seed {w['seed']}, {cells} regions) and parameters "
            f"(K={params['K']}, superpixel size and density as the workload), full schedule")
    return img.rgb, params, desc


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
def stage_alg_bytes(H, W, stage_counters, level_factor):
    """Algorithmic bytes of one stage's refinement launch: one read of the block-resolution
    label map per sweep, one 4-byte write per move, and one read of the stage's colour
    source (3 bytes per pixel at full resolution, 3 int32 sums per coarse cell above it)."""
    s = stage_counters.block
    nb = -(-W // s) * -(-H // s)
    f = level_factor[stage_counters.level]
    src = 3 * H * W if f == 1 else 12 * (-(-W // f)) * (-(-H // f))
    return 4 * nb * stage_counters.sweeps + 4 * stage_counters.moves + src


def kernel_traffic():
    """Per-launch DRAM bytes (ncu dram__bytes_read.sum + dram__bytes_write.sum) of the finest
    stage's launch from the committed ncu summary, when it was taken on the current kernel
    source; else None."""
    path = os.path.join(ROOT, "profiles", "stage_kernel_traffic.json")
    if not os.path.exists(path):
        return None, None
    d = json.load(open(path))
    if d.get("kernel_source_sha256") != kernel_source_sha256():
        return None, d
    return d.get("dram_bytes_per_launch"), d


def kernel_source_sha256():
    """Hash of the sources the stage kernel is compiled from."""
    csrc = os.path.join(ROOT, "paper_1704_02083_gb300", "csrc")
    h = hashlib.sha256()
    for name in ("k_stage.cu", "eval_tile.cuh", "rapid_dev.cuh"):
        h.update(open(os.path.join(csrc, name), "rb").read())
    return h.hexdigest()


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------- arms
def run_reference(args, rank, world):
    if rank != 0:
        return
    rgb, params, desc = cpu_sample(args.workload)
    npx = rgb.shape[0] * rgb.shape[1]
    ts = time_oracle(rgb, params, reps=args.warmup + args.steps)[args.warmup:]
    total = sum(ts)
    value = npx * len(ts) / total / 1e6
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(ts),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": args.workload, "sample": desc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_rapid(args, rank, world, local):
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

    w = synth.WORKLOADS[args.workload]
    H, W = w["H"], w["W"]
    params = dict(w["params"])
    img = synth.workload_image(args.workload)
    stream = torch.cuda.current_stream()
    rgb_dev = torch.from_numpy(img.rgb).cuda()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    ctx = pkg.Context(stream=stream, **params)
    ctx.set_image(rgb_dev)
    ctx.set_profiling(True)
    for _ in range(args.warmup):
        ctx.run()
    ctx.sync()
    c0 = ctx.counters()
    lf = {}
    L, C = params["num_levels"], params["ratio_C"]
    for l in range(1, L + 1):
        lf[l] = C ** (L - l)

    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    step_ms, stage_ms, stage_bytes = [], {}, {}
    for _ in range(args.steps):
        flush.zero_()  # L2 flush between steps (outside the timed events)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.run()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        c = ctx.counters()
        for i in range(c.num_stages):
            st = c.stage[i]
            stage_ms[i] = stage_ms.get(i, 0.0) + st.kernel_ms
            stage_bytes[i] = stage_bytes.get(i, 0) + stage_alg_bytes(H, W, st, lf)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    c1 = ctx.counters()
    launches_per_step = (c1.launches - c0.launches) / max(1, args.steps)

    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    npx = H * W
    value = world * npx * args.steps / (total_ms / 1e3) / 1e6

    # end to end through the C ABI from pinned host memory: H2D image, run, D2H labels + stats
    e2e = None
    if not args.no_e2e:
        pin = torch.from_numpy(img.rgb).pin_memory()
        lab_host = torch.empty((H, W), dtype=torch.int32).pin_memory()
        M = ctx.state()["M"]
        stats_host = np.zeros(M, pkg.SP_STATS_DTYPE)
        e2e_ctx = pkg.Context(stream=stream, **params)
        times = []
        for i in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            t = time.perf_counter()
            pkg.rapid_set_image(e2e_ctx.h, pin.data_ptr(), H, W, 3 * W, 0)
            pkg.rapid_run(e2e_ctx.h)
            pkg.rapid_read_labels(e2e_ctx.h, lab_host.data_ptr(), 4 * W, 0)
            pkg.rapid_read_stats(e2e_ctx.h, stats_host.ctypes.data, M)
            if i >= args.warmup:
                times.append(time.perf_counter() - t)
        e2e_ctx.close()
        tot = sum(times)
        if world > 1:
            t = torch.tensor([tot], dtype=torch.float64, device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            tot = float(t.item())
        e2e = {"value": world * npx * len(times) / tot / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": 3 * npx, "d2h_bytes_per_step": 4 * npx + M * pkg.SP_STATS_DTYPE.itemsize}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rgb_s, params_s, desc = cpu_sample(args.workload)
        ts = time_oracle(rgb_s, params_s, reps=1)
        cpu = {"value": rgb_s.shape[0] * rgb_s.shape[1] / ts[0] / 1e6, "unit": UNIT, "cores": 1,
               "kind": "oracle", "sample": desc}

    # roofline of the dominant launch: the stage launch with the largest device time (the
    # finest stage); its duration from CUDA events around each stage launch on ``stream``
    peak, peak_kind = measured_peak()
    dom = max(stage_ms, key=stage_ms.get)
    launch_ms = stage_ms[dom] / args.steps
    launch_bytes = stage_bytes[dom] / args.steps
    achieved = launch_bytes / (launch_ms / 1e3) / 1e9 if launch_ms > 0 else None
    all_ms, all_bytes = sum(stage_ms.values()), sum(stage_bytes.values())
    all_achieved = all_bytes / (all_ms / 1e3) / 1e9 if all_ms > 0 else None
    traffic, _ = kernel_traffic()
    st_dom = c1.stage[dom]
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "H": H, "W": W, "K": params["K"], "M": c1.M,
                       "levels": params["num_levels"], "ratio_C": params["ratio_C"],
                       "init_block": params["init_block"], "final_grain": params["final_grain"],
                       "size_mode": params["size_mode"], "predict": params["predict"], "reuse": params["reuse"],
                       "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write, untimed)",
                       "parallelism": f"replicas x{world}"},
            "roofline": {"kernel": f"stage_kernel, stage {dom} (level {st_dom.level}, block side {st_dom.block})",
                         "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": (achieved / peak) if achieved else None, "peak_source": peak_kind,
                         "traffic": traffic, "alg_bytes_per_launch": launch_bytes, "launch_ms": launch_ms,
                         "share_of_step": launch_ms / (total_ms / args.steps),
                         "all_stage_launches": {"launches_per_step": len(stage_ms),
                                                "ms_per_step": all_ms / args.steps,
                                                "alg_bytes_per_step": all_bytes / args.steps,
                                                "achieved": all_achieved,
                                                "frac": (all_achieved / peak) if all_achieved else None}},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(round(launches_per_step * args.steps)),
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
    run_rapid(args, rank, world, local)


if __name__ == "__main__":
    main()
