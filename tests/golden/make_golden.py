"""Write tests/golden/<workload>.json from the CPU oracle alone.

For each full-size workload: SHA-256 of the generated image, of the oracle's full-res
label map (int32 little-endian, row-major) and of its statistics (M x 7 int64: N, R, G, B,
X, Y, InitSize), the per-stage counters, and a few sampled labels.  A batch workload gets
the same record for each of its tiles, each refined alone (tiles run in parallel worker
processes); a slide workload one for each of its sampled tiles, generated alone from the
counter-based definition.  The CUDA path is never run here.
Usage: python tests/golden/make_golden.py [workload ...]
"""
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "oracle"))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1704_02083_gb300 import synth  # noqa: E402


def sha(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def record(rgb: np.ndarray, params: dict, n_samples: int = 64, omp: bool = False) -> dict:
    """The oracle's run on one image, as hashes, counters and n_samples sampled labels
    (omp: the oracle's all-core build, whose results equal the single-threaded one's)."""
    H, W = rgb.shape[:2]
    t = time.time()
    o = oracle.Oracle(rgb, omp=omp, **params).run()
    dt = time.time() - t
    lab = o.labels().astype("<i4")
    s, y, imp = o.stats()
    rng = np.random.default_rng(0)
    ys = rng.integers(0, H, n_samples)
    xs = rng.integers(0, W, n_samples)
    return {
        "image_sha256": sha(rgb),
        "labels_sha256": sha(lab),
        "stats_sha256": sha(s.astype("<i8")),
        "y_sha256": sha(y.astype("i1")),
        "important_sha256": sha(imp.astype("u1")),
        "M": int(s.shape[0]),
        "live_labels": int((s[:, 0] > 0).sum()),
        "counters": o.counters().tolist(),
        "samples": [[int(a), int(b), int(lab[a, b])] for a, b in zip(ys, xs)],
        "oracle_seconds_on_writer": round(dt, 2),
    }


def make(name: str) -> dict:
    w = synth.WORKLOADS[name]
    return {"workload": name, "params": w["params"], **record(synth.workload_image(name).rgb, w["params"])}


def _tile(job):
    name, i = job
    rgb, K = synth.batch_tile(name, i)
    return {"tile": i, "H": int(rgb.shape[0]), "W": int(rgb.shape[1]), "K": K,
            **record(rgb, dict(synth.BATCHES[name]["params"], K=K), n_samples=16)}


def make_batch(name: str, workers: int) -> dict:
    import multiprocessing as mp
    b = synth.BATCHES[name]
    jobs = [(name, i) for i in range(b["n"])]
    sizes = synth.batch_sizes(b["n"], b["seed"])
    jobs.sort(key=lambda j: -sizes[j[1]][0] * sizes[j[1]][1])  # largest first
    with mp.get_context("spawn").Pool(workers) as pool:
        tiles = sorted(pool.map(_tile, jobs, chunksize=1), key=lambda d: d["tile"])
    return {"workload": name, "params": b["params"], "tiles": tiles}


def seed_count(H: int, W: int, K: int, side0: int) -> int:
    """Superpixels of the seed grid on the first stage's blocks (the oracle's seeding rule):
    gx = round(sqrt(K W / H)), gy = round(K / gx), each at least 1 and at most the block
    grid's width or height."""
    import math
    nbx, nby = -(-W // side0), -(-H // side0)
    gx = max(1, math.floor(math.sqrt(K * W / H) + 0.5))
    gy = max(1, math.floor(K / gx + 0.5))
    return min(gx, nbx) * min(gy, nby)


def make_slide(name: str) -> dict:
    """Records of a slide's sampled tiles (the slide partitioned as rapid_refine_slide cuts
    it), each tile generated alone on the host from the counter-based definition and refined
    alone by the oracle; id_base is the tile's first slide-wide label id (the seed-grid
    sizes of the tiles before it)."""
    sd = synth.SLIDES[name]
    H, W = sd["H"], sd["W"]
    tiles = synth.slide_tiles(H, W, sd["max_tile"], sd["px_per_superpixel"])
    p = sd["params"]
    L, C = p["num_levels"], p["ratio_C"]
    side0 = max(p["init_block"], C ** (L - 1))
    bases = [0]
    for (_, _, h, w, K) in tiles:
        bases.append(bases[-1] + seed_count(h, w, K, side0))
    out = []
    for t in sd["sample_tiles"]:
        r0, c0, h, w, K = tiles[t]
        img = synth.slide_gen(H, W, sd["seed"], x0=c0, y0=r0, h=h, w=w, px_per_cell=sd["px_per_cell"],
                              white_frac=sd["white_frac"], fold_frac=sd["fold_frac"])
        rec = record(img.rgb, dict(p, K=K), n_samples=16, omp=True)
        out.append({"tile": t, "row0": r0, "col0": c0, "H": h, "W": w, "K": K, "id_base": bases[t], **rec})
        print(name, "tile", t, rec["labels_sha256"][:16], rec["oracle_seconds_on_writer"], flush=True)
    return {"workload": name, "params": p, "tiles_total": len(tiles), "M_total": bases[-1], "sampled": out}


if __name__ == "__main__":
    names = sys.argv[1:] or ["he4096_k4096_l3"]
    for n in names:
        if n in synth.BATCHES:
            d = make_batch(n, max(1, min(8, os.cpu_count() or 1)))
            summary = (len(d["tiles"]), round(sum(t["oracle_seconds_on_writer"] for t in d["tiles"]), 1))
        elif n in synth.SLIDES:
            d = make_slide(n)
            summary = (len(d["sampled"]), d["M_total"])
        else:
            d = make(n)
            summary = (d["labels_sha256"][:16], d["oracle_seconds_on_writer"])
        with open(os.path.join(HERE, f"{n}.json"), "w") as f:
            json.dump(d, f, indent=None if ("tiles" in d or "sampled" in d) else 1)
        print(n, *summary)
