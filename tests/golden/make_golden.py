"""Write tests/golden/<workload>.json from the CPU oracle alone.

For each full-size workload: SHA-256 of the generated image, of the oracle's full-res
label map (int32 little-endian, row-major) and of its statistics (M x 7 int64: N, R, G, B,
X, Y, InitSize), the per-stage counters, and a few sampled labels.  The CUDA path is
never run here.  Usage: python tests/golden/make_golden.py [workload ...]
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


def make(name: str) -> dict:
    w = synth.WORKLOADS[name]
    img = synth.workload_image(name)
    t = time.time()
    o = oracle.Oracle(img.rgb, **w["params"]).run()
    dt = time.time() - t
    lab = o.labels().astype("<i4")
    s, y, imp = o.stats()
    rng = np.random.default_rng(0)
    ys = rng.integers(0, w["H"], 64)
    xs = rng.integers(0, w["W"], 64)
    return {
        "workload": name,
        "params": w["params"],
        "image_sha256": sha(img.rgb),
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


if __name__ == "__main__":
    names = sys.argv[1:] or ["he4096_k4096_l3"]
    for n in names:
        d = make(n)
        with open(os.path.join(HERE, f"{n}.json"), "w") as f:
            json.dump(d, f, indent=1)
        print(n, d["labels_sha256"][:16], d["oracle_seconds_on_writer"], "s")
