"""Training and evaluation of the learned block scorer: a host driver over the C ABI.

Training data are the move logs of plain runs (rapid_set_logging) on tiles of the 4096^2
tile's generator and schedule with other seeds; training is rapid_trainer_fit.  The plain
method is the reference it is measured against: boundary recall and undersegmentation error
against the generator's ground truth, and the fraction of pixels whose label differs from
the plain run's.
"""
from __future__ import annotations

import time

import numpy as np

from . import Context, Trainer, quality, synth

# Training tiles: seeds 100..107 of the generator, 2048^2 each, one Voronoi cell per 8192 px
# and one superpixel per 4096 px, with the 3-level schedule of the 4096^2 workload.
TRAIN_SEEDS = tuple(range(100, 108))
TRAIN_SIDE = 2048
SCHEDULE = dict(num_levels=3, ratio_C=4, init_block=32, final_grain=1, size_mode=2, predict=1, reuse=1)


def training_tiles(side: int = TRAIN_SIDE, seeds=TRAIN_SEEDS):
    imgs, K = [], []
    for s in seeds:
        imgs.append(synth.he_image(side, side, max(1, side * side // 8192), s).rgb)
        K.append(max(1, side * side // 4096))
    return imgs, K


def collect_and_train(imgs, K, params=SCHEDULE, stream=None, capacity=4_000_000, neg_rate=0.05, epochs=8,
                      batch=4096, lr=3e-3, pos_weight=None, seed=0):
    """Log one plain run over the tiles, then fit the net.  Returns (weights, info)."""
    import torch

    t0 = time.perf_counter()
    with Trainer(capacity, neg_rate) as tr:
        with Context(stream=stream, **params) as ctx:
            ctx.set_logging(tr)
            ctx.set_images([torch.from_numpy(x).cuda() for x in imgs], K)
            ctx.run()
            ctx.sync()
            ctx.set_logging(None)
        n, pos = tr.count()
        pw = float(pos_weight) if pos_weight else float(max(n - pos, 1)) / float(max(pos, 1))
        w, loss = tr.fit(epochs=epochs, batch=batch, lr=lr, pos_weight=pw, seed=seed)
    info = dict(samples=int(n), positives=int(pos), neg_rate=neg_rate, pos_weight=pw, epochs=epochs,
                epoch_loss=[round(float(x), 5) for x in loss], seconds=round(time.perf_counter() - t0, 2))
    return w, info


def refine(rgb_dev, K, params, weights=None, threshold=0.0, stream=None):
    """One run; returns (labels, ms, counters array)."""
    import torch

    with Context(stream=stream, **params) as ctx:
        ctx.set_images([rgb_dev], [K])
        if weights is not None:
            ctx.set_scorer(weights, threshold)
        ctx.run()  # warm-up
        ctx.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s = torch.cuda.current_stream() if stream is None else stream
        e0.record(s)
        ctx.run()
        e1.record(s)
        e1.synchronize()
        return ctx.image_labels(0), e0.elapsed_time(e1), ctx.counters_array(0)


def evaluate(weights, thresholds, img: synth.SynthImage, K: int, params=SCHEDULE, stream=None):
    """The plain run and one pruned run per threshold on one image: quality against the
    ground truth and against the plain labels, time and blocks evaluated."""
    import torch

    rgb = torch.from_numpy(img.rgb).cuda()
    plab, pms, pcnt = refine(rgb, K, params, stream=stream)
    out = {"plain": dict(br=quality.boundary_recall(plab, img.regions),
                         ue=quality.undersegmentation_error(plab, img.regions), ms=pms,
                         evaluated=int(pcnt[:, 4].sum()))}
    for t in thresholds:
        lab, ms, cnt = refine(rgb, K, params, weights, t, stream=stream)
        out[f"{t:g}"] = dict(br=quality.boundary_recall(lab, img.regions),
                             ue=quality.undersegmentation_error(lab, img.regions), ms=ms,
                             evaluated=int(cnt[:, 4].sum()), disagreement=quality.disagreement(lab, plab))
    return out


def main():
    import argparse
    import json

    import __graft_entry__

    ap = argparse.ArgumentParser(description="train the block scorer and sweep its threshold")
    ap.add_argument("--side", type=int, default=TRAIN_SIDE)
    ap.add_argument("--thresholds", default="0.05,0.1,0.2,0.3,0.5")
    args = ap.parse_args()
    __graft_entry__.build()
    w, info = collect_and_train(*training_tiles(args.side))
    img = synth.workload_image("he4096_k4096_l3")
    res = evaluate(w, [float(x) for x in args.thresholds.split(",")], img, 4096)
    print(json.dumps({"train": info, "eval_he4096_k4096_l3": res}))


if __name__ == "__main__":
    main()
