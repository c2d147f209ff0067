"""Fitting and judging the linear classifier of Eq. predict over the superpixel features
(the F in R^4 of Sec. 4.1), a host driver over the C ABI.

Training data: at the prediction point (entry to level 2) of runs on tiles of the 4096^2
tile's generator with other seeds, each superpixel's 4 features (read through
rapid_read_features) and its ground-truth class: ROI when at least half of its pixels lie
in the generator's ROI mask.  Training follows Sec. 4.1's sampling, half positive and half
negative superpixels drawn at random, and fits a logistic regression by Newton's method.
The brightness stand-in (h = 3 T N - (R + G + B)) is the reference it is judged against:
class accuracy at the prediction point, boundary recall of the final superpixels on the
ROI boundary and on all region boundaries, and time.
"""
from __future__ import annotations

import time

import numpy as np

from . import Context, quality, synth

TRAIN_SEEDS = tuple(range(100, 108))
TRAIN_SIDE = 1024
SCHEDULE = dict(num_levels=3, ratio_C=4, init_block=32, final_grain=1, size_mode=2, predict=1, reuse=1)
T_STANDIN = 150.0
STANDIN_THETA = (3 * T_STANDIN, -3.0, 0.0, 0.0, 0.0)  # the stand-in's sign, as a linear classifier


def _tile(side, seed):
    return synth.he_image(side, side, max(1, side * side // 8192), seed), max(1, side * side // 4096)


def at_prediction(rgb_dev, K, params, theta=STANDIN_THETA, stream=None):
    """Refine up to the prediction and run it; returns (features M x 4, full-res labels at
    the prediction, y)."""
    with Context(stream=stream, K=K, **params) as ctx:
        ctx.set_classifier(theta)
        ctx.set_image(rgb_dev)
        ctx.seed()
        ctx.refine_stage()
        st = ctx.state()
        while True:
            lv_next = ctx.counters().stage[st["stage"] + 1].level
            level_now = st["level"]
            ctx.split()
            if level_now < 2 <= lv_next:
                break
            ctx.refine_stage()
            st = ctx.state()
        F = ctx.features(0)
        return F, ctx.labels(), ctx.stats()["y"].astype(np.int8)


def ground_truth(labels, roi, M):
    """Per superpixel: +1 when at least half its pixels are ROI, else -1; and pixel counts."""
    n = np.bincount(labels.ravel(), minlength=M)
    r = np.bincount(labels.ravel(), weights=roi.ravel().astype(np.float64), minlength=M)
    return np.where(2 * r >= n, 1, -1).astype(np.int8), n


def collect(seeds=TRAIN_SEEDS, side=TRAIN_SIDE, params=SCHEDULE, stream=None):
    import torch

    Fs, ys = [], []
    for s in seeds:
        img, K = _tile(side, s)
        F, lab, _ = at_prediction(torch.from_numpy(img.rgb).cuda(), K, params, stream=stream)
        y, n = ground_truth(lab, img.roi, F.shape[0])
        live = n > 0
        Fs.append(F[live])
        ys.append(y[live])
    return np.concatenate(Fs), np.concatenate(ys)


def fit(F, y, seed=0, l2=1e-3, iters=50):
    """Logistic regression on a balanced sample (as many negatives as positives, drawn at
    random), on standardised features; returns theta in the features' own units."""
    rng = np.random.default_rng(seed)
    pos, neg = np.flatnonzero(y > 0), np.flatnonzero(y < 0)
    m = min(len(pos), len(neg))
    if m == 0:
        raise ValueError("the training superpixels hold one class only")
    idx = np.concatenate([rng.choice(pos, m, replace=False), rng.choice(neg, m, replace=False)])
    X, t = F[idx], (y[idx] > 0).astype(np.float64)
    mu, sd = X.mean(0), X.std(0)
    sd[sd == 0] = 1.0
    Z = np.hstack([np.ones((len(X), 1)), (X - mu) / sd])
    w = np.zeros(Z.shape[1])
    for _ in range(iters):
        p = 1.0 / (1.0 + np.exp(-Z @ w))
        g = Z.T @ (p - t) + l2 * np.r_[0.0, w[1:]]
        Hm = (Z * (p * (1 - p))[:, None]).T @ Z + l2 * np.diag(np.r_[0.0, np.ones(len(w) - 1)])
        step = np.linalg.solve(Hm, g)
        w -= step
        if np.abs(step).max() < 1e-10:
            break
    theta = np.empty(5)
    theta[1:] = w[1:] / sd
    theta[0] = w[0] - np.sum(w[1:] * mu / sd)
    return theta, dict(samples=int(2 * m), positives=int(len(pos)), negatives=int(len(neg)))


def balanced_accuracy(pred, y):
    pos, neg = y > 0, y < 0
    return 0.5 * (float((pred[pos] > 0).mean()) + float((pred[neg] < 0).mean()))


def evaluate(theta, img, K, params=SCHEDULE, stream=None):
    """The stand-in and theta on one image: class accuracy at the prediction, then whole
    runs (time, evaluated blocks, boundary recall on the ROI boundary and on all regions)."""
    import torch

    rgb = torch.from_numpy(img.rgb).cuda()
    roi_map = img.roi.astype(np.int32)
    out = {}
    for name, th in (("standin", None), ("linear", theta)):
        F, lab, y = at_prediction(rgb, K, params, th if th is not None else STANDIN_THETA, stream)
        gt, n = ground_truth(lab, img.roi, F.shape[0])
        live = n > 0
        acc = balanced_accuracy(y[live], gt[live])
        with Context(stream=stream, K=K, **params) as ctx:
            if th is not None:
                ctx.set_classifier(th)
            ctx.set_image(rgb)
            ctx.run()
            ctx.sync()
            s = torch.cuda.current_stream() if stream is None else stream
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            ctx.run()
            e1.record(s)
            e1.synchronize()
            labels = ctx.labels()
            out[name] = dict(balanced_accuracy=round(acc, 4), ms=round(e0.elapsed_time(e1), 3),
                             evaluated=int(ctx.counters_array()[:, 4].sum()),
                             br_roi=round(quality.boundary_recall(labels, roi_map), 4),
                             br=round(quality.boundary_recall(labels, img.regions), 4),
                             ue=round(quality.undersegmentation_error(labels, img.regions), 4))
    return out


def train(seeds=TRAIN_SEEDS, side=TRAIN_SIDE, params=SCHEDULE, stream=None, seed=0):
    t0 = time.perf_counter()
    F, y = collect(seeds, side, params, stream)
    theta, info = fit(F, y, seed)
    info.update(superpixels=int(len(y)), train_balanced_accuracy=round(
        balanced_accuracy(np.where((((theta[0] + theta[1] * F[:, 0]) + theta[2] * F[:, 1]) + theta[3] * F[:, 2])
                                   + theta[4] * F[:, 3] >= 0, 1, -1), y), 4),
        seconds=round(time.perf_counter() - t0, 2), theta=[float(x) for x in theta])
    return theta, info


def main():
    import argparse
    import json

    import __graft_entry__

    ap = argparse.ArgumentParser(description="fit the linear classifier of Eq. predict and judge it")
    ap.add_argument("--side", type=int, default=TRAIN_SIDE)
    args = ap.parse_args()
    __graft_entry__.build()
    theta, info = train(side=args.side)
    img = synth.workload_image("he4096_k4096_l3")
    print(json.dumps({"train": info, "eval_he4096_k4096_l3": evaluate(theta, img, 4096)}))


if __name__ == "__main__":
    main()
