"""Shared helpers of the GPU tests: run the CUDA path through the C ABI and the CPU
oracle on the same seeded input, and compare."""
from __future__ import annotations

import numpy as np

import oracle

STAT_FIELDS = ("n", "sum_r", "sum_g", "sum_b", "sum_x", "sum_y", "init_size")


def gpu_run(rgb: np.ndarray, device_input: bool = True, theta=None, **params):
    import torch

    import paper_1704_02083_gb300 as pkg

    stream = torch.cuda.current_stream()
    with pkg.Context(stream=stream, **params) as ctx:
        if theta is not None:
            ctx.set_classifier(theta)
        if device_input:
            ctx.set_image(torch.from_numpy(np.ascontiguousarray(rgb)).cuda())
        else:
            ctx.set_image(rgb)
        ctx.run()
        lab = ctx.labels()
        st = ctx.stats()
        cnt = ctx.counters_array()
    stats = np.stack([st[f] for f in STAT_FIELDS], 1)
    return lab, stats, st["y"].astype(np.int8), st["important"].astype(np.uint8), cnt


def oracle_run(rgb: np.ndarray, theta=None, **params):
    p = {k: v for k, v in params.items() if k in oracle.DEFAULTS}
    if theta is None:
        return oracle.run(rgb, **p)
    o = oracle.Oracle(rgb, **p).set_classifier(theta).run()
    s, y, imp = o.stats()
    return o.labels(), s, y, imp, o.counters()


def gpu_counters(rgb: np.ndarray, **params):
    """Full rapid_counters of one run (for the implementation counters)."""
    import torch

    import paper_1704_02083_gb300 as pkg

    with pkg.Context(stream=torch.cuda.current_stream(), **params) as ctx:
        ctx.set_image(torch.from_numpy(np.ascontiguousarray(rgb)).cuda())
        ctx.run()
        c = ctx.counters()
        return [c.stage[i] for i in range(c.num_stages)], ctx.labels()


def assert_parity(rgb, theta=None, **params):
    lab, st, y, imp, cnt = gpu_run(rgb, theta=theta, **params)
    rlab, rst, ry, rimp, rcnt = oracle_run(rgb, theta=theta, **params)
    assert lab.shape == rlab.shape
    diff = np.argwhere(lab != rlab)
    assert diff.size == 0, f"{len(diff)} labels differ, first at {diff[:3].tolist()}"
    np.testing.assert_array_equal(st, rst)
    if params.get("predict", 0):
        np.testing.assert_array_equal(y, ry)
        np.testing.assert_array_equal(imp, rimp)
    np.testing.assert_array_equal(cnt, rcnt)
    return lab, st, cnt
