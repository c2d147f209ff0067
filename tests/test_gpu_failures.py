"""Failure handling without a GPU fault: the library's device allocations are made to fail
one at a time (rapid_debug_fail_alloc), and whichever call meets the failure must return
RAPID_ENOMEM, leave the context destroyable, and leave the library working: a fresh context
afterwards refines bit-exactly as the oracle does."""
import ctypes as C

import numpy as np
import pytest

from gpu_common import oracle_run
from paper_1704_02083_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _sequence(pkg, rgb, params, trainer=False):
    """create, image, scorer, run, read; returns the first failing status (or 0) and
    whether the run completed."""
    import torch

    L = pkg.lib()
    p = pkg.rapid_default_params(**params)
    h = C.c_void_p()
    stream = torch.cuda.Stream()  # a graph needs a stream other than the legacy default one
    st = L.rapid_create(C.byref(p), C.c_void_p(stream.cuda_stream), C.byref(h))
    if st != 0:
        assert h.value is None
        return (st, "create"), False
    try:
        dev = torch.from_numpy(np.ascontiguousarray(rgb)).cuda()
        H, W = rgb.shape[:2]
        lab = np.zeros((H, W), np.int32)
        for name, call in (("set_image", lambda: L.rapid_set_image(h, C.c_void_p(dev.data_ptr()), H, W, 3 * W, 1)),
                           ("set_graph", lambda: L.rapid_set_graph(h, 1)),
                           ("run", lambda: L.rapid_run(h)),
                           ("replay", lambda: L.rapid_run(h)),
                           ("sync", lambda: L.rapid_sync(h)),
                           ("read_labels", lambda: L.rapid_read_labels(h, C.c_void_p(lab.ctypes.data), 4 * W, 0))):
            st = call()
            if st != 0:
                return (st, name), False
        return (0, None), True
    finally:
        L.rapid_destroy(h)


def test_every_allocation_failure_is_reported_and_recoverable():
    import paper_1704_02083_gb300 as pkg

    rgb = synth.he_image(96, 128, 6, 3).rgb
    params = dict(num_levels=2, ratio_C=4, init_block=16, K=24, predict=1)
    seen = 0
    try:
        for n in range(1, 64):
            pkg.rapid_debug_fail_alloc(n)
            (st, where), done = _sequence(pkg, rgb, params)
            if done:  # the n-th allocation was never reached: every one has been failed once
                break
            assert st == pkg.RAPID_ENOMEM, (n, st, where)
            seen += 1
    finally:
        pkg.rapid_debug_fail_alloc(0)
    assert seen >= 8  # control block, label arrays, image copy, sum levels, label maps, bitmaps, ...
    # the library still works afterwards, bit-exactly
    import torch

    with pkg.Context(stream=torch.cuda.current_stream(), **params) as ctx:
        ctx.set_image(torch.from_numpy(rgb).cuda()).run()
        lab = ctx.labels()
    np.testing.assert_array_equal(lab, oracle_run(rgb, **params)[0])


def test_trainer_allocation_failures():
    import paper_1704_02083_gb300 as pkg

    L = pkg.lib()
    try:
        for n in (1, 2, 3, 4):
            pkg.rapid_debug_fail_alloc(n)
            h = C.c_void_p()
            assert L.rapid_trainer_create(1000, C.c_float(0.5), C.byref(h)) == pkg.RAPID_ENOMEM
            assert h.value is None
    finally:
        pkg.rapid_debug_fail_alloc(0)
    with pkg.Trainer(1000, 0.5) as tr:
        assert tr.count() == (0, 0)
