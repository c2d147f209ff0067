"""GB300 (sm_103a) implementation of the coarse-to-fine topology-preserving superpixel
refinement of RAPID (Sulimowicz & Ahmad, ICME 2017).

This module is the thin Python binding of the C ABI declared in include/rapid.h: the
functions below have the C names and only marshal arguments.  Every step of the method
runs in the CUDA kernels of ``_build/librapid.so``; there is no CPU path, and importing
the binding fails loudly when the library is missing.  PyTorch is used only for device
memory and streams.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librapid.so")

RAPID_OK, RAPID_EINVAL, RAPID_ENOMEM, RAPID_ECUDA, RAPID_ESTATE, RAPID_ETIMEOUT, RAPID_ERANGE = range(7)
RAPID_MAX_STAGES = 32


class RapidError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {rapid_status_string(status)}")


class rapid_params(C.Structure):
    _fields_ = [
        ("num_levels", C.c_int32), ("ratio_C", C.c_int32), ("init_block", C.c_int32),
        ("final_grain", C.c_int32), ("K", C.c_int32), ("size_mode", C.c_int32),
        ("lambda_pos0", C.c_double), ("lambda_b", C.c_double),
        ("lo_num", C.c_int32), ("lo_den", C.c_int32), ("hi_num", C.c_int32), ("hi_den", C.c_int32),
        ("predict", C.c_int32), ("reuse", C.c_int32), ("importance_rule", C.c_int32),
        ("max_sweeps", C.c_int32), ("h_T", C.c_int64), ("spin_limit_ns", C.c_int64),
        ("use_filter", C.c_int32), ("skip_tiles", C.c_int32), ("verify_filter", C.c_int32), ("schedule", C.c_int32),
    ]


class rapid_sp_stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("sum_r", C.c_int64), ("sum_g", C.c_int64), ("sum_b", C.c_int64),
                ("sum_x", C.c_int64), ("sum_y", C.c_int64), ("init_size", C.c_int64),
                ("y", C.c_int32), ("important", C.c_int32)]


class rapid_stage_counters(C.Structure):
    _fields_ = [("level", C.c_int32), ("block", C.c_int32), ("sweeps", C.c_int32), ("pad", C.c_int32),
                ("eligible", C.c_int64), ("evaluated", C.c_int64), ("moves", C.c_int64),
                ("merge_requests", C.c_int64), ("merges", C.c_int64), ("fp64_fallbacks", C.c_int64),
                ("filter_mismatches", C.c_int64), ("tiles_scanned", C.c_int64), ("tiles_skipped", C.c_int64),
                ("merge_searches", C.c_int64), ("merge_cache_hits", C.c_int64),
                ("kernel_ms", C.c_float),
                ("section_ms", C.c_float * 5), ("pad2", C.c_float)]


class rapid_synth_params(C.Structure):
    _fields_ = [("H", C.c_int64), ("W", C.c_int64), ("seed", C.c_uint64), ("px_per_cell", C.c_int32),
                ("pad", C.c_int32), ("white_frac", C.c_double), ("fold_frac", C.c_double),
                ("nucleus_density", C.c_double)]


class rapid_counters(C.Structure):
    _fields_ = [("num_stages", C.c_int32), ("M", C.c_int32), ("launches", C.c_int64),
                ("stage", rapid_stage_counters * RAPID_MAX_STAGES)]


# numpy view of rapid_sp_stats (same layout)
SP_STATS_DTYPE = np.dtype([("n", "<i8"), ("sum_r", "<i8"), ("sum_g", "<i8"), ("sum_b", "<i8"),
                           ("sum_x", "<i8"), ("sum_y", "<i8"), ("init_size", "<i8"), ("y", "<i4"),
                           ("important", "<i4")])
assert SP_STATS_DTYPE.itemsize == C.sizeof(rapid_sp_stats)

_lib = None


def lib() -> C.CDLL:
    """Load librapid.so (built by ``build.build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run paper_1704_02083_gb300.build.build() first "
                          "(there is no CPU fallback)")
    L = C.CDLL(LIB_PATH)
    P, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    pi32, pi64 = C.POINTER(C.c_int32), C.POINTER(C.c_int64)
    sig = {
        "rapid_default_params": (None, [C.POINTER(rapid_params)]),
        "rapid_create": (i32, [C.POINTER(rapid_params), P, C.POINTER(P)]),
        "rapid_set_image": (i32, [P, P, i32, i32, i64, i32]),
        "rapid_seed_grid": (i32, [P, pi32]),
        "rapid_refine_stage": (i32, [P, pi32, pi64, pi64]),
        "rapid_split": (i32, [P]),
        "rapid_run": (i32, [P]),
        "rapid_get_state": (i32, [P, pi32, pi32, pi32, pi32]),
        "rapid_read_labels": (i32, [P, P, i64, i32]),
        "rapid_read_block_labels": (i32, [P, P, i64, pi32, pi32]),
        "rapid_read_stats": (i32, [P, P, i64, pi64]),
        "rapid_read_counters": (i32, [P, C.POINTER(rapid_counters)]),
        "rapid_set_profiling": (i32, [P, i32]),
        "rapid_sync": (i32, [P]),
        "rapid_simple_table": (i32, [P]),
        "rapid_run_static": (i32, [C.POINTER(rapid_params), P, i32, i32, i64, P, i64, P, i64, pi32, P]),
        "rapid_set_images": (i32, [P, i32, C.POINTER(P), pi32, pi32, pi64, pi32, i32]),
        "rapid_get_image_info": (i32, [P, i32, pi32, pi32, pi32]),
        "rapid_read_image_labels": (i32, [P, i32, P, i64, i32]),
        "rapid_read_image_stats": (i32, [P, i32, P, i64, pi64]),
        "rapid_read_image_counters": (i32, [P, i32, C.POINTER(rapid_counters)]),
        "rapid_set_graph": (i32, [P, i32]),
        "rapid_set_stage_grids": (i32, [P, pi32, i32]),
        "rapid_set_scorer": (i32, [P, P, C.c_float]),
        "rapid_set_keep_mask": (i32, [P, i32, i32, P, i64, i32]),
        "rapid_set_scorer_stages": (i32, [P, P, i32]),
        "rapid_debug_fail_alloc": (None, [i64]),
        "rapid_set_race_check": (i32, [P, i32]),
        "rapid_read_race_violations": (i32, [P, pi64]),
        "rapid_race_selftest": (i32, [pi64]),
        "rapid_synth_slide": (i32, [C.POINTER(rapid_synth_params), P, i64, P, i64, P]),
        "rapid_set_classifier": (i32, [P, P]),
        "rapid_read_features": (i32, [P, i32, P]),
        "rapid_refine_slide": (i32, [P, P, i64, i64, i64, i32, i32, i32, P, i64, P, i64, pi64, pi32]),
        "rapid_scorer_features": (i32, [P, i32, P]),
        "rapid_scorer_scores": (i32, [P, i32, P, P]),
        "rapid_trainer_create": (i32, [i64, C.c_float, C.POINTER(P)]),
        "rapid_trainer_samples": (i32, [P, i64, i32, P, P, P]),
        "rapid_trainer_gradient": (i32, [P, P, i64, i32, C.c_float, P, P]),
        "rapid_set_logging": (i32, [P, P]),
        "rapid_trainer_count": (i32, [P, pi64, pi64]),
        "rapid_trainer_fit": (i32, [P, i32, i32, C.c_float, C.c_float, C.c_uint64, P, P, P]),
        "rapid_trainer_destroy": (None, [P]),
        "rapid_autotune": (i32, [P, pi32, pi32]),
        "rapid_set_stage_shapes": (i32, [P, pi32, i32]),
        "rapid_status_string": (C.c_char_p, [i32]),
        "rapid_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(status: int, what: str):
    if status != RAPID_OK:
        raise RapidError(status, what)


# ------------------------------------------------------------------ C-named functions
def rapid_status_string(status: int) -> str:
    return lib().rapid_status_string(status).decode()


def rapid_default_params(**overrides) -> rapid_params:
    p = rapid_params()
    lib().rapid_default_params(C.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def rapid_create(params: rapid_params, cuda_stream: int = 0) -> int:
    h = C.c_void_p()
    _check(lib().rapid_create(C.byref(params), C.c_void_p(cuda_stream), C.byref(h)), "rapid_create")
    return h.value


def rapid_set_image(ctx: int, rgb_ptr: int, H: int, W: int, row_pitch_bytes: int, rgb_is_device: int):
    _check(lib().rapid_set_image(ctx, rgb_ptr, H, W, row_pitch_bytes, rgb_is_device), "rapid_set_image")


def rapid_seed_grid(ctx: int) -> int:
    M = C.c_int32()
    _check(lib().rapid_seed_grid(ctx, C.byref(M)), "rapid_seed_grid")
    return M.value


def rapid_refine_stage(ctx: int, sync: bool = False):
    if not sync:
        _check(lib().rapid_refine_stage(ctx, None, None, None), "rapid_refine_stage")
        return None
    s, m, g = C.c_int32(), C.c_int64(), C.c_int64()
    _check(lib().rapid_refine_stage(ctx, C.byref(s), C.byref(m), C.byref(g)), "rapid_refine_stage")
    return s.value, m.value, g.value


def rapid_split(ctx: int):
    _check(lib().rapid_split(ctx), "rapid_split")


def rapid_run(ctx: int):
    _check(lib().rapid_run(ctx), "rapid_run")


def rapid_get_state(ctx: int):
    v = [C.c_int32() for _ in range(4)]
    _check(lib().rapid_get_state(ctx, *[C.byref(x) for x in v]), "rapid_get_state")
    return dict(zip(("stage", "level", "block", "M"), [x.value for x in v]))


def rapid_read_labels(ctx: int, dst_ptr: int, row_pitch_bytes: int, dst_is_device: int):
    _check(lib().rapid_read_labels(ctx, dst_ptr, row_pitch_bytes, dst_is_device), "rapid_read_labels")


def rapid_read_block_labels(ctx: int, dst_ptr: int, capacity: int):
    nbx, nby = C.c_int32(), C.c_int32()
    _check(lib().rapid_read_block_labels(ctx, dst_ptr, capacity, C.byref(nbx), C.byref(nby)),
           "rapid_read_block_labels")
    return nbx.value, nby.value


def rapid_read_stats(ctx: int, dst_ptr: int, capacity: int) -> int:
    M = C.c_int64()
    _check(lib().rapid_read_stats(ctx, dst_ptr, capacity, C.byref(M)), "rapid_read_stats")
    return M.value


def rapid_read_counters(ctx: int) -> rapid_counters:
    c = rapid_counters()
    _check(lib().rapid_read_counters(ctx, C.byref(c)), "rapid_read_counters")
    return c


RAPID_MAX_BATCH = 64


def rapid_refine_slide(ctx: int, rgb_dev_ptr: int, H: int, W: int, rgb_pitch_bytes: int, max_tile: int,
                       px_per_superpixel: int, autotune: bool, labels_dev_ptr: int, labels_pitch_bytes: int,
                       stats_dev_ptr: int = 0, stats_capacity: int = 0):
    """Whole slide in tiles of at most max_tile px (device buffers); returns (M, tiles)."""
    M, T = C.c_int64(), C.c_int32()
    _check(lib().rapid_refine_slide(ctx, rgb_dev_ptr, H, W, rgb_pitch_bytes, max_tile, px_per_superpixel,
                                    1 if autotune else 0, labels_dev_ptr, labels_pitch_bytes, stats_dev_ptr or None,
                                    stats_capacity, C.byref(M), C.byref(T)), "rapid_refine_slide")
    return M.value, T.value


def rapid_set_images(ctx: int, rgb_ptrs, H, W, row_pitch_bytes, K, rgb_is_device: int):
    """n images at once (pointer, height, width, row pitch per image; K per image or None)."""
    n = len(rgb_ptrs)
    ptrs = (C.c_void_p * n)(*rgb_ptrs)
    h = (C.c_int32 * n)(*H)
    w = (C.c_int32 * n)(*W)
    pitch = (C.c_int64 * n)(*row_pitch_bytes)
    k = (C.c_int32 * n)(*K) if K is not None else None
    _check(lib().rapid_set_images(ctx, n, ptrs, h, w, pitch, k, rgb_is_device), "rapid_set_images")


def rapid_get_image_info(ctx: int, i: int):
    v = [C.c_int32() for _ in range(3)]
    _check(lib().rapid_get_image_info(ctx, i, *[C.byref(x) for x in v]), "rapid_get_image_info")
    return dict(zip(("H", "W", "M"), [x.value for x in v]))


def rapid_read_image_labels(ctx: int, i: int, dst_ptr: int, row_pitch_bytes: int, dst_is_device: int):
    _check(lib().rapid_read_image_labels(ctx, i, dst_ptr, row_pitch_bytes, dst_is_device),
           "rapid_read_image_labels")


def rapid_read_image_stats(ctx: int, i: int, dst_ptr: int, capacity: int) -> int:
    M = C.c_int64()
    _check(lib().rapid_read_image_stats(ctx, i, dst_ptr, capacity, C.byref(M)), "rapid_read_image_stats")
    return M.value


def rapid_read_image_counters(ctx: int, i: int) -> rapid_counters:
    c = rapid_counters()
    _check(lib().rapid_read_image_counters(ctx, i, C.byref(c)), "rapid_read_image_counters")
    return c


def rapid_set_graph(ctx: int, on: bool):
    _check(lib().rapid_set_graph(ctx, 1 if on else 0), "rapid_set_graph")


def rapid_set_stage_grids(ctx: int, grids):
    n = len(grids)
    arr = (C.c_int32 * max(1, n))(*grids)
    _check(lib().rapid_set_stage_grids(ctx, arr, n), "rapid_set_stage_grids")


def rapid_set_stage_shapes(ctx: int, shapes):
    n = len(shapes)
    arr = (C.c_int32 * max(1, n))(*shapes)
    _check(lib().rapid_set_stage_shapes(ctx, arr, n), "rapid_set_stage_shapes")


def rapid_autotune(ctx: int):
    """Per-stage grid sizes and tile shapes chosen by timing (RAPID_MAX_STAGES entries each)."""
    grids = (C.c_int32 * RAPID_MAX_STAGES)()
    shapes = (C.c_int32 * RAPID_MAX_STAGES)()
    _check(lib().rapid_autotune(ctx, grids, shapes), "rapid_autotune")
    return list(grids), list(shapes)


RAPID_SCORER_PARAMS = 3777
RAPID_SCORER_FEATURES = 9


def _f32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.size != RAPID_SCORER_PARAMS:
        raise ValueError(f"expected {RAPID_SCORER_PARAMS} scorer parameters")
    return a


def rapid_set_scorer(ctx: int, weights, threshold: float):
    """Pruned refinement with the learned scorer (weights None = off)."""
    if weights is None:
        _check(lib().rapid_set_scorer(ctx, None, 0.0), "rapid_set_scorer")
        return
    w = _f32(weights)
    _check(lib().rapid_set_scorer(ctx, w.ctypes.data, float(threshold)), "rapid_set_scorer")


def rapid_synth_slide(params: rapid_synth_params, rgb_dev_ptr: int, rgb_pitch_bytes: int, regions_dev_ptr,
                      regions_pitch_bytes: int, cuda_stream: int = 0):
    """The counter-based synthetic slide into device buffers (see include/rapid.h)."""
    _check(lib().rapid_synth_slide(C.byref(params), rgb_dev_ptr, rgb_pitch_bytes, regions_dev_ptr,
                                   regions_pitch_bytes, cuda_stream), "rapid_synth_slide")


def synth_slide_device(H: int, W: int, seed: int, regions: bool = False, px_per_cell: int = 8192,
                       white_frac: float = 0.40, fold_frac: float = 0.05, nucleus_density: float = 1.0 / 400.0,
                       stream=None):
    """The counter-based synthetic slide made on the device (rapid_synth_slide): an H x W x 3
    uint8 CUDA tensor, and its ground-truth region ids (int32) when `regions`."""
    import torch

    rgb = torch.empty((H, W, 3), dtype=torch.uint8, device="cuda")
    reg = torch.empty((H, W), dtype=torch.int32, device="cuda") if regions else None
    p = rapid_synth_params(H=H, W=W, seed=seed, px_per_cell=px_per_cell, pad=0, white_frac=white_frac,
                           fold_frac=fold_frac, nucleus_density=nucleus_density)
    s = (stream or torch.cuda.current_stream()).cuda_stream
    rapid_synth_slide(p, rgb.data_ptr(), 3 * W, reg.data_ptr() if reg is not None else None, 4 * W, s)
    return (rgb, reg) if regions else rgb


def rapid_set_race_check(ctx: int, on: bool):
    _check(lib().rapid_set_race_check(ctx, 1 if on else 0), "rapid_set_race_check")


def rapid_read_race_violations(ctx: int) -> int:
    v = C.c_int64()
    _check(lib().rapid_read_race_violations(ctx, C.byref(v)), "rapid_read_race_violations")
    return v.value


def rapid_race_selftest():
    """Violations the race check finds on its three scripted write sequences."""
    v = (C.c_int64 * 3)()
    _check(lib().rapid_race_selftest(v), "rapid_race_selftest")
    return list(v)


def rapid_debug_fail_alloc(n: int):
    """Test hook: the n-th device allocation of the library from now on fails (0 = off)."""
    lib().rapid_debug_fail_alloc(int(n))


def rapid_set_scorer_stages(ctx: int, on):
    """Which stages the scorer prunes (a sequence of 0/1 per stage; later stages are pruned)."""
    a = np.ascontiguousarray(on, dtype=np.int32)
    _check(lib().rapid_set_scorer_stages(ctx, a.ctypes.data if a.size else None, a.size), "rapid_set_scorer_stages")


def rapid_set_keep_mask(ctx: int, i: int, s: int, mask):
    """Pruned sweeps of stage s with image i's keep mask (nby x nbx uint8, nonzero = kept;
    a numpy array or a CUDA tensor); mask None (with i = s = -1) clears every mask."""
    if mask is None:
        _check(lib().rapid_set_keep_mask(ctx, i, s, None, 0, 0), "rapid_set_keep_mask")
        return
    if hasattr(mask, "data_ptr"):
        m = mask.contiguous()
        _check(lib().rapid_set_keep_mask(ctx, i, s, m.data_ptr(), m.numel(), 1 if m.is_cuda else 0),
               "rapid_set_keep_mask")
        return
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    _check(lib().rapid_set_keep_mask(ctx, i, s, m.ctypes.data, m.size, 0), "rapid_set_keep_mask")


def rapid_set_classifier(ctx: int, theta):
    """Eq. predict with h = theta[0] + theta[1:] . F over the superpixel features (None: the
    brightness stand-in)."""
    if theta is None:
        _check(lib().rapid_set_classifier(ctx, None), "rapid_set_classifier")
        return
    t = np.ascontiguousarray(theta, dtype=np.float64)
    if t.shape != (5,):
        raise ValueError("theta has 5 entries")
    _check(lib().rapid_set_classifier(ctx, t.ctypes.data), "rapid_set_classifier")


def rapid_read_features(ctx: int, i: int, M: int) -> np.ndarray:
    out = np.zeros((M, 4), np.float64)
    _check(lib().rapid_read_features(ctx, i, out.ctypes.data), "rapid_read_features")
    return out


def rapid_scorer_features(ctx: int, i: int, dst_dev_ptr: int):
    _check(lib().rapid_scorer_features(ctx, i, dst_dev_ptr), "rapid_scorer_features")


def rapid_scorer_scores(ctx: int, i: int, weights, dst_dev_ptr: int):
    w = _f32(weights)
    _check(lib().rapid_scorer_scores(ctx, i, w.ctypes.data, dst_dev_ptr), "rapid_scorer_scores")


def rapid_trainer_create(capacity: int, neg_rate: float) -> int:
    h = C.c_void_p()
    _check(lib().rapid_trainer_create(capacity, float(neg_rate), C.byref(h)), "rapid_trainer_create")
    return h.value


def rapid_set_logging(ctx: int, trainer: int | None):
    _check(lib().rapid_set_logging(ctx, trainer), "rapid_set_logging")


def rapid_trainer_count(trainer: int):
    n, p = C.c_int64(), C.c_int64()
    _check(lib().rapid_trainer_count(trainer, C.byref(n), C.byref(p)), "rapid_trainer_count")
    return n.value, p.value


def rapid_trainer_fit(trainer: int, epochs: int, batch: int, lr: float, pos_weight: float, seed: int,
                      init=None):
    """Returns (weights, per-epoch mean loss)."""
    w = np.zeros(RAPID_SCORER_PARAMS, np.float32)
    loss = np.zeros(epochs, np.float32)
    keep = _f32(init) if init is not None else None  # held until the call returns
    ip = keep.ctypes.data if keep is not None else None
    _check(lib().rapid_trainer_fit(trainer, epochs, batch, float(lr), float(pos_weight), seed, ip, w.ctypes.data,
                                   loss.ctypes.data), "rapid_trainer_fit")
    del keep
    return w, loss


def rapid_trainer_samples(trainer: int, first: int, count: int):
    """Stored samples first .. first + count - 1: patches (count x 7 x 7 x 9 float32),
    in-image masks (count uint64, bit p = patch position p) and labels (count float32)."""
    x = np.zeros((count, 7, 7, 9), np.float32)
    inb = np.zeros(count, np.uint64)
    y = np.zeros(count, np.float32)
    _check(lib().rapid_trainer_samples(trainer, first, count, x.ctypes.data, inb.ctypes.data, y.ctypes.data),
           "rapid_trainer_samples")
    return x, inb, y


def rapid_trainer_gradient(trainer: int, weights, first: int, count: int, pos_weight: float):
    """Summed gradient (RAPID_SCORER_PARAMS float32) and loss of samples first .. first +
    count - 1 at the master weights `weights`."""
    w = _f32(weights)
    g = np.zeros(RAPID_SCORER_PARAMS, np.float32)
    loss = C.c_float()
    _check(lib().rapid_trainer_gradient(trainer, w.ctypes.data, first, count, float(pos_weight), g.ctypes.data,
                                        C.byref(loss)), "rapid_trainer_gradient")
    return g, loss.value


def rapid_trainer_destroy(trainer: int):
    if trainer:
        lib().rapid_trainer_destroy(trainer)


def rapid_set_profiling(ctx: int, on: bool):
    _check(lib().rapid_set_profiling(ctx, 1 if on else 0), "rapid_set_profiling")


def rapid_sync(ctx: int):
    _check(lib().rapid_sync(ctx), "rapid_sync")


def rapid_simple_table() -> np.ndarray:
    out = np.zeros(256, np.uint8)
    _check(lib().rapid_simple_table(out.ctypes.data), "rapid_simple_table")
    return out


def rapid_destroy(ctx: int):
    if ctx:
        lib().rapid_destroy(ctx)


RAPID_STATIC_MAX_PIXELS = 1 << 19
RAPID_STATIC_MAX_LABELS = 1 << 13


def rapid_run_static(params: rapid_params, rgb_dev_ptr: int, H: int, W: int, rgb_pitch_bytes: int,
                     labels_dev_ptr: int, labels_pitch_bytes: int, stats_dev_ptr: int, stats_capacity: int,
                     cuda_stream: int = 0) -> int:
    """Whole refinement without any GPU allocation (for callers that cannot call cudaMalloc);
    all buffers are the caller's device memory.  Returns M."""
    M = C.c_int32()
    _check(lib().rapid_run_static(C.byref(params), rgb_dev_ptr, H, W, rgb_pitch_bytes, labels_dev_ptr,
                                  labels_pitch_bytes, stats_dev_ptr, stats_capacity, C.byref(M),
                                  C.c_void_p(cuda_stream)), "rapid_run_static")
    return M.value


# ------------------------------------------------------------------ convenience wrapper
class Context:
    """One rapid_ctx bound to the current CUDA device and a torch stream.

    ``Context(params).set_image(rgb)`` accepts a numpy H x W x 3 uint8 array (host copy) or
    a CUDA torch tensor of that shape (device copy).  ``labels()`` returns a host int32
    H x W array (or writes into a CUDA int32 tensor with ``labels(out=t)``).
    """

    def __init__(self, params: rapid_params | None = None, stream=None, **overrides):
        if params is None:
            params = rapid_default_params(**overrides)
        elif overrides:
            for k, v in overrides.items():
                setattr(params, k, v)
        self.params = params
        self._stream = stream
        handle = 0
        if stream is not None:
            handle = int(getattr(stream, "cuda_stream", stream))
        self.h = rapid_create(params, handle)
        self.H = self.W = 0

    def close(self):
        if getattr(self, "h", 0):
            rapid_destroy(self.h)
            self.h = 0

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_image(self, rgb):
        if isinstance(rgb, np.ndarray):
            rgb = np.ascontiguousarray(rgb, dtype=np.uint8)
            if rgb.ndim != 3 or rgb.shape[2] != 3:
                raise ValueError("expected H x W x 3 uint8")
            H, W = rgb.shape[:2]
            rapid_set_image(self.h, rgb.ctypes.data, H, W, rgb.strides[0], 0)
        else:  # torch CUDA tensor, uint8, H x W x 3 with contiguous rows
            if str(rgb.dtype) != "torch.uint8" or rgb.dim() != 3 or rgb.shape[2] != 3 or not rgb.is_cuda:
                raise ValueError("expected a CUDA uint8 tensor of shape H x W x 3")
            if rgb.stride(2) != 1 or rgb.stride(1) != 3:
                raise ValueError("rows must be interleaved RGB (stride(1) == 3, stride(2) == 1)")
            H, W = int(rgb.shape[0]), int(rgb.shape[1])
            rapid_set_image(self.h, rgb.data_ptr(), H, W, rgb.stride(0), 1)
        self.H, self.W = int(H), int(W)
        self.sizes = [(self.H, self.W)]
        return self

    def seed(self) -> int:
        return rapid_seed_grid(self.h)

    def refine_stage(self, sync: bool = True):
        return rapid_refine_stage(self.h, sync)

    def split(self):
        rapid_split(self.h)

    def run(self):
        rapid_run(self.h)
        return self

    def state(self):
        return rapid_get_state(self.h)

    def labels(self, out=None):
        if out is None:
            a = np.empty((self.H, self.W), np.int32)
            rapid_read_labels(self.h, a.ctypes.data, a.strides[0], 0)
            return a
        rapid_read_labels(self.h, out.data_ptr(), out.stride(0) * 4, 1)
        return out

    def block_labels(self):
        st = self.state()
        s = st["block"]
        nbx, nby = -(-self.W // s), -(-self.H // s)
        a = np.empty((nby, nbx), np.int32)
        rapid_read_block_labels(self.h, a.ctypes.data, a.size)
        return a

    def stats(self) -> np.ndarray:
        M = self.state()["M"]
        a = np.zeros(max(M, 1), SP_STATS_DTYPE)
        rapid_read_stats(self.h, a.ctypes.data, a.size)
        return a[:M]

    def counters(self, i: int = 0) -> rapid_counters:
        return rapid_read_image_counters(self.h, i)

    def counters_array(self, i: int = 0) -> np.ndarray:
        """num_stages x 8 int64: level, block, sweeps, eligible, evaluated, moves, merge
        requests, merges (the oracle's counter layout)."""
        c = self.counters(i)
        rows = []
        for i in range(c.num_stages):
            s = c.stage[i]
            rows.append([s.level, s.block, s.sweeps, s.eligible, s.evaluated, s.moves, s.merge_requests, s.merges])
        return np.array(rows, np.int64).reshape(-1, 8)

    def set_profiling(self, on: bool = True):
        rapid_set_profiling(self.h, on)

    # ---- batches (rapid_set_images): image i's results
    def set_images(self, images, K=None):
        """A batch: a list of numpy H x W x 3 uint8 arrays (host copies) or of CUDA uint8
        tensors of that shape (device copies); K: superpixels per image (None: params.K)."""
        if len(images) == 0:
            raise ValueError("empty batch")
        on_device = not isinstance(images[0], np.ndarray)
        ptrs, H, W, pitch, keep = [], [], [], [], []
        for rgb in images:
            if isinstance(rgb, np.ndarray):
                if on_device:
                    raise ValueError("mixed host and device images")
                rgb = np.ascontiguousarray(rgb, dtype=np.uint8)
                if rgb.ndim != 3 or rgb.shape[2] != 3:
                    raise ValueError("expected H x W x 3 uint8")
                ptrs.append(rgb.ctypes.data)
                pitch.append(rgb.strides[0])
            else:
                if not on_device or str(rgb.dtype) != "torch.uint8" or rgb.dim() != 3 or rgb.shape[2] != 3 \
                        or not rgb.is_cuda or rgb.stride(2) != 1 or rgb.stride(1) != 3:
                    raise ValueError("expected CUDA uint8 tensors of shape H x W x 3 with interleaved rows")
                ptrs.append(rgb.data_ptr())
                pitch.append(rgb.stride(0))
            keep.append(rgb)
            H.append(int(rgb.shape[0]))
            W.append(int(rgb.shape[1]))
        rapid_set_images(self.h, ptrs, H, W, pitch, None if K is None else [int(k) for k in K],
                         1 if on_device else 0)
        self.sizes = list(zip(H, W))
        self.H, self.W = self.sizes[0]
        return self

    def image_info(self, i: int):
        return rapid_get_image_info(self.h, i)

    def image_labels(self, i: int) -> np.ndarray:
        H, W = self.sizes[i]
        a = np.empty((H, W), np.int32)
        rapid_read_image_labels(self.h, i, a.ctypes.data, a.strides[0], 0)
        return a

    def image_stats(self, i: int) -> np.ndarray:
        M = self.image_info(i)["M"]
        a = np.zeros(max(M, 1), SP_STATS_DTYPE)
        rapid_read_image_stats(self.h, i, a.ctypes.data, a.size)
        return a[:M]

    def set_graph(self, on: bool = True):
        rapid_set_graph(self.h, on)

    def set_scorer(self, weights, threshold: float = 0.3):
        rapid_set_scorer(self.h, weights, threshold)

    def set_race_check(self, on: bool = True):
        rapid_set_race_check(self.h, on)
        return self

    def race_violations(self) -> int:
        return rapid_read_race_violations(self.h)

    def set_scorer_stages(self, on):
        rapid_set_scorer_stages(self.h, on)
        return self

    def set_keep_mask(self, i: int, s: int, mask):
        """Image i's keep mask for stage s (pruned sweeps); None with i = s = -1 clears."""
        rapid_set_keep_mask(self.h, i, s, mask)
        return self

    def set_classifier(self, theta):
        """theta (5 floats) for Eq. predict over the superpixel features, or None."""
        rapid_set_classifier(self.h, theta)
        return self

    def features(self, i: int = 0) -> np.ndarray:
        """Image i's superpixel features of the last prediction (M x 4: absolute brightness,
        comparative brightness, extra-region and intra-region dissimilarity)."""
        return rapid_read_features(self.h, i, self.image_info(i)["M"])

    def set_logging(self, trainer):
        rapid_set_logging(self.h, trainer.h if trainer is not None else None)

    def set_stage_grids(self, grids):
        rapid_set_stage_grids(self.h, grids)

    def refine_slide(self, rgb, max_tile: int = 8192, px_per_superpixel: int = 4096, autotune: bool = False,
                     labels=None, stats=None):
        """Whole slide: rgb is a CUDA uint8 tensor H x W x 3 with interleaved rows; labels (a
        CUDA int32 H x W tensor, allocated when None) receives slide-wide ids; stats (a CUDA
        uint8 tensor of capacity x 64 bytes, optional) their statistics.  Returns
        (labels, M, tiles)."""
        import torch
        H, W = int(rgb.shape[0]), int(rgb.shape[1])
        if labels is None:
            labels = torch.empty((H, W), dtype=torch.int32, device=rgb.device)
        cap = 0 if stats is None else stats.numel() // SP_STATS_DTYPE.itemsize
        M, T = rapid_refine_slide(self.h, rgb.data_ptr(), H, W, rgb.stride(0), max_tile, px_per_superpixel, autotune,
                                  labels.data_ptr(), labels.stride(0) * 4, 0 if stats is None else stats.data_ptr(),
                                  cap)
        return labels, M, T

    def set_stage_shapes(self, shapes):
        rapid_set_stage_shapes(self.h, shapes)

    def autotune(self):
        """Time the schedule with each tile shape and grid size and keep the fastest per
        stage; returns (grids, shapes) per stage."""
        g, s = rapid_autotune(self.h)
        n = max(1, self.counters().num_stages)
        return g[:n], s[:n]

    def sync(self):
        rapid_sync(self.h)


class Trainer:
    """Training samples of the learned block scorer (rapid_trainer) on the device."""

    def __init__(self, capacity: int, neg_rate: float = 0.1):
        self.h = rapid_trainer_create(capacity, neg_rate)

    def count(self):
        return rapid_trainer_count(self.h)

    def fit(self, epochs=8, batch=2048, lr=3e-3, pos_weight=4.0, seed=0, init=None):
        return rapid_trainer_fit(self.h, epochs, batch, lr, pos_weight, seed, init)

    def samples(self, first: int, count: int):
        return rapid_trainer_samples(self.h, first, count)

    def gradient(self, weights, first: int, count: int, pos_weight: float = 4.0):
        return rapid_trainer_gradient(self.h, weights, first, count, pos_weight)

    def close(self):
        if getattr(self, "h", 0):
            rapid_trainer_destroy(self.h)
            self.h = 0

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
