"""ctypes wrapper of the CPU oracle (TEST INFRASTRUCTURE ONLY).

Only the tests, ``__graft_entry__.smoke()`` and the bench's CPU-baseline / reference leg
import this module.  The product path never does.
"""
from __future__ import annotations

import ctypes as C
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import build as _build  # noqa: E402

NCOUNT = 8
COUNTER_NAMES = ("level", "side", "sweeps", "eligible", "evaluated", "moves", "merge_requests", "merges")


class OrcParams(C.Structure):
    _fields_ = [
        ("num_levels", C.c_int32), ("ratio_C", C.c_int32), ("init_block", C.c_int32),
        ("final_grain", C.c_int32), ("K", C.c_int32), ("size_mode", C.c_int32),
        ("lambda_pos0", C.c_double), ("lambda_b", C.c_double),
        ("lo_num", C.c_int32), ("lo_den", C.c_int32), ("hi_num", C.c_int32), ("hi_den", C.c_int32),
        ("predict", C.c_int32), ("reuse", C.c_int32), ("importance_rule", C.c_int32),
        ("max_sweeps", C.c_int32), ("h_T", C.c_int64), ("schedule", C.c_int32), ("pad", C.c_int32),
    ]


# Defaults: lambda_pos0 = 400 and lambda_b = 50 (the paper states no weights), l = 1/4
# (Sec. 3.1), u = 3/2, T = 150, 64 sweeps per stage.
DEFAULTS = dict(num_levels=1, ratio_C=4, init_block=16, final_grain=1, K=200, size_mode=2,
                lambda_pos0=400.0, lambda_b=50.0, lo_num=1, lo_den=4, hi_num=3, hi_den=2,
                predict=0, reuse=1, importance_rule=0, max_sweeps=64, h_T=150, schedule=0)

_lib = None


def _load(path):
    """Bind the oracle functions of the shared library at ``path``."""
    if True:
        L = C.CDLL(path)
        P = C.c_void_p
        i32p, i64p = C.POINTER(C.c_int32), C.POINTER(C.c_int64)
        L.orc_create.restype = P
        L.orc_create.argtypes = [P, C.c_int32, C.c_int32, C.POINTER(OrcParams), i32p]
        L.orc_destroy.argtypes = [P]
        L.orc_destroy.restype = None
        for name in ("orc_num_stages", "orc_seed", "orc_refine_stage", "orc_next_stage", "orc_run",
                     "orc_run_fifo"):
            getattr(L, name).argtypes = [P]
            getattr(L, name).restype = C.c_int32
        L.orc_stage_info.argtypes = [P, C.c_int32, i32p, i32p]
        L.orc_phase.argtypes = [P, C.c_int32, i64p, i64p]
        L.orc_phase_moves.argtypes = [P, C.c_int32, i64p, i64p]
        L.orc_phase_merges.argtypes = [P, i64p]
        L.orc_pending_requests.argtypes = [P, P, P, C.c_int64]
        for name in ("orc_phase_moves", "orc_phase_merges", "orc_pending_requests"):
            getattr(L, name).restype = C.c_int32
        L.orc_get_grid.argtypes = [P, i32p, i32p, i32p, i32p, i32p, i32p]
        L.orc_read_block_labels.argtypes = [P, P]
        L.orc_read_labels.argtypes = [P, P]
        L.orc_read_stats.argtypes = [P, P, P, P]
        L.orc_read_counters.argtypes = [P, P]
        L.orc_read_pyramid.argtypes = [P, C.c_int32, P]
        L.orc_level_dims.argtypes = [P, C.c_int32, i32p, i32p, i32p]
        L.orc_lambda_pos.argtypes = [P]
        L.orc_lambda_pos.restype = C.c_double
        L.orc_simple_lut.argtypes = [P]
        L.orc_set_classifier.argtypes = [P, P]
        L.orc_set_keep_mask.argtypes = [P, C.c_int32, P, C.c_int64]
        L.orc_set_keep_mask.restype = C.c_int32
        L.orc_read_features.argtypes = [P, P]
        for name in ("orc_stage_info", "orc_phase", "orc_get_grid", "orc_read_block_labels",
                     "orc_read_labels", "orc_read_stats", "orc_read_counters", "orc_read_pyramid",
                     "orc_level_dims", "orc_simple_lut", "orc_set_classifier", "orc_read_features"):
            getattr(L, name).restype = C.c_int32
        L.orc_set_threads.argtypes = [C.c_int32]
        L.orc_set_threads.restype = C.c_int32
    return L


def lib():
    """The oracle (single-threaded build)."""
    global _lib
    if _lib is None:
        _lib = _load(_build.build())
    return _lib


_lib_omp = None


def lib_omp():
    """The same oracle with the decisions of a phase on all cores (OpenMP build); its
    results equal lib()'s for any thread count."""
    global _lib_omp
    if _lib_omp is None:
        _lib_omp = _load(_build.build(openmp=True))
    return _lib_omp


def params(**kw) -> OrcParams:
    d = dict(DEFAULTS)
    for k, v in kw.items():
        if k not in d:
            raise KeyError(k)
        d[k] = v
    return OrcParams(**d)


def simple_lut() -> np.ndarray:
    out = np.zeros(256, np.uint8)
    lib().orc_simple_lut(out.ctypes.data)
    return out


class Oracle:
    """One image, one parameter set; mirrors the steps of Algorithm RAPID."""

    def __init__(self, rgb: np.ndarray, omp: bool = False, threads: int = 0, **kw):
        """omp: the OpenMP build (phase decisions on `threads` cores, 0 = all)."""
        self._L = lib_omp() if omp else lib()
        if omp:
            self.threads = self._L.orc_set_threads(int(threads))
        rgb = np.ascontiguousarray(rgb, dtype=np.uint8)
        assert rgb.ndim == 3 and rgb.shape[2] == 3
        self.H, self.W = int(rgb.shape[0]), int(rgb.shape[1])
        self.p = params(**kw)
        st = C.c_int32(0)
        self._rgb = rgb
        self.h = self._L.orc_create(rgb.ctypes.data, self.H, self.W, C.byref(self.p), C.byref(st))
        if not self.h:
            raise ValueError(f"orc_create failed with status {st.value}")

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self._L.orc_destroy(h)
            self.h = None

    def _ok(self, r):
        if r != 0:
            raise RuntimeError(f"oracle call failed with status {r}")

    def num_stages(self) -> int:
        return self._L.orc_num_stages(self.h)

    def stages(self):
        out = []
        for i in range(self.num_stages()):
            lv, s = C.c_int32(), C.c_int32()
            self._ok(self._L.orc_stage_info(self.h, i, C.byref(lv), C.byref(s)))
            out.append((lv.value, s.value))
        return out

    def seed(self):
        self._ok(self._L.orc_seed(self.h))

    def phase(self, ph: int):
        mv, mg = C.c_int64(), C.c_int64()
        self._ok(self._L.orc_phase(self.h, ph, C.byref(mv), C.byref(mg)))
        return mv.value, mg.value

    def phase_moves(self, ph: int):
        mv, rq = C.c_int64(), C.c_int64()
        self._ok(self._L.orc_phase_moves(self.h, ph, C.byref(mv), C.byref(rq)))
        return mv.value, rq.value

    def phase_merges(self):
        mg = C.c_int64()
        self._ok(self._L.orc_phase_merges(self.h, C.byref(mg)))
        return mg.value

    def pending_requests(self, cap: int = 1 << 20):
        blk = np.empty(cap, np.int64)
        lab = np.empty(cap, np.int32)
        n = self._L.orc_pending_requests(self.h, blk.ctypes.data, lab.ctypes.data, cap)
        return blk[:n].copy(), lab[:n].copy()

    def refine_stage(self):
        self._ok(self._L.orc_refine_stage(self.h))

    def next_stage(self):
        self._ok(self._L.orc_next_stage(self.h))

    def run(self):
        self._ok(self._L.orc_run(self.h))
        return self

    def run_fifo(self):
        self._ok(self._L.orc_run_fifo(self.h))
        return self

    def set_classifier(self, theta):
        """Eq. predict with h = theta[0] + theta[1:] . F (None: the brightness stand-in)."""
        if theta is None:
            self._ok(self._L.orc_set_classifier(self.h, None))
            return self
        self._theta = np.ascontiguousarray(theta, dtype=np.float64)
        assert self._theta.shape == (5,)
        self._ok(self._L.orc_set_classifier(self.h, self._theta.ctypes.data))
        return self

    def set_keep_mask(self, stage: int, mask):
        """Pruned sweeps of stage `stage` with this keep mask over its block grid (nby x nbx,
        nonzero = kept); None sweeps the stage in full."""
        if mask is None:
            self._ok(self._L.orc_set_keep_mask(self.h, stage, None, 0))
            return self
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        self._ok(self._L.orc_set_keep_mask(self.h, stage, m.ctypes.data, m.size))
        return self

    def features(self) -> np.ndarray:
        """M x 4 features of the last prediction: absolute brightness, comparative
        brightness, extra-region dissimilarity, intra-region dissimilarity."""
        out = np.zeros((self.grid()["M"], 4), np.float64)
        self._ok(self._L.orc_read_features(self.h, out.ctypes.data))
        return out

    def grid(self):
        v = [C.c_int32() for _ in range(6)]
        self._L.orc_get_grid(self.h, *[C.byref(x) for x in v])
        return dict(zip(("stage", "nbx", "nby", "side", "level", "M"), [x.value for x in v]))

    def block_labels(self) -> np.ndarray:
        g = self.grid()
        out = np.empty((g["nby"], g["nbx"]), np.int32)
        self._ok(self._L.orc_read_block_labels(self.h, out.ctypes.data))
        return out

    def labels(self) -> np.ndarray:
        out = np.empty((self.H, self.W), np.int32)
        self._ok(self._L.orc_read_labels(self.h, out.ctypes.data))
        return out

    def stats(self):
        """(M x 7 int64 [N, R, G, B, X, Y, InitSize], y int8, important uint8)."""
        M = self.grid()["M"]
        s = np.empty((M, 7), np.int64)
        y = np.empty(M, np.int8)
        imp = np.empty(M, np.uint8)
        self._ok(self._L.orc_read_stats(self.h, s.ctypes.data, y.ctypes.data, imp.ctypes.data))
        return s, y, imp

    def counters(self) -> np.ndarray:
        n = self.num_stages()
        out = np.zeros((n, NCOUNT), np.int64)
        self._ok(self._L.orc_read_counters(self.h, out.ctypes.data))
        return out

    def lambda_pos(self) -> float:
        return self._L.orc_lambda_pos(self.h)

    def level_dims(self, level: int):
        Wl, Hl, f = C.c_int32(), C.c_int32(), C.c_int32()
        self._ok(self._L.orc_level_dims(self.h, level, C.byref(Wl), C.byref(Hl), C.byref(f)))
        return Wl.value, Hl.value, f.value

    def pyramid(self, level: int) -> np.ndarray:
        Wl, Hl, _ = self.level_dims(level)
        out = np.empty((Hl, Wl, 6), np.int64)
        self._ok(self._L.orc_read_pyramid(self.h, level, out.ctypes.data))
        return out


def run(rgb: np.ndarray, **kw):
    """Whole schedule; returns (full-res labels, stats M x 7, y, important, counters)."""
    o = Oracle(rgb, **kw).run()
    s, y, imp = o.stats()
    return o.labels(), s, y, imp, o.counters()
