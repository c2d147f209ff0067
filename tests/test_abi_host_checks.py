"""Argument checks of the C ABI that run before any CUDA call, exercised on the CPU.

Every entry point refuses a NULL context or handle with RAPID_EINVAL (the destroy calls
accept NULL).  rapid_create and rapid_run_static refuse every parameter set that
include/rapid.h calls invalid.  rapid_run_static refuses an image above its pixel limit
with RAPID_ERANGE before launching anything.  Without a GPU, a valid rapid_create reports
RAPID_ECUDA: there is no CPU fallback."""
import ctypes as C

import pytest


@pytest.fixture(scope="module")
def pkg():
    from paper_1704_02083_gb300 import build
    build.build()
    import paper_1704_02083_gb300 as p
    p.lib()
    return p


def _null_calls(pkg):
    i32, i64 = C.c_int32(), C.c_int64()
    buf = (C.c_uint8 * 4096)()
    ctr = pkg.rapid_counters()
    return {
        "rapid_set_image": (None, buf, 8, 8, 24, 0),
        "rapid_seed_grid": (None, C.byref(i32)),
        "rapid_refine_stage": (None, None, None, None),
        "rapid_split": (None,),
        "rapid_run": (None,),
        "rapid_sync": (None,),
        "rapid_get_state": (None, None, None, None, None),
        "rapid_read_labels": (None, buf, 32, 0),
        "rapid_read_block_labels": (None, buf, 16, None, None),
        "rapid_read_stats": (None, buf, 1, None),
        "rapid_read_counters": (None, C.byref(ctr)),
        "rapid_set_profiling": (None, 1),
        "rapid_set_images": (None, 1, None, None, None, None, None, 1),
        "rapid_get_image_info": (None, 0, None, None, None),
        "rapid_read_image_labels": (None, 0, buf, 32, 0),
        "rapid_read_image_stats": (None, 0, buf, 1, None),
        "rapid_read_image_counters": (None, 0, C.byref(ctr)),
        "rapid_set_graph": (None, 0),
        "rapid_set_stage_grids": (None, None, 0),
        "rapid_set_stage_shapes": (None, None, 0),
        "rapid_autotune": (None, None, None),
        "rapid_set_scorer": (None, None, C.c_float(0.5)),
        "rapid_set_keep_mask": (None, 0, 0, buf, 16, 0),
        "rapid_set_scorer_stages": (None, None, 0),
        "rapid_set_race_check": (None, 1),
        "rapid_read_race_violations": (None, C.byref(i64)),
        "rapid_set_classifier": (None, None),
        "rapid_read_features": (None, 0, buf),
        "rapid_scorer_features": (None, 0, buf),
        "rapid_scorer_scores": (None, 0, buf, buf),
        "rapid_set_logging": (None, None),
        "rapid_trainer_count": (None, C.byref(i64), C.byref(i64)),
        "rapid_trainer_fit": (None, 1, 1, C.c_float(1e-3), C.c_float(1.0), 0, None, buf, None),
        "rapid_trainer_samples": (None, 0, 1, buf, buf, buf),
        "rapid_trainer_gradient": (None, buf, 0, 1, C.c_float(1.0), buf, None),
        "rapid_refine_slide": (None, buf, 8, 8, 24, 64, 16, 0, buf, 32, None, 0, None, None),
        "rapid_simple_table": (None,),
        "rapid_create": (None, None, None),
    }


def test_null_handles_are_refused(pkg):
    L = pkg.lib()
    calls = _null_calls(pkg)
    for name, args in calls.items():
        assert getattr(L, name)(*args) == pkg.RAPID_EINVAL, name
    L.rapid_destroy(None)
    L.rapid_trainer_destroy(None)
    L.rapid_default_params(None)
    # every ctx-taking entry point of the header is covered here
    import test_abi
    takes_handle = {n for n in test_abi.declared_functions()
                    if n not in ("rapid_default_params", "rapid_status_string", "rapid_destroy",
                                 "rapid_trainer_destroy", "rapid_trainer_create", "rapid_run_static",
                                 "rapid_synth_slide", "rapid_debug_fail_alloc", "rapid_race_selftest")}
    assert takes_handle <= set(calls), sorted(takes_handle - set(calls))


def test_static_entry_refuses_non_boolean_flags(pkg):
    """rapid_run_static takes the same 0/1 flags as rapid_create and refuses other values
    before any CUDA call."""
    L = pkg.lib()
    fake = C.c_void_p(256)
    M = C.c_int32()
    for flag in ("use_filter", "skip_tiles", "verify_filter", "predict", "reuse", "importance_rule", "schedule"):
        p = pkg.rapid_default_params(**{flag: 2})
        assert L.rapid_run_static(C.byref(p), fake, 8, 8, 24, fake, 32, fake, 16, C.byref(M), None) == \
            pkg.RAPID_EINVAL, flag


BAD = [dict(num_levels=0), dict(num_levels=9), dict(num_levels=2, ratio_C=3), dict(num_levels=2, ratio_C=1),
       dict(num_levels=8, ratio_C=16), dict(init_block=3), dict(init_block=1 << 21), dict(final_grain=6),
       dict(K=0), dict(size_mode=-1), dict(size_mode=3), dict(max_sweeps=0), dict(lo_den=0), dict(hi_den=0),
       dict(lo_num=-1), dict(hi_num=-1), dict(lambda_pos0=float("inf")), dict(lambda_b=float("nan")),
       dict(predict=2), dict(reuse=-1), dict(importance_rule=2), dict(schedule=2), dict(spin_limit_ns=-1),
       dict(h_T=-1), dict(h_T=(1 << 40) + 1)]


@pytest.mark.parametrize("bad", BAD, ids=[",".join(f"{k}={v}" for k, v in b.items()) for b in BAD])
def test_invalid_parameters_are_refused_before_any_cuda_call(pkg, bad):
    L = pkg.lib()
    h = C.c_void_p(123)
    p = pkg.rapid_default_params(**bad)
    assert L.rapid_create(C.byref(p), None, C.byref(h)) == pkg.RAPID_EINVAL
    assert h.value is None  # *out is cleared
    fake = C.c_void_p(256)  # never dereferenced: the checks come first
    M = C.c_int32()
    assert L.rapid_run_static(C.byref(p), fake, 8, 8, 24, fake, 32, fake, 16, C.byref(M), None) == pkg.RAPID_EINVAL


def test_static_entry_checks_sizes_before_launching(pkg):
    L = pkg.lib()
    p = pkg.rapid_default_params()
    fake = C.c_void_p(256)
    M = C.c_int32()
    assert L.rapid_run_static(C.byref(p), None, 8, 8, 24, fake, 32, fake, 16, C.byref(M), None) == pkg.RAPID_EINVAL
    assert L.rapid_run_static(C.byref(p), fake, 8, 8, 23, fake, 32, fake, 16, C.byref(M), None) == pkg.RAPID_EINVAL
    assert L.rapid_run_static(C.byref(p), fake, 8, 8, 24, fake, 30, fake, 16, C.byref(M), None) == pkg.RAPID_EINVAL
    assert L.rapid_run_static(C.byref(p), fake, 0, 8, 24, fake, 32, fake, 16, C.byref(M), None) == pkg.RAPID_EINVAL
    big = 1 << 10  # 1024 x 1024 > 2^19 pixels
    assert L.rapid_run_static(C.byref(p), fake, big, big, 3 * big, fake, 4 * big, fake, 16, C.byref(M),
                              None) == pkg.RAPID_ERANGE


def test_trainer_arguments(pkg):
    L = pkg.lib()
    h = C.c_void_p()
    for cap, rate in ((0, 0.1), ((1 << 30) + 1, 0.1), (100, -0.5), (100, 1.5), (100, float("nan"))):
        assert L.rapid_trainer_create(cap, C.c_float(rate), C.byref(h)) == pkg.RAPID_EINVAL
    assert L.rapid_trainer_create(100, C.c_float(0.1), None) == pkg.RAPID_EINVAL


def test_valid_create_without_a_gpu_reports_ecuda(pkg):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    L = pkg.lib()
    h = C.c_void_p()
    p = pkg.rapid_default_params()
    assert L.rapid_create(C.byref(p), None, C.byref(h)) == pkg.RAPID_ECUDA
    assert h.value is None


def test_slide_generator_checks_its_arguments_before_any_cuda_call(pkg):
    L = pkg.lib()
    fake = C.c_void_p(256)
    good = dict(H=512, W=768, seed=5, px_per_cell=8192, pad=0, white_frac=0.4, fold_frac=0.05,
                nucleus_density=1 / 400)
    for bad in (dict(H=0), dict(W=-1), dict(px_per_cell=0), dict(white_frac=1.5), dict(fold_frac=-0.1),
                dict(nucleus_density=float("nan"))):
        p = pkg.rapid_synth_params(**dict(good, **bad))
        assert L.rapid_synth_slide(C.byref(p), fake, 3 * 768, None, 0, None) == pkg.RAPID_EINVAL, bad
    p = pkg.rapid_synth_params(**good)
    assert L.rapid_synth_slide(None, fake, 3 * 768, None, 0, None) == pkg.RAPID_EINVAL
    assert L.rapid_synth_slide(C.byref(p), None, 3 * 768, None, 0, None) == pkg.RAPID_EINVAL
    assert L.rapid_synth_slide(C.byref(p), fake, 3 * 768 - 1, None, 0, None) == pkg.RAPID_EINVAL
    assert L.rapid_synth_slide(C.byref(p), fake, 3 * 768, fake, 4 * 768 - 4, None) == pkg.RAPID_EINVAL
    dense = pkg.rapid_synth_params(**dict(good, px_per_cell=1024))  # 16 seeds per bucket
    assert L.rapid_synth_slide(C.byref(dense), fake, 3 * 768, None, 0, None) == pkg.RAPID_ERANGE
