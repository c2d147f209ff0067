"""rapid_run_static, the entry point for callers that cannot call cudaMalloc (for example a
service whose GPU memory is fully reserved by its own pool allocator): the whole refinement
runs with every byte of working memory taken from one fixed array inside the library.

Checked through the C ABI against the allocating path (rapid_run + reads) on two calls in
a row, bit for bit (labels and int64 statistics are exact on both paths), plus the size
limit.  This file is collected last so a failure here comes after every other test."""
import ctypes as C

import numpy as np
import pytest

from paper_1704_02083_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1704_02083_gb300 as pkg
    return torch, pkg


def _reference(torch, pkg, rgb, params):
    with pkg.Context(stream=torch.cuda.current_stream(), **params) as ctx:
        ctx.set_image(rgb).run()
        return ctx.labels(), ctx.stats()


def _static(torch, pkg, rgb, params, fill):
    H, W = rgb.shape[:2]
    dev_rgb = torch.from_numpy(np.ascontiguousarray(rgb)).cuda()
    labels = torch.full((H, W), fill, dtype=torch.int32, device="cuda")
    cap = 1 << 13
    stats = torch.full((cap * C.sizeof(pkg.rapid_sp_stats),), fill & 0xFF, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    M = pkg.rapid_run_static(pkg.rapid_default_params(**params), dev_rgb.data_ptr(), H, W, 3 * W,
                             labels.data_ptr(), 4 * W, stats.data_ptr(), cap, stream.cuda_stream)
    st = np.frombuffer(stats.cpu().numpy().tobytes(), dtype=pkg.SP_STATS_DTYPE)[:M]
    return labels.cpu().numpy(), st


CASES = [
    ("he321x481_k200", synth.WORKLOADS["he321x481_k200"]["params"]),
    ("he384x512_l3", dict(num_levels=3, ratio_C=4, init_block=32, K=192, predict=1, size_mode=2)),
    ("he321x481_k200_frontier", synth.WORKLOADS["he321x481_k200_frontier"]["params"]),
]


def test_static_entry_matches_allocating_path_twice_in_a_row(env):
    torch, pkg = env
    for (name, params), fill in zip(CASES, (-7, 123, 5)):
        if name in synth.WORKLOADS:
            rgb = synth.workload_image(name).rgb
        else:
            rgb = synth.he_image(384, 512, 24, seed=17).rgb
        ref_lab, ref_st = _reference(torch, pkg, rgb, params)
        lab, st = _static(torch, pkg, rgb, params, fill)
        np.testing.assert_array_equal(lab, ref_lab)
        assert st.shape == ref_st.shape
        for f in pkg.SP_STATS_DTYPE.names:
            np.testing.assert_array_equal(st[f], ref_st[f], err_msg=f)


def test_static_entry_rejects_oversize(env):
    torch, pkg = env
    H, W = 1024, 1024  # 2^20 pixels > RAPID_STATIC_MAX_PIXELS
    rgb = torch.zeros((H, W, 3), dtype=torch.uint8, device="cuda")
    lab = torch.zeros((H, W), dtype=torch.int32, device="cuda")
    st = torch.zeros((64 * C.sizeof(pkg.rapid_sp_stats),), dtype=torch.uint8, device="cuda")
    with pytest.raises(pkg.RapidError) as e:
        pkg.rapid_run_static(pkg.rapid_default_params(), rgb.data_ptr(), H, W, 3 * W, lab.data_ptr(), 4 * W,
                             st.data_ptr(), 64)
    assert e.value.status == pkg.RAPID_ERANGE
    # the array is still usable afterwards
    small = synth.he_image(64, 96, 4, seed=2).rgb
    params = dict(K=12, init_block=8)
    ref_lab, _ = _reference(torch, pkg, small, params)
    got, _ = _static(torch, pkg, small, params, 0)
    np.testing.assert_array_equal(got, ref_lab)
