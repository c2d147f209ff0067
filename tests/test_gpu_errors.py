"""Error behaviour of the C ABI on the GPU: out-of-order calls, invalid arguments, and a
device-side wait that gives up (spin limit 0) returning RAPID_ETIMEOUT instead of
hanging."""
import numpy as np
import pytest

from paper_1704_02083_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1704_02083_gb300 as p
    return p


def test_out_of_order_calls(pkg):
    buf = np.zeros((4, 4), np.int32)
    with pkg.Context() as ctx:
        for fn in (ctx.seed, lambda: ctx.refine_stage(sync=True), ctx.split,
                   lambda: pkg.rapid_read_labels(ctx.h, buf.ctypes.data, 16, 0)):
            with pytest.raises(pkg.RapidError) as e:
                fn()
            assert e.value.status == pkg.RAPID_ESTATE
        ctx.set_image(synth.he_image(32, 32, 3, 1).rgb)
        with pytest.raises(pkg.RapidError) as e:
            ctx.refine_stage(sync=True)
        assert e.value.status == pkg.RAPID_ESTATE


def test_invalid_arguments(pkg):
    with pytest.raises(pkg.RapidError) as e:
        pkg.rapid_create(pkg.rapid_default_params(init_block=3))
    assert e.value.status == pkg.RAPID_EINVAL
    with pytest.raises(pkg.RapidError) as e:
        pkg.rapid_create(pkg.rapid_default_params(num_levels=2, ratio_C=3))
    assert e.value.status == pkg.RAPID_EINVAL
    with pkg.Context(K=16, init_block=2) as ctx:
        rgb = np.zeros((8, 8, 3), np.uint8)
        for H, W, pitch in ((0, 8, 24), (8, 0, 24), (8, 8, 23)):
            with pytest.raises(pkg.RapidError) as e:
                pkg.rapid_set_image(ctx.h, rgb.ctypes.data, H, W, pitch, 0)
            assert e.value.status == pkg.RAPID_EINVAL
        ctx.set_image(rgb).run()
        small = np.zeros(3, pkg.SP_STATS_DTYPE)
        M = ctx.state()["M"]
        assert M > 3
        with pytest.raises(pkg.RapidError) as e:
            pkg.rapid_read_stats(ctx.h, small.ctypes.data, 3)
        assert e.value.status == pkg.RAPID_EINVAL
        out = np.zeros((8, 8), np.int32)
        with pytest.raises(pkg.RapidError) as e:
            pkg.rapid_read_labels(ctx.h, out.ctypes.data, 16, 0)
        assert e.value.status == pkg.RAPID_EINVAL


def test_level_sums_that_would_overflow_are_refused(pkg):
    """A level cell of 4096 x 4096 pixels could hold a channel sum of 255 * 2^24 > 2^31 - 1:
    rapid_set_image refuses it with RAPID_ERANGE before copying anything."""
    rgb = np.zeros((4096, 4096, 3), np.uint8)
    with pkg.Context(num_levels=2, ratio_C=4096, init_block=4096, K=1) as ctx:
        with pytest.raises(pkg.RapidError) as e:
            ctx.set_image(rgb)
        assert e.value.status == pkg.RAPID_ERANGE
    with pkg.Context(num_levels=2, ratio_C=2048, init_block=2048, K=4) as ctx:
        ctx.set_image(rgb[:2048, :2048]).run()  # 255 * 2^22 fits
        ctx.sync()
        assert ctx.state()["M"] == 1  # the first stage has a single 2048-px block


def test_barrier_give_up_reports_timeout(pkg):
    """spin_limit_ns = 0: every grid-barrier wait gives up at once; the launch returns,
    the context reports RAPID_ETIMEOUT, and a fresh context still works."""
    rgb = synth.he_image(64, 64, 4, 3).rgb
    with pkg.Context(spin_limit_ns=0, K=16, init_block=8) as ctx:
        ctx.set_image(rgb).run()
        with pytest.raises(pkg.RapidError) as e:
            ctx.sync()
        assert e.value.status == pkg.RAPID_ETIMEOUT
        with pytest.raises(pkg.RapidError) as e:  # sticky
            ctx.labels()
        assert e.value.status == pkg.RAPID_ETIMEOUT
    with pkg.Context(K=16, init_block=8) as ctx:
        ctx.set_image(rgb).run()
        ctx.sync()
        assert ctx.labels().shape == (64, 64)
