"""The device slide generator (rapid_synth_slide) against its host restatement
(synth.slide_gen): the same bytes and ground-truth ids, for slides of several sizes (ragged
against the 128-px buckets, narrow, with folds and nuclei crossing bucket edges), and a
window of a larger slide generated alone on the host."""
import numpy as np
import pytest

from paper_1704_02083_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("H,W,seed", [(700, 1000, 5), (333, 517, 9), (129, 257, 1), (1, 300, 2), (200, 1, 3),
                                      (640, 384, 11)])
def test_device_slide_equals_the_host_restatement(H, W, seed):
    import paper_1704_02083_gb300 as pkg

    rgb, reg = pkg.synth_slide_device(H, W, seed, regions=True)
    host = synth.slide_gen(H, W, seed)
    got = rgb.cpu().numpy()
    diff = np.argwhere((got != host.rgb).any(-1))
    assert diff.size == 0, f"{len(diff)} pixels differ, first at {diff[:3].tolist()}"
    np.testing.assert_array_equal(reg.cpu().numpy(), host.regions.astype(np.int32))


def test_window_of_a_large_slide():
    """A 512 x 640 window at an odd offset of a 6000 x 5000 slide: the host makes the window
    alone, the device the whole slide."""
    import paper_1704_02083_gb300 as pkg

    H, W, seed = 6000, 5000, 5
    rgb = pkg.synth_slide_device(H, W, seed)
    y0, x0, h, w = 2701, 1333, 512, 640
    host = synth.slide_gen(H, W, seed, x0=x0, y0=y0, h=h, w=w)
    np.testing.assert_array_equal(rgb[y0:y0 + h, x0:x0 + w].cpu().numpy(), host.rgb)


def test_slide_recipe():
    """The stated recipe on a 2048 x 3072 slide: about 40% white area, folds covering a few
    percent, purple and nuclei as ROI share, noise of sigma 6 inside a flat cell."""
    import paper_1704_02083_gb300 as pkg

    H, W = 2048, 3072
    rgb, reg = pkg.synth_slide_device(H, W, 7, regions=True)
    rgb, reg = rgb.cpu().numpy().astype(np.int64), reg.cpu().numpy()
    lay = synth.gen_layout(H, W)
    fold = reg >= lay["n_cells"] + lay["n_nuclei"]
    assert 0.01 < fold.mean() < 0.10
    white = (np.abs(rgb - 245).max(-1) <= 30) & ~fold
    assert 0.25 < white.mean() < 0.55
