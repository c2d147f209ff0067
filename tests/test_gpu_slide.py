"""Whole slides (rapid_refine_slide): the slide is cut into even row and column bands of at
most max_tile pixels (Eq. parallel_spit on both axes) and the tiles are refined in batches.
Every tile must come out exactly as the same tile refined alone (and as the oracle), with
slide-wide ids numbered tile by tile in row-major order."""
import numpy as np
import pytest

from gpu_common import oracle_run
from paper_1704_02083_gb300 import synth

pytestmark = pytest.mark.gpu

PARAMS = dict(num_levels=2, ratio_C=4, init_block=16, size_mode=2, predict=1)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _bands(n_px, max_tile):
    n = -(-n_px // max_tile)
    return [(n_px * i // n, n_px * (i + 1) // n) for i in range(n)]


def _seed_count(H, W, K, s0=16):
    """M of a tile: the regular seed grid gx x gy for K superpixels (as the oracle seeds it)."""
    gx = max(1, int(np.floor(np.sqrt(K * W / H) + 0.5)))
    gy = max(1, int(np.floor(K / gx + 0.5)))
    return min(gx, -(-W // s0)) * min(gy, -(-H // s0))


def _single(rgb, K, **params):
    import torch

    import paper_1704_02083_gb300 as pkg

    with pkg.Context(stream=torch.cuda.current_stream(), K=K, **params) as ctx:
        ctx.set_image(torch.from_numpy(np.ascontiguousarray(rgb)).cuda()).run()
        return ctx.labels(), ctx.state()["M"], ctx.stats()


@pytest.mark.parametrize("schedule", [0, 1], ids=["sweeps", "queue"])
@pytest.mark.parametrize("H,W,max_tile,ppsp,check", [(600, 900, 256, 1024, "all"), (300, 310, 32, 256, "some")],
                         ids=["12_tiles", "100_tiles_two_batches"])
def test_slide_tiles_equal_single_runs(H, W, max_tile, ppsp, check, schedule):
    import torch

    import paper_1704_02083_gb300 as pkg

    img = synth.slide_image(H, W, 7)
    rgb = torch.from_numpy(img.rgb).cuda()
    params = dict(PARAMS, schedule=schedule)
    with pkg.Context(stream=torch.cuda.current_stream(), **params) as ctx:
        stats = torch.zeros((200000 * pkg.SP_STATS_DTYPE.itemsize,), dtype=torch.uint8, device="cuda")
        labels, M, T = ctx.refine_slide(rgb, max_tile=max_tile, px_per_superpixel=ppsp, stats=stats)
        torch.cuda.synchronize()
    lab = labels.cpu().numpy()
    st = stats.cpu().numpy()[: M * pkg.SP_STATS_DTYPE.itemsize].view(pkg.SP_STATS_DTYPE)
    rows, cols = _bands(H, max_tile), _bands(W, max_tile)
    assert T == len(rows) * len(cols)
    offset, n_checked = 0, 0
    for i, (r0, r1) in enumerate(rows):
        for j, (c0, c1) in enumerate(cols):
            K = max(1, (r1 - r0) * (c1 - c0) // ppsp)
            t = i * len(cols) + j
            tile = np.ascontiguousarray(img.rgb[r0:r1, c0:c1])
            sub = lab[r0:r1, c0:c1]
            if check == "all" or t % 17 == 0 or t == T - 1:
                slab, m, sst = _single(tile, K, **params)
                np.testing.assert_array_equal(sub - offset, slab, err_msg=f"tile {t}")
                np.testing.assert_array_equal(st[offset:offset + m]["n"], sst["n"])
                np.testing.assert_array_equal(st[offset:offset + m]["sum_x"], sst["sum_x"])
                n_checked += 1
            else:
                m = _seed_count(r1 - r0, c1 - c0, K)
            assert m == _seed_count(r1 - r0, c1 - c0, K)
            assert sub.min() >= offset and sub.max() < offset + m
            offset += m
    assert offset == M and n_checked >= 3


def test_slide_tile_against_oracle():
    import torch

    import paper_1704_02083_gb300 as pkg

    img = synth.slide_image(200, 260, 9)
    with pkg.Context(stream=torch.cuda.current_stream(), **PARAMS) as ctx:
        labels, M, T = ctx.refine_slide(torch.from_numpy(img.rgb).cuda(), max_tile=128, px_per_superpixel=512)
    lab = labels.cpu().numpy()
    assert T == 2 * 3
    # the first tile: rows 0..100, columns 0..86
    tile = np.ascontiguousarray(img.rgb[0:100, 0:86])
    rlab = oracle_run(tile, K=max(1, 100 * 86 // 512), **PARAMS)[0]
    np.testing.assert_array_equal(lab[0:100, 0:86], rlab)


def test_counter_slide_on_the_device_tiles_against_the_oracle():
    """The whole-slide workload's pipeline at a small size: the slide made on the device by
    the counter-based generator, refined by rapid_refine_slide with the full-size workload's
    schedule; sampled tiles, each generated alone on the host from the same definition, against
    the oracle (labels, and the statistics of their slide-wide ids)."""
    import torch

    import paper_1704_02083_gb300 as pkg

    sd = synth.SLIDES["slide100k_l3"]
    H, W, max_tile, pps = 2600, 2100, 1024, 16384
    params = dict(sd["params"])
    rgb = pkg.synth_slide_device(H, W, 13)
    with pkg.Context(stream=torch.cuda.current_stream(), **params) as ctx:
        stats = torch.zeros((20000 * pkg.SP_STATS_DTYPE.itemsize,), dtype=torch.uint8, device="cuda")
        labels, M, T = ctx.refine_slide(rgb, max_tile=max_tile, px_per_superpixel=pps, stats=stats)
        torch.cuda.synchronize()
    tiles = synth.slide_tiles(H, W, max_tile, pps)
    assert T == len(tiles) == 9
    lab = labels.cpu().numpy()
    st = stats.cpu().numpy()[: M * pkg.SP_STATS_DTYPE.itemsize].view(pkg.SP_STATS_DTYPE)
    bases = np.cumsum([0] + [_seed_count(h, w, K, s0=32) for (_, _, h, w, K) in tiles])
    assert bases[-1] == M
    for t in (0, 4, 8):
        r0, c0, h, w, K = tiles[t]
        host = synth.slide_gen(H, W, 13, x0=c0, y0=r0, h=h, w=w)
        np.testing.assert_array_equal(rgb[r0:r0 + h, c0:c0 + w].cpu().numpy(), host.rgb)
        rlab, rst, _, _, _ = oracle_run(host.rgb, K=K, **params)
        np.testing.assert_array_equal(lab[r0:r0 + h, c0:c0 + w] - bases[t], rlab, err_msg=f"tile {t}")
        got = np.stack([st[bases[t]:bases[t + 1]][f] for f in ("n", "sum_r", "sum_g", "sum_b", "sum_x", "sum_y",
                                                                 "init_size")], 1)
        np.testing.assert_array_equal(got, rst, err_msg=f"tile {t}")
