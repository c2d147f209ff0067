"""The learned block scorer: features and scores against plain NumPy restatements of their
definitions, pruning that reduces to the plain method at threshold 0, training-data
logging and training, and pruned batches equal to pruned single runs."""
import numpy as np
import pytest

from gpu_common import STAT_FIELDS
from helpers import count_components_per_label, stats_from_labels
from paper_1704_02083_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


PARAMS = dict(num_levels=2, ratio_C=4, init_block=16, K=40, size_mode=2, predict=1)


def _bf16(x):
    """Round float32 to bfloat16 (nearest even) and back."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = (((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16).astype(np.uint32)
    return r.view(np.float32)


def _net(F, W):
    """The scorer's net on a feature map F (H x W x 9): three 3x3 convolutions with zero
    padding, ReLU, sigmoid; bf16 weights and activations."""
    w1, b1 = _bf16(W[:1296]).reshape(16, 9, 3, 3), W[1296:1312]
    w2, b2 = _bf16(W[1312:3616]).reshape(16, 16, 3, 3), W[3616:3632]
    w3, b3 = _bf16(W[3632:3776]).reshape(1, 16, 3, 3), W[3776:3777]

    def conv(x, w, b):
        H, Wd, _ = x.shape
        xp = np.pad(x.astype(np.float64), ((1, 1), (1, 1), (0, 0)))
        out = np.zeros((H, Wd, w.shape[0]))
        for ky in range(3):
            for kx in range(3):
                out += xp[ky:ky + H, kx:kx + Wd, :] @ w[:, :, ky, kx].T.astype(np.float64)
        return out + b

    h1 = _bf16(np.maximum(conv(_bf16(F), w1, b1), 0).astype(np.float32))
    h2 = _bf16(np.maximum(conv(h1, w2, b2), 0).astype(np.float32))
    z = conv(h2, w3, b3)[..., 0]
    return 1.0 / (1.0 + np.exp(-z))


def _features(rgb, blab, side, level, L, stats, imp_on):
    """The 9 features of every block, from their definitions (float64)."""
    H, W = rgb.shape[:2]
    nby, nbx = blab.shape
    mean = np.zeros((nby, nbx, 3))
    for by in range(nby):
        for bx in range(nbx):
            mean[by, bx] = rgb[by * side:(by + 1) * side, bx * side:(bx + 1) * side].reshape(-1, 3).mean(0)
    n = stats["n"].astype(np.float64)
    lm = np.stack([stats["sum_r"], stats["sum_g"], stats["sum_b"]], 1) / np.maximum(n, 1)[:, None]
    F = np.zeros((nby, nbx, 9))
    for by in range(nby):
        for bx in range(nbx):
            a = blab[by, bx]
            da = np.linalg.norm(mean[by, bx] - lm[a])
            nb = [blab[by - 1, bx] if by > 0 else -1, blab[by, bx - 1] if bx > 0 else -1,
                  blab[by, bx + 1] if bx + 1 < nbx else -1, blab[by + 1, bx] if by + 1 < nby else -1]
            cnt = 0
            for j, k in enumerate(nb):
                if k < 0 or k == a:
                    continue
                cnt += 1
                F[by, bx, j] = (da - np.linalg.norm(mean[by, bx] - lm[k])) / 64
            F[by, bx, 4] = cnt / 4
            F[by, bx, 5] = level / L
            F[by, bx, 6] = stats["important"][a] if imp_on else 1.0
            F[by, bx, 7] = np.log2(side) / 8
            F[by, bx, 8] = da / 64
    return F


def _ctx_at_stage(rgb, stage, **params):
    import torch

    import paper_1704_02083_gb300 as pkg

    ctx = pkg.Context(stream=torch.cuda.current_stream(), **params)
    ctx.set_image(torch.from_numpy(np.ascontiguousarray(rgb)).cuda())
    ctx.seed()
    ctx.refine_stage()
    for _ in range(stage):
        ctx.split()
        ctx.refine_stage()
    return ctx


def _random_weights(seed):
    rng = np.random.default_rng(seed)
    w = rng.normal(0, 0.35, 3777).astype(np.float32)
    w[1296:1312] = 0.1
    w[3616:3632] = 0.1
    return w


def test_features_and_scores_match_definitions():
    import torch

    import paper_1704_02083_gb300 as pkg

    rgb = synth.he_image(96, 144, 6, 31).rgb
    ctx = _ctx_at_stage(rgb, 3, **PARAMS)  # level 2 (after prediction), block side 2
    st = ctx.state()
    blab = ctx.block_labels()
    stats = ctx.stats()
    nby, nbx = blab.shape
    feat = torch.zeros(nby * nbx * 9, dtype=torch.float32, device="cuda")
    pkg.rapid_scorer_features(ctx.h, 0, feat.data_ptr())
    torch.cuda.synchronize()
    F = feat.cpu().numpy().reshape(nby, nbx, 9)
    ref = _features(rgb, blab, st["block"], st["level"], PARAMS["num_levels"], stats, True)
    np.testing.assert_allclose(F, ref, atol=2e-4)
    for seed in range(3):
        W = _random_weights(seed)
        sc = torch.zeros(nby * nbx, dtype=torch.float32, device="cuda")
        pkg.rapid_scorer_scores(ctx.h, 0, W, sc.data_ptr())
        torch.cuda.synchronize()
        got = sc.cpu().numpy().reshape(nby, nbx)
        want = _net(F, W)
        assert 0.01 < want.mean() < 0.99  # the weights exercise the net
        np.testing.assert_allclose(got, want, atol=3e-3)
    ctx.close()


def _run(rgb, weights=None, thr=0.0, **params):
    import torch

    import paper_1704_02083_gb300 as pkg

    with pkg.Context(stream=torch.cuda.current_stream(), **params) as ctx:
        ctx.set_image(torch.from_numpy(np.ascontiguousarray(rgb)).cuda())
        if weights is not None:
            ctx.set_scorer(weights, thr)
        ctx.run()
        st = ctx.stats()
        return ctx.labels(), np.stack([st[f] for f in STAT_FIELDS], 1), ctx.counters_array()


def test_threshold_zero_keeps_every_block():
    rgb = synth.he_image(128, 160, 8, 32).rgb
    lab, st, cnt = _run(rgb, **PARAMS)
    plab, pst, pcnt = _run(rgb, _random_weights(5), 0.0, **PARAMS)
    np.testing.assert_array_equal(plab, lab)
    np.testing.assert_array_equal(pst, st)
    np.testing.assert_array_equal(pcnt[:, 5], cnt[:, 5])  # the same moves


def _train(imgs, K, epochs=6):
    import torch

    import paper_1704_02083_gb300 as pkg

    with pkg.Trainer(200_000, neg_rate=0.3) as tr:
        with pkg.Context(stream=torch.cuda.current_stream(), **PARAMS) as ctx:
            ctx.set_logging(tr)
            ctx.set_images([torch.from_numpy(x).cuda() for x in imgs], K)
            ctx.run()
            ctx.sync()
            ctx.set_logging(None)
        n, pos = tr.count()
        w, loss = tr.fit(epochs=epochs, batch=1024, lr=3e-3, pos_weight=4.0, seed=1)
    return n, pos, w, loss


def test_logging_training_and_pruned_refinement():
    imgs = [synth.he_image(192, 192, 12, 40 + i).rgb for i in range(3)]
    n, pos, w, loss = _train(imgs, [80, 80, 80])
    assert n > 1000 and 0 < pos < n
    assert np.isfinite(w).all() and np.isfinite(loss).all()
    assert loss[-1] < loss[0]
    rgb = synth.he_image(192, 192, 12, 50).rgb
    plab, pst, pcnt = _run(rgb, **PARAMS)
    lab, st, cnt = _run(rgb, w, 0.3, **PARAMS)
    # every move is still exact: S equals recomputation, superpixels stay connected
    M = st.shape[0]
    np.testing.assert_array_equal(st[:, :6], stats_from_labels(rgb, lab, M)[:, :6])
    alive = int((st[:, 0] > 0).sum())
    assert count_components_per_label(lab) == alive
    # the scorer's mask keeps eligible blocks from the exact tests: the gap between eligible
    # and evaluated blocks grows (the evaluated total itself can rise: pruned sweeps end
    # with full sweeps, and training sums float gradients in no fixed order)
    assert (cnt[:, 3] - cnt[:, 4]).sum() > (pcnt[:, 3] - pcnt[:, 4]).sum()
    assert (lab != plab).mean() < 0.2


def test_pruned_batch_equals_pruned_single_runs():
    import torch

    import paper_1704_02083_gb300 as pkg

    imgs = [synth.he_image(96, 128, 6, 60 + i).rgb for i in range(3)]
    K = [30, 20, 40]
    W = _random_weights(9)
    with pkg.Context(stream=torch.cuda.current_stream(), **PARAMS) as ctx:
        ctx.set_scorer(W, 0.5)
        ctx.set_images([torch.from_numpy(x).cuda() for x in imgs], K)
        ctx.run()
        got = [(ctx.image_labels(i), ctx.counters_array(i)) for i in range(3)]
    for i, (x, k) in enumerate(zip(imgs, K)):
        p = dict(PARAMS)
        p["K"] = k
        lab, _, cnt = _run(x, W, 0.5, **p)
        np.testing.assert_array_equal(got[i][0], lab)
        np.testing.assert_array_equal(got[i][1], cnt)


def _log(imgs, K, trainer):
    import torch

    import paper_1704_02083_gb300 as pkg

    with pkg.Context(stream=torch.cuda.current_stream(), **PARAMS) as ctx:
        ctx.set_logging(trainer)
        ctx.set_images([torch.from_numpy(x).cuda() for x in imgs], K)
        ctx.run()
        ctx.sync()
        ctx.set_logging(None)


def test_logging_and_training_are_reproducible():
    """The same runs log the same samples in the same slots, and the same seed trains
    bit-identical weights (samples take their slots in block order, gradients are summed
    in a fixed order)."""
    import paper_1704_02083_gb300 as pkg

    imgs = [synth.he_image(160, 160, 10, 70 + i).rgb for i in range(2)]
    K = [60, 60]
    out = []
    for rep in range(2):
        with pkg.Trainer(100_000, neg_rate=0.3) as tr:
            _log(imgs, K, tr)
            n, pos = tr.count()
            x, inb, y = tr.samples(0, int(n))
            w, loss = tr.fit(epochs=3, batch=512, lr=3e-3, pos_weight=3.0, seed=5)
            out.append((n, x, inb, y, w, loss))
    (n0, x0, i0, y0, w0, l0), (n1, x1, i1, y1, w1, l1) = out
    assert n0 == n1 and n0 > 500
    np.testing.assert_array_equal(x0, x1)
    np.testing.assert_array_equal(i0, i1)
    np.testing.assert_array_equal(y0, y1)
    assert w0.tobytes() == w1.tobytes()
    assert l0.tobytes() == l1.tobytes()


def _bits(v, p):
    return (int(v) >> p) & 1


def _grad_float64(W, x, inb, y, pos_weight):
    """Summed loss gradient of samples (x: n x 7 x 7 x 9 patches, inb: in-image bits, y:
    labels), restated from the net's definition in float64: bf16 weights, inputs and
    activations, fp32 biases, zero padding outside the image at every layer, the roundings
    passed through by the backward pass.  Layout of W: w1 (16 x 9 x 3 x 3), b1 (16),
    w2 (16 x 16 x 3 x 3), b2 (16), w3 (16 x 3 x 3), b3."""
    w1 = _bf16(W[:1296]).reshape(16, 9, 3, 3).astype(np.float64)
    b1 = W[1296:1312].astype(np.float64)
    w2 = _bf16(W[1312:3616]).reshape(16, 16, 3, 3).astype(np.float64)
    b2 = W[3616:3632].astype(np.float64)
    w3 = _bf16(W[3632:3776]).reshape(16, 3, 3).astype(np.float64)
    b3 = float(W[3776])
    g = dict(w1=np.zeros_like(w1), b1=np.zeros(16), w2=np.zeros_like(w2), b2=np.zeros(16), w3=np.zeros_like(w3),
             b3=0.0)
    loss = 0.0
    for s in range(x.shape[0]):
        X = _bf16(x[s]).astype(np.float64)  # 7 x 7 x 9
        inside = np.array([[_bits(inb[s], r * 7 + c) for c in range(7)] for r in range(7)], bool)
        z1 = np.zeros((7, 7, 16))
        h1 = np.zeros((7, 7, 16))
        for r in range(1, 6):
            for c in range(1, 6):
                z1[r, c] = b1 + np.einsum("abk,kcab->c", X[r - 1:r + 2, c - 1:c + 2], w1.transpose(1, 0, 2, 3))
                if inside[r, c]:
                    h1[r, c] = _bf16(np.maximum(z1[r, c], 0).astype(np.float32))
        z2 = np.zeros((7, 7, 16))
        h2 = np.zeros((7, 7, 16))
        for r in range(2, 5):
            for c in range(2, 5):
                z2[r, c] = b2 + np.einsum("abk,kcab->c", h1[r - 1:r + 2, c - 1:c + 2], w2.transpose(1, 0, 2, 3))
                if inside[r, c]:
                    h2[r, c] = _bf16(np.maximum(z2[r, c], 0).astype(np.float32))
        z3 = b3 + np.einsum("abk,kab->", h2[2:5, 2:5], w3)
        p = 1.0 / (1.0 + np.exp(-z3))
        pos = y[s] > 0.5
        # the loss as training reports it: p in float32, whose 1 - p saturates (clamped at 1e-12)
        p32 = np.float32(1) / (np.float32(1) + np.exp(np.float32(-z3)))
        loss += -pos_weight * np.log(max(float(p32), 1e-12)) if pos else -np.log(max(float(np.float32(1) - p32), 1e-12))
        dz3 = pos_weight * (p - 1.0) if pos else p
        g["b3"] += dz3
        g["w3"] += dz3 * h2[2:5, 2:5].transpose(2, 0, 1)
        d2 = np.zeros((7, 7, 16))
        for r in range(2, 5):
            for c in range(2, 5):
                if inside[r, c]:
                    d2[r, c] = np.where(z2[r, c] > 0, dz3 * w3[:, r - 2, c - 2], 0.0)
        d1 = np.zeros((7, 7, 16))
        for r in range(2, 5):
            for c in range(2, 5):
                g["b2"] += d2[r, c]
                g["w2"] += np.einsum("o,abi->oiab", d2[r, c], h1[r - 1:r + 2, c - 1:c + 2])
                for ty in range(3):
                    for tx in range(3):
                        d1[r - 1 + ty, c - 1 + tx] += w2[:, :, ty, tx].T @ d2[r, c]
        for r in range(1, 6):
            for c in range(1, 6):
                d1[r, c] = np.where(inside[r, c] & (z1[r, c] > 0), d1[r, c], 0.0)
                g["b1"] += d1[r, c]
                g["w1"] += np.einsum("o,abi->oiab", d1[r, c], X[r - 1:r + 2, c - 1:c + 2])
    flat = np.concatenate([g["w1"].ravel(), g["b1"], g["w2"].ravel(), g["b2"], g["w3"].ravel(), [g["b3"]]])
    return flat, loss


def test_training_gradient_matches_a_float64_restatement():
    """rapid_trainer_gradient (the gradient training follows) against the net's forward and
    backward pass restated in float64, on 48 logged samples at seeded weights with active
    units in every layer.  Tolerance: per parameter group, 2e-3 of the group's largest
    gradient (float32 sums against float64; an activation on a bf16 rounding boundary can
    round the other way)."""
    import paper_1704_02083_gb300 as pkg

    imgs = [synth.he_image(128, 128, 8, 90).rgb]
    with pkg.Trainer(50_000, neg_rate=0.5) as tr:
        _log(imgs, [40], tr)
        n, pos = tr.count()
        assert n >= 48 and pos > 0
        x, inb, y = tr.samples(0, 48)
        W = _random_weights(17)
        g, loss = tr.gradient(W, 0, 48, pos_weight=2.5)
        g2, _ = tr.gradient(W, 0, 48, pos_weight=2.5)
    assert g.tobytes() == g2.tobytes()
    ref, rloss = _grad_float64(W, x, inb, y, 2.5)
    assert abs(loss - rloss) <= 1e-3 * abs(rloss) + 1e-3
    groups = [(0, 1296), (1296, 1312), (1312, 3616), (3616, 3632), (3632, 3776), (3776, 3777)]
    for a, b in groups:
        scale = np.abs(ref[a:b]).max()
        assert scale > 0, (a, b)
        err = np.abs(g[a:b] - ref[a:b]).max()
        assert err <= 2e-3 * scale + 1e-6, f"parameters {a}..{b}: {err} against scale {scale}"
