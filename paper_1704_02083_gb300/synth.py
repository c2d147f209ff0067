"""Seeded synthetic H&E-like images: the input generator shared by tests and the bench.

The paper evaluates on BSD500 and on NLST whole-slide H&E images (Sec. 4.1); neither is
available here, so every input is generated from a seed with the shapes and structure of
those workloads:

* tissue regions: a Voronoi partition of ``n_cells`` uniform seed points (exact Euclidean
  nearest seed, from ``scipy.ndimage.distance_transform_edt``);
* region class: pink (230,150,190) 45 %, purple (120,70,150) 35 %, white (245,245,245) 20 %
  (``white_frac`` moves the white share and rescales the other two); per-region mean
  colour = base + U{-15..15} per channel (white: U{-5..5});
* nuclei: round(area * ``nucleus_density``) discs (a Poisson process conditioned on its
  mean count) with uniform centres, radius U{3..8}, colour (60,30,90) + U{-10..10}, placed only where the centre
  falls in a non-white region;
* noise: a discrete Gaussian of standard deviation 6 per channel (integer offsets -30..30
  with probability proportional to exp(-v^2/72), drawn by table inversion of uniform 32-bit
  integers), clamped to [0, 255].

Only integer operations of numpy's PCG64 stream and an exact Euclidean distance transform
are used, so a seed gives the same bytes on x86-64 and AArch64.

It also returns the ground-truth region map (regions, then nuclei) and the ROI mask
(purple regions and nuclei), which the quality metrics use.  This module holds none of the
superpixel method's arithmetic: it only makes pixels.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.ndimage as ndi

PINK = (230, 150, 190)
PURPLE = (120, 70, 150)
WHITE = (245, 245, 245)
NUCLEUS = (60, 30, 90)


@dataclasses.dataclass
class SynthImage:
    rgb: np.ndarray        # H x W x 3 uint8, C-contiguous (interleaved RGB)
    regions: np.ndarray    # H x W int32 ground-truth region id
    roi: np.ndarray        # H x W bool, purple regions and nuclei
    n_regions: int


# Cumulative thresholds (out of 2^32) of the discrete Gaussian noise, sigma = 6, support
# -30..30: offset v = -30 + #(thresholds <= u) for a uniform 32-bit u.
_NOISE_CDF = np.array([
    1064, 3479, 8809, 20251, 44139, 92645, 188445, 372463, 716254, 1340945, 2444952, 4342595,
    7515037, 12673366, 20830933, 33378184, 52148550, 79459272, 118107525, 171301547, 242510082,
    335222422, 452625448, 597221792, 770431245, 972231699, 1200901570, 1452919839, 1723061373,
    2004696593, 2290270703, 2571905923, 2842047457, 3094065726, 3322735597, 3524536051,
    3697745504, 3842341848, 3959744874, 4052457214, 4123665749, 4176859771, 4215508024,
    4242818746, 4261589112, 4274136363, 4282293930, 4287452259, 4290624701, 4292522344,
    4293626351, 4294251042, 4294594833, 4294778851, 4294874651, 4294923157, 4294947045,
    4294958487, 4294963817, 4294966232], np.uint32)
_NOISE_LO = -30


def he_image(H: int, W: int, n_cells: int, seed: int, nucleus_density: float = 1.0 / 400.0,
             white_frac: float = 0.20) -> SynthImage:
    """Generate one H x W synthetic H&E-like tile (see the module docstring)."""
    if H <= 0 or W <= 0:
        raise ValueError("image must be non-empty")
    rng = np.random.default_rng(seed)
    n_cells = max(1, int(n_cells))

    # Voronoi seeds: distinct pixels (duplicates collapse into one region).
    sy = rng.integers(0, H, n_cells)
    sx = rng.integers(0, W, n_cells)
    flat = np.unique(sy.astype(np.int64) * W + sx)
    sy, sx = (flat // W).astype(np.int64), (flat % W).astype(np.int64)
    n = flat.size
    seed_id = np.full((H, W), -1, np.int32)
    seed_id[sy, sx] = np.arange(n, dtype=np.int32)
    notseed = seed_id < 0
    if notseed.all():  # cannot happen (n >= 1) but keeps the EDT call well defined
        raise RuntimeError("no Voronoi seed")
    iy, ix = ndi.distance_transform_edt(notseed, return_distances=False, return_indices=True)
    cell = seed_id[iy, ix]
    del iy, ix

    # class by integer thresholds on U{0..9999}: white, then purple, then pink
    u = rng.integers(0, 10000, size=n)
    n_white = int(round(white_frac * 10000))
    n_purple = int(round((1.0 - white_frac) * 0.4375 * 10000))  # 35 % of 80 %
    cls = np.where(u < n_white, 2, np.where(u < n_white + n_purple, 1, 0))
    base = np.array([PINK, PURPLE, WHITE], np.int32)[cls]
    jit = rng.integers(-15, 16, size=(n, 3))
    jit_w = rng.integers(-5, 6, size=(n, 3))
    mean = base + np.where((cls == 2)[:, None], jit_w, jit)

    img = mean[cell].astype(np.int32)              # H x W x 3
    regions = cell.astype(np.int32)
    roi = (cls == 1)[cell]

    # Nuclei.
    n_nuc = int(H * W * nucleus_density + 0.5)
    cy = rng.integers(0, H, n_nuc)
    cx = rng.integers(0, W, n_nuc)
    rad = rng.integers(3, 9, n_nuc)
    ncol = np.array(NUCLEUS, np.int32)[None, :] + rng.integers(-10, 11, size=(n_nuc, 3))
    keep = cls[cell[cy, cx]] != 2
    for r in range(3, 9):
        sel = np.nonzero(keep & (rad == r))[0]
        if sel.size == 0:
            continue
        dy, dx = np.mgrid[-r:r + 1, -r:r + 1]
        inside = dy * dy + dx * dx <= r * r
        dy, dx = dy[inside], dx[inside]
        yy = cy[sel][:, None] + dy[None, :]
        xx = cx[sel][:, None] + dx[None, :]
        ok = (yy >= 0) & (yy < H) & (xx >= 0) & (xx < W)
        which = np.broadcast_to(sel[:, None], yy.shape)[ok]
        yy, xx = yy[ok], xx[ok]
        img[yy, xx] = ncol[which]
        regions[yy, xx] = n + which
        roi[yy, xx] = True

    # Noise, row band by row band to bound memory.
    out = np.empty((H, W, 3), np.uint8)
    band = max(1, (1 << 22) // max(1, W))
    for y0 in range(0, H, band):
        y1 = min(H, y0 + band)
        u = rng.integers(0, 1 << 32, size=(y1 - y0, W, 3), dtype=np.uint64).astype(np.uint32)
        noise = np.searchsorted(_NOISE_CDF, u, side="right").astype(np.int32) + _NOISE_LO
        out[y0:y1] = np.clip(img[y0:y1] + noise, 0, 255).astype(np.uint8)
    return SynthImage(rgb=out, regions=regions, roi=roi, n_regions=int(n + n_nuc))


FOLD = (80, 40, 110)


def slide_image(H: int, W: int, seed: int, px_per_cell: int = 8192, white_frac: float = 0.40,
                fold_frac: float = 0.05) -> SynthImage:
    """A whole-slide stand-in: the tile generator over the whole slide with ``white_frac``
    white background, then tissue folds painted over it until they cover about
    ``fold_frac`` of the area: straight dark-purple bands (colour FOLD + U{-10..10}, the
    same noise) of width U{20..80} px, uniform angle and centre, length U[0.3, 1.0] x the
    shorter side.  Each band is one more ground-truth region (not ROI)."""
    img = he_image(H, W, max(1, (H * W) // px_per_cell), seed, white_frac=white_frac)
    rgb, regions, roi = img.rgb, img.regions, img.roi
    rng = np.random.default_rng(seed + 7919)
    covered, target, band = 0, fold_frac * H * W, 0
    while covered < target and band < 10000:
        width = int(rng.integers(20, 81))
        length = (0.3 + 0.7 * float(rng.integers(0, 1 << 20)) / float(1 << 20)) * min(H, W)
        theta = np.pi * float(rng.integers(0, 1 << 20)) / float(1 << 20)
        cy, cx = float(rng.integers(0, H)), float(rng.integers(0, W))
        dy, dx = np.sin(theta), np.cos(theta)
        # pixels p with |n.(p - c)| <= width / 2 and |d.(p - c)| <= length / 2, row by row
        ext = 0.5 * (abs(dy) * length + abs(dx) * width) + 1
        ys = np.arange(max(0, int(cy - ext)), min(H, int(cy + ext) + 1))
        if ys.size == 0:
            band += 1
            continue
        # for a row y the constraints are two intervals in x; intersect them
        lo = np.full(ys.size, -np.inf)
        hi = np.full(ys.size, np.inf)
        # d.(p - c) = dx (x - cx) + dy (y - cy);  n.(p - c) = -dy (x - cx) + dx (y - cy)
        for a, by, half in ((dx, dy, 0.5 * length), (-dy, dx, 0.5 * width)):
            b = by * (ys - cy)  # the y part of the projection
            if abs(a) < 1e-12:
                bad = np.abs(b) > half
                lo[bad], hi[bad] = np.inf, -np.inf
                continue
            x1 = (-half - b) / a + cx
            x2 = (half - b) / a + cx
            lo = np.maximum(lo, np.minimum(x1, x2))
            hi = np.minimum(hi, np.maximum(x1, x2))
        xl = np.clip(np.ceil(lo), 0, W).astype(np.int64)
        xr = np.clip(np.floor(hi) + 1, 0, W).astype(np.int64)
        n = np.maximum(xr - xl, 0)
        if n.sum() == 0:
            band += 1
            continue
        yy = np.repeat(ys, n)
        xx = np.repeat(xl, n) + (np.arange(n.sum()) - np.repeat(np.cumsum(n) - n, n))
        col = np.array(FOLD, np.int32) + rng.integers(-10, 11, size=3)
        u = rng.integers(0, 1 << 32, size=(yy.size, 3), dtype=np.uint64).astype(np.uint32)
        noise = np.searchsorted(_NOISE_CDF, u, side="right").astype(np.int32) + _NOISE_LO
        rgb[yy, xx] = np.clip(col[None, :] + noise, 0, 255).astype(np.uint8)
        regions[yy, xx] = img.n_regions + band
        roi[yy, xx] = False
        covered += int(n.sum())
        band += 1
    return SynthImage(rgb=rgb, regions=regions, roi=roi, n_regions=img.n_regions + band)


def flat_image(H: int, W: int, colour=(128, 128, 128)) -> np.ndarray:
    """A constant-colour image (closed-form test cases)."""
    out = np.empty((H, W, 3), np.uint8)
    out[...] = np.array(colour, np.uint8)
    return out


def two_colour_image(H: int, W: int, x0: int, left=(230, 150, 190), right=(120, 70, 150)) -> np.ndarray:
    """Columns [0, x0) in one colour, [x0, W) in another (closed-form test cases)."""
    out = np.empty((H, W, 3), np.uint8)
    out[:, :x0] = np.array(left, np.uint8)
    out[:, x0:] = np.array(right, np.uint8)
    return out


def random_image(H: int, W: int, seed: int, levels: int = 256) -> np.ndarray:
    """Uniform random pixels (tiny fuzz cases); ``levels`` < 256 quantises to make ties likely."""
    rng = np.random.default_rng(seed)
    v = rng.integers(0, levels, size=(H, W, 3))
    if levels < 256:
        v = v * (255 // max(1, levels - 1))
    return v.astype(np.uint8)


# The workloads the tests and the bench use, by what they are.
WORKLOADS = {
    # BSD500-sized single image, single level, blocks 16 -> 1 px.
    "he321x481_k200": dict(H=321, W=481, n_cells=40, seed=1,
                           params=dict(num_levels=1, ratio_C=4, init_block=16, final_grain=1,
                                       K=200, size_mode=2, predict=0, reuse=1)),
    # One 4096^2 tile, 3-level box pyramid x16/x4/x1, 4096 superpixels, init block 32 px.
    "he4096_k4096_l3": dict(H=4096, W=4096, n_cells=2000, seed=2,
                            params=dict(num_levels=3, ratio_C=4, init_block=32, final_grain=1,
                                        K=4096, size_mode=2, predict=1, reuse=1)),
}
# The same images refined with the frontier schedule (schedule 1: the boundary queue of
# Sec. 2.1 as one flag per block, popped by the phases and refilled around every move).
for _name in list(WORKLOADS):
    WORKLOADS[_name + "_frontier"] = dict(WORKLOADS[_name], params=dict(WORKLOADS[_name]["params"], schedule=1))


# Batches of uneven tiles (the adaptive data partitioning of whole slides, Sec. 3.3): tile
# sizes, one generator call per tile with cell count and superpixel count proportional to
# its area.
BATCHES = {
    # 64 tiles, long side from {512, 1024, 2048, 3072, 4096}, aspect U[1, 2] with the short
    # side rounded down to a multiple of 32, 1 Voronoi cell per 8192 px and 1 superpixel per
    # 4096 px; the 4096^2 tile's 3-level schedule.
    "batch64_l3": dict(n=64, seed=3, px_per_cell=8192, px_per_superpixel=4096,
                       params=dict(num_levels=3, ratio_C=4, init_block=32, final_grain=1,
                                   size_mode=2, predict=1, reuse=1)),
}


# Whole slides (scaled-down stand-ins for 100000 x 80000 NLST slides): size, seed, the
# tile limit of the partition, superpixel density and the 3-level schedule.
SLIDES = {
    "slide16k_l3": dict(H=16384, W=12288, seed=5, max_tile=8192, px_per_superpixel=4096,
                        params=dict(num_levels=3, ratio_C=4, init_block=32, final_grain=1, size_mode=2,
                                    predict=1, reuse=1)),
}
# The same batch and slide refined with the queue schedule.
for _d in (BATCHES, SLIDES):
    for _name in list(_d):
        _d[_name + "_frontier"] = dict(_d[_name], params=dict(_d[_name]["params"], schedule=1))


def batch_sizes(n: int, seed: int):
    """(H, W) of each tile of a batch, from the seed alone."""
    rng = np.random.default_rng(seed)
    sizes = []
    for _ in range(n):
        long_side = int(rng.choice(np.array([512, 1024, 2048, 3072, 4096])))
        aspect = 1.0 + float(rng.integers(0, 1 << 20)) / float(1 << 20)  # U[1, 2)
        short_side = max(32, int(long_side / aspect) // 32 * 32)
        if rng.integers(0, 2):
            sizes.append((short_side, long_side))
        else:
            sizes.append((long_side, short_side))
    return sizes


def batch_tile(name: str, i: int):
    """Tile i of a batch workload: its RGB array and superpixel count K."""
    b = BATCHES[name]
    H, W = batch_sizes(b["n"], b["seed"])[i]
    cells = max(1, (H * W) // b["px_per_cell"])
    return he_image(H, W, cells, b["seed"] * 1000 + i).rgb, max(1, (H * W) // b["px_per_superpixel"])


def batch_workload(name: str, count: int | None = None):
    """The tiles of a batch workload (the first ``count`` when given): RGB arrays and the
    superpixel count K of each."""
    n = BATCHES[name]["n"] if count is None else min(count, BATCHES[name]["n"])
    tiles = [batch_tile(name, i) for i in range(n)]
    return [t[0] for t in tiles], [t[1] for t in tiles]


def workload_image(name: str) -> SynthImage:
    w = WORKLOADS[name]
    return he_image(w["H"], w["W"], w["n_cells"], w["seed"])
