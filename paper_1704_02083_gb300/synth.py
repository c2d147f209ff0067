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
    # The whole-slide workload at its full size: 100000 x 80000 (24 GB of RGB), made on the
    # device by the counter-based generator (slide_gen restates it on the host), 40% white,
    # folds over about 5%, one Voronoi cell per 8192 px, one superpixel per 16384 px (about
    # 488k), tiles of at most 8192^2 (Eq. parallel_spit on both axes: 13 x 10 tiles); the
    # oracle's records cover the sampled tiles.
    "slide100k_l3": dict(H=100000, W=80000, seed=5, max_tile=8192, px_per_superpixel=16384, generator="counter",
                         px_per_cell=8192, white_frac=0.40, fold_frac=0.05, sample_tiles=(0, 65, 129),
                         geometry="152,152,152,152,152,152:4,4,4,4,4,4",
                         params=dict(num_levels=3, ratio_C=4, init_block=32, final_grain=1, size_mode=2,
                                     predict=1, reuse=1)),
}


def slide_tiles(H: int, W: int, max_tile: int, px_per_superpixel: int):
    """The tiles of a slide as rapid_refine_slide cuts it: even row and column bands of at
    most max_tile px (Eq. parallel_spit on both axes), row-major; per tile (row0, col0,
    height, width, K)."""
    nr, nc = -(-H // max_tile), -(-W // max_tile)
    out = []
    for t in range(nr * nc):
        i, j = divmod(t, nc)
        r0, r1, c0, c1 = H * i // nr, H * (i + 1) // nr, W * j // nc, W * (j + 1) // nc
        out.append((r0, c0, r1 - r0, c1 - c0, max(1, (r1 - r0) * (c1 - c0) // px_per_superpixel)))
    return out
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


# ---------------------------------------------------------------- counter-based slide generator
# The whole-slide stand-in at full size (100000 x 80000, 24 GB of RGB) is generated on the
# device (rapid_synth_slide) from the definition below, which this host function restates
# pixel for pixel, so that both give the same bytes: every random quantity is a hash of
# (seed, stream, index), never a stream position, and every geometric test is exact
# integer arithmetic.  Any window of the slide can therefore be generated alone.
#
# hash: h(seed, s, i) = mix(mix(mix(seed) ^ s) ^ i) on unsigned 64-bit words, where mix is
# the SplitMix64 output function (z += 0x9E3779B97F4A7C15; z = (z ^ z >> 30) *
# 0xBF58476D1CE4E5B9; z = (z ^ z >> 27) * 0x94D049BB133111EB; z ^ z >> 31).
#
# * Buckets: B x B pixels (B = 128), bucket (bx, by) spans [B bx, min(B bx + B, W)) x ...
#   (edge buckets are clipped); bucket index q = by * nbx + bx.
# * Voronoi cells: kc = max(1, round(B^2 / px_per_cell)) seeds per bucket; seed id
#   = q kc + j at (B bx + h(seed, 1, id) % bw_q, B by + h(seed, 2, id) % bh_q) (bw_q, bh_q the
#   clipped bucket size).  A pixel belongs to the seed of least squared distance (ties: the
#   smaller id); since every bucket holds a seed, the nearest lies within 2 buckets.
# * Cell classes: u = h(seed, 3, id) % 10000: white below round(10000 white_frac), purple
#   below that plus round(10000 (1 - white_frac) 0.4375), else pink; mean = base colour +
#   h(seed, 4 + c, id) % 31 - 15 per channel c (white: % 11 - 5).
# * Nuclei: kn = round(B^2 nucleus_density) per bucket, id = q kn + j, centre (B bx +
#   h(seed, 10, id) % bw_q, B by + h(seed, 11, id) % bh_q), radius 3 + h(seed, 12, id) % 6,
#   colour NUCLEUS + h(seed, 13 + c, id) % 21 - 10; kept when the centre's cell is not white.
#   A pixel within the radius (squared distance <= r^2) of kept nuclei takes the largest id.
# * Folds: nf = max(1, round(fold_frac H W / (50 * 0.65 * min(H, W)))) bands; band b: width
#   20 + h(seed, 30, b) % 61, direction (ax, ay) = (h(seed, 31, b) % 2049 - 1024, h(seed, 32,
#   b) % 2049 - 1024) ((1, 0) when both are 0), centre (h(seed, 33, b) % W, h(seed, 34, b) %
#   H), length min(H, W) (300 + h(seed, 35, b) % 701) // 1000, colour FOLD + h(seed, 36 + c,
#   b) % 21 - 10.  With d = p - centre and n2 = ax^2 + ay^2, a pixel is in the band when
#   4 (ax dx + ay dy)^2 <= length^2 n2 and 4 (ay dx - ax dy)^2 <= width^2 n2; the largest b
#   wins, over nuclei and cells.
# * Noise: channel c of pixel (x, y) adds -30 + #{t in the discrete Gaussian table, t <= u},
#   u = h(seed, 20, 3 (y W + x) + c) >> 32; the sum is clamped to [0, 255].
# * Ground truth: cell id, then n_cells + nucleus id, then n_cells + n_nuclei + band id; ROI =
#   purple cells and nuclei (folds are not ROI).
GEN_BUCKET = 128
_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _mix(z):
    z = (z + np.uint64(0x9E3779B97F4A7C15)) & _M64
    z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
    z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
    return z ^ (z >> np.uint64(31))


def gen_hash(seed: int, stream: int, idx):
    """h(seed, stream, idx) of the counter-based generator (idx: int or integer array)."""
    with np.errstate(over="ignore"):
        k = _mix(_mix(np.uint64(seed)) ^ np.uint64(stream))
        return _mix(k ^ np.asarray(idx, dtype=np.uint64))


def gen_layout(H: int, W: int, px_per_cell: int = 8192, nucleus_density: float = 1.0 / 400.0,
               fold_frac: float = 0.05):
    """Bucket grid and counts of the counter-based slide generator."""
    B = GEN_BUCKET
    nbx, nby = -(-W // B), -(-H // B)
    kc = max(1, int(round(B * B / px_per_cell)))
    kn = int(round(B * B * nucleus_density))
    nf = max(1, int(round(fold_frac * H * W / (50.0 * 0.65 * min(H, W)))))
    return dict(B=B, nbx=nbx, nby=nby, kc=kc, kn=kn, nf=nf, n_cells=nbx * nby * kc, n_nuclei=nbx * nby * kn)


def _bucket_dims(q, nbx, H, W, B):
    bx, by = q % nbx, q // nbx
    return bx, by, np.minimum(B, W - B * bx), np.minimum(B, H - B * by)


def _cell_pos(seed, ids, kc, nbx, H, W, B):
    """Seed positions of the cells with the given ids."""
    q = ids // kc
    bx, by, bw, bh = _bucket_dims(q, nbx, H, W, B)
    x = B * bx + (gen_hash(seed, 1, ids) % bw.astype(np.uint64)).astype(np.int64)
    y = B * by + (gen_hash(seed, 2, ids) % bh.astype(np.uint64)).astype(np.int64)
    return x, y


def _cells(seed, ids, kc, nbx, H, W, B, white_frac):
    """Position, class and mean colour of the cells with the given ids."""
    x, y = _cell_pos(seed, ids, kc, nbx, H, W, B)
    u = (gen_hash(seed, 3, ids) % np.uint64(10000)).astype(np.int64)
    n_white = int(round(white_frac * 10000))
    n_purple = int(round((1.0 - white_frac) * 0.4375 * 10000))
    cls = np.where(u < n_white, 2, np.where(u < n_white + n_purple, 1, 0))
    base = np.array([PINK, PURPLE, WHITE], np.int64)[cls]
    jit = np.stack([(gen_hash(seed, 4 + c, ids) % np.uint64(31)).astype(np.int64) - 15 for c in range(3)], -1)
    jit_w = np.stack([(gen_hash(seed, 4 + c, ids) % np.uint64(11)).astype(np.int64) - 5 for c in range(3)], -1)
    mean = base + np.where((cls == 2)[..., None], jit_w, jit)
    return x, y, cls, mean


def slide_gen(H: int, W: int, seed: int, x0: int = 0, y0: int = 0, h: int | None = None, w: int | None = None,
              px_per_cell: int = 8192, white_frac: float = 0.40, fold_frac: float = 0.05,
              nucleus_density: float = 1.0 / 400.0) -> SynthImage:
    """The window [x0, x0 + w) x [y0, y0 + h) of the counter-based slide (see above)."""
    h = H - y0 if h is None else h
    w = W - x0 if w is None else w
    if not (0 <= x0 and 0 <= y0 and w > 0 and h > 0 and x0 + w <= W and y0 + h <= H):
        raise ValueError("window outside the slide")
    lay = gen_layout(H, W, px_per_cell, nucleus_density, fold_frac)
    B, nbx, nby, kc, kn, nf = lay["B"], lay["nbx"], lay["nby"], lay["kc"], lay["kn"], lay["nf"]
    n_cells, n_nuc = lay["n_cells"], lay["n_nuclei"]
    ys = np.arange(y0, y0 + h, dtype=np.int64)
    xs = np.arange(x0, x0 + w, dtype=np.int64)
    # Voronoi: candidate seeds of the buckets within 2 of each pixel's bucket (seed
    # positions computed once per bucket of the window's neighbourhood)
    cell = np.empty((h, w), np.int64)
    gx0, gx1 = max(0, x0 // B - 2), min(nbx - 1, (x0 + w - 1) // B + 2)
    gy0, gy1 = max(0, y0 // B - 2), min(nby - 1, (y0 + h - 1) // B + 2)
    gq = (np.arange(gy0, gy1 + 1)[:, None] * nbx + np.arange(gx0, gx1 + 1)[None, :]).astype(np.int64)
    spos = [_cell_pos(seed, gq * kc + j, kc, nbx, H, W, B) for j in range(kc)]
    band = max(1, (1 << 20) // w)
    for r0 in range(0, h, band):
        yy = ys[r0:r0 + band][:, None]
        xx = xs[None, :]
        best_d = np.full((yy.shape[0], w), np.iinfo(np.int64).max, np.int64)
        best_id = np.full((yy.shape[0], w), -1, np.int64)
        pbx, pby = xx // B, yy // B
        for dby in range(-2, 3):
            for dbx in range(-2, 3):
                qbx, qby = pbx + dbx, pby + dby
                ok = (qbx >= 0) & (qbx < nbx) & (qby >= 0) & (qby < nby)
                lx = np.clip(qbx - gx0, 0, gx1 - gx0)
                ly = np.clip(qby - gy0, 0, gy1 - gy0)
                q = np.where(ok, qby * nbx + qbx, 0)
                for j in range(kc):
                    ids = q * kc + j
                    sx, sy = spos[j][0][ly, lx], spos[j][1][ly, lx]
                    d = (sx - xx) ** 2 + (sy - yy) ** 2
                    better = ok & ((d < best_d) | ((d == best_d) & (ids < best_id)))
                    best_d = np.where(better, d, best_d)
                    best_id = np.where(better, ids, best_id)
        cell[r0:r0 + band] = best_id
    _, _, ccls, cmean = _cells(seed, cell, kc, nbx, H, W, B, white_frac)
    colour = cmean.copy()
    regions = cell.copy()
    roi = ccls == 1
    # nuclei whose disc can reach the window, painted in ascending id order
    qx0, qx1 = max(0, (x0 - 8) // B), min(nbx - 1, (x0 + w - 1 + 8) // B)
    qy0, qy1 = max(0, (y0 - 8) // B), min(nby - 1, (y0 + h - 1 + 8) // B)
    qs = np.array([qy * nbx + qx for qy in range(qy0, qy1 + 1) for qx in range(qx0, qx1 + 1)], np.int64)
    nid = (qs[:, None] * kn + np.arange(kn, dtype=np.int64)[None, :]).ravel()
    nid.sort()
    if nid.size:
        q = nid // kn
        bx, by, bw, bh = _bucket_dims(q, nbx, H, W, B)
        cx = B * bx + (gen_hash(seed, 10, nid) % bw.astype(np.uint64)).astype(np.int64)
        cy = B * by + (gen_hash(seed, 11, nid) % bh.astype(np.uint64)).astype(np.int64)
        rad = 3 + (gen_hash(seed, 12, nid) % np.uint64(6)).astype(np.int64)
        ncol = np.array(NUCLEUS, np.int64)[None, :] + np.stack(
            [(gen_hash(seed, 13 + c, nid) % np.uint64(21)).astype(np.int64) - 10 for c in range(3)], -1)
        # the centre's cell (its own Voronoi search, as for any pixel)
        centre = slide_cells_at(H, W, seed, cx, cy, px_per_cell, white_frac)
        _, _, ncls, _ = _cells(seed, centre, kc, nbx, H, W, B, white_frac)
        for t in np.nonzero(ncls != 2)[0]:
            r = int(rad[t])
            ya, yb = max(y0, int(cy[t]) - r), min(y0 + h, int(cy[t]) + r + 1)
            xa, xb = max(x0, int(cx[t]) - r), min(x0 + w, int(cx[t]) + r + 1)
            if ya >= yb or xa >= xb:
                continue
            gy, gx = np.mgrid[ya:yb, xa:xb]
            inside = (gx - cx[t]) ** 2 + (gy - cy[t]) ** 2 <= r * r
            sy, sx = gy[inside] - y0, gx[inside] - x0
            colour[sy, sx] = ncol[t]
            regions[sy, sx] = n_cells + nid[t]
            roi[sy, sx] = True
    # folds, painted in ascending band order
    for b in range(nf):
        fw = 20 + int(gen_hash(seed, 30, b) % np.uint64(61))
        ax = int(gen_hash(seed, 31, b) % np.uint64(2049)) - 1024
        ay = int(gen_hash(seed, 32, b) % np.uint64(2049)) - 1024
        if ax == 0 and ay == 0:
            ax = 1
        fcx, fcy = int(gen_hash(seed, 33, b) % np.uint64(W)), int(gen_hash(seed, 34, b) % np.uint64(H))
        flen = min(H, W) * (300 + int(gen_hash(seed, 35, b) % np.uint64(701))) // 1000
        fcol = np.array(FOLD, np.int64) + np.array(
            [int(gen_hash(seed, 36 + c, b) % np.uint64(21)) - 10 for c in range(3)], np.int64)
        ext = (flen + fw) // 2 + 2  # the band lies within this distance of its centre
        ya, yb = max(y0, fcy - ext), min(y0 + h, fcy + ext + 1)
        xa, xb = max(x0, fcx - ext), min(x0 + w, fcx + ext + 1)
        if ya >= yb or xa >= xb:
            continue
        n2 = ax * ax + ay * ay
        for r0 in range(ya, yb, 256):
            gy, gx = np.mgrid[r0:min(yb, r0 + 256), xa:xb]
            dx, dy = gx.astype(np.int64) - fcx, gy.astype(np.int64) - fcy
            along, across = ax * dx + ay * dy, ay * dx - ax * dy
            inside = (4 * along * along <= flen * flen * n2) & (4 * across * across <= fw * fw * n2)
            sy, sx = gy[inside] - y0, gx[inside] - x0
            colour[sy, sx] = fcol
            regions[sy, sx] = n_cells + n_nuc + b
            roi[sy, sx] = False
    # noise
    pix = (ys[:, None] * W + xs[None, :])[..., None] * 3 + np.arange(3, dtype=np.int64)[None, None, :]
    u = (gen_hash(seed, 20, pix) >> np.uint64(32)).astype(np.uint32)
    noise = np.searchsorted(_NOISE_CDF, u, side="right").astype(np.int64) + _NOISE_LO
    rgb = np.clip(colour + noise, 0, 255).astype(np.uint8)
    return SynthImage(rgb=np.ascontiguousarray(rgb), regions=regions.astype(np.int64), roi=roi,
                      n_regions=int(n_cells + n_nuc + nf))


def slide_cells_at(H, W, seed, px, py, px_per_cell=8192, white_frac=0.40):
    """Voronoi cell id of pixels (px, py) (integer arrays) of the counter-based slide."""
    lay = gen_layout(H, W, px_per_cell)
    B, nbx, nby, kc = lay["B"], lay["nbx"], lay["nby"], lay["kc"]
    px, py = np.asarray(px, np.int64), np.asarray(py, np.int64)
    best_d = np.full(px.shape, np.iinfo(np.int64).max, np.int64)
    best_id = np.full(px.shape, -1, np.int64)
    for dby in range(-2, 3):
        for dbx in range(-2, 3):
            qbx, qby = px // B + dbx, py // B + dby
            ok = (qbx >= 0) & (qbx < nbx) & (qby >= 0) & (qby < nby)
            q = np.where(ok, qby * nbx + qbx, 0)
            for j in range(kc):
                ids = q * kc + j
                sx, sy = _cell_pos(seed, ids, kc, nbx, H, W, B)
                d = (sx - px) ** 2 + (sy - py) ** 2
                better = ok & ((d < best_d) | ((d == best_d) & (ids < best_id)))
                best_d = np.where(better, d, best_d)
                best_id = np.where(better, ids, best_id)
    return best_id
