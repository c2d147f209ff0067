"""Brute force on tiny images: every decision of a phase re-derived from the per-pixel
energy of Eq. equa:energy1, in exact rational arithmetic, with the phase's snapshot means.

For block p with label a and each label k of its 4-neighbours, the whole-map energy
E = sum_p |I(p) - c_{s_p}|^2 + lambda_pos |p - mu_{s_p}|^2 + lambda_b sum_p sum_{q in N4(p)} [s_p != s_q]
is evaluated with p relabelled k and compared with p kept (Eq. operation).  Topology uses
the classical simple-point definition (plus the interior case), independent of the oracle's
table.  Ties and near-ties of the double-precision arithmetic are skipped."""
from fractions import Fraction

import numpy as np
import pytest
import scipy.ndimage as ndi

import helpers
import oracle
from paper_1704_02083_gb300 import synth

RING = [(-1, -1), (0, -1), (1, -1), (1, 0), (1, 1), (0, 1), (-1, 1), (-1, 0)]


def simple_classical(blab, bx, by):
    a = blab[by, bx]
    H, W = blab.shape
    g = np.zeros((3, 3), bool)
    for dx, dy in RING:
        x, y = bx + dx, by + dy
        if 0 <= x < W and 0 <= y < H and blab[y, x] == a:
            g[1 + dy, 1 + dx] = True
    if g.sum() == 8:
        return True
    lab, _ = ndi.label(g, ndi.generate_binary_structure(2, 1))
    t4 = len({lab[r, c] for (r, c) in ((0, 1), (1, 2), (2, 1), (1, 0)) if lab[r, c] > 0})
    bg = ~g
    bg[1, 1] = False
    _, t8 = ndi.label(bg, ndi.generate_binary_structure(2, 2))
    return t4 == 1 and t8 == 1


def pixel_energy(rgb, lab, means, lam_pos, lam_b):
    H, W = lab.shape
    E = Fraction(0)
    for y in range(H):
        for x in range(W):
            k = lab[y, x]
            c, mx, my = means[k]
            E += sum((Fraction(int(rgb[y, x, ch])) - c[ch]) ** 2 for ch in range(3))
            E += lam_pos * ((Fraction(x) - mx) ** 2 + (Fraction(y) - my) ** 2)
    E += 2 * lam_b * helpers.unequal_pairs(lab)
    return E


@pytest.mark.parametrize("seed", range(6))
def test_phase_decisions_match_exact_energy(seed):
    H, W = 7, 9
    rgb = synth.random_image(H, W, seed, levels=4)
    o = oracle.Oracle(rgb, K=6, init_block=2, size_mode=0, lambda_pos0=400.0, lambda_b=50.0)
    o.seed()
    lam_pos = Fraction(o.lambda_pos())
    lam_b = Fraction(50.0)
    checked = skipped = 0
    for st in range(o.num_stages()):
        if st > 0:
            o.next_stage()
        for sw in range(3):
            for ph in range(9):
                g = o.grid()
                side = g["side"]
                bl = o.block_labels()
                s, _, _ = o.stats()
                # snapshot means exactly as doubles (Fractions of the rounded values)
                means = {}
                for k in range(g["M"]):
                    if s[k, 0] > 0:
                        n = float(s[k, 0])
                        means[k] = ([Fraction(float(s[k, 1 + ch]) / n) for ch in range(3)],
                                    Fraction(float(s[k, 4]) / n), Fraction(float(s[k, 5]) / n))
                lab = helpers.upsample(bl, side, H, W)
                E0 = pixel_energy(rgb, lab, means, lam_pos, lam_b)
                expect = bl.copy()
                py, px = divmod(ph, 3)
                nby, nbx = bl.shape
                for by in range(py, nby, 3):
                    for bx in range(px, nbx, 3):
                        a = bl[by, bx]
                        nbrs = [bl[y, x] for x, y in ((bx, by - 1), (bx - 1, by), (bx + 1, by), (bx, by + 1))
                                if 0 <= x < nbx and 0 <= y < nby]
                        if all(k == a for k in nbrs):
                            continue
                        if not simple_classical(bl, bx, by):
                            continue
                        dEs = {}
                        for k in sorted(set(nbrs) - {a}):
                            t = bl.copy()
                            t[by, bx] = k
                            dEs[k] = pixel_energy(rgb, helpers.upsample(t, side, H, W), means, lam_pos, lam_b) - E0
                        best = min(dEs.values())
                        ties = sorted(dEs.values())
                        near = abs(best) < abs(E0) * Fraction(1, 10**9) or (
                            len(ties) > 1 and ties[1] - ties[0] < abs(E0) * Fraction(1, 10**9))
                        if near:
                            skipped += 1
                            expect[by, bx] = -1
                            continue
                        if best < 0:
                            expect[by, bx] = min(k for k, v in dEs.items() if v == best)
                        checked += 1
                o.phase(ph)
                got = o.block_labels()
                m = expect >= 0
                np.testing.assert_array_equal(got[m], expect[m], err_msg=f"stage {st} sweep {sw} phase {ph}")
    assert checked > 20
