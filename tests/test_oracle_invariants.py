"""Invariants of the oracle, checked after every phase / sweep with independent numpy code:
the statistics equal their recomputation from the label map (int64, exact); every live
superpixel is one 4-connected component (E_topo, Eq. equa:energy1); with no merging the
energy of Eq. equa:energy1 never rises (Eq. operation only takes lower-energy labels)."""
import numpy as np
import pytest

import helpers
import oracle
from paper_1704_02083_gb300 import synth


def _image():
    return synth.he_image(72, 100, n_cells=8, seed=11).rgb


def _walk(o, rgb, check_energy, max_sweeps=20):
    """Run every stage phase by phase; yields after each phase."""
    H, W = rgb.shape[:2]
    o.seed()
    nst = o.num_stages()
    for st in range(nst):
        if st > 0:
            o.next_stage()
        for sw in range(max_sweeps):
            changes = 0
            for ph in range(9):
                g = o.grid()
                before = helpers.upsample(o.block_labels(), g["side"], H, W)
                mv, mg = o.phase(ph)
                changes += mv + mg
                yield st, sw, ph, before, mv, mg
            if changes == 0:
                break


@pytest.mark.parametrize("size_mode", [0, 1, 2])
def test_stats_and_connectivity(size_mode):
    rgb = _image()
    H, W = rgb.shape[:2]
    o = oracle.Oracle(rgb, K=24, init_block=16, size_mode=size_mode)
    n_phases = 0
    for st, sw, ph, before, mv, mg in _walk(o, rgb, False):
        g = o.grid()
        lab = helpers.upsample(o.block_labels(), g["side"], H, W)
        s, _, _ = o.stats()
        ref = helpers.stats_from_labels(rgb, lab, g["M"])
        np.testing.assert_array_equal(s[:, :6], ref)
        live = np.unique(lab)
        assert (s[live, 0] > 0).all()
        dead = np.setdiff1d(np.arange(g["M"]), live)
        assert (s[dead, :6] == 0).all()
        if size_mode != 2:
            assert mg == 0 and len(live) == g["M"]
        if ph == 8:
            assert helpers.count_components_per_label(lab) == len(live)
        n_phases += 1
    assert n_phases > 50


@pytest.mark.parametrize("size_mode", [0, 1])
def test_energy_never_rises(size_mode):
    rgb = _image()
    H, W = rgb.shape[:2]
    o = oracle.Oracle(rgb, K=24, init_block=16, size_mode=size_mode)
    lam_pos, lam_b = None, o.p.lambda_b
    prev = None
    rises = 0
    for st, sw, ph, before, mv, mg in _walk(o, rgb, True, max_sweeps=6):
        if lam_pos is None:
            lam_pos = o.lambda_pos()
        g = o.grid()
        lab = helpers.upsample(o.block_labels(), g["side"], H, W)
        e_before = helpers.total_energy(rgb, before, lam_pos, lam_b)
        e_after = helpers.total_energy(rgb, lab, lam_pos, lam_b) if mv else e_before
        # decisions are taken in double precision: allow rounding-level slack only
        assert e_after <= e_before + abs(e_before) * 1e-12, (st, sw, ph, float(e_after - e_before))
        if mv:
            assert e_after < e_before or e_after <= e_before + abs(e_before) * 1e-12
        prev = e_after
    assert prev is not None


@pytest.mark.parametrize("size_mode,K,seed", [(1, 24, 11), (2, 24, 11), (2, 60, 4), (2, 100, 3)])
def test_size_rule_against_phase_start_counts(size_mode, K, seed):
    """Sec. 3.1, judged against the counts at the start of the phase (the snapshot every
    block of the phase decides against): no executed move takes its superpixel below
    l * InitSize (case 2, lambda_s infinite, and the merge mode alike), and every merge
    request comes from a block whose removal would (the merge mode).  Blocks of one label
    that move in the same phase must not see each other's moves."""
    rgb = synth.he_image(72, 100, n_cells=8, seed=seed).rgb
    H, W = rgb.shape[:2]
    o = oracle.Oracle(rgb, K=K, init_block=16, size_mode=size_mode)
    o.seed()
    checked = 0
    for st in range(o.num_stages()):
        if st > 0:
            o.next_stage()
        for sw in range(6):
            for ph in range(9):
                side = o.grid()["side"]
                bl0 = o.block_labels()
                s0, _, _ = o.stats()

                def w(by, bx):
                    return (min(side * (bx + 1), W) - side * bx) * (min(side * (by + 1), H) - side * by)

                o.phase_moves(ph)
                bl1 = o.block_labels()
                for by, bx in np.argwhere(bl0 != bl1):
                    a = bl0[by, bx]
                    assert 4 * (s0[a, 0] - w(by, bx)) >= s0[a, 6]
                    checked += 1
                blk, lab = o.pending_requests()
                nbx = bl0.shape[1]
                for b, a in zip(blk.tolist(), lab.tolist()):
                    by, bx = divmod(b, nbx)
                    assert bl0[by, bx] == a and 4 * (s0[a, 0] - w(by, bx)) < s0[a, 6]
                    checked += 1
                if size_mode == 1:
                    assert len(blk) == 0
                o.phase_merges()
    assert checked > 100


def test_counters_consistent():
    rgb = _image()
    o = oracle.Oracle(rgb, K=24, init_block=16, size_mode=2).run()
    c = o.counters()
    assert (c[:, oracle.COUNTER_NAMES.index("evaluated")] <= c[:, oracle.COUNTER_NAMES.index("eligible")]).all()
    assert (c[:, 7] <= c[:, 6]).all()                # merges <= requests
    assert (c[:, 2] >= 1).all() and (c[:, 2] <= 64).all()
    assert [tuple(r[:2]) for r in c] == [(1, 16), (1, 8), (1, 4), (1, 2), (1, 1)]
