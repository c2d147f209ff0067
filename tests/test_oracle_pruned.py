"""Pins of the oracle's pruned sweeps (the mode the learned block scorer drives): a stage
with a keep mask tests and decides only the kept eligible blocks until a sweep changes
nothing, then falls back to full sweeps until a full sweep changes nothing, within
max_sweeps.  The mask only prunes which eligible blocks get the exact tests (the pruning
idea of Sec. 3.2, boundary superpixels only, taken to a per-block mask); it never decides a
move.

Pinned against what the definition fixes, not against the oracle itself:
* a mask that keeps every block sweeps exactly as the plain run, plus one full sweep after
  the pruned sweeps converge (the same labels, S, moves and merges);
* a mask that keeps no block makes one sweep that tests nothing (its eligible blocks are
  counted, none evaluated), after which the run is the plain run;
* with a random mask, every decision of a phase is re-derived from the per-pixel energy in
  exact rationals: the kept blocks decide as in the plain method, the others stay put;
* a stage that converged under the mask is followed by full sweeps (the fallback) that
  find the moves the mask hid."""
import numpy as np
import pytest

import helpers
import oracle
import test_oracle_bruteforce as bf
from paper_1704_02083_gb300 import synth

C_SWEEPS, C_ELIG, C_EVAL, C_MOVES, C_REQ, C_MERGES = 2, 3, 4, 5, 6, 7


def _grids(o):
    """Block-grid shapes (nby, nbx) of every stage."""
    H, W = o.H, o.W
    return [(-(-H // side), -(-W // side)) for _, side in o.stages()]


def _run(rgb, masks=None, **p):
    o = oracle.Oracle(rgb, **p)
    if masks is not None:
        for i, m in enumerate(masks):
            if m is not None:
                o.set_keep_mask(i, m)
    o.run()
    s, y, imp = o.stats()
    return o.labels(), s, o.counters(), (y, imp)


def _eligible_count(bl, imp_on, imp, y, rule):
    """Eligible blocks of a block-label map (Eq. bound; with prediction on also the
    boundary-superpixel rule, or the pair rule of Eq. new_bound): the count one sweep that
    moves nothing sees."""
    H, W = bl.shape
    pad = np.pad(bl, 1, constant_values=-1)
    nb = [pad[:-2, 1:-1], pad[1:-1, :-2], pad[1:-1, 2:], pad[2:, 1:-1]]
    bnd = np.zeros(bl.shape, bool)
    for n in nb:
        bnd |= (n >= 0) & (n != bl)
    if not imp_on:
        return int(bnd.sum())
    if rule == 0:
        return int((bnd & (imp[bl] != 0)).sum())
    pair = np.zeros(bl.shape, bool)
    for n in nb:
        pair |= (n >= 0) & (n != bl) & (y[np.maximum(n, 0)] != y[bl])
    return int((bnd & pair).sum())


CASES = [
    dict(H=40, W=56, levels=6, seed=1, p=dict(K=12, init_block=8, size_mode=2, max_sweeps=40)),
    dict(H=33, W=47, levels=4, seed=2, p=dict(K=9, init_block=4, size_mode=1, max_sweeps=40)),
    dict(H=48, W=48, levels=8, seed=3, p=dict(num_levels=2, ratio_C=2, init_block=8, K=16, size_mode=2,
                                              predict=1, max_sweeps=40)),
    dict(H=50, W=37, levels=5, seed=4, p=dict(num_levels=2, ratio_C=2, init_block=8, K=10, size_mode=0,
                                              predict=1, importance_rule=1, max_sweeps=40)),
]


def _case(c):
    rgb = synth.random_image(c["H"], c["W"], c["seed"], levels=c["levels"])
    return rgb, c["p"]


@pytest.mark.parametrize("c", CASES, ids=[f"case{i}" for i in range(len(CASES))])
def test_keep_everything_is_the_plain_run_plus_one_full_sweep(c):
    rgb, p = _case(c)
    lab, s, cnt, _ = _run(rgb, **p)
    o = oracle.Oracle(rgb, **p)
    ones = [np.ones(g, np.uint8) for g in _grids(o)]
    lab1, s1, cnt1, _ = _run(rgb, ones, **p)
    np.testing.assert_array_equal(lab1, lab)
    np.testing.assert_array_equal(s1, s)
    np.testing.assert_array_equal(cnt1[:, [C_MOVES, C_REQ, C_MERGES]], cnt[:, [C_MOVES, C_REQ, C_MERGES]])
    for st in range(cnt.shape[0]):
        if cnt[st, C_SWEEPS] < p["max_sweeps"]:  # the plain stage converged: one more sweep, which repeats it
            assert cnt1[st, C_SWEEPS] == cnt[st, C_SWEEPS] + 1
            assert cnt1[st, C_ELIG] > cnt[st, C_ELIG] or cnt[st, C_ELIG] == 0
        else:
            assert cnt1[st, C_SWEEPS] == cnt[st, C_SWEEPS]


@pytest.mark.parametrize("c", CASES, ids=[f"case{i}" for i in range(len(CASES))])
def test_keep_nothing_is_one_idle_sweep_then_the_plain_run(c):
    rgb, p = _case(c)
    o = oracle.Oracle(rgb, **p)
    zeros = [np.zeros(g, np.uint8) for g in _grids(o)]
    # the plain run, stage by stage, with the eligible blocks of each stage's starting map
    o.seed()
    start_elig = []
    for st in range(o.num_stages()):
        if st > 0:
            o.next_stage()
        s, y, imp = o.stats()
        imp_on = p.get("predict", 0) and o.stages()[st][0] >= 2
        start_elig.append(_eligible_count(o.block_labels(), imp_on, imp, y, p.get("importance_rule", 0)))
        o.refine_stage()
    lab, s, cnt = o.labels(), o.stats()[0], o.counters()
    lab0, s0, cnt0, _ = _run(rgb, zeros, **p)
    np.testing.assert_array_equal(lab0, lab)
    np.testing.assert_array_equal(s0, s)
    assert (cnt[:, C_SWEEPS] < p["max_sweeps"]).all()
    np.testing.assert_array_equal(cnt0[:, C_SWEEPS], cnt[:, C_SWEEPS] + 1)
    np.testing.assert_array_equal(cnt0[:, C_EVAL], cnt[:, C_EVAL])
    np.testing.assert_array_equal(cnt0[:, C_ELIG], cnt[:, C_ELIG] + np.array(start_elig))
    np.testing.assert_array_equal(cnt0[:, [C_MOVES, C_REQ, C_MERGES]], cnt[:, [C_MOVES, C_REQ, C_MERGES]])


RCASES = [(7, 9, 6, 2, 50.0, s, m, 4) for s in range(3) for m in (0, 1, 2)] + \
         [(11, 13, 4, 4, 2000.0, s, 2, 4) for s in range(2)] + [(12, 12, 9, 4, 10.0, 9, 1, 4)]


@pytest.mark.parametrize("H,W,K,ib,lamb,seed,size_mode,levels", RCASES)
def test_pruned_phase_decisions_match_exact_energy(H, W, K, ib, lamb, seed, size_mode, levels):
    """Every phase of the first two pruned sweeps of every stage, re-derived in rationals
    (test_oracle_bruteforce's per-pixel energy), with the blocks the random mask leaves out
    kept as they are and never requesting a merge."""
    from fractions import Fraction
    rgb = synth.random_image(H, W, seed, levels=levels)
    o = oracle.Oracle(rgb, K=K, init_block=ib, size_mode=size_mode, lambda_pos0=400.0, lambda_b=lamb)
    rng = np.random.default_rng(1000 + seed)
    masks = [(rng.random(g) < 0.5).astype(np.uint8) for g in _grids(o)]
    for i, m in enumerate(masks):
        o.set_keep_mask(i, m)
    o.seed()
    lam_pos, lam_b = Fraction(o.lambda_pos()), Fraction(lamb)
    checked = masked_movers = 0
    for st in range(o.num_stages()):
        if st > 0:
            o.next_stage()
        for sw in range(2):
            for ph in range(9):
                g = o.grid()
                bl = o.block_labels()
                s, _, _ = o.stats()
                expect, requests, decidable = bf._rederive(rgb, bl, s, g["side"], ph, lam_pos, lam_b, size_mode)
                keep = masks[st].astype(bool)
                masked_movers += int(((expect != bl) & ~keep).sum())
                expect = np.where(keep, expect, bl)
                requests = [r for r in requests if keep.flat[r]]
                decidable = decidable | ~keep
                o.phase_moves(ph)
                got = o.block_labels()
                np.testing.assert_array_equal(got[decidable], expect[decidable],
                                              err_msg=f"stage {st} sweep {sw} phase {ph}")
                blk, _ = o.pending_requests()
                if decidable.all():
                    assert sorted(blk.tolist()) == requests
                checked += int(decidable.sum())
                o.phase_merges()
    assert checked > 20
    # the mask matters: some blocks the plain method would move are held back by it
    PRUNE_HITS.append(masked_movers)


PRUNE_HITS = []


def test_pruned_cases_hold_back_moves():
    if len(PRUNE_HITS) < len(RCASES):
        pytest.skip("runs after the rational re-derivations in the same process")
    assert sum(PRUNE_HITS) > 10


def test_fallback_finds_what_the_mask_hid():
    """A mask that keeps only one phase class converges early; the full sweeps that follow
    reach the plain run's quality of convergence: the final state is a fixed point of a full
    sweep (one more full sweep by hand changes nothing)."""
    rgb = synth.random_image(40, 56, 1, levels=6)
    p = dict(K=12, init_block=8, size_mode=2, max_sweeps=60)
    o = oracle.Oracle(rgb, **p)
    masks = []
    for nby, nbx in _grids(o):
        m = np.zeros((nby, nbx), np.uint8)
        m[0::3, 0::3] = 1
        masks.append(m)
    for i, m in enumerate(masks):
        o.set_keep_mask(i, m)
    o.seed()
    for st in range(o.num_stages()):
        if st > 0:
            o.next_stage()
        o.refine_stage()
        assert o.counters()[st, C_SWEEPS] < p["max_sweeps"]
        o.set_keep_mask(st, None)  # full sweeps now; the state must already be their fixed point
        before = o.block_labels()
        changes = 0
        for ph in range(9):
            mv, mg = o.phase(ph)
            changes += mv + mg
        assert changes == 0
        np.testing.assert_array_equal(o.block_labels(), before)
    s, _, _ = o.stats()
    np.testing.assert_array_equal(s[:, :6], helpers.stats_from_labels(rgb, o.labels(), s.shape[0])[:, :6])


def test_keep_mask_checks_its_size_and_schedule():
    rgb = synth.random_image(20, 24, 5, levels=4)
    o = oracle.Oracle(rgb, K=4, init_block=4)
    nby, nbx = _grids(o)[0]
    with pytest.raises(RuntimeError):
        o.set_keep_mask(0, np.ones((nby, nbx + 1), np.uint8))
    with pytest.raises(RuntimeError):
        o.set_keep_mask(o.num_stages(), np.ones((nby, nbx), np.uint8))
    q = oracle.Oracle(rgb, K=4, init_block=4, schedule=1)
    with pytest.raises(RuntimeError):
        q.set_keep_mask(0, np.ones((nby, nbx), np.uint8))
