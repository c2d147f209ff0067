"""The oracle's frontier schedule (schedule 1: the boundary queue of Sec. 2.1 kept as one
flag per block), pinned against an independent model of the queue and the exact energy.

Phase by phase on tiny images, a plain Python queue model follows the definition: every
block is queued when a stage starts; a phase takes the queued blocks of its class off the
queue; a block that moved, and the first requesting block of each accepted merge, queue
their 4-neighbours.  Each queued block's decision is re-derived from the per-pixel energy
of Eq. equa:energy1 in rationals (as for the sweep schedule); blocks that are not queued
must not move or request, and the eligible / evaluated counters must count exactly the
popped blocks that pass the boundary test (Eq. bound) and the classical simple-point test."""
import numpy as np
import pytest

import helpers
import oracle
from paper_1704_02083_gb300 import synth
from test_oracle_bruteforce import _rederive, simple_classical

C_ELIG, C_EVAL = 3, 4


def _push(q, bx, by):
    nby, nbx = q.shape
    for x, y in ((bx, by - 1), (bx - 1, by), (bx + 1, by), (bx, by + 1)):
        if 0 <= x < nbx and 0 <= y < nby:
            q[y, x] = True


def _boundary(bl, bx, by):
    nby, nbx = bl.shape
    a = bl[by, bx]
    return any(bl[y, x] != a for x, y in ((bx, by - 1), (bx - 1, by), (bx + 1, by), (bx, by + 1))
               if 0 <= x < nbx and 0 <= y < nby)


CASES = [(7, 9, 6, 2, 50.0, s, m, 4) for s in range(3) for m in (0, 1, 2)] + \
        [(11, 13, 4, 4, 2000.0, s, 2, 4) for s in range(3)] + \
        [(8, 12, 6, 2, 10.0, 9, m, 2) for m in (1, 2)]


def _walk(H, W, K, ib, lamb, seed, size_mode, levels):
    """Check every phase of the first 4 sweeps of each stage; returns the accepted merges."""
    from fractions import Fraction

    rgb = synth.random_image(H, W, seed, levels=levels)
    o = oracle.Oracle(rgb, K=K, init_block=ib, size_mode=size_mode, lambda_pos0=400.0, lambda_b=lamb, schedule=1)
    o.seed()
    lam_pos, lam_b = Fraction(o.lambda_pos()), Fraction(lamb)
    checked = popped_total = merges_seen = 0
    for st in range(o.num_stages()):
        if st > 0:
            o.next_stage()
        g = o.grid()
        q = np.ones((g["nby"], g["nbx"]), bool)
        for sw in range(4):
            for ph in range(9):
                bl = o.block_labels()
                s, _, _ = o.stats()
                c0 = o.counters()[st]
                expect, requests, decidable = _rederive(rgb, bl, s, g["side"], ph, lam_pos, lam_b, size_mode)
                py, px = divmod(ph, 3)
                popped = np.zeros_like(q)
                popped[py::3, px::3] = q[py::3, px::3]
                q[py::3, px::3] = False
                # blocks not on the queue keep their label and raise no request
                expect = np.where(popped, expect, bl)
                requests = [r for r in requests if popped.flat[r]]
                o.phase_moves(ph)
                got = o.block_labels()
                np.testing.assert_array_equal(got[decidable], expect[decidable],
                                              err_msg=f"stage {st} sweep {sw} phase {ph}")
                blk, lab = o.pending_requests()
                if decidable.all():
                    assert sorted(blk.tolist()) == requests
                # counters: popped blocks passing the boundary test, then the topology test
                elig = [(x, y) for y, x in zip(*np.nonzero(popped)) if _boundary(bl, x, y)]
                ev = [(x, y) for x, y in elig if simple_classical(bl, x, y)]
                c1 = o.counters()[st]
                assert c1[C_ELIG] - c0[C_ELIG] == len(elig)
                assert c1[C_EVAL] - c0[C_EVAL] == len(ev)
                for y, x in zip(*np.nonzero(got != bl)):
                    _push(q, x, y)
                n_before = o.stats()[0][:, 0].copy()
                o.phase_merges()
                n_after = o.stats()[0][:, 0]
                for a in np.nonzero((n_before > 0) & (n_after == 0))[0]:  # accepted merges
                    first = int(blk[lab == a].min())
                    _push(q, first % g["nbx"], first // g["nbx"])
                    merges_seen += 1
                checked += int(decidable.sum())
                popped_total += int(popped.sum())
    assert checked > 20 and popped_total > 0
    return merges_seen


@pytest.mark.parametrize("H,W,K,ib,lamb,seed,size_mode,levels", CASES)
def test_frontier_phases_match_queue_model_and_exact_energy(H, W, K, ib, lamb, seed, size_mode, levels):
    _walk(H, W, K, ib, lamb, seed, size_mode, levels)


def test_frontier_cases_include_accepted_merges():
    assert sum(_walk(*c) for c in CASES if c[6] == 2) > 0


@pytest.mark.parametrize("size_mode", [0, 2])
def test_frontier_first_sweep_is_a_full_sweep(size_mode):
    """Every block is queued when a stage starts, so with one sweep per stage the two
    schedules visit the same blocks with the same states."""
    rgb = synth.he_image(64, 80, n_cells=6, seed=5).rgb
    kw = dict(K=20, init_block=16, size_mode=size_mode, max_sweeps=1, num_levels=2, predict=1)
    a = oracle.Oracle(rgb, schedule=0, **kw).run()
    b = oracle.Oracle(rgb, schedule=1, **kw).run()
    np.testing.assert_array_equal(a.labels(), b.labels())
    np.testing.assert_array_equal(a.counters(), b.counters())


def test_frontier_stage_ends_with_an_empty_queue():
    """A stage stops after a sweep without changes; the queue is then empty, so a further
    sweep pops nothing (no eligible block counted, no move)."""
    rgb = synth.he_image(64, 96, n_cells=6, seed=8).rgb
    o = oracle.Oracle(rgb, K=24, init_block=16, schedule=1)
    o.seed()
    converged = 0
    for st in range(o.num_stages()):
        if st > 0:
            o.next_stage()
        o.refine_stage()
        c = o.counters()[st]
        if c[2] < 64:  # converged before max_sweeps
            converged += 1
            before = o.block_labels()
            for ph in range(9):
                assert o.phase(ph) == (0, 0)
            assert o.counters()[st][C_ELIG] == c[C_ELIG]
            np.testing.assert_array_equal(o.block_labels(), before)
    assert converged > 0


def test_frontier_invariants():
    """S equals its recomputation and every superpixel stays 4-connected (E_topo)."""
    rgb = synth.he_image(72, 100, n_cells=8, seed=11).rgb
    H, W = rgb.shape[:2]
    for size_mode in (0, 2):
        o = oracle.Oracle(rgb, K=24, init_block=16, size_mode=size_mode, schedule=1).run()
        lab = o.labels()
        s, _, _ = o.stats()
        np.testing.assert_array_equal(s[:, :6], helpers.stats_from_labels(rgb, lab, o.grid()["M"]))
        live = np.unique(lab)
        assert helpers.count_components_per_label(lab) == len(live)
