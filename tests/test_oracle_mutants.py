"""Planted mistakes in the oracle: each must make one of its pins fail.

Every mutant below is one plausible slip in ``oracle/rapid_oracle.c``: a dropped term, a
wrong sign, a transposed operand or index, an off-by-one in a bound, a missing queue push.
It is planted by a textual replacement in a copy of the source, which must match the
oracle exactly once, and built into a library of its own in a temporary folder.  The pins
named beside it then run against that library in a separate process, so that a mistake
that corrupts memory cannot take this one down.  At least one of them must fail with an
assertion.  The copy without a planted mistake, built and run the same way over every pin
file named here, must pass (the control).

Test infrastructure only: nothing here is part of the library.
"""
from __future__ import annotations

import json
import os
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor
from typing import NamedTuple

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
ORACLE_DIR = os.path.join(ROOT, "oracle")
RESULT_TAG = "MUTANT-RESULT "

BF = "test_oracle_bruteforce.py"
CF = "test_oracle_closed_forms.py"
FR = "test_oracle_frontier.py"
FT = "test_oracle_features.py"
INV = "test_oracle_invariants.py"
LV = "test_oracle_levels.py"
MG = "test_oracle_merge.py"
FF = "test_oracle_fifo.py"
SP = "test_oracle_simple_point.py"
PR = "test_oracle_pruned.py"


class Mutant(NamedTuple):
    name: str
    passage: str   # what the planted line gets wrong
    original: str  # text of the oracle, matched exactly once
    planted: str
    pins: tuple    # pin files (or node ids) expected to catch it, cheapest first


ENERGY = "return (ec + lam_pos * ep) + lam_b2 * (double)Bk;"
SIZE_RULE = "(int64_t)st->p.lo_den * (N0[a] - b[0]) < (int64_t)st->p.lo_num * st->init[a]) {"
MERGE_ZERO = ("        st->N[a] = st->R[a] = st->G[a] = st->B[a] = st->X[a] = st->Y[a] = 0;\n"
              "      }\n    }\n    free(tgt); free(inv); free(to);")

MUTANTS = [
    # Eq. equa:energy1 and Eq. operation: the block energy and the choice of label
    Mutant("colour_term_drops_blue", "E_col sums three channels",
           "double ec = (eR + eG) + eB;", "double ec = eR + eG;", (BF,)),
    Mutant("position_term_sign", "E_pos is added",
           ENERGY, "return (ec - lam_pos * ep) + lam_b2 * (double)Bk;", (BF,)),
    Mutant("boundary_term_dropped", "E_b is part of the energy",
           ENERGY, "return ec + lam_pos * ep;", (BF,)),
    Mutant("colour_cross_term_halved", "sum |I - c|^2 expands to sum I^2 - 2 S.c + w |c|^2",
           "double eR = (w * cR) * cR - (double)(2 * b[1]) * cR;",
           "double eR = (w * cR) * cR - (double)(b[1]) * cR;", (BF,)),
    Mutant("y_position_uses_x_sum", "E_pos takes the y sums for the y mean",
           "double ey = (w * my) * my - (double)(2 * b[5]) * my;",
           "double ey = (w * my) * my - (double)(2 * b[4]) * my;", (BF,)),
    Mutant("boundary_pairs_counted_once", "E_b sums over p and over q in N4(p): each pair twice",
           "st->lam_b2 = 2.0 * st->p.lambda_b;", "st->lam_b2 = st->p.lambda_b;", (BF,)),
    Mutant("boundary_length_against_own_label", "E_b of candidate k counts edges not labelled k",
           "if (nb[i] >= 0 && nb[i] != k) Bk += len[i];",
           "if (nb[i] >= 0 && nb[i] != a) Bk += len[i];", (BF,)),
    Mutant("edge_lengths_transposed", "N and S edges are the block's width, W and E its height",
           "int32_t len[4] = {bw, bh, bh, bw};", "int32_t len[4] = {bh, bw, bw, bh};", (BF,)),
    Mutant("argmin_takes_the_largest", "Eq. operation takes the lowest energy",
           "if (bestk < 0 || dE < best || (dE == best && k < bestk)) {",
           "if (bestk < 0 || dE > best || (dE == best && k < bestk)) {", (BF,)),
    Mutant("phase_classes_transposed", "phase (py, px) in raster order",
           "int32_t py = phase / 3, px = phase % 3, M = st->M;",
           "int32_t px = phase / 3, py = phase % 3, M = st->M;", (BF,)),
    Mutant("size_rule_reads_live_counts", "the size rule reads the phase-start counts",
           "r[j] = (int8_t)decide(st, bx, by, cR, cG, cB, mX, mY, N0, &kk[j], &e, &v);",
           "r[j] = (int8_t)decide(st, bx, by, cR, cG, cB, mX, mY, N0, &kk[j], &e, &v);"
           " if (r[j] == 1) { int64_t bb[6]; block_sums(st, bx, by, bb); N0[st->lab[blk]] -= bb[0]; }",
           (BF, INV)),
    Mutant("evaluated_counts_topology_failures", "a block counts as evaluated once it passes E_topo",
           "if (!st->lut[neighbour_mask(st, bx, by, a)]) return 0;\n  (*eval)++;",
           "(*eval)++;\n  if (!st->lut[neighbour_mask(st, bx, by, a)]) return 0;", (FR,)),
    Mutant("full_res_position_transposed", "a full-resolution pixel adds x to the x sum",
           "c[4] = X; c[5] = Y;", "c[4] = Y; c[5] = X;", (INV, BF)),
    # E_topo: the simple-point test
    Mutant("topology_test_skipped", "a move must keep the superpixel connected",
           "if (!st->lut[neighbour_mask(st, bx, by, a)]) return 0;",
           "if (!st->lut[neighbour_mask(st, bx, by, a)] && 0) return 0;", (INV, BF)),
    Mutant("topology_west_neighbour_unchecked", "every 4-neighbour labelled a must stay joined",
           "  for (int j = 0; j < 4; j++)\n    if (grid[1 + fy[j]][1 + fx[j]] && !seen",
           "  for (int j = 0; j < 3; j++)\n    if (grid[1 + fy[j]][1 + fx[j]] && !seen", (SP,)),
    Mutant("topology_isolated_block_removable", "a block with no 4-neighbour labelled a is not simple",
           "if (start < 0) return 0;", "if (start < 0) return 1;", (SP,)),
    Mutant("neighbour_mask_diagonal_only", "the window reads (dx, dy) around the block",
           "if (label_at(st, bx + RING_DX[i], by + RING_DY[i]) == a) m |= 1u << i;",
           "if (label_at(st, bx + RING_DX[i], by + RING_DX[i]) == a) m |= 1u << i;", (INV, BF)),
    # Eq. bound and Eq. new_bound: which blocks are tested
    Mutant("south_neighbour_not_a_boundary", "Eq. bound looks at all four neighbours",
           "label_at(st, bx, by + 1)};\n  int boundary = 0;", "-1};\n  int boundary = 0;", (BF,)),
    Mutant("eligibility_ignores_importance", "Eq. new_bound: only boundary superpixels from level 2",
           "if (st->p.importance_rule == 0) return st->imp[a] != 0;",
           "if (st->p.importance_rule == 0) return 1;", (LV,)),
    Mutant("pair_rule_ignores_classes", "the literal pair rule wants a neighbour of the other class",
           "if (nb[j] >= 0 && nb[j] != a && st->y[nb[j]] != st->y[a]) return 1;",
           "if (nb[j] >= 0 && nb[j] != a) return 1;", (LV,)),
    # Sec. 3.1: the size rule and the merge
    Mutant("size_rule_ignores_the_block", "the count after removing the block is compared",
           SIZE_RULE, "(int64_t)st->p.lo_den * N0[a] < (int64_t)st->p.lo_num * st->init[a]) {", (BF,)),
    Mutant("size_rule_not_strict", "the bound is 'smaller than' l InitSize",
           SIZE_RULE, SIZE_RULE.replace(") < (", ") <= ("), (BF,)),
    Mutant("size_mode_1_requests_merges", "with lambda_s infinite the move is refused, no merge",
           "return st->p.size_mode == 2 ? 2 : 0;", "return 2;", (INV, BF)),
    Mutant("initsize_doubled", "InitSize is the seeded superpixel's pixel count",
           "for (int32_t k = 0; k < st->M; k++) st->init[k] = st->N[k];",
           "for (int32_t k = 0; k < st->M; k++) st->init[k] = 2 * st->N[k];", (CF,)),
    Mutant("ward_unweighted", "Eq. eqa:merge weighs by Na Nn / (Na + Nn)",
           "double t = ((double)st->N[a] * (double)st->N[n]) / (double)(st->N[a] + st->N[n]);",
           "double t = 1.0;", (MG,)),
    Mutant("ward_drops_position", "Eq. eqa:merge has a position term",
           "return t * (dc + st->lam_pos * dm);", "return t * dc;", (MG,)),
    Mutant("upper_bound_on_source", "Eq. condtion bounds the target's InitSize",
           "> (int64_t)st->p.hi_num * st->init[n]) continue;",
           "> (int64_t)st->p.hi_num * st->init[a]) continue;", (MG,)),
    Mutant("merge_takes_the_worst", "the target has the least merge cost",
           "if (best < 0 || w < bw || (w == bw && n < best)) {",
           "if (best < 0 || w > bw || (w == bw && n < best)) {", (MG,)),
    Mutant("merge_target_taken_twice", "a superpixel takes part in one merge per phase",
           "if (n < 0 || inv[a] || inv[n]) continue;", "if (n < 0 || inv[a]) continue;", (MG,)),
    Mutant("merged_source_keeps_its_sums", "S_n += S_a, then S_a = 0",
           MERGE_ZERO, MERGE_ZERO.split("\n", 1)[1], (INV, MG)),
    # Algorithm RAPID "update mu and c": statistics after a move
    Mutant("move_adds_x_to_y", "a move carries the block's y sum",
           "st->X[k] += b[4]; st->Y[k] += b[5];", "st->X[k] += b[4]; st->Y[k] += b[4];", (INV,)),
    Mutant("move_leaves_source_count", "a move takes the block off its old superpixel",
           "st->N[a] -= b[0]; ", "", (INV,)),
    # Sec. 2.2, Eq. eq:mu: levels, stages and reuse
    Mutant("pyramid_y_sums_x", "a coarse pixel keeps the y sum of its footprint",
           "c[4] += x; c[5] += y;", "c[4] += x; c[5] += x;", (LV,)),
    Mutant("level_factor_one_too_many", "f_l = C^(L - l)",
           "for (int32_t i = 0; i < st->L - l; i++) f *= (st->L > 1 ? p->ratio_C : 1);",
           "for (int32_t i = 0; i <= st->L - l; i++) f *= (st->L > 1 ? p->ratio_C : 1);", (LV,)),
    Mutant("stage_level_off_by_one", "a side belongs to the coarsest level whose factor is <= it",
           "if (st->f[l] <= s) { lev = l; break; }", "if (st->f[l] < s) { lev = l; break; }", (LV,)),
    Mutant("lambda_pos_not_scaled", "lambda_pos per unit of initial superpixel area",
           "st->lam_pos = st->p.lambda_pos0 * ((double)st->M / ((double)st->H * (double)st->W));",
           "st->lam_pos = st->p.lambda_pos0;", (CF,)),
    # Algorithm RAPID: seeding
    Mutant("seed_columns_transposed", "gx = round(sqrt(K W / H))",
           "sqrt((double)st->p.K * (double)st->W / (double)st->H)",
           "sqrt((double)st->p.K * (double)st->H / (double)st->W)", (CF,)),
    Mutant("seed_rows_truncated", "gy = round(K / gx)",
           "int32_t gy = (int32_t)floor((double)st->p.K / (double)gx + 0.5);",
           "int32_t gy = (int32_t)((double)st->p.K / (double)gx);", (CF,)),
    # Eq. predict and Sec. 4.1: prediction, importance and the features
    Mutant("prediction_at_wrong_level", "the prediction runs on entering level 2",
           "st->st_level[nxt] >= 2 && prev_level < 2", "st->st_level[nxt] >= 3 && prev_level < 3", (LV,)),
    Mutant("brightness_not_averaged_over_channels", "f1 = (R + G + B) / (3 N)",
           "f[0] = (double)(st->R[k] + st->G[k] + st->B[k]) / (double)(3 * st->N[k]);",
           "f[0] = (double)(st->R[k] + st->G[k] + st->B[k]) / (double)(st->N[k]);", (FT,)),
    Mutant("prediction_tie_not_roi", "h >= 0 is ROI", "pos = h >= 0;", "pos = h > 0;", (LV,)),
    Mutant("prediction_sign_flipped", "the stand-in calls dark superpixels ROI",
           "int64_t h = 3 * st->p.h_T * st->N[k] - (st->R[k] + st->G[k] + st->B[k]);",
           "int64_t h = (st->R[k] + st->G[k] + st->B[k]) - 3 * st->p.h_T * st->N[k];", (LV,)),
    Mutant("importance_marks_one_side", "both superpixels of a mixed pair are boundary superpixels",
           "if (e >= 0 && e != a && st->y[e] != st->y[a]) st->imp[a] = st->imp[e] = 1;",
           "if (e >= 0 && e != a && st->y[e] != st->y[a]) st->imp[a] = 1;", (LV,)),
    Mutant("classifier_weights_swapped", "theta_3 weighs f3 and theta_4 weighs f4",
           "t[3] * f[2]) + t[4] * f[3];", "t[3] * f[3]) + t[4] * f[2];", (FT,)),
    Mutant("comparative_brightness_one_side", "each pair adds to both superpixels' f2",
           "sb[b] += ((st->R[a] + st->G[a] + st->B[a]) << 16) / (3 * st->N[a]);", "", (FT,)),
    Mutant("comparative_brightness_sign", "f2 = own brightness minus the neighbours'",
           "f[1] = f[0] - ((double)sb[k] / (double)np[k]) / 65536.0;",
           "f[1] = ((double)sb[k] / (double)np[k]) / 65536.0 - f[0];", (FT,)),
    Mutant("extra_dissimilarity_green_twice", "f3 is the distance over all three channels",
           "eb = cb[a] - cb[b];", "eb = cg[a] - cg[b];", (FT,)),
    Mutant("intra_dissimilarity_unweighted", "f4 weighs each block by its pixel count",
           "double v = w * (dr * dr + dg * dg + db * db);",
           "double v = (dr * dr + dg * dg + db * db);", (FT,)),
    # the queue schedule: the boundary queue of Sec. 2.1 as one flag per block
    Mutant("queue_no_push_after_move", "a moved block queues its 4-neighbours",
           "if (st->p.schedule == 1) queue_neighbours(st, mv[i].blk);", "", (FR,)),
    Mutant("queue_no_push_after_merge", "an accepted merge queues the requesting block's neighbours",
           "if (st->p.schedule == 1) queue_neighbours(st, st->req_blk[i]);", "", (FR,)),
    Mutant("queue_never_pops", "a popped block leaves the queue", "st->queued[blk] = 0;", "", (FR,)),
    Mutant("queue_push_misses_west", "all four neighbours are queued",
           "if (bx > 0) st->queued[blk - 1] = 1;", "", (FR,)),
]

MUTANTS += [
    # the sequential FIFO (Sec. 2.1, Algorithm RAPID's order), the quality comparator
    Mutant("fifo_no_push_after_merge", "a merge re-queues the requesting block's neighbours",
           "      c[C_MERGES]++;\n    } else {", "      c[C_MERGES]++;\n      continue;\n    } else {", (FF,)),
    Mutant("fifo_move_skips_statistics", "statistics follow every move at once",
           "      apply_move(st, i, a, k);\n      c[C_MOVES]++;", "      st->lab[i] = k;\n      c[C_MOVES]++;", (FF,)),
    Mutant("fifo_queues_duplicates", "a block is on the queue at most once",
           "      if (inq[ni]) continue;\n", "", (FF,)),
    Mutant("fifo_push_order_reversed", "neighbours are queued N, W, E, S",
           "    const int dx[4] = {0, -1, 1, 0}, dy[4] = {-1, 0, 0, 1};\n    for (int j = 0; j < 4; j++) {\n      int32_t nx",
           "    const int dx[4] = {0, 1, -1, 0}, dy[4] = {1, 0, 0, -1};\n    for (int j = 0; j < 4; j++) {\n      int32_t nx",
           (FF,)),
    Mutant("fifo_queues_every_block", "the first queue holds the boundary blocks",
           "      if (eligible(st, bx, by, label_at(st, bx, by))) {", "      {", (FF,)),
]

MUTANTS += [
    # pruned sweeps (a keep mask per stage, the mode the learned scorer drives)
    Mutant("keep_mask_ignored", "a block the mask leaves out is not tested",
           "if (st->pruned && !st->keep[st->cur][(int64_t)by * st->nbx + bx]) return 0;", "", (PR,)),
    Mutant("keep_mask_before_eligible_count", "pruned blocks still count as eligible",
           "  (*elig)++;\n  /* pruned sweeps",
           "  if (st->pruned && !st->keep[st->cur][(int64_t)by * st->nbx + bx]) return 0;\n  (*elig)++;\n  /* pruned sweeps",
           (PR,)),
    Mutant("pruned_no_fallback", "a converged pruned stage goes on with full sweeps",
           "      st->pruned = 0; /* the fallback: full sweeps from here on */", "      break;", (PR,)),
    Mutant("pruned_fallback_skipped_sweep_count", "every sweep counts against max_sweeps",
           "    st->cnt[st->cur][C_SWEEPS]++;\n    if (changes == 0) {\n      if (!st->pruned) break;",
           "    if (changes == 0) {\n      if (!st->pruned) { st->cnt[st->cur][C_SWEEPS]++; break; }",
           (PR,)),
]

CONTROL_PINS = tuple(sorted({p for m in MUTANTS for p in m.pins}))


def _build(tmp: str, name: str, original: str | None, planted: str | None) -> str:
    sys.path.insert(0, ORACLE_DIR)
    import build as oracle_build  # oracle/build.py

    with open(os.path.join(ORACLE_DIR, "rapid_oracle.c")) as f:
        src = f.read()
    if original is not None:
        assert src.count(original) == 1, f"{name}: the planted text must match the oracle exactly once"
        src = src.replace(original, planted)
    d = os.path.join(tmp, name)
    os.makedirs(d)
    with open(os.path.join(d, "rapid_oracle.c"), "w") as f:
        f.write(src)
    with open(os.path.join(ORACLE_DIR, "rapid_oracle.h")) as f, open(os.path.join(d, "rapid_oracle.h"), "w") as g:
        g.write(f.read())
    return oracle_build.compile_to(os.path.join(d, "liboracle.so"), [os.path.join(d, "rapid_oracle.c")])


def _run(tmp: str, name: str, original: str | None, planted: str | None, pins) -> dict:
    lib = _build(tmp, name, original, planted)
    args = [os.path.join(HERE, p) for p in pins]
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), lib] + args, cwd=ROOT,
                           capture_output=True, text=True, timeout=600)
    except subprocess.TimeoutExpired:
        return {"rc": None, "failed": [], "note": "timed out"}
    for line in r.stdout.splitlines():
        if line.startswith(RESULT_TAG):
            return json.loads(line[len(RESULT_TAG):])
    return {"rc": r.returncode, "failed": [], "note": (r.stdout + r.stderr)[-2000:]}


@pytest.fixture(scope="module")
def outcomes():
    jobs = [("control", None, None, CONTROL_PINS)] + [(m.name, m.original, m.planted, m.pins) for m in MUTANTS]
    with tempfile.TemporaryDirectory(prefix="oracle-mutants-") as tmp:
        with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
            res = list(ex.map(lambda j: _run(tmp, *j), jobs))
    return {j[0]: r for j, r in zip(jobs, res)}


def test_unplanted_copy_passes_every_pin(outcomes):
    r = outcomes["control"]
    assert r["rc"] == 0 and not r["failed"], r


@pytest.mark.parametrize("m", MUTANTS, ids=[m.name for m in MUTANTS])
def test_planted_mistake_fails_a_pin(outcomes, m):
    r = outcomes[m.name]
    caught = [n for n, kind in r["failed"] if kind == "AssertionError"]
    assert r["rc"] == 1 and caught, f"{m.name} ({m.passage}) survived its pins {m.pins}: {r}"


def _child(lib: str, test_args: list) -> int:
    """Run the given pin tests against the oracle library ``lib`` and print what failed."""
    for p in (ROOT, ORACLE_DIR, HERE):
        if p not in sys.path:
            sys.path.insert(0, p)
    import oracle

    oracle._build.build = lambda force=False: lib
    assert oracle.lib()._name == lib

    class Record:
        def __init__(self):
            self.failed = []

        def pytest_runtest_makereport(self, item, call):
            if call.excinfo is not None and call.when in ("setup", "call"):
                self.failed.append([item.nodeid, call.excinfo.typename])

    rec = Record()
    rc = pytest.main(test_args + ["-x", "-q", "-m", "not gpu", "-p", "no:cacheprovider", "--no-header",
                                  "-o", "addopts="], plugins=[rec])
    print(RESULT_TAG + json.dumps({"rc": int(rc), "failed": rec.failed}))
    return 0


if __name__ == "__main__":
    sys.exit(_child(sys.argv[1], sys.argv[2:]))
