"""Properties of the oracle's whole runs over the parameter space, drawn by hypothesis
(derandomized: the same examples every time).

Any image size from 1 x 1 up, any K, initial block, final grain, level count and ratio,
each size mode with several bounds l and u, prediction with either importance rule, reuse
on or off, both schedules.
After the run:
  * the statistics equal their recomputation from the label map (exact int64);
  * every live superpixel is one 4-connected region (E_topo) and every label id lies in
    [0, M); retired labels hold zero sums;
  * InitSize is the superpixel's pixel count at seeding, and never changes;
  * the counters are consistent: evaluated <= eligible, merges <= requests, at least one
    sweep and at most max_sweeps per stage, the stage list as scheduled;
  * without the size term nothing is requested or merged, and M never changes."""
import numpy as np
import pytest

import helpers
import oracle
from paper_1704_02083_gb300 import synth

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")

PARAMS = st.fixed_dictionaries({
    "H": st.integers(1, 64), "W": st.integers(1, 64), "seed": st.integers(0, 10_000),
    "kind": st.sampled_from(["he", "random", "levels2"]),
    "K": st.integers(1, 40), "init_block": st.sampled_from([1, 2, 4, 8, 16]),
    "final_grain": st.sampled_from([1, 1, 2, 4]), "num_levels": st.integers(1, 3),
    "ratio_C": st.sampled_from([2, 4]), "size_mode": st.integers(0, 2), "predict": st.integers(0, 1),
    "importance_rule": st.integers(0, 1), "reuse": st.integers(0, 1), "schedule": st.integers(0, 1),
    "max_sweeps": st.sampled_from([1, 3, 64]),
    "lo": st.sampled_from([(1, 4), (1, 2), (3, 4)]), "hi": st.sampled_from([(3, 2), (2, 1), (4, 1)]),
})


def _image(p):
    if p["kind"] == "he":
        return synth.he_image(p["H"], p["W"], 3, p["seed"]).rgb
    return synth.random_image(p["H"], p["W"], p["seed"], levels=256 if p["kind"] == "random" else 2)


@hyp.settings(max_examples=500, deadline=None, derandomize=True, database=None)
@hyp.given(PARAMS)
def test_whole_runs_keep_their_invariants(p):
    rgb = _image(p)
    H, W = rgb.shape[:2]
    kw = {k: v for k, v in p.items() if k not in ("H", "W", "seed", "kind", "lo", "hi")}
    kw.update(lo_num=p["lo"][0], lo_den=p["lo"][1], hi_num=p["hi"][0], hi_den=p["hi"][1])
    o = oracle.Oracle(rgb, **kw)
    o.seed()
    seeded = o.block_labels().copy()
    side0 = o.grid()["side"]
    M = o.grid()["M"]
    init = helpers.stats_from_labels(rgb, helpers.upsample(seeded, side0, H, W), M)[:, 0]
    o.refine_stage()
    while o.grid()["stage"] + 1 < o.num_stages():
        o.next_stage()
        o.refine_stage()
    lab = o.labels()
    s, y, imp = o.stats()
    assert o.grid()["M"] == M and lab.min() >= 0 and lab.max() < M
    np.testing.assert_array_equal(s[:, :6], helpers.stats_from_labels(rgb, lab, M))
    np.testing.assert_array_equal(s[:, 6], init)
    live = np.unique(lab)
    assert (s[live, 0] > 0).all()
    assert (s[np.setdiff1d(np.arange(M), live), :6] == 0).all()
    assert helpers.count_components_per_label(lab) == len(live)
    c = o.counters()
    assert [tuple(r[:2]) for r in c] == [tuple(x) for x in o.stages()]
    assert (c[:, 4] <= c[:, 3]).all() and (c[:, 7] <= c[:, 6]).all()
    assert (c[:, 2] >= 1).all() and (c[:, 2] <= p["max_sweeps"]).all()
    if p["size_mode"] != 2:
        assert c[:, 6].sum() == 0 and c[:, 7].sum() == 0 and len(live) == M
    SEEN["moves"] += int(c[:, 5].sum() > 0)
    SEEN["merges"] += int(c[:, 7].sum() > 0)
    SEEN["predicted"] += int(p["predict"] and (y != 0).any())


SEEN = {"moves": 0, "merges": 0, "predicted": 0}


def test_the_examples_move_merge_and_predict():
    """Runs after the property: the drawn examples exercise moves, merges and the prediction."""
    assert SEEN["moves"] > 100 and SEEN["merges"] > 5 and SEEN["predicted"] > 20, SEEN
