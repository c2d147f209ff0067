"""Quality of the phased schedules against the paper's own sequential order (soft checks):
the 9-phase sweep schedule with phase snapshots, the queue schedule (schedule 1) and the
FIFO queue with live statistics (Algorithm RAPID, Sec. 2.1) must give superpixels of
similar boundary recall (2 px tolerance) and undersegmentation error against the
generator's ground-truth regions, and all must follow the regions far better than the seed
grid.

The bound is 1.5 points of BR and of UE on a 640 x 768 tile with 600 to 1200 superpixels.
The schedules reach different local optima of the same energy, so the gap is a sampling
effect of how many superpixels are compared: measured at this size it is at most 1.2 points
(two seeds, the three parameter sets below), while on 160 x 192 tiles with 60 superpixels it
reached 3.3 points."""
import pytest

import oracle
from helpers import boundary_recall, undersegmentation_error
from paper_1704_02083_gb300 import synth

CASES = [
    dict(K=600, init_block=16, size_mode=2),
    dict(K=600, init_block=16, size_mode=0),
    dict(K=1200, init_block=8, size_mode=2, num_levels=2, ratio_C=4, predict=1),
]
IDS = ["merge", "no_size_term", "two_levels_predict"]
BOUND = 0.015
_RUNS = {}


def _runs(i):
    """Labels of the sweep, queue and FIFO schedules and of the seed grid, and the
    evaluated-block counts of the two phased schedules (computed once per case)."""
    if i not in _RUNS:
        p = CASES[i]
        img = synth.he_image(640, 768, 120, 21)
        sweeps = oracle.Oracle(img.rgb, omp=True, **p).run()
        queue = oracle.Oracle(img.rgb, omp=True, schedule=1, **p).run()
        fifo = oracle.Oracle(img.rgb, **p).run_fifo()
        seeded = oracle.Oracle(img.rgb, **p)
        seeded.seed()
        labs = [x.labels() for x in (sweeps, queue, fifo, seeded)]
        _RUNS[i] = dict(br=[boundary_recall(x, img.regions) for x in labs],
                        ue=[undersegmentation_error(x, img.regions) for x in labs],
                        evaluated=(int(sweeps.counters()[:, 4].sum()), int(queue.counters()[:, 4].sum())))
    return _RUNS[i]


@pytest.mark.parametrize("i", range(len(CASES)), ids=IDS)
def test_phased_schedule_quality_matches_fifo(i):
    r = _runs(i)
    br, ue = r["br"], r["ue"]
    print(f"BR sweeps {br[0]:.4f} fifo {br[2]:.4f} grid {br[3]:.4f}; UE sweeps {ue[0]:.4f} fifo {ue[2]:.4f} "
          f"grid {ue[3]:.4f}")
    assert abs(br[0] - br[2]) <= BOUND and abs(ue[0] - ue[2]) <= BOUND
    assert min(br[0], br[2]) > br[3] + 0.2
    assert max(ue[0], ue[2]) < ue[3]


@pytest.mark.parametrize("i", range(len(CASES)), ids=IDS)
def test_frontier_schedule_quality_matches_sweeps_and_fifo(i):
    """The queue schedule re-evaluates only the 4-neighbours of what moved, like the
    paper's queue: similar quality to the sweeps and to the FIFO, with far fewer block
    evaluations than the sweeps."""
    r = _runs(i)
    br, ue = r["br"], r["ue"]
    print(f"BR sweeps {br[0]:.4f} queue {br[1]:.4f} fifo {br[2]:.4f}; UE sweeps {ue[0]:.4f} queue {ue[1]:.4f} "
          f"fifo {ue[2]:.4f}")
    assert abs(br[1] - br[0]) <= BOUND and abs(ue[1] - ue[0]) <= BOUND
    assert abs(br[1] - br[2]) <= BOUND and abs(ue[1] - ue[2]) <= BOUND
    assert r["evaluated"][1] < 0.5 * r["evaluated"][0]
