"""Quality of the phased schedule against the paper's own sequential order (soft checks,
reported rather than exact): the 9-phase schedule with phase snapshots and the FIFO queue
with live statistics (Algorithm RAPID, Sec. 2.1) must give superpixels of similar boundary
recall (2 px tolerance) and undersegmentation error against the generator's ground-truth
regions, and both must follow the regions far better than the seed grid."""
import numpy as np
import pytest

import oracle
from helpers import boundary_recall, undersegmentation_error
from paper_1704_02083_gb300 import synth

CASES = [
    dict(K=60, init_block=16, size_mode=2),
    dict(K=60, init_block=16, size_mode=0),
    dict(K=120, init_block=8, size_mode=2, num_levels=2, ratio_C=4, predict=1),
]


@pytest.mark.parametrize("params", CASES, ids=["merge", "no_size_term", "two_levels_predict"])
def test_phased_schedule_quality_matches_fifo(params):
    img = synth.he_image(160, 192, 12, 21)
    phased = oracle.run(img.rgb, **params)[0]
    fifo = oracle.Oracle(img.rgb, **params).run_fifo().labels()
    seeded = oracle.Oracle(img.rgb, **params)
    seeded.seed()
    grid = seeded.labels()
    br = [boundary_recall(x, img.regions) for x in (phased, fifo, grid)]
    ue = [undersegmentation_error(x, img.regions) for x in (phased, fifo, grid)]
    print(f"BR phased {br[0]:.3f} fifo {br[1]:.3f} grid {br[2]:.3f}; "
          f"UE phased {ue[0]:.3f} fifo {ue[1]:.3f} grid {ue[2]:.3f}")
    assert abs(br[0] - br[1]) <= 0.05 and abs(ue[0] - ue[1]) <= 0.05
    assert min(br[0], br[1]) > br[2] + 0.2
    assert max(ue[0], ue[1]) < ue[2]


@pytest.mark.parametrize("params", CASES, ids=["merge", "no_size_term", "two_levels_predict"])
def test_frontier_schedule_quality_matches_sweeps_and_fifo(params):
    """The frontier schedule (schedule 1) re-evaluates only the 4-neighbours of what moved,
    like the paper's queue: similar quality to the sweeps and to the FIFO, with far fewer
    block evaluations than the sweeps."""
    img = synth.he_image(160, 192, 12, 21)
    sweeps = oracle.Oracle(img.rgb, **params).run()
    front = oracle.Oracle(img.rgb, schedule=1, **params).run()
    fifo = oracle.Oracle(img.rgb, **params).run_fifo()
    labs = [x.labels() for x in (sweeps, front, fifo)]
    br = [boundary_recall(x, img.regions) for x in labs]
    ue = [undersegmentation_error(x, img.regions) for x in labs]
    print(f"BR sweeps {br[0]:.3f} frontier {br[1]:.3f} fifo {br[2]:.3f}; "
          f"UE sweeps {ue[0]:.3f} frontier {ue[1]:.3f} fifo {ue[2]:.3f}")
    assert abs(br[1] - br[0]) <= 0.05 and abs(ue[1] - ue[0]) <= 0.05
    assert abs(br[1] - br[2]) <= 0.05 and abs(ue[1] - ue[2]) <= 0.05
    assert front.counters()[:, 4].sum() < 0.5 * sweeps.counters()[:, 4].sum()
