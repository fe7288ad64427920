"""The server's admission planner (pure host logic, no GPU): budget, LRU
eviction of idle grids, per-trajectory order and no overtaking."""
import pytest

from paper_1704_02745_gb300 import build as pbbuild
from paper_1704_02745_gb300 import pb


@pytest.fixture(scope="module", autouse=True)
def lib():
    pbbuild.build()
    pb.load()


def slot(traj, dims=(33, 33, 33), nbytes=100, busy=False, last=0):
    return {"trajectory_id": traj, "dims": dims, "bytes": nbytes, "busy": busy, "last_used": last}


def test_fits_without_eviction():
    admit, evict = pb.pb_plan_admission(1000, [], [(1, (33, 33, 33), 300), (2, (33, 33, 33), 300)])
    assert admit == [-1, -1] and evict == []


def test_reuses_idle_grid_of_the_trajectory():
    admit, evict = pb.pb_plan_admission(1000, [slot(7)], [(7, (33, 33, 33), 100)])
    assert admit == [0] and evict == [0]


def test_busy_trajectory_gets_another_grid():
    admit, evict = pb.pb_plan_admission(1000, [slot(7, busy=True)],
                                        [(7, (33, 33, 33), 100), (8, (33, 33, 33), 100),
                                         (7, (33, 33, 33), 100)])
    assert admit == [-1, -1, -1] and evict == [0]


def test_reuses_the_most_recent_idle_grid():
    slots = [slot(7, last=3), slot(7, last=9), slot(7, busy=True, last=12)]
    admit, evict = pb.pb_plan_admission(1000, slots, [(7, (33, 33, 33), 100), (7, (33, 33, 33), 100)])
    assert admit == [1, 0] and evict == [0, 0, 0]


def test_lru_eviction_of_idle_grids_only():
    slots = [slot(1, nbytes=400, last=5), slot(2, nbytes=400, last=1), slot(3, nbytes=150, busy=True)]
    admit, evict = pb.pb_plan_admission(1000, slots, [(9, (65, 65, 65), 400)])
    # 950 used; 400 more needs one eviction: the least recently used idle grid (traj 2)
    assert admit == [-1] and evict == [0, 1, 0]


def test_no_overtaking_after_a_blocked_request():
    slots = [slot(1, nbytes=800, busy=True)]
    admit, evict = pb.pb_plan_admission(1000, slots, [(2, (65, 65, 65), 500), (3, (33, 33, 33), 100)])
    assert admit == [-2, -2] and evict == [0]


def test_changed_dims_replace_the_stale_grid():
    slots = [slot(4, dims=(33, 33, 33), nbytes=300, last=3)]
    admit, evict = pb.pb_plan_admission(500, slots, [(4, (49, 49, 49), 450)])
    assert admit == [-1] and evict == [1]


def test_untagged_requests_never_share():
    admit, evict = pb.pb_plan_admission(1000, [slot(-1)], [(-1, (33, 33, 33), 100)])
    assert admit == [-1] and evict == [0]
