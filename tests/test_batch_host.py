"""Host logic of the brick autotuner: the ranking of candidate shapes (no GPU)."""
from paper_2409_09399_gb300.batch import CANDIDATE_BRICKS, rank_shapes


def test_shapes_every_system_takes_come_first_then_by_time():
    table = {
        (8, 8, 8): {0: None, 1: 0.010},          # one system cannot take it
        (4, 4, 8): {0: 0.030, 1: 0.020},         # 0.050 in total
        (4, 4, 4): {0: 0.020, 1: 0.020},         # 0.040 in total: fastest
        (2, 2, 2): {0: None, 1: None},           # no system takes it
    }
    assert rank_shapes(table) == [(4, 4, 4), (4, 4, 8), (8, 8, 8), (2, 2, 2)]


def test_ties_keep_the_candidate_order():
    table = {b: {0: 1.0} for b in CANDIDATE_BRICKS}
    assert rank_shapes(table) == list(CANDIDATE_BRICKS)


def test_candidates_fit_the_tensor_core_point_limit():
    # the exact form takes at most 512 points per brick, the three-product form 1024
    assert all(bx * by * bz <= 512 for bx, by, bz in CANDIDATE_BRICKS)
