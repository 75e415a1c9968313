"""Algorithm 1 (Sec. IV-B) in the oracle, pinned on hand-worked cases and on
the special cases that reduce it to GCC_0; the box-world scene generator
(Sec. V-B) against its definition."""
import numpy as np
import pytest

import oracle
from paper_2402_15281_gb300 import synth as S


def test_first_loop_returns_first_confirmed_prediction():
    # eps = 0: m0 predicted free but collides, m1 predicted colliding (skipped),
    # m2 predicted free and free -> returned by the first loop after 2 exact checks
    r = oracle.search_first_free([0.1, -0.2, 0.3, 0.5], [-0.1, 0.2, 0.05, 0.4], 0.0)
    assert r == {"motion": 2, "loop": 1, "n_exact": 2, "n_nn_seq": 3}


def test_second_loop_orders_by_decreasing_prediction():
    # only m0 is predicted free and it collides; the rest by decreasing d_hat:
    # m3 (-0.01, collides), m1 (-0.05, free) -> m1 after 3 exact checks
    r = oracle.search_first_free([0.2, -0.05, -0.3, -0.01], [-0.1, 0.02, 0.4, -0.2], 0.0)
    assert r == {"motion": 1, "loop": 2, "n_exact": 3, "n_nn_seq": 4}


def test_second_loop_ties_keep_the_given_order():
    r = oracle.search_first_free([-0.1, -0.1, -0.1], [-1.0, 0.5, 0.7], 0.0)
    assert r["motion"] == 1 and r["n_exact"] == 2


def test_margin_tie_is_a_collision():
    # free iff > eps (a distance equal to the margin is a collision), and a
    # prediction equal to the margin is not "predicted free"
    r = oracle.search_first_free([0.05, 0.06], [0.05, 0.07], 0.05)
    assert r == {"motion": 1, "loop": 1, "n_exact": 1, "n_nn_seq": 2}


def test_no_free_motion():
    r = oracle.search_first_free([1.0, -1.0], [-0.5, -0.5], 0.0)
    assert r == {"motion": -1, "loop": 0, "n_exact": 2, "n_nn_seq": 2}
    assert oracle.search_gcc0([-0.5, -0.5], 0.0) == {"motion": -1, "n_exact": 2}


@pytest.mark.parametrize("seed", range(5))
def test_special_cases_reduce_to_gcc0(seed):
    rng = np.random.default_rng(seed)
    delta = rng.uniform(-0.2, 0.1, 40)
    g = oracle.search_gcc0(delta, 0.0)
    # a predictor that calls everything free (or everything colliding) checks in the given order
    for dhat in (np.full(40, np.inf), np.full(40, -np.inf)):
        r = oracle.search_first_free(dhat, delta, 0.0)
        assert (r["motion"], r["n_exact"]) == (g["motion"], g["n_exact"])
    # a perfect predictor needs one exact check when a free motion exists
    r = oracle.search_first_free(delta, delta, 0.0)
    if g["motion"] >= 0:
        assert r["motion"] == g["motion"] and r["n_exact"] == 1
    else:
        assert r["motion"] == -1


@pytest.mark.parametrize("seed", [0, 7])
def test_box_world_follows_its_definition(seed):
    pts, centres, rots, sides = S.box_world(seed)
    assert len(centres) == 50
    assert np.all(centres >= S.BOX_LO) and np.all(centres <= S.BOX_HI)
    assert np.all((sides >= 0.01) & (sides <= 0.10))
    assert np.abs(np.einsum("nij,nkj->nik", rots, rots) - np.eye(3)).max() < 1e-12
    assert np.all(np.abs(np.linalg.det(rots) - 1) < 1e-12)
    area_cm2 = 2 * (sides[:, 0] * sides[:, 1] + sides[:, 1] * sides[:, 2] + sides[:, 0] * sides[:, 2]) * 1e4
    counts = np.round(area_cm2 * 0.1).astype(int)
    assert len(pts) == counts.sum()
    # every point lies on the surface of its box: in the box frame one coordinate
    # is at +-half a side, the others within the face
    xyz = pts[:, :3].astype(np.float64)
    start = np.concatenate([[0], np.cumsum(counts)])
    for b in range(50):
        loc = (xyz[start[b]:start[b + 1]] - centres[b]) @ rots[b]
        rel = np.abs(loc) / (sides[b] / 2)
        assert np.all(rel <= 1 + 5e-5)           # float32 points
        assert np.all(np.abs(rel.max(axis=1) - 1) <= 5e-5)


def test_box_world_motions_share_one_start():
    robot = S.make_robot(1)
    q0, q1 = S.box_world_motions(robot, 100, seed=3)
    assert q0.shape == q1.shape == (100, 6)
    assert np.all(q0 == q0[0])
    assert np.all(q1 >= robot.qmin) and np.all(q1 <= robot.qmax)


def test_sorted_search_hand_worked():
    # by decreasing prediction: m2 (0.4, collides), m0 (0.1, free) -> m0 after 2 checks
    assert oracle.search_sorted([0.1, -0.3, 0.4], [0.2, 0.5, -0.1], 0.0) == {"motion": 0, "n_exact": 2}
    assert oracle.search_sorted([0.1, 0.1], [-1.0, -1.0], 0.0) == {"motion": -1, "n_exact": 2}


@pytest.mark.parametrize("seed", range(4))
def test_sorted_search_special_cases(seed):
    rng = np.random.default_rng(seed)
    delta = rng.uniform(-0.2, 0.1, 30)
    g = oracle.search_gcc0(delta, 0.0)
    # a constant prediction keeps the given order: GCC_0
    assert oracle.search_sorted(np.zeros(30), delta, 0.0) == g
    # a perfect predictor finds a free motion (the farthest one) with one check
    r = oracle.search_sorted(delta, delta, 0.0)
    if g["motion"] >= 0:
        assert r == {"motion": int(np.argmax(delta)), "n_exact": 1}
