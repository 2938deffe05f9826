"""The autotuner's choice among timed candidates (no GPU): the fastest, except that a
later candidate must be more than 2 % faster to replace an earlier one."""
from paper_2606_00444_gb300.tune import _pick


def c(v, ms):
    return dict(lanes=1, variant=v, ms=ms)


def test_fastest_wins_by_a_clear_margin():
    assert _pick([c(0, 0.42), c(2, 0.39), c(5, 0.45)])["variant"] == 2


def test_near_ties_keep_the_earlier_candidate():
    assert _pick([c(0, 0.42), c(2, 0.3908), c(5, 0.3904)])["variant"] == 2
    assert _pick([c(0, 0.42), c(2, 0.3908), c(5, 0.3820)])["variant"] == 5


def test_single_candidate():
    assert _pick([c(7, 1.0)])["variant"] == 7


def test_candidates_cover_leaf_sizes_blocks_and_lanes():
    from paper_2606_00444_gb300.tune import LEAF_SIZES, closest_point_candidates
    cands = closest_point_candidates()
    assert {x["leaf"] for x in cands} == set(LEAF_SIZES) == {1, 2, 4, 8}
    assert {x["block"] for x in cands if x["lanes"] == 1} == {32, 64, 128}
    assert {x["lanes"] for x in cands} == {1, 2, 4, 8, 16, 32}
    # blocks other than 128 only for the variants compiled in them
    assert {x["variant"] for x in cands if x["block"] != 128} == {0, 2, 3, 13}
    assert {x["variant"] for x in cands if x["lanes"] == 1} == set(range(14))
    # every configuration is tried once per leaf size
    per_leaf = [x for x in cands if x["leaf"] == 1]
    assert len(per_leaf) == len({(x["lanes"], x["variant"], x["block"]) for x in per_leaf}) == 27
