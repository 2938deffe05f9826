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
