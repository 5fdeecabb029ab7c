"""Host logic of the precision autotuner (no GPU): the candidate settings are walked from the
cheapest up, so the first one that meets the targets is the cheapest that does."""
from paper_2311_08050_gb300 import tune


def test_candidates_are_ordered_by_their_gemm_cost():
    costs = [tune.candidate_cost(c) for c in tune.CANDIDATES]
    assert all(a <= b + 1e-9 for a, b in zip(costs, costs[1:])), list(zip(tune.CANDIDATES, costs))


def test_candidates_are_distinct_valid_slice_counts_ending_at_the_six_slice_rung():
    assert len(set(tune.CANDIDATES)) == len(tune.CANDIDATES)
    for setting in tune.CANDIDATES:
        assert len(setting) == 5 and all(2 <= k <= 6 for k in setting)
    # the most expensive candidate is the FP64-accurate rung everywhere it matters
    assert tune.CANDIDATES[-1] == (6, 6, 6, 4, 6)


def test_cost_counts_gemm_passes_per_phase():
    # one more slice in a phase adds (S + 1) passes of that phase's work
    base = tune.candidate_cost((4, 4, 4, 3, 4))
    assert abs(tune.candidate_cost((5, 4, 4, 3, 4)) - base - 2 * 5 / 3) < 1e-12
    assert abs(tune.candidate_cost((4, 5, 4, 3, 4)) - base - 5 / 3) < 1e-12
    assert abs(tune.candidate_cost((4, 4, 4, 4, 4)) - base - tune.NEWTON_WEIGHT * 4) < 1e-12
