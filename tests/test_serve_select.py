"""Host-side tests of the serving loop's iteration choice (tfhe_serve_select):
which admitted requests run their next level in one batched launch.

The rule: rank requests by levels left plus iterations waited (ties in
admission order), take next levels in that order while the gate cap allows
(passing over a level that does not fit, always taking the first), then keep
the prefix with the most gates per estimated millisecond.  The estimate is
the autotuner's level time of the width bucket while a level fits one wave
of 4 bootstraps per SM, whole waves above; untuned, fixed fractions of a
wave.  The paper evaluates one circuit at a time, so this has no
counterpart there; results of the served requests never depend on it."""
import numpy as np
import pytest

from paper_2005_01945_gb300 import api

SMS = 152
W4 = 4 * SMS
EDGES = [152, 304, 608, 1216, 2432, 4864, 9728]


def cost(g, level_ms=None, wave_ms=0.0):
    """The estimate the header states, written out for the checks below."""
    t4 = wave_ms if wave_ms > 0 else 1.0
    if g > W4:
        return -(-g // W4) * t4
    if level_ms is not None and wave_ms > 0:
        b = next((i for i, e in enumerate(EDGES) if g <= e), 7)
        if level_ms[b] > 0:
            return float(np.float32(level_ms[b]))
    if g <= SMS:
        return 0.35 * t4
    if g <= 2 * SMS:
        return 0.55 * t4
    return t4


def test_rank_by_levels_left_plus_wait_ties_in_admission_order():
    # remaining + waited: 5, 7, 7, 3 -> order 1, 2, 0, 3 (1 before 2: admitted first)
    got = api.serve_select([10, 10, 10, 10], [5, 7, 2, 3], [0, 0, 5, 0], cap=10000, num_sms=SMS)
    assert list(got) == [1, 2, 0, 3]


def test_waiting_promotes_a_shallow_request():
    got = api.serve_select([10, 10], [5, 1], [0, 10], cap=10000, num_sms=SMS)
    assert list(got) == [1, 0]


def test_cap_passes_over_levels_that_do_not_fit_and_always_takes_the_first():
    # ranked 0, 1, 2: 2432 + 2500 > 4864, so 1 is passed over and 2 fits (four
    # full waves, then five: the same rate, and the longer list is kept)
    got = api.serve_select([2432, 2500, 608], [9, 8, 7], [0, 0, 0], cap=4864, num_sms=SMS)
    assert list(got) == [0, 2]
    # a single level wider than the cap still runs
    got = api.serve_select([9000, 10], [9, 1], [0, 0], cap=4864, num_sms=SMS)
    assert list(got) == [0]


def test_spill_into_a_second_wave_is_left_for_the_next_iteration():
    # 600 gates fill one wave; 20 more would take a second wave for 20 gates
    got = api.serve_select([600, 20], [10, 1], [0, 0], cap=4864, num_sms=SMS)
    assert list(got) == [0]
    # a second wave is kept when the two waves hold more gates per wave
    # (1208 / 2 = 604 > 600); 1100 / 2 = 550 is not
    got = api.serve_select([600, 608], [10, 1], [0, 0], cap=4864, num_sms=SMS)
    assert list(got) == [0, 1]
    got = api.serve_select([600, 500], [10, 1], [0, 0], cap=4864, num_sms=SMS)
    assert list(got) == [0]


def test_narrow_widths_use_the_narrow_level_times():
    # untuned: 100 gates cost 0.35 waves (285.7 gates per wave-time), 160 gates
    # 0.55 (290.9): both requests run
    assert list(api.serve_select([100, 60], [5, 3], [0, 0], cap=4864, num_sms=SMS)) == [0, 1]
    # 140 + 20 = 160 -> 160 / 0.55 = 290.9 < 140 / 0.35 = 400: only the first
    assert list(api.serve_select([140, 20], [5, 3], [0, 0], cap=4864, num_sms=SMS)) == [0]


def test_measured_level_times_replace_the_untuned_model():
    lv = [2.65, 4.32, 7.85, 15.65, 31.33, 62.61, 125.05, 211.01]
    # with these times 160 gates cost 4.32 ms (37 per ms) against 2.65 ms for
    # 140 (52.8 per ms): only the first
    assert list(api.serve_select([140, 20], [5, 3], [0, 0], cap=4864, num_sms=SMS,
                                 level_ms=lv, wave_ms=7.85)) == [0]
    # a 304-gate level at 4.32 ms (70.4 per ms) beats 152 at 2.65 (57.4 per ms)
    assert list(api.serve_select([152, 152], [5, 3], [0, 0], cap=4864, num_sms=SMS,
                                 level_ms=lv, wave_ms=7.85)) == [0, 1]
    # without wave_ms the measured table is not used
    assert list(api.serve_select([152, 152], [5, 3], [0, 0], cap=4864, num_sms=SMS,
                                 level_ms=lv, wave_ms=0.0)) == [0, 1]


@pytest.mark.parametrize("seed", range(40))
def test_random_cases_follow_the_rule(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 40))
    width = rng.choice([1, 2, 3, 20, 31, 63, 136, 528], size=n)
    rem = rng.integers(1, 120, size=n)
    wait = rng.integers(0, 4, size=n)
    tuned = seed % 2 == 1
    lv = [2.65, 4.32, 7.85, 15.65, 31.33, 62.61, 125.05, 211.01] if tuned else None
    wave = 7.85 if tuned else 0.0
    cap = int(rng.choice([608, 2432, 4864]))
    got = list(api.serve_select(width, rem, wait, cap=cap, num_sms=SMS, level_ms=lv,
                                wave_ms=wave))
    rank = sorted(range(n), key=lambda i: (-(int(rem[i]) + int(wait[i])), i))
    greedy, total = [], 0
    for i in rank:
        if greedy and total + width[i] > cap:
            continue
        greedy.append(i)
        total += int(width[i])
    assert got == greedy[:len(got)] and len(got) >= 1
    sums = np.cumsum([int(width[i]) for i in greedy])
    rates = [s / cost(int(s), lv, wave) for s in sums]
    best = max(rates)
    assert rates[len(got) - 1] >= best * (1 - 1e-6)
    assert all(r < best * (1 - 1e-6) for r in rates[len(got):])


def _iterations_until_taken(rem, shrink):
    width = [608, 608, 608, 608, 5]
    rem = list(rem)
    wait = [0] * 5
    for it in range(1, 1000):
        got = list(api.serve_select(width, rem, wait, cap=4 * 608, num_sms=SMS))
        if 4 in got:
            return it
        for i in range(5):
            wait[i] = 0 if i in got else wait[i] + 1
            if shrink and i in got:
                rem[i] -= 1
    return None


def test_a_shallow_request_is_not_starved():
    # four deep requests whose levels fill the cap sit at the top of the
    # ranking; a one-level request behind them runs once its rank (1 + the
    # iterations it waited) exceeds theirs, so after at most 100 waits even if
    # their levels left never shrank
    assert _iterations_until_taken([100, 100, 100, 100, 1], shrink=False) == 101
    # as they run their rank falls while the waiting one's rises: they meet
    # half way
    assert _iterations_until_taken([100, 100, 100, 100, 1], shrink=True) == 51


def test_empty_and_invalid_inputs():
    assert len(api.serve_select([], [], [], cap=10, num_sms=SMS)) == 0
    for bad in [dict(width=[0], remaining=[1], waited=[0]),
                dict(width=[5], remaining=[0], waited=[0]),
                dict(width=[5], remaining=[1], waited=[-1])]:
        with pytest.raises(api.TFHEError):
            api.serve_select(bad["width"], bad["remaining"], bad["waited"], cap=10, num_sms=SMS)
    with pytest.raises(api.TFHEError):
        api.serve_select([5], [1], [0], cap=0, num_sms=SMS)
    with pytest.raises(api.TFHEError):
        api.serve_select([5], [1], [0], cap=10, num_sms=0)
    with pytest.raises(ValueError):
        api.serve_select([5, 6], [1], [0], cap=10, num_sms=SMS)
