"""Host side of the environment kernel's phase trace: the summary of a
trace table (paper_2510_18221_gb300.phase_trace.summarise) on a table
written by hand."""
import numpy as np

from paper_2510_18221_gb300.phase_trace import summarise


def _row(start, arrive, passes, end, step, claimants):
    r = np.zeros(16, np.uint64)
    r[0] = start
    for k, (a, p) in enumerate(zip(arrive, passes)):
        r[1 + k] = start + a
        r[5 + k] = start + p
    r[9] = start + end
    r[10] = step
    r[11] = claimants
    r[12] = len(arrive)
    return r


def test_summarise_hand_written_table():
    t = np.zeros((64, 16), np.uint64)
    # three steps, three barriers each; times in ns from each step's start
    t[5] = _row(10_000, [5_000, 10_000, 15_000], [6_000, 11_000, 16_000], 25_000, 5, 2)
    t[6] = _row(50_000, [6_000, 12_000, 18_000], [7_000, 13_000, 19_000], 21_000, 6, 0)
    t[7] = _row(90_000, [4_000, 8_000, 12_000], [5_000, 9_000, 13_000], 29_000, 7, 4)
    s = summarise(t)
    assert s["steps"] == 3
    assert s["arrive_0"] == {"median": 5.0, "min": 4.0, "max": 6.0}
    assert s["pass_2"] == {"median": 16.0, "min": 13.0, "max": 19.0}
    assert s["end"]["median"] == 25.0
    assert s["end_with_claimants"] == {"median": 27.0, "min": 25.0, "max": 29.0}
    assert s["end_without_claimants"] == {"median": 21.0, "min": 21.0, "max": 21.0}
    assert s["claimants_median"] == 2.0
    assert "arrive_3" not in s


def test_summarise_empty_table():
    assert summarise(np.zeros((64, 16), np.uint64)) == {"steps": 0}
