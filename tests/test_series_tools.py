"""Host-side helpers of the time-series tool (no GPU): peak finding on sampled curves."""
import math

from paper_2608_13437_gb300.tgv_series import local_maxima, moving_average


def test_local_maxima_finds_the_peaks_of_a_noisy_two_peak_curve():
    t = [0.01 * i for i in range(1001)]  # 0 .. 10
    v = [math.exp(-(x - 2.5) ** 2) + 1.2 * math.exp(-(x - 6.5) ** 2)
         + 1e-3 * math.sin(97.0 * x) for x in t]
    peaks = local_maxima(t, v, 1.0)
    assert len(peaks) == 2
    (t1, v1), (t2, v2) = peaks
    assert abs(t1 - 2.5) < 0.05 and abs(t2 - 6.5) < 0.05
    assert abs(v1 / v2 - 1.0 / 1.2) < 0.01


def test_local_maxima_ignores_the_ends_and_plateau_neighbours():
    assert local_maxima([0, 1, 2, 3], [5, 1, 1, 5], 1.0) == []
    assert local_maxima([0, 1, 2, 3, 4], [0, 2, 1, 2, 0], 1.0) == [(1, 2), (3, 2)]


def test_moving_average_keeps_a_line_and_damps_alternation():
    t = [0.1 * i for i in range(21)]
    line = [3.0 + 2.0 * x for x in t]
    avg = moving_average(t, line, 0.15)  # one neighbour each side inside the series
    for x, a in zip(t[1:-1], avg[1:-1]):
        assert abs(a - (3.0 + 2.0 * x)) < 1e-12
    alt = [1.0 + (-1) ** i for i in range(21)]
    inner = moving_average(t, alt, 0.15)[1:-1]
    assert max(abs(a - 1.0) for a in inner) <= 1.0 / 3.0 + 1e-12
