"""Pins of the event-detection oracle (Section 4.1 pre-processing: event
detection, adaptor trimming) against facts that do not come from the oracle:
hand-worked statistics, scipy's Welch t-test, noiseless step signals whose
boundaries and means are known exactly, invariance under a change of the
ADC scale and offset, and a hand-derived tie."""
import numpy as np
import pytest

import oracle
import synth
from tests.conftest import read_golden


@pytest.mark.parametrize("row", read_golden("events_hand.txt"))
def test_tstat_hand_worked(row):
    xs, w, i, num, den = row
    x = np.array([int(v) for v in xs.split()], dtype=np.int16)
    n_, d_ = oracle.event_tstat(x, int(w))
    assert (n_[int(i)], d_[int(i)]) == (int(num), int(den))
    # undefined outside [w, n - w]
    w = int(w)
    assert all(d_[j] == 0 for j in range(x.shape[0] + 1) if j < w or j > x.shape[0] - w)


def test_tstat_is_welch_t_test():
    """With sample variances, Welch's t (scipy) is t * sqrt((w - 1) / w) of
    this statistic (population variances), wherever the variance floor is
    not in play."""
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(31)
    for w in (3, 6, 9):
        x = synth.to_adc(rng.normal(90, 3, 400) + np.repeat(rng.normal(0, 10, 40), 10))
        num, den = oracle.event_tstat(x, w)
        for i in range(w, x.shape[0] - w + 1, 7):
            a, b = x[i - w:i].astype(np.float64), x[i:i + w].astype(np.float64)
            if den[i] <= 1:
                continue
            welch = stats.ttest_ind(b, a, equal_var=False).statistic
            assert np.isclose(num[i] / den[i] * (w - 1) / w, welch ** 2, rtol=1e-9, atol=0)


def step_signal(rng, nseg, lo=13, hi=40):
    lengths = rng.integers(lo, hi, nseg)
    levels = np.cumsum(rng.choice([-1, 1], nseg) * rng.integers(1, 300, nseg)) + 2000
    x = np.repeat(levels, lengths).astype(np.int16)
    return x, np.cumsum(lengths)[:-1], levels


def test_noiseless_steps_are_exact():
    """A piecewise-constant signal whose segments are longer than twice the
    long window: every change point is a boundary, nothing else is, and each
    event's mean is its level."""
    rng = np.random.default_rng(32)
    for _ in range(20):
        x, cuts, levels = step_signal(rng, int(rng.integers(2, 40)))
        np.testing.assert_array_equal(oracle.event_boundaries(x), cuts)
        np.testing.assert_array_equal(oracle.read_events(x, trim=0, max_events=10 ** 6),
                                      levels.astype(np.float32))


def test_trim_and_prefix():
    """The query is events [trim, trim + max_events): a slice of the levels."""
    rng = np.random.default_rng(33)
    x, _, levels = step_signal(rng, 60)
    lv = levels.astype(np.float32)
    for trim, m in ((0, 5), (10, 20), (55, 250), (59, 1), (60, 3), (70, 3)):
        np.testing.assert_array_equal(oracle.read_events(x, trim=trim, max_events=m), lv[trim:trim + m])


def test_affine_change_of_adc_scale_keeps_boundaries():
    """t is a ratio of a squared mean difference to a variance: scaling the
    samples by a > 0 and shifting them leaves every boundary in place."""
    rng = np.random.default_rng(34)
    for _ in range(10):
        x = synth.to_adc(rng.normal(90, 2.5, 3000) + np.repeat(rng.normal(0, 12, 300), 10))
        y = (3 * x.astype(np.int32) - 700).astype(np.int16)
        np.testing.assert_array_equal(oracle.event_boundaries(y), oracle.event_boundaries(x))


def test_tie_goes_to_the_first_position():
    """a a ... a m b b ... b with m midway: the statistics one position either
    side of m's left edge are mirror images (equal), so both windows peak
    twice with equal values; the boundary is the first of the two, at m."""
    x = np.array([100] * 20 + [150] + [200] * 20, dtype=np.int16)
    for w in (3, 6):
        num, den = oracle.event_tstat(x, w)
        assert num[20] * den[21] == num[21] * den[20]
    np.testing.assert_array_equal(oracle.event_boundaries(x), [20])
    np.testing.assert_array_equal(oracle.read_events(x, trim=0, max_events=9),
                                  np.array([100.0, 4150.0 / 21.0], dtype=np.float32))


def test_noise_only_gives_few_long_events():
    """Gaussian noise around one level has no steps: the long window never
    fires (its threshold is far above noise), short-window peaks are at least
    w1 + 1 = 4 samples apart, and every event mean lies within the samples'
    range."""
    rng = np.random.default_rng(35)
    x = synth.to_adc(rng.normal(90, 2.5, 5000))
    b = oracle.event_boundaries(x)
    assert (np.diff(b) >= 4).all() and b.min() >= 3 and b.max() <= 5000 - 3
    num, den = oracle.event_tstat(x, 6)
    ok = den > 0
    assert (num[ok] * 10000 <= 900 * 900 * den[ok]).all()
    ev = oracle.read_events(x, trim=0, max_events=10 ** 6)
    assert ev.shape[0] == b.shape[0] + 1 and ev.min() >= x.min() and ev.max() <= x.max()


def test_signal_batch_composes_reads():
    g, m, k, R = synth.signal_workload("sars_signal_32x250", nreads=6)
    ev, off = oracle.signal_events(R.samples, R.offsets, threads=3)
    for r in range(R.nreads):
        np.testing.assert_array_equal(ev[off[r]:off[r + 1]], oracle.read_events(R.read(r)))
    assert (np.diff(off.astype(np.int64)) == 250).all()


def test_boundaries_of_simulated_reads_keep_their_spacing():
    """On simulated R9.4-like reads (steps between pore-model levels under
    noise) both windows fire, often a few samples apart at the same step:
    keeping only long-window peaks there leaves every pair of boundaries at
    least w1 + 1 = 4 samples apart, and a boundary never sits within the
    first or last w1 samples of the read."""
    g, m, k, R = synth.signal_workload("sars_signal_32x250", nreads=8)
    for r in range(R.nreads):
        x = R.read(r)
        b = oracle.event_boundaries(x)
        assert (np.diff(b) >= 4).all()
        assert b.min() >= 3 and b.max() <= x.shape[0] - 3
