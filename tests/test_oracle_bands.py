"""Pins of the oracle's bands method (trial-period extraction, Section 3.1)
against closed forms, brute force and invariants -- never against itself.

Steps (Section 3.1): derivatives d_i; ten equal-count magnitude bands;
D_j = sum |d_i| per band; the N_b bands of largest D; the spectral window of
Eq. (bands) per band; the N_t highest local maxima, one-day periods left out.
"""
import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("n", [2, 3, 5, 9, 10, 11, 15, 23, 100, 601])
def test_band_partition_counts_and_magnitude_order(n):
    rng = np.random.default_rng(n)
    y = rng.normal(size=n)
    band = oracle.bands_of(y)
    counts = np.bincount(band, minlength=10)
    want = [((k + 1) * n) // 10 - (k * n) // 10 for k in range(10)]
    assert counts.tolist() == want
    assert counts.sum() == n
    for k in range(9):                      # every sample of band k is below every sample of a higher band
        lo, hi = y[band == k], y[band > k]
        if lo.size and hi.size:
            assert lo.max() < hi.min()


def test_band_ties_go_by_sample_index():
    y = np.full(20, 17.0)
    assert oracle.bands_of(y).tolist() == [i // 2 for i in range(20)]
    y = np.array([3.0, 1.0, 3.0, 1.0, 2.0, 2.0, 3.0, 1.0, 2.0, 3.0])
    # ascending ranks: 1.0 at samples 1, 3, 7; 2.0 at 4, 5, 8; 3.0 at 0, 2, 6, 9
    want = np.empty(10, int)
    for r, i in enumerate([1, 3, 7, 4, 5, 8, 0, 2, 6, 9]):
        want[i] = r
    assert oracle.bands_of(y).tolist() == want.tolist()


@pytest.mark.parametrize("slope", [0.37, -1.9])
def test_derivative_sums_of_a_linear_ramp(slope):
    """y = a t + b: every d_i = a; the ranks follow the time order (reversed
    for a < 0), so D_k = |a| times the number of samples i < N-1 in band k."""
    n = 57
    rng = np.random.default_rng(3)
    t = np.cumsum(rng.uniform(0.1, 3.0, n))
    y = slope * t + 12.0
    band = oracle.bands_of(y)
    D = oracle.band_derivative_sums(t, y, band)
    rank = np.arange(n) if slope > 0 else np.arange(n)[::-1]
    b_of_rank = np.array([next(k for k in range(10) if r < ((k + 1) * n) // 10) for r in range(n)])
    assert np.array_equal(band, b_of_rank[rank])
    want = np.array([abs(slope) * np.sum(band[:-1] == k) for k in range(10)])
    np.testing.assert_allclose(D, want, rtol=1e-12)


def test_derivative_of_equal_times_is_zero_and_d_scales():
    t = np.array([0.0, 0.0, 1.0, 2.0, 2.0, 5.0])
    y = np.array([1.0, 9.0, 3.0, 4.0, 8.0, 2.0])
    band = oracle.bands_of(y)
    D = oracle.band_derivative_sums(t, y, band)
    # d = [0 (equal times), (3-9)/1, (4-3)/1, 0 (equal times), (2-8)/3]
    want = np.zeros(10)
    for i, d in enumerate([0.0, -6.0, 1.0, 0.0, -2.0]):
        want[band[i]] += abs(d)
    np.testing.assert_allclose(D, want, rtol=0, atol=0)
    # magnitudes scaled by c > 0 keep the bands and scale D by c; times scaled by s divide D by s
    np.testing.assert_array_equal(oracle.bands_of(2.5 * y), band)
    np.testing.assert_allclose(oracle.band_derivative_sums(t, 2.5 * y, band), 2.5 * D, rtol=1e-15)
    np.testing.assert_allclose(oracle.band_derivative_sums(4.0 * t, y, band), D / 4.0, rtol=1e-15)


def test_band_order_descending_and_stable():
    D = np.array([1.0, 3.0, 3.0, 0.0, 7.0, 1.0, 0.0, 2.0, 3.0, 0.5])
    assert oracle.band_order(D).tolist() == [4, 1, 2, 8, 7, 0, 5, 9, 3, 6]


def test_spectral_window_of_an_arithmetic_progression():
    """Band times t0 + i*dt, i < m: S(f) = sin^2(pi f m dt) / sin^2(pi f dt),
    m^2 where f dt is an integer (the Dirichlet kernel)."""
    m, dt, t0 = 13, 0.7, 1234.5
    t = t0 + dt * np.arange(m)
    band = np.zeros(m, np.int32)
    f0, df, nk = 0.003, 0.0111, 400
    S = oracle.spectral_window(t, band, 0, f0, df, nk)
    f = f0 + df * np.arange(nk)
    x = np.pi * f * dt
    want = np.where(np.abs(np.sin(x)) < 1e-12, m * m, np.sin(m * x) ** 2 / np.maximum(np.sin(x) ** 2, 1e-300))
    np.testing.assert_allclose(S, want, rtol=1e-9, atol=1e-9)
    S0 = oracle.spectral_window(t, band, 0, 0.0, 1.0 / dt, 3)
    np.testing.assert_allclose(S0, [m * m] * 3, rtol=1e-12)


def test_spectral_window_ignores_other_bands_and_time_shifts():
    rng = np.random.default_rng(5)
    t = np.sort(rng.uniform(0, 900, 80))
    band = rng.integers(0, 10, 80).astype(np.int32)
    S = oracle.spectral_window(t, band, 4, 0.01, 1e-3, 700)
    S_shift = oracle.spectral_window(t + 4321.0, band, 4, 0.01, 1e-3, 700)
    np.testing.assert_allclose(S_shift, S, rtol=1e-8, atol=1e-9)
    only = band == 4
    S_alone = oracle.spectral_window(t[only], np.full(only.sum(), 4, np.int32), 4, 0.01, 1e-3, 700)
    np.testing.assert_allclose(S_alone, S, rtol=1e-12, atol=1e-12)
    assert np.all(S <= only.sum() ** 2 * (1 + 1e-12))


def _brute_trials(S, f_min, df, n_t):
    K = len(S)
    cand = []
    for k in range(K):
        left = k == 0 or S[k] > S[k - 1]
        right = k == K - 1 or S[k] >= S[k + 1]
        f = f_min + k * df
        one_day = f > 0 and abs(1.0 / f - 1.0) < 1e-4
        if left and right and not one_day:
            cand.append((-S[k], k))
    cand.sort()
    ks = [k for _, k in cand[:n_t]]
    return ks + [-1] * (n_t - len(ks))


@pytest.mark.parametrize("seed", range(6))
def test_window_trials_match_brute_force(seed):
    rng = np.random.default_rng(seed)
    K = int(rng.integers(1, 400))
    S = np.round(rng.uniform(0, 6, K)) * 1.5            # coarse values: plateaus and exact ties
    f_min, df = 0.9990, 1e-5                            # the grid crosses the one-day window
    for n_t in (1, 5, 40, 400):
        got = oracle.window_trials(S, f_min, df, n_t).tolist()
        assert got == _brute_trials(S, f_min, df, n_t)


def test_one_day_frequencies_are_left_out():
    assert oracle.is_one_day(1.0) and oracle.is_one_day(1.00009) and oracle.is_one_day(0.99991)
    assert not oracle.is_one_day(1.00011) and not oracle.is_one_day(0.9998) and not oracle.is_one_day(0.0)
    # nightly sampling: the window's highest local maximum sits at f = 1 and must not be chosen
    rng = np.random.default_rng(7)
    t = np.arange(300, dtype=np.float64) + rng.normal(0, 0.02, 300)
    band = np.zeros(300, np.int32)
    f_min, df, nk = 0.5, 1e-4, 10001                    # f = 1 is grid point 5000
    S = oracle.spectral_window(t, band, 0, f_min, df, nk)
    assert int(np.argmax(S)) in (4999, 5000, 5001)
    trials = oracle.window_trials(S, f_min, df, 10)
    for k in trials:
        assert not oracle.is_one_day(f_min + k * df)
    assert 5000 not in trials.tolist()


def test_bands_method_recovers_an_injected_period():
    """A clean eclipsing-like signal: the trial list contains the full-grid
    best frequency, so the bands search and the full search agree."""
    rng = np.random.default_rng(11)
    n = 240
    t = np.sort(synth.seasonal_times(rng, np.array([n]), 1000.0)[:n])
    P = 2.7183
    phase = (t / P) % 1.0
    y = 17.0 + 0.6 * np.exp(-0.5 * ((phase - 0.5) / 0.04) ** 2) + rng.normal(0, 0.02, n)
    e = np.full(n, 0.02)
    b = synth.Batch(times=t, mags=y.astype(np.float32), errs=e.astype(np.float32),
                    offsets=np.array([0, n], np.int64), period=np.array([P]), periodic=np.array([True]),
                    kind=np.array([0], np.int8))
    g = synth.Grid(0.02, 4e-4, 7451, bands=True, n_bands=3, trials_per_band=150)
    v = oracle.batch_nckp(b, 0.2, g.freqs())[0]           # the full grid, for comparison
    k_full = int(np.argmax(v))
    bands = oracle.batch_best(b, g, sigma_t=0.2)
    trials = oracle.batch_bands_trials(b, g)
    assert k_full in trials[0]
    assert bands["best_idx"][0] == k_full
    assert bands["best_stat"][0] == pytest.approx(v[k_full], rel=1e-12)
    f_best = bands["best_freq"][0]
    assert min(abs(f_best - r / P) for r in (1, 2, 3)) < 2 * 4e-4
