"""Pins of the oracle's spurious-period exclusion windows (Section 6.1,
Filtering of spurious periods; Table tab:spuriousperiods lists the periods,
the paper does not give its mask widths, so the caller supplies closed
frequency intervals).  The best period is the best admissible frequency;
the coarse-then-fine search also skips excluded coarse peaks; the bands
method's trial lists are unchanged and the windows filter the best trial.

Each pin recomputes the choice independently: numpy masks built from the
interval bounds, numpy argmax, and a brute-force local-maximum scan."""
import numpy as np
import pytest

import oracle
import synth


def mask(f, exclude):
    f = np.asarray(f, np.float64)
    m = np.zeros(f.shape, bool)
    for lo, hi in exclude:
        m |= (f >= lo) & (f <= hi)
    return m


def test_intervals_are_closed_and_compared_exactly():
    ex = [(0.25, 0.5), (2.0, 2.0)]
    assert oracle.is_excluded(0.25, ex) and oracle.is_excluded(0.5, ex) and oracle.is_excluded(2.0, ex)
    assert not oracle.is_excluded(np.nextafter(0.25, 0.0), ex)
    assert not oracle.is_excluded(np.nextafter(0.5, 1.0), ex)
    assert not oracle.is_excluded(np.nextafter(2.0, 3.0), ex)
    assert not oracle.is_excluded(1.0, [])


def test_full_grid_best_is_the_masked_argmax():
    b = synth.ragged_batch(4, seed=61, n_lo=30, n_hi=80, span=600.0)
    g0 = synth.Grid(0.05, 2.5e-3, 400)
    free = oracle.batch_best(b, g0, sigma_t=0.3)
    f = g0.freqs()
    for c in range(b.n_curves):
        fb = free["best_freq"][c]
        # a window around the unrestricted best, one ending exactly on a grid point, one elsewhere
        ex = ((fb - 0.01, fb + 0.012), (f[37], f[40]), (0.9, 0.95))
        g = synth.Grid(g0.f_min, g0.df, g0.n_freq, exclude=ex)
        r = oracle.batch_best(b.subset([c]), g, sigma_t=0.3)
        t, m, e = b.curve(c)
        v = oracle.nckp(t, m.astype(np.float64), oracle.median(e.astype(np.float64)), 0.3, f)
        vm = np.where(mask(f, ex), -np.inf, v)
        k = int(np.argmax(vm))
        assert r["best_idx"][0] == k and r["best_freq"][0] == f[k]
        assert r["best_stat"][0] == pytest.approx(v[k], rel=1e-13)
        assert not mask([r["best_freq"][0]], ex)[0]


def _brute_top_maxima(v, f, top_k, ex):
    """Local maxima v[k] > v[k-1], v[k] >= v[k+1] (ends: one neighbour), excluded
    frequencies skipped as candidates, the top_k by value (ties: lower k)."""
    n = len(v)
    cand = [k for k in range(n)
            if (k == 0 or v[k] > v[k - 1]) and (k == n - 1 or v[k] >= v[k + 1]) and not mask([f[k]], ex)[0]]
    return sorted(cand, key=lambda k: (-v[k], k))[:top_k]


def test_coarse_peaks_skip_excluded_candidates_by_brute_force():
    rng = np.random.default_rng(62)
    for trial in range(40):
        # ties and plateaus, also among the highest values
        v = np.round(rng.normal(size=120), 1) if trial % 2 else rng.integers(0, 5, size=120).astype(np.float64)
        f = 0.1 + np.arange(120) * 0.01
        ex = ((f[5], f[9]), (f[60] - 1e-9, f[60] + 1e-9), (2.0, 3.0))
        got = oracle.top_local_maxima_excl(v, 7, 0.1, 0.01, ex)
        want = _brute_top_maxima(v, 0.1 + np.arange(120) * 0.01, 7, ex)
        assert list(got) == want


def test_coarse_then_fine_with_windows_by_composition():
    b = synth.ragged_batch(3, seed=63, n_lo=30, n_hi=60, span=400.0)
    g0 = synth.Grid(0.01, 1e-3, 991, True, 5e-3, 3, 1e-3, 4e-3)     # f_max = 1.0
    free = oracle.batch_best(b, g0, sigma_t=0.3)
    kc = int(np.floor((g0.f_max - g0.f_min) / g0.coarse_df + 0.5)) + 1
    J = int(np.floor(g0.fine_halfwidth / g0.fine_df + 0.5))
    for c in range(b.n_curves):
        fb = free["best_freq"][c]
        ex = ((fb - 0.0025, fb + 0.0015), (0.5, 0.52))
        g = synth.Grid(g0.f_min, g0.df, g0.n_freq, True, 5e-3, 3, 1e-3, 4e-3, exclude=ex)
        r = oracle.batch_best(b.subset([c]), g, sigma_t=0.3)
        t, m, e = b.curve(c)
        y, sy = m.astype(np.float64), oracle.median(e.astype(np.float64))
        fc = g.f_min + np.arange(kc) * g.coarse_df
        peaks = _brute_top_maxima(oracle.nckp(t, y, sy, 0.3, fc), fc, g.top_k, ex)
        cand = [g.f_min + p * g.coarse_df + j * g.fine_df for p in peaks for j in range(-J, J + 1)]
        cand = np.array([x for x in cand if g.f_min <= x <= g.f_max and not mask([x], ex)[0]])
        v = oracle.nckp(t, y, sy, 0.3, cand)
        assert r["best_freq"][0] == cand[int(np.argmax(v))]
        assert not mask([r["best_freq"][0]], ex)[0]


def test_fine_candidates_inside_a_window_are_skipped():
    """Windows that cover every fine point around the best coarse peak except
    the peak's own coarse frequency: that peak stays a candidate, its excluded
    neighbours do not."""
    b = synth.ragged_batch(3, seed=67, n_lo=30, n_hi=60, span=400.0)
    g0 = synth.Grid(0.01, 1e-3, 991, True, 5e-3, 3, 1e-3, 4e-3)
    kc = int(np.floor((g0.f_max - g0.f_min) / g0.coarse_df + 0.5)) + 1
    J = int(np.floor(g0.fine_halfwidth / g0.fine_df + 0.5))
    hits = 0
    for c in range(b.n_curves):
        t, m, e = b.curve(c)
        y, sy = m.astype(np.float64), oracle.median(e.astype(np.float64))
        fc = g0.f_min + np.arange(kc) * g0.coarse_df
        vc = oracle.nckp(t, y, sy, 0.3, fc)
        fp = fc[oracle.top_local_maxima(vc, 1)[0]]
        h = 0.5 * g0.fine_df
        ex = ((fp + h, fp + J * g0.fine_df + h), (fp - J * g0.fine_df - h, fp - h))
        g = synth.Grid(g0.f_min, g0.df, g0.n_freq, True, 5e-3, 3, 1e-3, 4e-3, exclude=ex)
        r = oracle.batch_best(b.subset([c]), g, sigma_t=0.3)
        peaks = _brute_top_maxima(vc, fc, g.top_k, ex)
        cand = [g.f_min + p * g.coarse_df + j * g.fine_df for p in peaks for j in range(-J, J + 1)]
        cand = np.array([x for x in cand if g.f_min <= x <= g.f_max and not mask([x], ex)[0]])
        v = oracle.nckp(t, y, sy, 0.3, cand)
        assert r["best_freq"][0] == cand[int(np.argmax(v))]
        hits += r["best_freq"][0] == fp
    assert hits >= 1          # the setting does exercise the window (the peak's own point wins)


def test_bands_windows_filter_the_best_trial_only():
    b = synth.ragged_batch(3, seed=64, n_lo=60, n_hi=120, span=900.0)
    g0 = synth.Grid(0.01, 2e-3, 700, bands=True, n_bands=2, trials_per_band=6)
    free = oracle.batch_best(b, g0, sigma_t=0.3)
    for c in range(b.n_curves):
        fb = free["best_freq"][c]
        ex = ((fb - 1e-3, fb + 1e-3),)
        g = synth.Grid(g0.f_min, g0.df, g0.n_freq, bands=True, n_bands=2, trials_per_band=6, exclude=ex)
        t, m, e = b.curve(c)
        y = m.astype(np.float64)
        trials = oracle.bands_trials(t, y, g.f_min, g.df, g.n_freq, 2, 6).reshape(-1)
        ks = trials[trials >= 0]
        fr = g.f_min + ks * g.df
        v = oracle.nckp(t, y, oracle.median(e.astype(np.float64)), 0.3, fr)
        q = int(np.argmax(np.where(mask(fr, ex), -np.inf, v)))
        r = oracle.batch_best(b.subset([c]), g, sigma_t=0.3)
        assert r["best_idx"][0] == ks[q] and r["best_freq"][0] == fr[q]


def test_everything_excluded_gives_no_best():
    b = synth.ragged_batch(2, seed=65, n_lo=20, n_hi=30, span=300.0)
    for g in (synth.Grid(0.1, 0.01, 50, exclude=((0.0, 10.0),)),
              synth.Grid(0.1, 0.01, 50, True, 0.05, 2, 0.01, 0.02, exclude=((0.0, 10.0),))):
        r = oracle.batch_best(b, g, sigma_t=0.3)
        assert np.all(r["best_idx"] == -1) and np.all(np.isnan(r["best_freq"])) and not r["is_periodic"].any()


def test_spurious_period_window_recovers_the_true_period():
    """A curve whose strongest signal sits at the sidereal-day period 0.9973 d
    (Table tab:spuriousperiods) on top of a real 2.7 d variation: the search
    picks the spurious frequency; with windows around it and its
    sub-multiples (the period multiples 2P, 3P, which the statistic also
    rewards) it picks the real one."""
    rng = np.random.default_rng(66)
    t = np.sort(rng.uniform(0.0, 600.0, 150))
    y = 17.0 + 0.5 * np.sin(2 * np.pi * t / 0.9973) + 0.25 * np.sin(2 * np.pi * t / 2.7) + rng.normal(0, 0.02, 150)
    b = synth.Batch(t, y.astype(np.float32), np.full(150, 0.02, np.float32), np.array([0, 150], np.int64),
                    np.array([2.7]), np.array([True]), np.array([2], np.int8))
    g0 = synth.grid_from_range(0.1, 1.2, 2e-4)
    r0 = oracle.batch_best(b, g0, sigma_t=0.3)
    fs = 1 / 0.9973
    assert abs(r0["best_freq"][0] - fs) < 2e-4
    ex = tuple((fs / m - 4e-3, fs / m + 4e-3) for m in (1, 2, 3))
    g = synth.Grid(g0.f_min, g0.df, g0.n_freq, exclude=ex)
    r = oracle.batch_best(b, g, sigma_t=0.3)
    assert abs(r["best_freq"][0] - 1 / 2.7) < 2e-4
