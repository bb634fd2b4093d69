"""Pins for the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage it follows.  They are chosen so that a plausible
mistake in the oracle (a dropped IP subtraction, a missing factor 2 or pi, a
dropped diagonal, a wrong sign, a transposed operand, an off-by-one
quantile) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
import scipy.stats

import oracle
from oracle.series import taylor_harmonic_coefficients
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SQ2PI = math.sqrt(2 * math.pi)


def rnd_curve(n, seed, span=800.0):
    rng = np.random.default_rng(seed)
    t = np.sort(rng.uniform(0, span, n))
    y = 17 + 0.4 * rng.standard_normal(n)
    return t, y


# --- Eq. (Gausskernel) -----------------------------------------------------
@pytest.mark.parametrize("sigma", [0.02, 0.1, 1.0, 3.0])
def test_gauss_matches_normal_pdf(sigma):
    for x in [0.0, 0.3 * sigma, -1.7 * sigma, 5 * sigma]:
        assert oracle.gauss(x, sigma) == pytest.approx(scipy.stats.norm.pdf(x, scale=sigma), rel=1e-13)
    assert oracle.gauss(0.0, sigma) == pytest.approx(1.0 / (SQ2PI * sigma), rel=1e-15)


# --- Eq. (periodickernel) via the warp u_f of Eq. (warp) --------------------
@pytest.mark.parametrize("f,sigma", [(0.27, 0.1), (1.3, 0.45), (0.002, 0.6)])
def test_periodic_kernel_is_gaussian_of_warp(f, sigma):
    rng = np.random.default_rng(3)
    for _ in range(20):
        z, y = rng.uniform(0, 2000, 2)
        uz = np.array([np.cos(2 * np.pi * f * z), np.sin(2 * np.pi * f * z)])
        uy = np.array([np.cos(2 * np.pi * f * y), np.sin(2 * np.pi * f * y)])
        d2 = float(np.sum((uz - uy) ** 2))
        via_warp = math.exp(-d2 / (2 * sigma * sigma)) / (SQ2PI * sigma)
        assert oracle.periodic_kernel(f, z - y, sigma) == pytest.approx(via_warp, rel=1e-9, abs=1e-300)
        # period 1/f in the lag
        assert oracle.periodic_kernel(f, z - y + 3.0 / f, sigma) == pytest.approx(
            oracle.periodic_kernel(f, z - y, sigma), rel=1e-8, abs=1e-300)


def test_kernel_matrices_symmetric_unit_diagonal():
    t, y = rnd_curve(9, 1)
    sy, st, f = 0.2, 0.3, 0.37
    Gy = np.array([[oracle.gauss(a - b, sy) * SQ2PI * sy for b in y] for a in y])
    Gt = np.array([[oracle.periodic_kernel(f, a - b, st) * SQ2PI * st for b in t] for a in t])
    for M in (Gy, Gt):
        assert np.array_equal(M, M.T)
        assert np.all(np.diag(M) == 1.0)


# --- Eq. (HP), (IP), (CKP): closed forms ------------------------------------
@pytest.mark.parametrize("seed", range(5))
def test_ckp_two_points_closed_form(seed):
    rng = np.random.default_rng(seed)
    t = rng.uniform(0, 500, 2)
    y = rng.uniform(16, 18, 2)
    sy, st = rng.uniform(0.05, 0.5), rng.uniform(0.1, 0.6)
    freqs = rng.uniform(0.002, 5, 7)
    G0, Gd = 1 / (SQ2PI * sy), oracle.gauss(y[0] - y[1], sy)
    At = 1 / (SQ2PI * st)
    E = np.exp(-2 * np.sin(np.pi * freqs * (t[0] - t[1])) ** 2 / st ** 2)
    want = At / 4 * (G0 - Gd) * (1 - E)       # N = 2, diagonal included
    got = oracle.ckp(t, y, sy, st, freqs)
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-15)
    ip = (G0 + Gd) / 2
    assert oracle.information_potential(y, sy) == pytest.approx(ip, rel=1e-14)
    np.testing.assert_allclose(oracle.nckp(t, y, sy, st, freqs), np.sqrt(2 * st) / ip * want, rtol=1e-11, atol=1e-15)


def test_ckp_zero_frequency_is_zero():
    t, y = rnd_curve(40, 2)
    v = oracle.ckp(t, y, 0.15, 0.3, [0.0])
    g = np.array([[oracle.gauss(a - b, 0.15) for b in y] for a in y])
    assert abs(v[0]) < 1e-13 * g.sum() / 40 ** 2


def test_ckp_integer_lattice_is_zero():
    rng = np.random.default_rng(4)
    t = np.sort(rng.choice(np.arange(0, 300), 25, replace=False)).astype(float)
    y = 17 + 0.3 * rng.standard_normal(25)
    v = oracle.ckp(t, y, 0.1, 0.2, [1.0, 2.0, 3.0])
    assert np.all(np.abs(v) < 1e-12)


def test_ckp_constant_magnitudes_is_zero():
    t, _ = rnd_curve(30, 5)
    y = np.full(30, 17.25)
    assert oracle.information_potential(y, 0.1) == pytest.approx(1 / (SQ2PI * 0.1), rel=1e-14)
    scale = (1 / (SQ2PI * 0.1)) * (1 / (SQ2PI * 0.3))
    assert np.all(np.abs(oracle.ckp(t, y, 0.1, 0.3, [0.1, 0.37, 2.5])) < 1e-13 * scale)


def test_invariances_shift_offset_permutation():
    t, y = rnd_curve(35, 6)
    f = np.array([0.013, 0.27, 1.9])
    base = oracle.nckp(t, y, 0.12, 0.25, f)
    np.testing.assert_allclose(oracle.nckp(t + 2451234.5, y, 0.12, 0.25, f), base, rtol=1e-6)
    np.testing.assert_allclose(oracle.nckp(t + 123.25, y, 0.12, 0.25, f), base, rtol=1e-10)
    np.testing.assert_allclose(oracle.nckp(t, y - 3.5, 0.12, 0.25, f), base, rtol=1e-10)
    p = np.random.default_rng(0).permutation(35)
    np.testing.assert_allclose(oracle.nckp(t[p], y[p], 0.12, 0.25, f), base, rtol=1e-10)


# --- Eq. (taylor): harmonic series of the periodic kernel -------------------
@pytest.mark.parametrize("st,nm", [(0.1, 100), (0.2, 50), (0.45, 30)])
def test_ckp_equals_taylor_harmonic_series(st, nm):
    """The direct CKP equals sum_m b_m C_m(f), C_m = sum_ij W_ij cos(2 pi m f dt_ij),
    with b_m from the paper's own series, Eq. (taylor), summed exactly."""
    t, y = rnd_curve(23, 7)
    sy = 0.2
    b = np.array(taylor_harmonic_coefficients(st, nm))
    assert b[0] + b[1:].sum() == pytest.approx(1.0, abs=1e-12)       # dt = 0 gives the kernel peak
    ip = oracle.information_potential(y, sy)
    W = np.array([[oracle.gauss(a - c, sy) - ip for c in y] for a in y])
    dt = np.subtract.outer(t, t)
    for f in [0.011, 0.31, 2.2]:
        C = np.array([np.sum(W * np.cos(2 * np.pi * m * f * dt)) for m in range(nm + 1)])
        via_series = (b @ C) / (SQ2PI * st) / len(t) ** 2
        assert oracle.ckp(t, y, sy, st, [f])[0] == pytest.approx(via_series, rel=1e-10, abs=1e-14)


def test_large_sigma_t_limit_is_cosine_periodogram():
    """Section 2.1: for large sigma_t the periodic kernel tends to a constant
    plus cos(2 pi f dt); with sum W = 0 the CKP tends to a W-weighted cosine
    periodogram: sigma_t^2 * CKP / A_t -> (1/N^2) sum W_ij cos(2 pi f dt_ij)."""
    t, y = rnd_curve(21, 8)
    sy, st = 0.3, 1e3
    ip = oracle.information_potential(y, sy)
    W = np.array([[oracle.gauss(a - c, sy) - ip for c in y] for a in y])
    dt = np.subtract.outer(t, t)
    for f in [0.05, 0.8]:
        lim = np.sum(W * np.cos(2 * np.pi * f * dt)) / 21 ** 2
        got = oracle.ckp(t, y, sy, st, [f])[0] * st ** 2 * (SQ2PI * st)
        assert got == pytest.approx(lim, rel=1e-5, abs=1e-9)


def test_independent_numpy_evaluation_small():
    """A second, independent evaluation (NumPy outer differences) on small N."""
    t, y = rnd_curve(48, 9)
    sy, st = 0.17, 0.33
    f = np.linspace(0.01, 3.0, 41)
    dy = np.subtract.outer(y, y)
    dt = np.subtract.outer(t, t)
    G = np.exp(-dy ** 2 / (2 * sy ** 2)) / (SQ2PI * sy)
    ip = G.mean()
    want = np.array([np.mean((G - ip) * np.exp(-2 * np.sin(np.pi * fk * dt) ** 2 / st ** 2) / (SQ2PI * st))
                     for fk in f]) * np.sqrt(48 * st) / ip
    np.testing.assert_allclose(oracle.nckp(t, y, sy, st, f), want, rtol=1e-11, atol=1e-13)


# --- order statistics, Eq. (pavlosrule), Eq. (pSNR), sigma_t rule ------------
@pytest.mark.parametrize("n", [1, 2, 3, 10, 11, 1000])
def test_median_quantile_match_numpy(n):
    x = np.random.default_rng(n).standard_normal(n)
    assert oracle.median(x) == np.median(x)
    for q in (0.25, 0.5, 0.75):
        assert oracle.quantile(x, q) == pytest.approx(np.percentile(x, 100 * q), rel=1e-15, abs=1e-15)


def test_psnr_known_values():
    y = np.arange(1.0, 10.0)            # 1..9: Q1 = 3, Q3 = 7 (linear), iqr = 4
    e = np.array([0.5, 0.1, 0.2, 0.2, 0.3, 0.2, 0.9, 0.2, 0.4])   # median 0.2
    assert oracle.psnr(y, e, 1.0) == pytest.approx(0.7413 * 4 / 0.2, rel=1e-14)
    assert oracle.psnr(y, e, 0.42) == pytest.approx(0.7413 * 4 / (0.42 * 0.2), rel=1e-14)


def test_bowley_skewness_and_sigma_t_rule():
    assert oracle.bowley_skewness(np.arange(1.0, 9.0)) == 0.0
    assert oracle.sigma_t_rule(np.arange(1.0, 9.0)) == pytest.approx(0.6, abs=1e-15)
    # [1,1,1,1,2,10]: halves [1,1,1] and [1,2,10] -> Q1 = 1, Q3 = 2, Q2 = 1 -> S = 1
    assert oracle.bowley_skewness(np.array([1, 1, 1, 1, 2, 10.0])) == pytest.approx(1.0)
    assert oracle.sigma_t_rule(np.array([1, 1, 1, 1, 2, 10.0])) == pytest.approx(0.1 + 0.5 * math.exp(-12), rel=1e-14)
    # odd N, middle excluded: [1,2,3,4,100] -> Q1 = 1.5, Q3 = 52, Q2 = 3
    S = (52 + 1.5 - 6) / 50.5
    assert oracle.bowley_skewness(np.array([1, 2, 3, 4, 100.0])) == pytest.approx(S, rel=1e-14)
    # the rule at an S other than 0 and +-1 (where S and S^2 agree)
    assert oracle.sigma_t_rule(np.array([1, 2, 3, 4, 100.0])) == pytest.approx(0.1 + 0.5 * math.exp(-12 * S * S),
                                                                                rel=1e-14)
    # mirrored data flips the sign; constant data gives 0 (Q3 == Q1)
    x = np.random.default_rng(1).lognormal(size=101)
    assert oracle.bowley_skewness(-x) == pytest.approx(-oracle.bowley_skewness(x), rel=1e-14)
    assert oracle.bowley_skewness(np.full(7, 2.0)) == 0.0


# --- Table tab:th ------------------------------------------------------------
def load_thresholds():
    rows = []
    for line in open(os.path.join(GOLDEN, "thresholds_tab_th.txt")):
        if line.startswith("#") or not line.strip():
            continue
        lo, hi, th = line.split()[:3]
        rows.append((float(lo), float(hi), float(th)))
    return rows


def test_threshold_table_from_paper():
    rows = load_thresholds()
    assert len(rows) == 8
    for b, (lo, hi, th) in enumerate(rows):
        for p in [lo, lo + 1e-9, (lo + min(hi, lo + 5)) / 2, np.nextafter(hi, -np.inf) if np.isfinite(hi) else 1e9]:
            assert oracle.snr_bin(p) == b
            assert oracle.threshold(p) == th


# --- best period, local maxima -------------------------------------------------
def test_argmax_ties_lowest_index():
    assert oracle.argmax([1.0, 3.0, 2.0, 3.0]) == 1
    assert oracle.argmax([0.0, 0.0, 0.0]) == 0


def brute_local_maxima(v, k):
    n = len(v)
    idx = [i for i in range(n) if (i == 0 or v[i] > v[i - 1]) and (i == n - 1 or v[i] >= v[i + 1])]
    idx.sort(key=lambda i: (-v[i], i))
    return idx[:k]


def test_top_local_maxima_brute_force():
    assert list(oracle.top_local_maxima([0, 2, 1, 3, 3, 0, 5], 10)) == [6, 3, 1]
    assert list(oracle.top_local_maxima([5, 5, 5], 3)) == [0]
    assert list(oracle.top_local_maxima([1.0], 4)) == [0]
    rng = np.random.default_rng(11)
    for trial in range(200):
        n = int(rng.integers(1, 60))
        v = rng.integers(0, 6, n).astype(float)   # many ties
        k = int(rng.integers(1, 12))
        assert list(oracle.top_local_maxima(v, k)) == brute_local_maxima(list(v), k)


def test_hierarchical_reduces_to_full_grid():
    """With coarse step = fine step = df and top_k covering every maximum, the
    coarse-then-fine search returns the full-grid best frequency and value."""
    b = synth.ragged_batch(3, seed=12, n_lo=20, n_hi=40, span=300.0)
    g = synth.grid_from_range(0.01, 1.0, 0.01)
    full = oracle.batch_best(b, g, sigma_t=0.3)
    gh = synth.Grid(g.f_min, g.df, g.n_freq, True, g.df, 200, g.df, 2 * g.df)
    hier = oracle.batch_best(b, gh, sigma_t=0.3)
    np.testing.assert_allclose(hier["best_freq"], full["best_freq"], rtol=0, atol=1e-12)
    # the two routes reach the same grid frequency up to one FP64 ulp (f_min + k df versus
    # f_peak + j fine_df); over a 300-day span that ulp moves nCKP by ~1e-13 relative
    np.testing.assert_allclose(hier["best_stat"], full["best_stat"], rtol=1e-12)


def test_hierarchical_search_by_brute_force():
    """Coarse-then-fine search with a fine step finer than the coarse one: the
    result equals the search composed by hand from pinned pieces -- nCKP on the
    coarse grid, its top-k local maxima, windows of +-round(halfwidth / fine_df)
    fine steps clipped to [f_min, f_max], the best value over all windows."""
    b = synth.ragged_batch(3, seed=13, n_lo=30, n_hi=60, span=400.0)
    g = synth.Grid(0.01, 1e-3, 991, True, 5e-3, 3, 1e-3, 4e-3)     # f_max = 1.0
    r = oracle.batch_best(b, g, sigma_t=0.3)
    kc = int(np.floor((g.f_max - g.f_min) / g.coarse_df + 0.5)) + 1
    J = int(np.floor(g.fine_halfwidth / g.fine_df + 0.5))
    assert J == 4
    for c in range(b.n_curves):
        t, m, e = b.curve(c)
        y, sy = m.astype(np.float64), oracle.median(e.astype(np.float64))
        fc = g.f_min + np.arange(kc) * g.coarse_df
        peaks = oracle.top_local_maxima(oracle.nckp(t, y, sy, 0.3, fc), g.top_k)
        cand = [g.f_min + p * g.coarse_df + j * g.fine_df for p in peaks for j in range(-J, J + 1)]
        cand = np.array([f for f in cand if g.f_min <= f <= g.f_max])
        v = oracle.nckp(t, y, sy, 0.3, cand)
        assert r["best_freq"][c] == cand[int(np.argmax(v))]
        assert r["best_stat"][c] == pytest.approx(v.max(), rel=1e-13)


def test_batch_nckp_equals_single_curve_nckp():
    """The batch evaluation (per-curve sigma_t, float32 inputs widened) is the
    single-curve Eq. (CKP) evaluation curve by curve."""
    b = synth.ragged_batch(4, seed=14, n_lo=2, n_hi=50, span=600.0)
    st = np.array([0.15, 0.3, 0.45, 0.6])
    fr = np.linspace(0.01, 2.0, 37)
    got = oracle.batch_nckp(b, st, fr)
    for c in range(b.n_curves):
        t, m, e = b.curve(c)
        ref = oracle.nckp(t, m.astype(np.float64), oracle.median(e.astype(np.float64)), st[c], fr)
        np.testing.assert_allclose(got[c], ref, rtol=1e-13, atol=1e-15)


def test_noiseless_sinusoid_recovered_within_one_step():
    """A noiseless 3.7 d sinusoid on the 150-point seasonal sampling peaks
    within one grid step of 1/3.7 on the 0.002-2.0, 2e-4 grid."""
    b = synth.single_curve(seed=0, noise=0.0)
    g = synth.grid_from_range(0.002, 2.0, 2e-4)
    assert g.n_freq == 9991
    r = oracle.batch_best(b, g, sigma_t=0.3)
    assert abs(r["best_freq"][0] - 1 / 3.7) <= g.df


def test_noisy_single_curve_recovered():
    b, g = synth.workload_single()
    r = oracle.batch_best(b, g, sigma_t=0.3)
    assert abs(r["best_freq"][0] - 1 / 3.7) <= g.df
    assert r["is_periodic"][0]
