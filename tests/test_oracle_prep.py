"""Pins of the oracle's preprocessing (Section 5.2): error-bar cut
e_i < mean(e) + 3 std(e), discard below 50 samples, weighted linear chi^2
fit of Eq. (chisquare) removed when corr(x, fit) > 0.5 -- against closed
forms and independent library routines."""
import numpy as np
import pytest

import oracle
import synth


def test_error_bar_cut_closed_form():
    e = np.array([1.0] * 20 + [20.0])
    t = np.arange(21, dtype=np.float64)
    x = np.zeros(21)
    ot, ox, oe, r = oracle.preprocess(t, x, e, min_n=1)
    m = 40.0 / 21.0
    sd = np.sqrt((20 * (1 - m) ** 2 + (20 - m) ** 2) / 21.0)     # population standard deviation
    assert r["e_mean"] == pytest.approx(m, rel=1e-15)
    assert r["e_std"] == pytest.approx(sd, rel=1e-14)
    assert r["n_out"] == 20 and np.all(oe == 1.0) and np.array_equal(ot, t[:20])


def test_cut_keeps_sample_order_and_values():
    rng = np.random.default_rng(1)
    n = 300
    t = np.sort(rng.uniform(0, 1000, n))
    x = rng.normal(17, 0.1, n)
    e = rng.uniform(0.05, 0.1, n)
    bad = [7, 100, 250]
    e[bad] = 3.0
    ot, ox, oe, r = oracle.preprocess(t, x, e)
    keep = np.ones(n, bool)
    keep[bad] = False
    assert np.array_equal(ot, t[keep]) and np.array_equal(oe, e[keep])
    if not r["detrended"]:
        assert np.array_equal(ox, x[keep])


@pytest.mark.parametrize("n,kept", [(49, 0), (50, 1), (51, 1)])
def test_discard_below_fifty(n, kept):
    t = np.arange(n, dtype=np.float64)
    _, _, _, r = oracle.preprocess(t, np.sin(t), np.full(n, 0.1))
    assert r["n_out"] == n and r["kept"] == kept


def test_chi2_line_matches_weighted_least_squares():
    rng = np.random.default_rng(2)
    n = 200
    t = np.sort(rng.uniform(0, 2500, n))
    e = rng.uniform(0.02, 0.3, n)
    x = 16.0 - 3e-4 * t + rng.normal(0, 1, n) * e
    a0, a1 = oracle.chi2_line(t, x, e)
    p1, p0 = np.polyfit(t, x, 1, w=1.0 / e)        # minimises sum ((x - p(t)) / e)^2
    assert a1 == pytest.approx(p1, rel=1e-9) and a0 == pytest.approx(p0, rel=1e-12)


def test_pearson_matches_numpy():
    rng = np.random.default_rng(3)
    u, v = rng.normal(size=77), rng.normal(size=77)
    v += 0.4 * u
    assert oracle.pearson(u, v) == pytest.approx(np.corrcoef(u, v)[0, 1], rel=1e-12)
    assert oracle.pearson(u, np.full(77, 2.0)) == 0.0


@pytest.mark.parametrize("slope", [4e-4, -4e-4])
def test_noiseless_trend_is_removed_for_either_sign(slope):
    t = np.linspace(0, 2500, 120)
    x = 17.0 + slope * t
    ot, ox, oe, r = oracle.preprocess(t, x, np.full(120, 0.05))
    assert r["r"] == pytest.approx(1.0, abs=1e-12) and r["detrended"] == 1
    assert np.max(np.abs(ox)) < 1e-9
    assert r["a1"] == pytest.approx(slope, rel=1e-9) and r["a0"] == pytest.approx(17.0, rel=1e-12)


def test_flat_noise_is_not_detrended():
    rng = np.random.default_rng(4)
    t = np.sort(rng.uniform(0, 2500, 400))
    x = rng.normal(17.0, 0.2, 400)
    ot, ox, oe, r = oracle.preprocess(t, x, np.full(400, 0.2))
    assert abs(r["r"]) < 0.5 and r["detrended"] == 0
    assert np.array_equal(ox, x)


def test_batch_offsets_and_discarded_curves():
    b = synth.ragged_batch(6, seed=5, n_lo=40, n_hi=120)
    ot, ox, oe, oo, res = oracle.batch_preprocess(b)
    for c in range(b.n_curves):
        t, m, e = b.curve(c)
        tt, xx, ee, r = oracle.preprocess(t, m.astype(np.float64), e.astype(np.float64))
        assert res[c] == r
        if r["kept"]:
            assert np.array_equal(ot[oo[c]:oo[c + 1]], tt) and np.array_equal(ox[oo[c]:oo[c + 1]], xx)
        else:
            assert oo[c + 1] == oo[c]
    assert any(not r["kept"] for r in res) and any(r["kept"] for r in res)
