"""Pins of the oracle's whitening (Section 7.1, multimodes): fold at P0, a
moving average of 30 folded samples as the template, subtract it, samples
back in time order -- against closed forms and invariants."""
import numpy as np
import pytest

import oracle


def test_constant_curve_whitens_to_zero():
    t = np.sort(np.random.default_rng(0).uniform(0, 900, 120))
    out = oracle.whiten(t, np.full(120, 17.25), 3.1)
    assert np.max(np.abs(out)) < 1e-12


@pytest.mark.parametrize("n,w", [(200, 30), (90, 30), (64, 16)])
def test_sinusoid_on_a_uniform_fold_matches_the_dirichlet_kernel(n, w):
    """Phases k/N (any order in time): the circular average of w samples over
    positions k - w/2 .. k - w/2 + w - 1 of A sin(2 pi k/N) is
    A D sin(2 pi (k + c)/N) with D = sin(pi w/N) / (w sin(pi/N)) and centre
    offset c = (w - 1)/2 - w/2."""
    P, A = 2.7, 0.6
    rng = np.random.default_rng(1)
    k = rng.permutation(n)                            # samples in a scrambled time order
    t = (k + 17 * n) * P / n + 1e-9                   # phase k/N (plus a tiny offset, no ties)
    x = A * np.sin(2 * np.pi * k / n)
    out = oracle.whiten(t, x, P, w)
    D = np.sin(np.pi * w / n) / (w * np.sin(np.pi / n))
    c = (w - 1) / 2.0 - w // 2
    want = x - A * D * np.sin(2 * np.pi * (k + c) / n)
    np.testing.assert_allclose(out, want, atol=1e-9)


def test_output_follows_the_input_order_and_is_linear():
    rng = np.random.default_rng(2)
    n = 150
    t = np.sort(rng.uniform(0, 2000, n))
    x = 17 + 0.3 * np.sin(2 * np.pi * t / 4.3) + rng.normal(0, 0.05, n)
    out = oracle.whiten(t, x, 4.3)
    perm = rng.permutation(n)
    np.testing.assert_allclose(oracle.whiten(t[perm], x[perm], 4.3), out[perm], rtol=0, atol=1e-12)
    np.testing.assert_allclose(oracle.whiten(t, 2.5 * x - 4.0, 4.3), 2.5 * out, atol=1e-12)
    # the periodic signal is removed: what is left is close to the noise
    assert np.std(out) < 0.5 * np.std(x)


def test_short_curve_uses_all_samples():
    t = np.array([0.1, 0.5, 1.3, 2.2])
    x = np.array([1.0, 2.0, 4.0, 8.0])
    np.testing.assert_allclose(oracle.whiten(t, x, 1.0), x - x.mean(), atol=1e-15)


def test_batch_whitening_matches_single_curves_and_passes_bad_periods_through():
    """The batch driver against the pinned single-curve whitening: every
    curve of a ragged CSR batch lands at its own offsets, and a curve whose
    period is <= 0, NaN or infinite comes back unchanged (FP32 magnitudes
    widened exactly)."""
    import synth
    rng = np.random.default_rng(3)
    sizes = [45, 7, 120, 31, 2, 66, 30, 89]
    t_parts, m_parts = [], []
    for n in sizes:
        t = np.sort(rng.uniform(0.0, 1500.0, n))
        t_parts.append(t)
        m_parts.append((16.0 + 0.4 * np.sin(2 * np.pi * t / 3.3) + rng.normal(0, 0.05, n)).astype(np.float32))
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    b = synth.Batch(np.concatenate(t_parts), np.concatenate(m_parts), np.ones(off[-1], np.float32), off,
                    np.zeros(len(sizes)), np.zeros(len(sizes), bool), np.zeros(len(sizes), np.int8))
    p0 = np.array([3.3, 0.0, 7.9, -2.0, 1.1, np.nan, np.inf, 0.61])
    out = oracle.batch_whiten(b, p0, w=30)
    assert out.shape == (off[-1],)
    for c, n in enumerate(sizes):
        t, m, _ = b.curve(c)
        got = out[off[c]:off[c + 1]]
        if p0[c] > 0 and np.isfinite(p0[c]):
            np.testing.assert_array_equal(got, oracle.whiten(t, m.astype(np.float64), p0[c], 30))
            assert n < 3 or np.any(got != m)
        else:
            np.testing.assert_array_equal(got, m.astype(np.float64))
