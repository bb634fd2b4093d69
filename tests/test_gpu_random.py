"""Randomised parity: small seeded batches with random sizes, time spans,
grids (including f_min = 0 and a single frequency), duplicated times and
sigma_t, through both forms of the pair sum, against the FP64 oracle.

The bar is the one of the other parity tests: per curve, peak-relative nCKP
error <= 1e-5 (direct FP32 form) and <= 1e-3 (tensor form, FP16 operands,
harmonics per curve; BF16 with both operands split on every third case), and
the c16 acceptance of the best index.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1412_1840_gb300 as cp  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def random_case(seed):
    rng = np.random.default_rng(seed)
    n_curves = int(rng.integers(1, 7))
    sizes = np.where(rng.uniform(size=n_curves) < 0.4, rng.integers(2, 41, n_curves),
                     rng.integers(41, 401, n_curves)).astype(np.int64)
    span = float(rng.choice([5.0, 100.0, 2500.0]))
    ts, ys, es = [], [], []
    for n in sizes:
        t = np.sort(rng.uniform(0.0, span, n))
        if n > 4 and rng.uniform() < 0.3:           # a few repeated epochs (pairs with dt = 0)
            k = int(rng.integers(1, max(2, n // 4)))
            src = rng.integers(0, n, k)
            dst = rng.integers(0, n, k)
            t[dst] = t[src]
            t = np.sort(t)
        ts.append(t)
        ys.append(15.0 + rng.normal(0.0, rng.uniform(0.01, 1.0), n))
        es.append(rng.uniform(0.005, 0.2, n))
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    b = synth.Batch(np.concatenate(ts), np.concatenate(ys).astype(np.float32), np.concatenate(es).astype(np.float32),
                    off, np.zeros(n_curves), np.zeros(n_curves, bool), np.zeros(n_curves, np.int8))
    f_min = 0.0 if rng.uniform() < 0.2 else float(rng.uniform(0.001, 3.0))
    df = float(10.0 ** rng.uniform(-5, -2))
    n_freq = 1 if rng.uniform() < 0.1 else int(rng.integers(2, 701))
    g = synth.Grid(f_min, df, n_freq)
    sigma_t = float(rng.uniform(0.1, 0.7))   # 0.1: the sigma_t rule's floor (48 harmonics)
    return b, g, sigma_t


def periodogram(b, g, **kw):
    with cp.Plan(b.times, b.mags, b.errs, b.offsets, cp.grid_from(g), **kw) as p:
        out = torch.empty((b.n_curves, g.n_freq), dtype=torch.float32, device="cuda")
        p.periodogram(out)
        p.sync()
        best = p.best_period()
    return out.cpu().numpy(), best


def check(out, best, ref, tol, tag):
    for c in range(ref.shape[0]):
        scale = np.max(np.abs(ref[c]))
        if scale == 0.0:
            assert np.all(out[c] == 0.0), tag
            continue
        err = np.max(np.abs(out[c] - ref[c])) / scale
        assert err <= tol, (tag, c, err)
        k, kstar = int(best["best_idx"][c]), int(np.argmax(ref[c]))
        assert ref[c, k] >= ref[c, kstar] - tol * abs(ref[c, kstar]), (tag, c, k, kstar)


@pytest.mark.parametrize("seed", range(24))
def test_random_batches_both_forms(seed):
    b, g, sigma_t = random_case(1000 + seed)
    st = float(np.float32(sigma_t))
    ref = oracle.batch_nckp(b, np.full(b.n_curves, st), g.freqs())
    out, best = periodogram(b, g, sigma_t=sigma_t)
    check(out, best, ref, 1e-5, "direct seed %d" % seed)
    out, best = periodogram(b, g, sigma_t=sigma_t, form=cp.CP_FORM_TENSOR, n_max=0)
    check(out, best, ref, 1e-3, "tensor seed %d" % seed)
    if seed % 3 == 0:   # BF16 with both operands split, on every third case
        out, best = periodogram(b, g, sigma_t=sigma_t, form=cp.CP_FORM_TENSOR, n_max=0,
                                dtype=cp.CP_DTYPE_BF16_SPLIT)
        check(out, best, ref, 1e-3, "tensor bf16 split seed %d" % seed)


@pytest.mark.parametrize("seed", range(12))
def test_random_bands_trial_lists(seed):
    """Bands method on random batches and grids (1-4 kept bands, 1-200 trials
    per band, grids of 50-20,000 points): the trial lists are index work and
    must equal the oracle's entry by entry wherever the oracle's band order is
    decided (its derivative sums separated)."""
    rng = np.random.default_rng(5000 + seed)
    b, _, _ = random_case(5000 + seed)
    n_bands = int(rng.integers(1, 5))
    n_t = int(rng.integers(1, 201))
    f_min = float(rng.uniform(0.0005, 1.0))
    df = float(10.0 ** rng.uniform(-4.5, -2.5))
    n_freq = int(rng.integers(50, 20001))
    g = synth.Grid(f_min, df, n_freq, bands=True, n_bands=n_bands, trials_per_band=n_t)
    with cp.Plan(b.times, b.mags, b.errs, b.offsets, cp.grid_from(g), sigma_t=0.3) as p:
        p.best_period()
        idx = p.trials()["trial_idx"].astype(np.int64)
    ref = oracle.batch_bands_trials(b, g)
    checked = 0
    for c in range(b.n_curves):
        t, m, _ = b.curve(c)
        y = m.astype(np.float64)
        D = np.sort(oracle.band_derivative_sums(t, y, oracle.bands_of(y)))[::-1]
        if not all(D[q] - D[q + 1] > 1e-9 * max(D[0], 1e-300) or D[q] == D[q + 1] == 0.0
                   for q in range(min(n_bands, 9))):
            continue
        np.testing.assert_array_equal(idx[c], ref[c], err_msg="seed %d curve %d" % (seed, c))
        checked += 1
    assert checked > 0 or b.n_curves == 0
