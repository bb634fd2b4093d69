"""Parity of the device preprocessing (Section 5.2) and whitening
(Section 7.1) with the FP64 oracle, and the two-level multimode search."""
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


def dirty_batch(seed=51):
    """Curves with error-bar outliers, strong linear trends on every third
    curve, and sizes around the 50-sample limit (some discarded after the cut)."""
    rng = np.random.default_rng(seed)
    sizes = np.array([45, 49, 50, 51, 52, 53, 55, 60, 120, 300, 500, 700, 64, 200, 333, 999, 51, 52, 54, 410])
    t = synth.seasonal_times(rng, sizes, 2500.0)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    m = 17.0 + 0.2 * np.sin(2 * np.pi * t / 3.3) + rng.normal(0, 0.05, t.shape[0])
    e = rng.uniform(0.03, 0.08, t.shape[0])
    for c in range(len(sizes)):
        a, z = off[c], off[c + 1]
        n = z - a
        bad = rng.choice(n, size=max(1, n // 25), replace=False)
        e[a + bad] *= rng.uniform(8, 20, bad.size)
        if c % 3 == 0:
            m[a:z] += rng.choice([-1, 1]) * rng.uniform(1e-3, 3e-3) * (t[a:z] - t[a])
    return synth.Batch(t, m.astype(np.float32), e.astype(np.float32), off, np.zeros(len(sizes)),
                       np.zeros(len(sizes), bool), np.zeros(len(sizes), np.int8))


def test_preprocess_matches_oracle():
    b = dirty_batch()
    ot, ox, oe, oo, res = oracle.batch_preprocess(b)
    d = cp.cp_preprocess(torch.from_numpy(b.times).cuda(), torch.from_numpy(b.mags).cuda(),
                         torch.from_numpy(b.errs).cuda(), b.offsets)
    flags = d["flags"]
    np.testing.assert_array_equal(d["offsets_all"], oo)
    np.testing.assert_array_equal(flags & 1, np.array([r["kept"] for r in res], np.uint8))
    for c, r in enumerate(res):
        if r["kept"] and abs(r["r"] - 0.5) > 1e-9:
            assert bool(flags[c] & 2) == bool(r["detrended"]), c
        np.testing.assert_allclose(d["fit"][c], [r["a0"], r["a1"], r["r"]], rtol=1e-9, atol=1e-12)
    assert any(not r["kept"] for r in res) and any(r["detrended"] for r in res)
    np.testing.assert_array_equal(d["times"].cpu().numpy(), ot)
    np.testing.assert_array_equal(d["errs"].cpu().numpy(), oe.astype(np.float32))
    np.testing.assert_allclose(d["mags"].cpu().numpy(), ox, rtol=0, atol=4e-6 * max(1.0, np.abs(ox).max()))
    # the kept-curve CSR plans directly
    kept = d["curve"]
    assert d["offsets"][-1] == d["times"].shape[0] and len(d["offsets"]) == len(kept) + 1
    with cp.Plan(d["times"], d["mags"], d["errs"], d["offsets"], cp.make_grid(0.01, 1e-3, 500)) as p:
        best = p.best_period()
    assert np.all(best["best_idx"] >= 0)


def test_whiten_matches_oracle():
    b = synth.ragged_batch(16, seed=52, n_lo=30, n_hi=900)
    rng = np.random.default_rng(52)
    p0 = rng.uniform(0.3, 40.0, b.n_curves)
    p0[3] = 0.0                                      # copied unchanged
    ref = oracle.batch_whiten(b, p0)
    out = cp.cp_whiten(torch.from_numpy(b.times).cuda(), torch.from_numpy(b.mags).cuda(), b.offsets, p0)
    got = out.cpu().numpy()
    np.testing.assert_allclose(got, ref, rtol=0, atol=4e-6 * np.abs(b.mags).max())
    a, z = b.offsets[3], b.offsets[4]
    np.testing.assert_array_equal(got[a:z], b.mags[a:z])
    # in place
    mags = torch.from_numpy(b.mags).cuda()
    cp.cp_whiten(torch.from_numpy(b.times).cuda(), mags, b.offsets, p0, out=mags)
    np.testing.assert_array_equal(mags.cpu().numpy(), got)


def test_two_level_search_finds_the_second_mode():
    """A double-mode curve: the search finds P0; after whitening at P0 it
    finds P1 (Section 7.1)."""
    rng = np.random.default_rng(53)
    n = 900
    t = np.sort(synth.seasonal_times(rng, np.array([n]), 2500.0)[:n])
    P0, P1 = 0.71, 3.37
    y = 17 + 0.5 * np.sin(2 * np.pi * t / P0) + 0.2 * np.sin(2 * np.pi * t / P1 + 1.0) + rng.normal(0, 0.03, n)
    e = np.full(n, 0.03, np.float32)
    off = np.array([0, n], np.int64)
    g = cp.make_grid(0.05, 2e-4, 9751)               # 0.05 .. 2.0 1/d
    td, md, ed = (torch.from_numpy(t).cuda(), torch.from_numpy(y.astype(np.float32)).cuda(),
                  torch.from_numpy(e).cuda())
    with cp.Plan(td, md, ed, off, g, sigma_t=0.4) as p:
        f0 = p.best_period()["best_freq"][0]
    assert abs(f0 - 1 / P0) < 3e-4
    w = cp.cp_whiten(td, md, off, [1.0 / f0])
    with cp.Plan(td, w, ed, off, g, sigma_t=0.4) as p:
        f1 = p.best_period()["best_freq"][0]
    assert abs(f1 - 1 / P1) < 3e-4, (f1, 1 / P1)
