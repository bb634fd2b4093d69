"""Seeded synthetic lightcurve batches shaped like the paper's workload.

This module is shared by the tests, the oracle-driven checks and ``bench.py``.
It holds no arithmetic of the periodogram itself: it only draws observation
times, magnitudes and error bars, and writes frequency-grid descriptions.

Shapes follow the paper's data description: seasonal sampling over a
multi-year baseline (EROS-2 spans about 2500 days, Section "Efficiency as a
function of parameters"), mean sample counts of a few hundred per curve
(Section "Description of the data"), periods between 0.2 and 1000 days
(Section "Synthetic lightcurves"), and per-point Gaussian errors.  The
signal-to-noise scaling of the two-band throughput batch follows the
synthetic-set recipe of Section "Synthetic lightcurves" (step 6:
Y = S * med(e) / (0.7413 * iqr(Y_s)) * Y_s + Y_n).

All arrays use the library's CSR layout: ``times`` float64[sum N],
``mags`` and ``errs`` float32[sum N], ``offsets`` int64[n_curves + 1].
"""
from __future__ import annotations

import dataclasses
import numpy as np

YEAR_D = 365.25          # days per observing year
SEASON_D = 243.5         # 8-month observing window at the start of each year


@dataclasses.dataclass
class Batch:
    times: np.ndarray     # float64 [sum N]
    mags: np.ndarray      # float32 [sum N]
    errs: np.ndarray      # float32 [sum N]
    offsets: np.ndarray   # int64 [n_curves + 1]
    period: np.ndarray    # float64 [n_curves], 0 for non-periodic curves
    periodic: np.ndarray  # bool [n_curves]
    kind: np.ndarray      # int8 [n_curves] shape code (see SHAPES)

    @property
    def n_curves(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def sizes(self) -> np.ndarray:
        return np.diff(self.offsets)

    def curve(self, c: int):
        a, b = int(self.offsets[c]), int(self.offsets[c + 1])
        return self.times[a:b], self.mags[a:b], self.errs[a:b]

    def subset(self, idx) -> "Batch":
        idx = np.asarray(idx, dtype=np.int64)
        parts_t, parts_m, parts_e, offs = [], [], [], [0]
        for c in idx:
            t, m, e = self.curve(int(c))
            parts_t.append(t); parts_m.append(m); parts_e.append(e)
            offs.append(offs[-1] + t.shape[0])
        return Batch(np.concatenate(parts_t) if parts_t else np.zeros(0),
                     np.concatenate(parts_m).astype(np.float32) if parts_m else np.zeros(0, np.float32),
                     np.concatenate(parts_e).astype(np.float32) if parts_e else np.zeros(0, np.float32),
                     np.asarray(offs, dtype=np.int64), self.period[idx].copy(),
                     self.periodic[idx].copy(), self.kind[idx].copy())


SHAPES = {0: "white noise", 1: "damped random walk", 2: "sinusoid (1-3 harmonics)",
          3: "sawtooth", 4: "eclipsing box dips", 5: "fixed sinusoid"}


@dataclasses.dataclass
class Grid:
    """Uniform trial-frequency grid f_k = f_min + k*df, k = 0..n_freq-1 (1/day),
    plus the coarse/fine parameters of the hierarchical search, or (bands=True)
    the band and trial counts of the bands method of Section 3.1, whose
    spectral windows run on this grid."""
    f_min: float
    df: float
    n_freq: int
    hierarchical: bool = False
    coarse_df: float = 0.0
    top_k: int = 0
    fine_df: float = 0.0
    fine_halfwidth: float = 0.0
    bands: bool = False
    n_bands: int = 0
    trials_per_band: int = 0
    exclude: tuple = ()          # spurious-period exclusion windows: ((f_lo, f_hi), ...) in 1/day

    @property
    def f_max(self) -> float:
        return self.f_min + (self.n_freq - 1) * self.df

    def freqs(self) -> np.ndarray:
        return self.f_min + np.arange(self.n_freq, dtype=np.float64) * self.df


def grid_from_range(f_min: float, f_max: float, df: float, **kw) -> Grid:
    """K = round((f_max - f_min)/df) + 1 points, f_k = f_min + k*df."""
    n = int(np.floor((f_max - f_min) / df + 0.5)) + 1
    return Grid(f_min=f_min, df=df, n_freq=n, **kw)


def seasonal_times(rng: np.random.Generator, sizes: np.ndarray, span: float) -> np.ndarray:
    """Sorted times, uniform on the union of yearly 8-month windows within [0, span].

    Sorted uniform samples come straight from normalised cumulative sums of
    exponential spacings (n + 1 per curve), mapped through the monotone
    window map, so no sort is needed."""
    starts = np.arange(0.0, span, YEAR_D)
    ends = np.minimum(starts + SEASON_D, span)
    lens = ends - starts
    cum = np.concatenate([[0.0], np.cumsum(lens)])
    n_c = sizes.shape[0]
    ext = sizes + 1
    e = rng.exponential(size=int(ext.sum()))
    cs = np.cumsum(e)
    eoff = np.concatenate([[0], np.cumsum(ext)])
    base = np.concatenate([[0.0], cs])[eoff[:-1]]          # cumulative sum before each curve
    tot = cs[eoff[1:] - 1] - base                           # sum of the curve's n + 1 spacings
    keep = np.ones(e.shape[0], bool)
    keep[eoff[1:] - 1] = False                              # drop each curve's last partial sum
    cid = np.repeat(np.arange(n_c), sizes)
    u = (cs[keep] - base[cid]) / tot[cid] * cum[-1]
    w = np.clip(np.searchsorted(cum, u, side="right") - 1, 0, len(lens) - 1)
    return starts[w] + (u - cum[w])


def _offsets(sizes: np.ndarray) -> np.ndarray:
    off = np.zeros(sizes.shape[0] + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    return off


def _errors(rng, sizes, e0):
    """Per-point error bars e_i = e0*(1 + 0.1*N(0,1)), clipped to >= 0.5*e0."""
    e0p = np.repeat(e0, sizes)
    e = e0p * (1.0 + 0.1 * rng.standard_normal(e0p.shape[0]))
    return np.maximum(e, 0.5 * e0p)


def _shape_values(rng, kinds, periods, t, cid, sizes):
    """Unit-amplitude signal shapes evaluated at the flat time array."""
    n_c = kinds.shape[0]
    ph0 = rng.uniform(0.0, 1.0, n_c)
    nharm = rng.integers(1, 4, n_c)
    hamp = rng.uniform(0.2, 0.6, (n_c, 3))
    hphs = rng.uniform(0.0, 1.0, (n_c, 3))
    duty = rng.uniform(0.02, 0.15, n_c)
    tau = rng.uniform(10.0, 300.0, n_c)
    out = np.zeros(t.shape[0], dtype=np.float64)
    pc = np.where(periods > 0, periods, 1.0)[cid]
    phase = np.mod(t / pc + ph0[cid], 1.0)
    k = kinds[cid]
    # sinusoid with 1-3 harmonics
    m = k == 2
    if m.any():
        s = np.sin(2 * np.pi * phase[m])
        for h in (2, 3):
            use = (nharm[cid[m]] >= h)
            s = s + use * hamp[cid[m], h - 1] * np.sin(2 * np.pi * h * phase[m] + 2 * np.pi * hphs[cid[m], h - 1])
        out[m] = s
    m = k == 3          # sawtooth (fast rise, linear decline)
    out[m] = 2.0 * phase[m] - 1.0
    m = k == 4          # box eclipses: primary dip and a shallower secondary at phase 0.5
    if m.any():
        d = duty[cid[m]]
        p = phase[m]
        prim = p < d
        sec = np.abs(p - 0.5) < 0.5 * d
        out[m] = np.where(prim, 1.0, np.where(sec, 0.4, 0.0))
    m = k == 5
    out[m] = np.sin(2 * np.pi * t[m] / pc[m])
    m = k == 0          # white noise
    out[m] = rng.standard_normal(int(m.sum()))
    m = k == 1          # damped random walk (Ornstein-Uhlenbeck), exact irregular-step update
    if m.any():
        drw = np.nonzero(kinds == 1)[0]
        off = np.concatenate([[0], np.cumsum(sizes)])
        starts, lens = off[drw], sizes[drw]
        x = rng.standard_normal(drw.shape[0])
        out[starts] = x
        # step i of every damped-random-walk curve at once (vectorised across curves)
        for i in range(1, int(lens.max()) if lens.size else 1):
            act = lens > i
            idx = starts[act] + i
            dec = np.exp(-(t[idx] - t[idx - 1]) / tau[drw[act]])
            x_act = x[act] * dec + np.sqrt(1.0 - dec * dec) * rng.standard_normal(idx.shape[0])
            x[act] = x_act
            out[idx] = x_act
    return out


def _iqr(x):
    q75, q25 = np.percentile(x, [75, 25])
    return q75 - q25


def single_curve(seed: int = 0, n: int = 150, span: float = 1000.0, period: float = 3.7,
                 amp: float = 0.3, noise: float = 0.1, base: float = 17.0) -> Batch:
    """One seasonal curve: y = base + amp*sin(2*pi*t/period) + N(0, noise^2), e_i = noise."""
    rng = np.random.default_rng(seed)
    sizes = np.array([n], dtype=np.int64)
    t = seasonal_times(rng, sizes, span)
    y = base + amp * np.sin(2 * np.pi * t / period)
    if noise > 0:
        y = y + rng.normal(0.0, noise, size=n)
    e = np.full(n, noise if noise > 0 else 0.1)
    return Batch(t, y.astype(np.float32), e.astype(np.float32), _offsets(sizes),
                 np.array([period]), np.array([True]), np.array([5], np.int8))


def ragged_batch(n_curves: int, seed: int = 1, n_lo: int = 300, n_hi: int = 1000,
                 span: float = 2500.0, p_lo: float = 0.2, p_hi: float = 500.0,
                 snr_scaling: bool = False, snr_lo: float = 0.2, snr_hi: float = 10.0) -> Batch:
    """Ragged batch: N ~ U{n_lo..n_hi}; 50% periodic (log-uniform period, shape in
    {multi-harmonic sinusoid, sawtooth, box eclipse}, amplitude 0.05-1.0 mag),
    50% non-periodic (white noise or damped random walk, tau 10-300 d); error bar
    scale e0 log-uniform in 0.02-0.3 mag.  With ``snr_scaling`` the signal is set
    to a log-uniform SNR in [snr_lo, snr_hi] by the paper's synthetic-set scaling."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(n_lo, n_hi + 1, n_curves).astype(np.int64)
    t = seasonal_times(rng, sizes, span)
    cid = np.repeat(np.arange(n_curves), sizes)
    periodic = rng.uniform(size=n_curves) < 0.5
    kinds = np.where(periodic, rng.integers(2, 5, n_curves), rng.integers(0, 2, n_curves)).astype(np.int8)
    periods = np.where(periodic, np.exp(rng.uniform(np.log(p_lo), np.log(p_hi), n_curves)), 0.0)
    amp = rng.uniform(0.05, 1.0, n_curves)
    e0 = np.exp(rng.uniform(np.log(0.02), np.log(0.3), n_curves))
    base = rng.uniform(15.0, 20.0, n_curves)
    shape = _shape_values(rng, kinds, periods, t, cid, sizes)
    err = _errors(rng, sizes, e0)
    noise = err * rng.standard_normal(err.shape[0])
    if snr_scaling:
        snr = np.exp(rng.uniform(np.log(snr_lo), np.log(snr_hi), n_curves))
        off = _offsets(sizes)
        scale = np.empty(n_curves)
        nmax = int(sizes.max())
        for c0 in range(0, n_curves, 4096):            # padded blocks of curves
            c1 = min(n_curves, c0 + 4096)
            nb = c1 - c0
            pos = np.arange(off[c0], off[c1]) - np.repeat(off[c0:c1], sizes[c0:c1])
            row = np.repeat(np.arange(nb), sizes[c0:c1])
            S = np.full((nb, nmax), np.nan)
            E = np.full((nb, nmax), np.nan)
            S[row, pos] = shape[off[c0]:off[c1]]
            E[row, pos] = err[off[c0]:off[c1]]
            S.sort(axis=1)                      # NaN padding sorts last
            E.sort(axis=1)
            nn = sizes[c0:c1]
            rows = np.arange(nb)

            def q_lin(A, q):
                pos = q * (nn - 1)
                lo = np.floor(pos).astype(np.int64)
                hi = np.minimum(lo + 1, nn - 1)
                return A[rows, lo] + (pos - lo) * (A[rows, hi] - A[rows, lo])
            iq = q_lin(S, 0.75) - q_lin(S, 0.25)
            med = q_lin(E, 0.5)
            scale[c0:c1] = np.where(iq > 0, snr[c0:c1] * med / (0.7413 * np.where(iq > 0, iq, 1.0)), 0.0)
        sig = scale[cid] * shape
    else:
        sig = amp[cid] * shape
    y = base[cid] + sig + noise
    return Batch(t, y.astype(np.float32), err.astype(np.float32), _offsets(sizes),
                 periods, periodic, kinds)


def two_band_batch(n_sources: int, seed: int = 5, n_lo: int = 200, n_hi: int = 1000,
                   span: float = 2500.0) -> Batch:
    """Two independent bands per source: curves 2s and 2s+1 are drawn with the
    same period, shape class and SNR recipe but independent sampling and noise;
    SNR log-uniform 0.2-10 by the paper's synthetic-set scaling."""
    a = ragged_batch(n_sources, seed=seed, n_lo=n_lo, n_hi=n_hi, span=span, snr_scaling=True)
    b = ragged_batch(n_sources, seed=seed + 1, n_lo=n_lo, n_hi=n_hi, span=span, snr_scaling=True)
    # interleave a's and b's curves: curve 2s from a, 2s+1 from b
    sizes = np.empty(2 * n_sources, dtype=np.int64)
    sizes[0::2] = a.sizes
    sizes[1::2] = b.sizes
    off = _offsets(sizes)
    total = int(off[-1])
    src_a = np.repeat(np.arange(n_sources) * 2, a.sizes)
    src_b = np.repeat(np.arange(n_sources) * 2 + 1, b.sizes)
    pos_a = off[src_a] + (np.arange(a.offsets[-1]) - np.repeat(a.offsets[:-1], a.sizes))
    pos_b = off[src_b] + (np.arange(b.offsets[-1]) - np.repeat(b.offsets[:-1], b.sizes))
    t = np.empty(total); m = np.empty(total, np.float32); e = np.empty(total, np.float32)
    t[pos_a], m[pos_a], e[pos_a] = a.times, a.mags, a.errs
    t[pos_b], m[pos_b], e[pos_b] = b.times, b.mags, b.errs
    return Batch(t, m, e, off, np.repeat(a.period, 2), np.repeat(a.periodic, 2), np.repeat(a.kind, 2))


def edge_batch(seed: int = 7) -> Batch:
    """Edge cases for parity tests: N = 2, 3, small ragged sizes, a constant-magnitude
    curve, integer times, and sizes just across tile boundaries."""
    rng = np.random.default_rng(seed)
    sizes = np.array([2, 3, 5, 31, 32, 33, 64, 65, 127, 129, 200], dtype=np.int64)
    t = seasonal_times(rng, sizes, 1500.0)
    y = 16.0 + 0.3 * rng.standard_normal(t.shape[0])
    e = 0.02 + 0.1 * rng.uniform(size=t.shape[0])
    off = _offsets(sizes)
    y[off[3]:off[4]] = 17.25                       # constant magnitudes: W == 0
    t[off[2]:off[3]] = np.array([0.0, 1.0, 3.0, 4.0, 9.0])  # integer times
    return Batch(t, y.astype(np.float32), e.astype(np.float32), off,
                 np.zeros(sizes.shape[0]), np.zeros(sizes.shape[0], bool), np.zeros(sizes.shape[0], np.int8))


# ---------------------------------------------------------------------------
# Named workloads (sizes as the benchmark configurations state them)
# ---------------------------------------------------------------------------

def workload_single():
    """150-point seasonal curve over 1000 d, 0.3 mag sinusoid of period 3.7 d,
    N(0, 0.1^2) noise; grid 0.002-2.0 1/d step 2e-4 (9,991 freqs); seed 0."""
    return single_curve(seed=0), grid_from_range(0.002, 2.0, 2e-4)


def workload_ragged(n_curves: int = 4096, seed: int = 1):
    """4096 curves, N ~ U{300..1000}, seasonal over 2500 d; grid 0.002-5 step 1e-4 (49,981)."""
    return ragged_batch(n_curves, seed=seed), grid_from_range(0.002, 5.0, 1e-4)


def workload_bands(n_curves: int = 4096, seed: int = 1):
    """Same batch; the bands method of Section 3.1 at the paper's operating
    point N_b = 3, N_t = 150, spectral windows on 0.00125-3 1/d (periods
    0.33-800 d) at step 1e-4 (29,988 frequencies; the paper gives no step)."""
    b = ragged_batch(n_curves, seed=seed)
    g = grid_from_range(0.00125, 3.0, 1e-4, bands=True, n_bands=3, trials_per_band=150)
    return b, g


def workload_throughput(n_sources: int = 100000, seed: int = 5):
    """100,000 two-band sources (200,000 curves, N ~ U{200..1000} per band,
    SNR 0.2-10, 50% periodic); hierarchical search: coarse step 1e-3 over
    0.002-5, top-10 refined at 1e-5 over +-2e-3."""
    b = two_band_batch(n_sources, seed=seed)
    g = grid_from_range(0.002, 5.0, 1e-4)
    g.hierarchical = True
    g.coarse_df = 1e-3
    g.top_k = 10
    g.fine_df = 1e-5
    g.fine_halfwidth = 2e-3
    return b, g


def workload_hierarchical(n_curves: int = 4096, seed: int = 1):
    """Same batch; coarse step 1e-3, top-10 local maxima refined at 1e-5 over +-2e-3."""
    b, g = workload_ragged(n_curves, seed)
    g.hierarchical = True
    g.coarse_df = 1e-3
    g.top_k = 10
    g.fine_df = 1e-5
    g.fine_halfwidth = 2e-3
    return b, g
