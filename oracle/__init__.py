"""FP64 CPU oracle for the correntropy kernelized periodogram (arXiv:1412.1840).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  It
shares no code with the CUDA implementation in ``paper_1412_1840_gb300``.

The arithmetic lives in ``ckp_oracle.c`` (plain C, FP64, libm, built without
fast-math); this module only compiles it and marshals arguments.  The exact
rational expansion of the periodic kernel, Eq. (taylor), is in ``series.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ckp_oracle.c")
_LIB = os.path.join(_HERE, "liborcckp.so")
_lock = threading.Lock()
_lib = None

D = ctypes.c_double
I64 = ctypes.c_int64
PD = ctypes.POINTER(ctypes.c_double)
PF = ctypes.POINTER(ctypes.c_float)
PI64 = ctypes.POINTER(ctypes.c_int64)
PI32 = ctypes.POINTER(ctypes.c_int32)


class OrcGrid(ctypes.Structure):
    _fields_ = [("f_min", D), ("df", D), ("n_freq", I64), ("hierarchical", ctypes.c_int),
                ("coarse_df", D), ("top_k", I64), ("fine_df", D), ("fine_halfwidth", D),
                ("n_bands", I64), ("trials_per_band", I64), ("n_exclude", I64), ("exclude", PD)]


class OrcOptions(ctypes.Structure):
    _fields_ = [("sigma_t_mode", ctypes.c_int), ("sigma_t", D), ("sigma_t_per_curve", PD),
                ("alpha", D)]


class OrcPrep(ctypes.Structure):
    _fields_ = [("n_in", I64), ("n_out", I64), ("kept", ctypes.c_int), ("detrended", ctypes.c_int),
                ("e_mean", D), ("e_std", D), ("a0", D), ("a1", D), ("r", D)]


class OrcResult(ctypes.Structure):
    _fields_ = [("best_idx", I64), ("best_freq", D), ("best_stat", D), ("is_periodic", ctypes.c_int),
                ("psnr", D), ("sigma_y", D), ("sigma_t", D), ("ip", D)]


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O2 -fopenmp, IEEE semantics, no fast-math)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + ".tmp%d" % os.getpid()
            subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                                   "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.orc_max_threads.restype = ctypes.c_int; L.orc_max_threads.argtypes = []
        L.orc_gauss.restype = D; L.orc_gauss.argtypes = [D, D]
        L.orc_periodic_kernel.restype = D; L.orc_periodic_kernel.argtypes = [D, D, D]
        L.orc_information_potential.restype = D; L.orc_information_potential.argtypes = [PD, I64, D]
        L.orc_ckp.restype = None; L.orc_ckp.argtypes = [PD, PD, I64, D, D, PD, I64, PD]
        L.orc_nckp.restype = None; L.orc_nckp.argtypes = [PD, PD, I64, D, D, PD, I64, PD]
        L.orc_median.restype = D; L.orc_median.argtypes = [PD, I64]
        L.orc_quantile.restype = D; L.orc_quantile.argtypes = [PD, I64, D]
        L.orc_psnr.restype = D; L.orc_psnr.argtypes = [PD, PD, I64, D]
        L.orc_bowley_skewness.restype = D; L.orc_bowley_skewness.argtypes = [PD, I64]
        L.orc_sigma_t_rule.restype = D; L.orc_sigma_t_rule.argtypes = [PD, I64]
        L.orc_snr_bin.restype = ctypes.c_int; L.orc_snr_bin.argtypes = [D]
        L.orc_threshold.restype = D; L.orc_threshold.argtypes = [D]
        L.orc_argmax.restype = I64; L.orc_argmax.argtypes = [PD, I64]
        L.orc_top_local_maxima.restype = I64; L.orc_top_local_maxima.argtypes = [PD, I64, I64, PI64]
        L.orc_is_excluded.restype = ctypes.c_int; L.orc_is_excluded.argtypes = [D, I64, PD]
        L.orc_top_local_maxima_excl.restype = I64
        L.orc_top_local_maxima_excl.argtypes = [PD, I64, I64, D, D, I64, PD, PI64]
        L.orc_curve_best.restype = None
        L.orc_curve_best.argtypes = [PD, PD, PD, I64, I64, ctypes.POINTER(OrcGrid),
                                     ctypes.POINTER(OrcOptions), ctypes.POINTER(OrcResult)]
        L.orc_batch_best.restype = None
        L.orc_batch_best.argtypes = [PD, PF, PF, PI64, I64, ctypes.POINTER(OrcGrid),
                                     ctypes.POINTER(OrcOptions), ctypes.POINTER(OrcResult)]
        L.orc_batch_nckp.restype = None
        L.orc_batch_nckp.argtypes = [PD, PF, PF, PI64, I64, PD, PD, I64, PD]
        L.orc_chi2_line.restype = None; L.orc_chi2_line.argtypes = [PD, PD, PD, I64, PD, PD]
        L.orc_pearson.restype = D; L.orc_pearson.argtypes = [PD, PD, I64]
        L.orc_preprocess.restype = OrcPrep; L.orc_preprocess.argtypes = [PD, PD, PD, I64, I64, PD, PD, PD]
        L.orc_batch_preprocess.restype = None
        L.orc_batch_preprocess.argtypes = [PD, PF, PF, PI64, I64, I64, PD, PD, PD, PI64, ctypes.POINTER(OrcPrep)]
        L.orc_whiten.restype = None; L.orc_whiten.argtypes = [PD, PD, I64, D, I64, PD]
        L.orc_batch_whiten.restype = None; L.orc_batch_whiten.argtypes = [PD, PF, PI64, I64, PD, I64, PD]
        L.orc_bands_of.restype = None; L.orc_bands_of.argtypes = [PD, I64, PI32]
        L.orc_band_derivative_sums.restype = None
        L.orc_band_derivative_sums.argtypes = [PD, PD, I64, PI32, PD]
        L.orc_band_order.restype = None; L.orc_band_order.argtypes = [PD, PI32]
        L.orc_spectral_window.restype = None
        L.orc_spectral_window.argtypes = [PD, I64, PI32, ctypes.c_int32, D, D, I64, PD]
        L.orc_is_one_day.restype = ctypes.c_int; L.orc_is_one_day.argtypes = [D]
        L.orc_window_trials.restype = I64; L.orc_window_trials.argtypes = [PD, I64, D, D, I64, PI64]
        L.orc_bands_trials.restype = None
        L.orc_bands_trials.argtypes = [PD, PD, I64, D, D, I64, I64, I64, PI64]
        L.orc_batch_bands_trials.restype = None
        L.orc_batch_bands_trials.argtypes = [PD, PF, PI64, I64, D, D, I64, I64, I64, PI64]
        _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(PD)


def gauss(x: float, sigma: float) -> float:
    return lib().orc_gauss(float(x), float(sigma))


def periodic_kernel(f: float, dt: float, sigma: float) -> float:
    return lib().orc_periodic_kernel(float(f), float(dt), float(sigma))


def information_potential(y, sigma_y: float) -> float:
    y, py = _d(y)
    return lib().orc_information_potential(py, y.shape[0], float(sigma_y))


def ckp(t, y, sigma_y, sigma_t, freqs) -> np.ndarray:
    t, pt = _d(t); y, py = _d(y); f, pf = _d(np.atleast_1d(freqs))
    out = np.empty(f.shape[0]); lib().orc_ckp(pt, py, t.shape[0], sigma_y, sigma_t, pf, f.shape[0], out.ctypes.data_as(PD))
    return out


def nckp(t, y, sigma_y, sigma_t, freqs) -> np.ndarray:
    t, pt = _d(t); y, py = _d(y); f, pf = _d(np.atleast_1d(freqs))
    out = np.empty(f.shape[0]); lib().orc_nckp(pt, py, t.shape[0], sigma_y, sigma_t, pf, f.shape[0], out.ctypes.data_as(PD))
    return out


def median(x) -> float:
    x, px = _d(x); return lib().orc_median(px, x.shape[0])


def quantile(x, q) -> float:
    x, px = _d(x); return lib().orc_quantile(px, x.shape[0], float(q))


def psnr(y, e, alpha=1.0) -> float:
    y, py = _d(y); e, pe = _d(e); return lib().orc_psnr(py, pe, y.shape[0], float(alpha))


def bowley_skewness(y) -> float:
    y, py = _d(y); return lib().orc_bowley_skewness(py, y.shape[0])


def sigma_t_rule(y) -> float:
    y, py = _d(y); return lib().orc_sigma_t_rule(py, y.shape[0])


def snr_bin(p) -> int:
    return lib().orc_snr_bin(float(p))


def threshold(p) -> float:
    return lib().orc_threshold(float(p))


def argmax(v) -> int:
    v, pv = _d(v); return lib().orc_argmax(pv, v.shape[0])


def top_local_maxima(v, top_k) -> np.ndarray:
    v, pv = _d(v); out = np.zeros(max(int(top_k), 1), dtype=np.int64)
    n = lib().orc_top_local_maxima(pv, v.shape[0], int(top_k), out.ctypes.data_as(PI64))
    return out[:n]


# ---- preprocessing, Section 5.2 --------------------------------------------


def chi2_line(t, x, e):
    t, pt = _d(t); x, px = _d(x); e, pe = _d(e); a0 = D(); a1 = D()
    lib().orc_chi2_line(pt, px, pe, t.shape[0], ctypes.byref(a0), ctypes.byref(a1))
    return a0.value, a1.value


def pearson(u, v) -> float:
    u, pu = _d(u); v, pv = _d(v)
    return lib().orc_pearson(pu, pv, u.shape[0])


def _prep_dict(r):
    return {k: getattr(r, k) for k, _ in OrcPrep._fields_}


def preprocess(t, x, e, min_n=50):
    """One curve: (kept t, x, e arrays, summary dict)."""
    t, pt = _d(t); x, px = _d(x); e, pe = _d(e)
    n = t.shape[0]
    ot, ox, oe = np.empty(max(n, 1)), np.empty(max(n, 1)), np.empty(max(n, 1))
    r = lib().orc_preprocess(pt, px, pe, n, int(min_n), ot.ctypes.data_as(PD), ox.ctypes.data_as(PD),
                             oe.ctypes.data_as(PD))
    k = r.n_out
    return ot[:k], ox[:k], oe[:k], _prep_dict(r)


def batch_preprocess(batch, min_n=50):
    """CSR batch -> (times, mags, errs as float64, out_offsets over the input curves, list of summaries)."""
    t = np.ascontiguousarray(batch.times, np.float64)
    m = np.ascontiguousarray(batch.mags, np.float32)
    e = np.ascontiguousarray(batch.errs, np.float32)
    off = np.ascontiguousarray(batch.offsets, np.int64)
    nc = off.shape[0] - 1
    n = max(int(off[-1]), 1)
    ot, ox, oe = np.empty(n), np.empty(n), np.empty(n)
    oo = np.empty(nc + 1, np.int64)
    res = (OrcPrep * max(nc, 1))()
    lib().orc_batch_preprocess(t.ctypes.data_as(PD), m.ctypes.data_as(PF), e.ctypes.data_as(PF),
                               off.ctypes.data_as(PI64), nc, int(min_n), ot.ctypes.data_as(PD),
                               ox.ctypes.data_as(PD), oe.ctypes.data_as(PD), oo.ctypes.data_as(PI64), res)
    k = int(oo[-1])
    return ot[:k], ox[:k], oe[:k], oo, [_prep_dict(res[c]) for c in range(nc)]


# ---- whitening, Section 7.1 -------------------------------------------------


def whiten(t, x, p0, w=30) -> np.ndarray:
    t, pt = _d(t); x, px = _d(x); out = np.empty(t.shape[0])
    lib().orc_whiten(pt, px, t.shape[0], float(p0), int(w), out.ctypes.data_as(PD))
    return out


def batch_whiten(batch, p0, w=30) -> np.ndarray:
    t = np.ascontiguousarray(batch.times, np.float64)
    m = np.ascontiguousarray(batch.mags, np.float32)
    off = np.ascontiguousarray(batch.offsets, np.int64)
    p = np.ascontiguousarray(p0, np.float64)
    out = np.empty(max(int(off[-1]), 1))
    lib().orc_batch_whiten(t.ctypes.data_as(PD), m.ctypes.data_as(PF), off.ctypes.data_as(PI64), off.shape[0] - 1,
                           p.ctypes.data_as(PD), int(w), out.ctypes.data_as(PD))
    return out[:int(off[-1])]


# ---- bands method, Section 3.1 ---------------------------------------------


def bands_of(y) -> np.ndarray:
    """Band 0..9 of every sample (ten equal-count magnitude bands)."""
    y, py = _d(y); out = np.empty(y.shape[0], np.int32)
    lib().orc_bands_of(py, y.shape[0], out.ctypes.data_as(PI32))
    return out


def band_derivative_sums(t, y, band) -> np.ndarray:
    t, pt = _d(t); y, py = _d(y); b = np.ascontiguousarray(band, np.int32); out = np.empty(10)
    lib().orc_band_derivative_sums(pt, py, t.shape[0], b.ctypes.data_as(PI32), out.ctypes.data_as(PD))
    return out


def band_order(D) -> np.ndarray:
    D, pD = _d(D); out = np.empty(10, np.int32)
    lib().orc_band_order(pD, out.ctypes.data_as(PI32))
    return out


def spectral_window(t, band, j, f_min, df, nk) -> np.ndarray:
    t, pt = _d(t); b = np.ascontiguousarray(band, np.int32); out = np.empty(int(nk))
    lib().orc_spectral_window(pt, t.shape[0], b.ctypes.data_as(PI32), int(j), float(f_min), float(df), int(nk),
                              out.ctypes.data_as(PD))
    return out


def is_one_day(f) -> bool:
    return bool(lib().orc_is_one_day(float(f)))


def window_trials(S, f_min, df, n_t) -> np.ndarray:
    S, pS = _d(S); out = np.empty(max(int(n_t), 1), np.int64)
    lib().orc_window_trials(pS, S.shape[0], float(f_min), float(df), int(n_t), out.ctypes.data_as(PI64))
    return out[:int(n_t)]


def bands_trials(t, y, f_min, df, nk, n_bands, n_t) -> np.ndarray:
    """[n_bands, n_t] trial grid indices of one curve (-1 = none)."""
    t, pt = _d(t); y, py = _d(y); out = np.empty((int(n_bands), int(n_t)), np.int64)
    lib().orc_bands_trials(pt, py, t.shape[0], float(f_min), float(df), int(nk), int(n_bands), int(n_t),
                           out.ctypes.data_as(PI64))
    return out


def batch_bands_trials(batch, grid) -> np.ndarray:
    """[n_curves, n_bands * trials_per_band] trial grid indices of a CSR batch."""
    t = np.ascontiguousarray(batch.times, np.float64)
    m = np.ascontiguousarray(batch.mags, np.float32)
    off = np.ascontiguousarray(batch.offsets, np.int64)
    nc = off.shape[0] - 1
    L = int(grid.n_bands) * int(grid.trials_per_band)
    out = np.empty((nc, L), np.int64)
    lib().orc_batch_bands_trials(t.ctypes.data_as(PD), m.ctypes.data_as(PF), off.ctypes.data_as(PI64), nc,
                                 float(grid.f_min), float(grid.df), int(grid.n_freq), int(grid.n_bands),
                                 int(grid.trials_per_band), out.ctypes.data_as(PI64))
    return out


def _exclude_array(g):
    ex = np.ascontiguousarray(np.asarray(getattr(g, "exclude", ()) or (), np.float64).reshape(-1))
    return ex, ex.shape[0] // 2


def _grid(g):
    """(OrcGrid, keepalive) of a synthetic grid description."""
    mode = 2 if getattr(g, "bands", False) else int(bool(g.hierarchical))
    ex, n_ex = _exclude_array(g)
    og = OrcGrid(g.f_min, g.df, g.n_freq, mode, g.coarse_df or 0.0,
                 int(g.top_k or 0), g.fine_df or 0.0, g.fine_halfwidth or 0.0,
                 int(getattr(g, "n_bands", 0) or 0), int(getattr(g, "trials_per_band", 0) or 0),
                 n_ex, ex.ctypes.data_as(PD) if n_ex else None)
    return og, ex


def is_excluded(f, exclude) -> bool:
    """Section 6.1 exclusion test of one frequency against [(lo, hi), ...]."""
    ex = np.ascontiguousarray(np.asarray(exclude, np.float64).reshape(-1))
    return bool(lib().orc_is_excluded(float(f), ex.shape[0] // 2, ex.ctypes.data_as(PD) if ex.size else None))


def top_local_maxima_excl(v, top_k, f_min, df, exclude) -> np.ndarray:
    v, pv = _d(v); out = np.zeros(max(int(top_k), 1), dtype=np.int64)
    ex = np.ascontiguousarray(np.asarray(exclude, np.float64).reshape(-1))
    n = lib().orc_top_local_maxima_excl(pv, v.shape[0], int(top_k), float(f_min), float(df), ex.shape[0] // 2,
                                        ex.ctypes.data_as(PD) if ex.size else None, out.ctypes.data_as(PI64))
    return out[:n]


def _opts(sigma_t_mode, sigma_t, per_curve, alpha):
    keep = None
    p = None
    if per_curve is not None:
        keep = np.ascontiguousarray(per_curve, dtype=np.float64)
        p = keep.ctypes.data_as(PD)
    return OrcOptions(int(sigma_t_mode), float(sigma_t), p, float(alpha)), keep


def batch_best(batch, grid, sigma_t_mode=0, sigma_t=0.3, sigma_t_per_curve=None, alpha=1.0):
    """Best period and discriminator for every curve of a CSR batch (dict of arrays)."""
    t = np.ascontiguousarray(batch.times, np.float64)
    m = np.ascontiguousarray(batch.mags, np.float32)
    e = np.ascontiguousarray(batch.errs, np.float32)
    off = np.ascontiguousarray(batch.offsets, np.int64)
    nc = off.shape[0] - 1
    g, gkeep = _grid(grid)
    o, keep = _opts(sigma_t_mode, sigma_t, sigma_t_per_curve, alpha)
    res = (OrcResult * max(nc, 1))()
    lib().orc_batch_best(t.ctypes.data_as(PD), m.ctypes.data_as(PF), e.ctypes.data_as(PF),
                         off.ctypes.data_as(PI64), nc, ctypes.byref(g), ctypes.byref(o), res)
    del keep, gkeep
    out = {k: np.array([getattr(res[c], k) for c in range(nc)]) for k, _ in OrcResult._fields_}
    out["best_idx"] = out["best_idx"].astype(np.int64)
    out["is_periodic"] = out["is_periodic"].astype(bool)
    return out


def max_threads() -> int:
    """OpenMP threads the oracle's parallel loops use."""
    return int(lib().orc_max_threads())


def batch_nckp(batch, sigma_t, freqs) -> np.ndarray:
    """nCKP of every curve at its own frequency list: freqs [n_curves, nf] (or [nf])."""
    t = np.ascontiguousarray(batch.times, np.float64)
    m = np.ascontiguousarray(batch.mags, np.float32)
    e = np.ascontiguousarray(batch.errs, np.float32)
    off = np.ascontiguousarray(batch.offsets, np.int64)
    nc = off.shape[0] - 1
    st = np.ascontiguousarray(np.broadcast_to(np.asarray(sigma_t, np.float64), (nc,)))
    f = np.asarray(freqs, np.float64)
    if f.ndim == 1:
        f = np.broadcast_to(f, (nc, f.shape[0]))
    f = np.ascontiguousarray(f)
    nf = f.shape[1]
    out = np.empty((nc, nf))
    lib().orc_batch_nckp(t.ctypes.data_as(PD), m.ctypes.data_as(PF), e.ctypes.data_as(PF),
                         off.ctypes.data_as(PI64), nc, st.ctypes.data_as(PD), f.ctypes.data_as(PD),
                         nf, out.ctypes.data_as(PD))
    return out


def curve_stats(batch, sigma_t_mode=0, sigma_t=0.3, sigma_t_per_curve=None, alpha=1.0):
    """sigma_y, sigma_t, IP and pSNR per curve (same conventions as batch_best)."""
    nc = batch.n_curves
    out = {"sigma_y": np.empty(nc), "sigma_t": np.empty(nc), "ip": np.empty(nc), "psnr": np.empty(nc)}
    for c in range(nc):
        t, m, e = batch.curve(c)
        y = m.astype(np.float64); ee = e.astype(np.float64)
        sy = median(ee)
        out["sigma_y"][c] = sy
        out["ip"][c] = information_potential(y, sy)
        out["psnr"][c] = psnr(y, ee, alpha)
        if sigma_t_mode == 1:
            out["sigma_t"][c] = sigma_t_per_curve[c]
        elif sigma_t_mode == 2:
            out["sigma_t"][c] = sigma_t_rule(y)
        else:
            out["sigma_t"][c] = sigma_t
    return out
