"""GB300 (sm_103a) correntropy kernelized periodogram of arXiv:1412.1840.

Thin Python binding of the C ABI in ``include/cp.h`` (library
``_lib/libcp.so``).  It only marshals arguments: every step of the method
runs in the library's CUDA kernels.  There is no CPU fallback; if the
library cannot be loaded or no CUDA device is present, calls raise.

Entry points carry the C names: ``cp_plan``, ``cp_periodogram``,
``cp_best_period``, ``cp_sync``, ``cp_curve_stats``, ``cp_get_plan_info``,
``cp_destroy``, ``cp_bessel_coefficients``, ``cp_max_points``,
``cp_trial_frequencies``, ``cp_preprocess``, ``cp_whiten``.  ``Plan`` wraps
a plan handle and keeps the bound input arrays alive.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libcp.so")

CP_OK, CP_EINVAL, CP_ENOMEM, CP_ECUDA, CP_ETIMEOUT, CP_ESTATE, CP_EUNSUPPORTED = range(7)
CP_FORM_DIRECT, CP_FORM_TENSOR = 0, 1
CP_DTYPE_FP16, CP_DTYPE_BF16, CP_DTYPE_BF16_SPLIT = 0, 1, 2
CP_SIGMA_T_FIXED, CP_SIGMA_T_PER_CURVE, CP_SIGMA_T_RULE = 0, 1, 2
CP_MEM_HOST, CP_MEM_DEVICE = 0, 1
CP_SEARCH_FULL, CP_SEARCH_COARSE_FINE, CP_SEARCH_BANDS = 0, 1, 2
CP_BANDS_MAX_TRIALS = 512
CP_MAX_EXCLUDE = 64


class CpError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__("%s: status %d (%s): %s" % (where, status, _status_name(status), msg))
        self.status = status


class cp_freq_grid(ctypes.Structure):
    _fields_ = [("f_min", ctypes.c_double), ("df", ctypes.c_double), ("n_freq", ctypes.c_int64),
                ("hierarchical", ctypes.c_int32), ("top_k", ctypes.c_int32), ("coarse_df", ctypes.c_double),
                ("fine_df", ctypes.c_double), ("fine_halfwidth", ctypes.c_double),
                ("n_bands", ctypes.c_int32), ("trials_per_band", ctypes.c_int32),
                ("n_exclude", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("exclude", ctypes.POINTER(ctypes.c_double))]


CP_TUNE_MAX_BUCKETS = 16


class cp_tuning(ctypes.Structure):
    _fields_ = [("n_buckets", ctypes.c_int32), ("bucket_max_n", ctypes.c_int32 * CP_TUNE_MAX_BUCKETS),
                ("direct_fc", ctypes.c_int32 * CP_TUNE_MAX_BUCKETS),
                ("tensor_classes", ctypes.c_int32 * CP_TUNE_MAX_BUCKETS)]


def tuning_from(table) -> cp_tuning:
    """cp_tuning from the autotuner's JSON table (a path or the loaded dict)."""
    if isinstance(table, (str, os.PathLike)):
        import json
        with open(table) as fh:
            table = json.load(fh)
    t = cp_tuning()
    buckets = table["buckets"]
    if len(buckets) > CP_TUNE_MAX_BUCKETS:
        raise ValueError("at most %d buckets" % CP_TUNE_MAX_BUCKETS)
    t.n_buckets = len(buckets)
    for i, bk in enumerate(buckets):
        t.bucket_max_n[i] = int(bk["max_n"])
        t.direct_fc[i] = int(bk["direct_fc"])
        t.tensor_classes[i] = sum(1 << k for k, cl in enumerate(("8", "16", "32", "12", "48"))
                                  if bk["tensor"].get(cl, True))
    return t


class cp_options(ctypes.Structure):
    _fields_ = [("sigma_t_mode", ctypes.c_int32), ("sigma_t", ctypes.c_float),
                ("sigma_t_per_curve", ctypes.POINTER(ctypes.c_float)), ("alpha", ctypes.c_float),
                ("form", ctypes.c_int32), ("dtype", ctypes.c_int32), ("n_max", ctypes.c_int32),
                ("input_memory", ctypes.c_int32), ("use_graph", ctypes.c_int32), ("device", ctypes.c_int32),
                ("tuning", ctypes.POINTER(cp_tuning))]


class cp_plan_info(ctypes.Structure):
    _fields_ = [("n_curves", ctypes.c_int64), ("n_points", ctypes.c_int64), ("pair_freq_full", ctypes.c_double),
                ("pair_freq_search", ctypes.c_double), ("launches_per_search", ctypes.c_int64),
                ("last_pair_kernel_ms", ctypes.c_float), ("last_step_ms", ctypes.c_float),
                ("n_sm", ctypes.c_int32), ("max_n", ctypes.c_int32), ("class_curves", ctypes.c_int64 * 7),
                ("last_tensor_kernel_ms", ctypes.c_float), ("last_direct_kernel_ms", ctypes.c_float),
                ("tensor_flops_search", ctypes.c_double), ("direct_pair_freq_search", ctypes.c_double),
                ("last_bands_kernel_ms", ctypes.c_float), ("reserved0", ctypes.c_float),
                ("window_terms_search", ctypes.c_double), ("w_bytes_direct", ctypes.c_double),
                ("w_bytes_tensor", ctypes.c_double), ("replans", ctypes.c_int64),
                ("bands_exact_scans", ctypes.c_int64)]


_lock = threading.Lock()
_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("CUDA library %s is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
        L.cp_default_options.argtypes = [ctypes.POINTER(cp_options)]
        L.cp_default_options.restype = None
        L.cp_plan.argtypes = [vp, vp, vp, vp, i64, ctypes.POINTER(cp_freq_grid), ctypes.POINTER(cp_options), vp,
                              ctypes.POINTER(vp)]
        L.cp_periodogram.argtypes = [vp, vp]
        L.cp_best_period.argtypes = [vp, vp, vp, vp, vp, vp]
        L.cp_sync.argtypes = [vp]
        L.cp_curve_stats.argtypes = [vp, vp, vp, vp, vp]
        L.cp_get_plan_info.argtypes = [vp, ctypes.POINTER(cp_plan_info)]
        L.cp_trial_frequencies.argtypes = [vp, vp, vp]
        L.cp_preprocess.argtypes = [vp, vp, vp, vp, i64, ctypes.c_int32, vp, vp, vp, vp, vp, vp, vp]
        L.cp_whiten.argtypes = [vp, vp, vp, i64, vp, ctypes.c_int32, vp, vp]
        L.cp_destroy.argtypes = [vp]
        L.cp_destroy.restype = None
        L.cp_max_points.restype = i64
        L.cp_bessel_coefficients.argtypes = [d, ctypes.c_int32, vp]
        L.cp_best_period_noalloc.argtypes = [vp, vp, vp, vp, i64, ctypes.POINTER(cp_freq_grid), ctypes.c_float, vp,
                                             vp, vp, vp, vp]
        L.cp_best_period_noalloc.restype = ctypes.c_int
        L.cp_status_string.argtypes = [ctypes.c_int]
        L.cp_status_string.restype = ctypes.c_char_p
        L.cp_last_error.restype = ctypes.c_char_p
        for fn in ("cp_plan", "cp_periodogram", "cp_best_period", "cp_sync", "cp_curve_stats",
                   "cp_get_plan_info", "cp_bessel_coefficients", "cp_trial_frequencies", "cp_preprocess",
                   "cp_whiten"):
            getattr(L, fn).restype = ctypes.c_int
        _lib = L
    return _lib


def lib():
    return _load()


def _status_name(s: int) -> str:
    try:
        return _load().cp_status_string(s).decode()
    except Exception:
        return str(s)


def _check(status: int, where: str):
    if status != CP_OK:
        raise CpError(status, where, (_load().cp_last_error() or b"").decode())


def _ptr(a):
    """(pointer, on_device, keepalive) of a numpy array or a torch tensor."""
    if a is None:
        return None, False, None
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), bool(a.is_cuda), a
    arr = np.ascontiguousarray(a)
    return arr.ctypes.data, False, arr


def cp_default_options() -> cp_options:
    o = cp_options()
    _load().cp_default_options(ctypes.byref(o))
    return o


def cp_max_points() -> int:
    return int(_load().cp_max_points())


def cp_bessel_coefficients(sigma_t: float, n_max: int) -> np.ndarray:
    out = np.zeros(n_max + 1, dtype=np.float64)
    _check(_load().cp_bessel_coefficients(float(sigma_t), int(n_max), out.ctypes.data), "cp_bessel_coefficients")
    return out


def make_grid(f_min, df, n_freq, hierarchical=False, coarse_df=0.0, top_k=0, fine_df=0.0, fine_halfwidth=0.0,
              bands=False, n_bands=0, trials_per_band=0, exclude=()):
    """cp_freq_grid; ``bands=True`` selects the bands method of Section 3.1
    (N_b = n_bands, N_t = trials_per_band) over the uniform grid; ``exclude``
    holds the spurious-period windows of Section 6.1 as (f_lo, f_hi) pairs."""
    mode = CP_SEARCH_BANDS if bands else (CP_SEARCH_COARSE_FINE if hierarchical else CP_SEARCH_FULL)
    ex = np.ascontiguousarray(np.asarray(exclude if exclude is not None else (), np.float64).reshape(-1))
    if ex.size % 2:
        raise ValueError("exclude holds (f_lo, f_hi) pairs")
    g = cp_freq_grid(float(f_min), float(df), int(n_freq), mode, int(top_k),
                     float(coarse_df), float(fine_df), float(fine_halfwidth), int(n_bands), int(trials_per_band),
                     int(ex.size // 2), 0, ex.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if ex.size else None)
    g._exclude_keep = ex          # the pointer above refers to this array
    return g


class Plan:
    """A cp_plan handle bound to a CSR lightcurve batch.

    times (float64), mags and errs (float32) are numpy arrays or torch
    tensors, all on the host or all on one CUDA device; offsets is a host
    int64 array of n_curves + 1 entries.  The arrays are kept alive by the
    plan, and every call reads their current contents."""

    def __init__(self, times, mags, errs, offsets, grid: cp_freq_grid, sigma_t=0.3, sigma_t_mode=None,
                 sigma_t_per_curve=None, alpha=1.0, form=CP_FORM_DIRECT, dtype=CP_DTYPE_FP16, n_max=0,
                 use_graph=True, device=None, stream=None, tuning=None):
        L = _load()
        pt, dev_t, kt = _ptr(times)
        pm, dev_m, km = _ptr(mags)
        pe, dev_e, ke = _ptr(errs)
        if not (dev_t == dev_m == dev_e):
            raise ValueError("times, mags and errs must all be on the host or all on the device")
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        self._keep = [kt, km, ke, off]
        o = cp_default_options()
        if sigma_t_mode is None:
            sigma_t_mode = CP_SIGMA_T_PER_CURVE if sigma_t_per_curve is not None else CP_SIGMA_T_FIXED
        o.sigma_t_mode = int(sigma_t_mode)
        o.sigma_t = float(sigma_t)
        if sigma_t_per_curve is not None:
            stpc = np.ascontiguousarray(np.asarray(sigma_t_per_curve, dtype=np.float32))
            self._keep.append(stpc)
            o.sigma_t_per_curve = stpc.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        o.alpha = float(alpha)
        o.form = int(form)
        o.dtype = int(dtype)
        o.n_max = int(n_max)
        o.input_memory = CP_MEM_DEVICE if dev_t else CP_MEM_HOST
        o.use_graph = 1 if use_graph else 0
        if tuning is not None:
            tt = tuning if isinstance(tuning, cp_tuning) else tuning_from(tuning)
            self._keep.append(tt)
            o.tuning = ctypes.pointer(tt)
        if device is None:
            device = times.device.index if dev_t and times.device.index is not None else 0
        o.device = int(device)
        if stream is None and dev_t:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        self.stream = stream
        self.n_curves = int(off.shape[0] - 1)
        self.grid = grid
        h = ctypes.c_void_p()
        _check(L.cp_plan(pt, pm, pe, off.ctypes.data, self.n_curves, ctypes.byref(grid), ctypes.byref(o),
                         ctypes.c_void_p(stream) if stream else None, ctypes.byref(h)), "cp_plan")
        self.handle = h

    # -- entry points ---------------------------------------------------------
    def periodogram(self, out=None):
        """Runs the uniform-grid pass; ``out`` is a CUDA float32 tensor
        [n_curves, n_freq] (or None).  Asynchronous on the plan's stream."""
        p = None
        if out is not None:
            p, on_dev, _ = _ptr(out)
            if not on_dev:
                raise ValueError("out must be a CUDA tensor")
        _check(_load().cp_periodogram(self.handle, p), "cp_periodogram")
        return out

    def best_period(self):
        n = self.n_curves
        idx = np.empty(n, np.int64); f = np.empty(n, np.float64); v = np.empty(n, np.float32)
        per = np.empty(n, np.uint8); ps = np.empty(n, np.float32)
        _check(_load().cp_best_period(self.handle, idx.ctypes.data, f.ctypes.data, v.ctypes.data, per.ctypes.data,
                                      ps.ctypes.data), "cp_best_period")
        return {"best_idx": idx, "best_freq": f, "best_stat": v, "is_periodic": per.astype(bool), "psnr": ps}

    def best_period_into(self, idx, f, v, per, ps):
        """Same as best_period, writing into caller-provided host numpy arrays."""
        _check(_load().cp_best_period(self.handle, idx.ctypes.data, f.ctypes.data, v.ctypes.data, per.ctypes.data,
                                      ps.ctypes.data), "cp_best_period")

    def sync(self):
        _check(_load().cp_sync(self.handle), "cp_sync")

    def trials(self):
        """Trial list of the last search of a bands-method plan:
        ``trial_idx`` [n_curves, n_bands * trials_per_band] grid indices
        (-1 = none) and ``trial_stat`` (nCKP at each, NaN where none)."""
        L = int(self.grid.n_bands) * int(self.grid.trials_per_band)
        idx = np.empty((self.n_curves, L), np.int32)
        st = np.empty((self.n_curves, L), np.float32)
        _check(_load().cp_trial_frequencies(self.handle, idx.ctypes.data, st.ctypes.data), "cp_trial_frequencies")
        return {"trial_idx": idx, "trial_stat": st}

    def curve_stats(self):
        n = self.n_curves
        sy = np.empty(n, np.float32); st = np.empty(n, np.float32); ip = np.empty(n, np.float64)
        ps = np.empty(n, np.float32)
        _check(_load().cp_curve_stats(self.handle, sy.ctypes.data, st.ctypes.data, ip.ctypes.data, ps.ctypes.data),
               "cp_curve_stats")
        return {"sigma_y": sy, "sigma_t": st, "ip": ip, "psnr": ps}

    def info(self) -> dict:
        i = cp_plan_info()
        _check(_load().cp_get_plan_info(self.handle, ctypes.byref(i)), "cp_get_plan_info")
        d = {k: getattr(i, k) for k, _ in cp_plan_info._fields_}
        d["class_curves"] = list(i.class_curves)
        return d

    def close(self):
        if getattr(self, "handle", None):
            _load().cp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def cp_plan(times, mags, errs, offsets, grid, **kw) -> Plan:
    return Plan(times, mags, errs, offsets, grid, **kw)


def cp_periodogram(plan: Plan, out=None):
    return plan.periodogram(out)


def cp_best_period(plan: Plan):
    return plan.best_period()


def cp_sync(plan: Plan):
    plan.sync()


def cp_curve_stats(plan: Plan):
    return plan.curve_stats()


def cp_get_plan_info(plan: Plan):
    return plan.info()


def cp_destroy(plan: Plan):
    plan.close()


def cp_trial_frequencies(plan: Plan):
    return plan.trials()


def cp_best_period_noalloc(times, mags, errs, offsets, grid: cp_freq_grid, sigma_t: float, best_idx=None,
                           best_freq=None, best_stat=None, is_periodic=None, stream=None):
    """Best-period search that allocates no device memory (for callers that
    cannot allocate at call time).  Inputs and outputs are contiguous CUDA
    tensors on the current device: times float64, mags and errs float32 with
    offsets[-1] elements; outputs int64, float64, float32, uint8 with
    n_curves elements (any may be None).  offsets is a host int64 array.
    Synchronous.  Arguments of the wrong type, size or device raise
    ValueError before anything reaches the GPU."""
    import torch
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    if off.ndim != 1 or off.shape[0] < 2:
        raise ValueError("offsets must hold n_curves + 1 entries")
    n_pts, n_cur = int(off[-1]), int(off.shape[0] - 1)
    cur = torch.cuda.current_device()

    def dev_arg(a, name, dtype, count):
        if not (isinstance(a, torch.Tensor) and a.is_cuda):
            raise ValueError("%s must be a CUDA tensor" % name)
        if a.device.index != cur:
            raise ValueError("%s is on cuda:%s, the current device is cuda:%d" % (name, a.device.index, cur))
        if a.dtype != dtype:
            raise ValueError("%s must be %s, not %s" % (name, dtype, a.dtype))
        if not a.is_contiguous() or a.numel() != count:
            raise ValueError("%s must be contiguous with %d elements (it has %d)" % (name, count, a.numel()))
        return a.data_ptr()

    pt = dev_arg(times, "times", torch.float64, n_pts)
    pm = dev_arg(mags, "mags", torch.float32, n_pts)
    pe = dev_arg(errs, "errs", torch.float32, n_pts)
    outs = []
    for o, name, dt in ((best_idx, "best_idx", torch.int64), (best_freq, "best_freq", torch.float64),
                        (best_stat, "best_stat", torch.float32), (is_periodic, "is_periodic", torch.uint8)):
        outs.append(None if o is None else dev_arg(o, name, dt, n_cur))
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    _check(_load().cp_best_period_noalloc(pt, pm, pe, off.ctypes.data, int(off.shape[0] - 1), ctypes.byref(grid),
                                          float(sigma_t), ctypes.c_void_p(stream) if stream else None, *outs),
           "cp_best_period_noalloc")


def _device_tensor(a, name):
    p, on_dev, keep = _ptr(a)
    if not on_dev:
        raise ValueError("%s must be a CUDA tensor" % name)
    return p, keep


def cp_preprocess(times, mags, errs, offsets, min_n=50, stream=None):
    """Section 5.2 cleaning on the device (see include/cp.h).  times (float64),
    mags and errs (float32) are CUDA tensors; offsets a host int64 array.
    Returns a dict: the kept samples ``times``, ``mags``, ``errs`` (CUDA
    tensors), ``offsets`` over the kept curves (host), ``curve`` (input index
    of each kept curve), ``flags`` and ``fit`` per input curve."""
    import torch
    pt, _ = _device_tensor(times, "times")
    pm, _ = _device_tensor(mags, "mags")
    pe, _ = _device_tensor(errs, "errs")
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    nc = off.shape[0] - 1
    n = int(off[-1])
    ot = torch.empty(max(n, 1), dtype=torch.float64, device=times.device)
    om = torch.empty(max(n, 1), dtype=torch.float32, device=times.device)
    oe = torch.empty(max(n, 1), dtype=torch.float32, device=times.device)
    oo = np.empty(nc + 1, np.int64)
    flags = np.empty(nc, np.uint8)
    fit = np.empty((nc, 3), np.float64)
    if stream is None:
        stream = torch.cuda.current_stream(times.device).cuda_stream
    _check(_load().cp_preprocess(pt, pm, pe, off.ctypes.data, nc, int(min_n), ot.data_ptr(), om.data_ptr(),
                                 oe.data_ptr(), oo.ctypes.data, flags.ctypes.data, fit.ctypes.data,
                                 ctypes.c_void_p(stream) if stream else None), "cp_preprocess")
    kept = np.nonzero(flags & 1)[0]
    k = int(oo[-1])
    return {"times": ot[:k], "mags": om[:k], "errs": oe[:k],
            "offsets": np.concatenate([[0], np.cumsum(oo[kept + 1] - oo[kept])]).astype(np.int64),
            "offsets_all": oo, "curve": kept, "flags": flags, "fit": fit}


def cp_whiten(times, mags, offsets, p0, window=30, out=None, stream=None):
    """Section 7.1 whitening on the device (see include/cp.h); returns ``out``
    (a new CUDA float32 tensor unless given; may be ``mags`` itself)."""
    import torch
    pt, _ = _device_tensor(times, "times")
    pm, _ = _device_tensor(mags, "mags")
    if out is None:
        out = torch.empty_like(mags)
    po, _ = _device_tensor(out, "out")
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    p = np.ascontiguousarray(np.asarray(p0, dtype=np.float64))
    if stream is None:
        stream = torch.cuda.current_stream(times.device).cuda_stream
    _check(_load().cp_whiten(pt, pm, off.ctypes.data, off.shape[0] - 1, p.ctypes.data, int(window), po,
                             ctypes.c_void_p(stream) if stream else None), "cp_whiten")
    return out


def grid_from(g) -> cp_freq_grid:
    """cp_freq_grid from any object with the synthetic-grid attribute names."""
    return make_grid(g.f_min, g.df, g.n_freq, g.hierarchical, g.coarse_df, g.top_k, g.fine_df, g.fine_halfwidth,
                     getattr(g, "bands", False), getattr(g, "n_bands", 0), getattr(g, "trials_per_band", 0),
                     getattr(g, "exclude", ()))
