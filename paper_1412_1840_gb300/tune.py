"""Autotuner of the launch choices the plan makes per curve size:

* frequencies per work unit of the direct form (2, 4, 8 or 16), and
* for each harmonic class of the tensor form (8, 12, 16, 32, 48 harmonics)
  whether the tensor form or the direct form is faster at that curve size (the
  tensor form pads a curve to 128-row tiles, which costs most for small N).
  Classes 8, 12 and 16 are compared with the direct form's cos-form exponent
  (sigma_t 0.3), classes 32 and 48, which serve sigma_t < 0.25, with its
  sin-form exponent (sigma_t 0.2), the one those curves run in.

It times the pair kernels through the public API on synthetic curves of
each size bucket (results do not depend on the data, only on N and the grid
size) and writes a JSON table that ``tuning_from`` turns into the C ABI's
``cp_tuning``:

    python -m paper_1412_1840_gb300.tune --out paper_1412_1840_gb300/tuning_gb300.json

``--merge TABLE --classes 32,48`` keeps TABLE's direct-form frequencies per
unit and its other classes and times only the listed classes (and the
sin-form direct rate they are compared with).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import (CP_FORM_DIRECT, CP_FORM_TENSOR, CP_SIGMA_T_FIXED, Plan, cp_max_points, make_grid,
               tuning_from)

# (lowest, highest] curve sizes of each bucket
BUCKETS = [(2, 96), (96, 192), (192, 320), (320, 512), (512, 768), (768, 1024), (1024, 1536),
           (1536, 2048), (2048, 3072), (3072, 4096)]
TABLE_BYTES = 196608        # shared trig table of the direct kernel (12 B per point and frequency)


def fc_fits(n: int, fc: int) -> bool:
    npad = (n + 31) // 32 * 32
    return npad * fc * 12 <= TABLE_BYTES


def synthetic_batch(rng, lo: int, hi: int, n_curves: int):
    sizes = rng.integers(lo + 1, hi + 1, n_curves)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    t = np.concatenate([np.sort(rng.uniform(0.0, 2500.0, s)) for s in sizes])
    y = (17.0 + 0.2 * rng.standard_normal(off[-1])).astype(np.float32)
    e = np.full(off[-1], 0.05, np.float32)
    return t, y, e, off, sizes


SIN_FORM_CLASSES = (32, 48)   # harmonic classes whose curves take the direct form's sin-form exponent


def timed(t, y, e, off, grid, reps: int = 2, sigma_t: float = 0.3, **kw) -> dict:
    """Pair-kernel time of one best-period search (the last of `reps`)."""
    with Plan(t, y, e, off, grid, sigma_t=sigma_t, sigma_t_mode=CP_SIGMA_T_FIXED, **kw) as p:
        for _ in range(reps):
            p.best_period()
        info = p.info()
    ms = info["last_tensor_kernel_ms"] if kw.get("form") == CP_FORM_TENSOR else info["last_direct_kernel_ms"]
    return {"ms": ms, "pair_freq_per_s": info["pair_freq_search"] / (ms * 1e-3)}


def tune(n_freq: int = 2048, target_pair_freq: float = 4e10, seed: int = 0, device: int = 0, log=print,
         classes=(8, 12, 16, 32, 48), base: dict | None = None) -> dict:
    rng = np.random.default_rng(seed)
    grid = make_grid(0.01, 1e-3, n_freq)
    out = {"n_freq": n_freq, "buckets": []}
    try:
        import torch
        out["device"] = torch.cuda.get_device_name(device)
    except Exception:
        out["device"] = "unknown"
    t_start = time.time()
    for lo, hi in BUCKETS:
        if lo >= cp_max_points():
            break
        hi = min(hi, cp_max_points())
        mean_pairs = ((lo + hi) / 2.0) ** 2 / 2.0
        n_curves = int(np.clip(target_pair_freq / (mean_pairs * n_freq), 8, 4096))
        t, y, e, off, sizes = synthetic_batch(rng, lo, hi, n_curves)
        prev = None
        if base is not None:
            prev = next(b for b in base["buckets"] if b["max_n"] == hi)
            assert prev["n_curves"] == n_curves, "the merged table was made with other settings"
        if prev is not None:
            entry = dict(prev, direct=dict(prev["direct"]), tensor_rate=dict(prev["tensor_rate"]),
                         tensor=dict(prev["tensor"]))
            best_fc = prev["direct_fc"]
            best_rate = prev["direct"][str(best_fc)]
        else:
            entry = {"max_n": hi, "n_curves": n_curves, "direct": {}, "tensor_rate": {}, "tensor": {}}
            best_fc, best_rate = None, 0.0
            for fc in (16, 8, 4, 2):
                if not fc_fits(hi, fc):
                    continue
                one = tuning_from({"buckets": [{"max_n": cp_max_points(), "direct_fc": fc, "tensor": {}}]})
                r = timed(t, y, e, off, grid, form=CP_FORM_DIRECT, tuning=one, device=device)
                entry["direct"][str(fc)] = r["pair_freq_per_s"]
                if r["pair_freq_per_s"] > best_rate:
                    best_fc, best_rate = fc, r["pair_freq_per_s"]
            entry["direct_fc"] = best_fc
        sin_rate = None
        if any(c in SIN_FORM_CLASSES for c in classes):
            one = tuning_from({"buckets": [{"max_n": cp_max_points(), "direct_fc": best_fc, "tensor": {}}]})
            sin_rate = timed(t, y, e, off, grid, form=CP_FORM_DIRECT, tuning=one, device=device,
                             sigma_t=0.2)["pair_freq_per_s"]
            entry["direct_sin_form"] = sin_rate
        for cls in classes:
            r = timed(t, y, e, off, grid, form=CP_FORM_TENSOR, n_max=cls, device=device)
            entry["tensor_rate"][str(cls)] = r["pair_freq_per_s"]
            ref = sin_rate if cls in SIN_FORM_CLASSES else best_rate
            entry["tensor"][str(cls)] = bool(r["pair_freq_per_s"] > ref)
        out["buckets"].append(entry)
        log("N in (%d, %d]: %d curves; direct fc %d at %.3e pair*freq/s; tensor %s" % (
            lo, hi, n_curves, best_fc, best_rate,
            ", ".join("%s: %.3e%s" % (k, v, "*" if entry["tensor"][k] else "") for k, v in entry["tensor_rate"].items())))
    out["seconds"] = time.time() - t_start
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--out", required=True)
    ap.add_argument("--n-freq", type=int, default=2048)
    ap.add_argument("--device", type=int, default=0)
    ap.add_argument("--classes", default="8,12,16,32,48", help="harmonic classes to time")
    ap.add_argument("--merge", default=None, help="an earlier table whose other entries are kept")
    args = ap.parse_args()
    base = None
    if args.merge:
        with open(args.merge) as fh:
            base = json.load(fh)
    table = tune(n_freq=base["n_freq"] if base else args.n_freq, device=args.device,
                 classes=tuple(int(c) for c in args.classes.split(",")), base=base)
    with open(args.out, "w") as fh:
        json.dump(table, fh, indent=1)
    print("wrote %s (%.1f s)" % (args.out, table["seconds"]))


if __name__ == "__main__":
    main()
