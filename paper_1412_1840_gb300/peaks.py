"""Instruction-rate probes of the pipes that bound the pair kernels, run on
the target GPU (a measurement tool of the package; not part of the method):

* MUFU ``ex2.approx.f32`` (the direct form does one per pair-frequency
  evaluation), also with a negated operand and as ``ex2.approx.f16x2``;
* FP32 FFMA, packed f32x2 FFMA2 and FP64 DFMA;
* the direct form's two pair-term instruction mixes (sin form: three f32x2
  operations and one accumulate per two evaluations; cos form: two and one);
* ``tcgen05.mma`` kind::f16 (M 128, N 256, K 16) issued back to back by one
  thread per SM: the tensor pipe as the tensor-form kernel drives it;
* cuBLAS FP16 and BF16 GEMMs (8192^3 through torch), for comparison with the
  BF16 figures measured by the same method.

Each rate is reported per clock per SM (clock from clock64 over %globaltimer
inside the probe) and as an absolute rate at that clock and at 2,070 MHz.
The JSON it writes is read by ``bench.py`` for the direct form's roofline:

    python -m paper_1412_1840_gb300.peaks --out paper_1412_1840_gb300/peaks_gb300.json
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import time

from .build import PROBE_LIB

SM_MAX_MHZ = 2070.0
KINDS = {
    "ex2_f32": (0, "MUFU ex2.approx.ftz.f32, x <- ex2(x)", 30000),
    "ex2_f32_neg": (1, "MUFU ex2.approx.ftz.f32, x <- ex2(-x)", 30000),
    "ffma_f32": (2, "FFMA, x <- x a + b", 100000),
    "ffma2_f32x2": (3, "packed fma.rn.f32x2 (lane-ops)", 100000),
    "dfma_f64": (4, "DFMA", 2000),
    "pair_sin_form": (5, "direct-form sin-form term (pair-frequency evaluations)", 16000),
    "pair_cos_form": (6, "direct-form cos-form term (pair-frequency evaluations)", 16000),
    "ex2_f16x2": (7, "MUFU ex2.approx.f16x2 (values)", 12000),
    "tcgen05_mma_f16": (8, "tcgen05.mma kind::f16 M128 N256 K16, one issuing thread per SM (flops)", 200000),
}


def _lib():
    if not os.path.exists(PROBE_LIB):
        raise RuntimeError("probe library %s is missing: run paper_1412_1840_gb300.build" % PROBE_LIB)
    L = ctypes.CDLL(PROBE_LIB)
    L.cp_probe_rate.argtypes = [ctypes.c_int, ctypes.c_longlong, ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.cp_probe_rate.restype = ctypes.c_int
    return L


def probe(L, kind: int, iters: int, reps: int = 3) -> dict:
    """Best of `reps` runs after one warm-up: operations per second and the SM clock."""
    best = None
    for r in range(reps + 1):
        ms, ops, mhz = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        rc = L.cp_probe_rate(kind, iters, ctypes.byref(ms), ctypes.byref(ops), ctypes.byref(mhz))
        if rc != 0:
            raise RuntimeError("probe %d failed with code %d" % (kind, rc))
        if r == 0:
            continue
        rate = ops.value / (ms.value * 1e-3)
        if best is None or rate > best["ops_per_s"]:
            best = {"ops_per_s": rate, "ms": ms.value, "sm_mhz": mhz.value}
    return best


def gemm_rate(dtype_name: str, n: int = 8192, reps: int = 10) -> dict:
    import torch
    dt = getattr(torch, dtype_name)
    a = torch.randn(n, n, device="cuda", dtype=dt)
    b = torch.randn(n, n, device="cuda", dtype=dt)
    for _ in range(3):
        torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 0.0
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, 2.0 * n ** 3 / (e0.elapsed_time(e1) * 1e-3))
    return {"flops_per_s": best, "how": "torch.matmul %s %d^3, best of %d (burst)" % (dtype_name, n, reps)}


def measure(log=print) -> dict:
    import torch
    L = _lib()
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    out = {"device": torch.cuda.get_device_name(0), "n_sm": n_sm, "sm_max_mhz": SM_MAX_MHZ,
           "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()), "rates": {}}
    for name, (kind, what, iters) in KINDS.items():
        r = probe(L, kind, iters)
        per_clk_sm = r["ops_per_s"] / (n_sm * r["sm_mhz"] * 1e6)
        out["rates"][name] = {"what": what, "per_clk_per_sm": per_clk_sm, "ops_per_s": r["ops_per_s"],
                              "sm_mhz": r["sm_mhz"], "ops_per_s_at_max_clock": per_clk_sm * n_sm * SM_MAX_MHZ * 1e6,
                              "ms": r["ms"]}
        log("%-16s %8.2f /clk/SM  %.4e /s at %.0f MHz" % (name, per_clk_sm, r["ops_per_s"], r["sm_mhz"]))
    for dt in ("float16", "bfloat16"):
        g = gemm_rate(dt)
        out["rates"]["cublas_" + dt] = g
        log("cublas %-9s %.1f TFLOP/s" % (dt, g["flops_per_s"] / 1e12))
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--out", required=True)
    args = ap.parse_args()
    table = measure()
    with open(args.out, "w") as fh:
        json.dump(table, fh, indent=1)
    print("wrote %s" % args.out)


if __name__ == "__main__":
    main()
