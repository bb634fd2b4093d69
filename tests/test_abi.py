"""C-ABI checks that need no GPU: the library loads, exports every function
include/cp.h declares, validates arguments before touching a device, and its
host-side Bessel coefficients match the paper's series (Eq. (taylor))."""
import ctypes
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

import paper_1412_1840_gb300 as cp
from oracle.series import taylor_harmonic_coefficients

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cp_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = cp.lib()
    names = declared_functions()
    assert "cp_plan" in names and "cp_periodogram" in names and "cp_best_period" in names
    for name in names:
        assert hasattr(L, name), name


def _c_layout(struct, fields):
    """sizeof and offsetof of a header struct, from a C program compiled against include/cp.h."""
    body = 'printf("%%zu", sizeof(%s));' % struct
    for f in fields:
        body += 'printf(" %%zu", offsetof(%s, %s));' % (struct, f)
    src = '#include <stdio.h>\n#include <stddef.h>\n#include "cp.h"\nint main(void){%s return 0;}\n' % body
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "l.c")
        exe = os.path.join(d, "l")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        return [int(x) for x in subprocess.check_output([exe]).split()]


@pytest.mark.parametrize("cls,name", [(cp.cp_freq_grid, "cp_freq_grid"), (cp.cp_options, "cp_options"),
                                      (cp.cp_plan_info, "cp_plan_info"), (cp.cp_tuning, "cp_tuning")])
def test_binding_structs_match_header_layout(cls, name):
    fields = [f for f, _ in cls._fields_]
    got = _c_layout(name, fields)
    want = [ctypes.sizeof(cls)] + [getattr(cls, f).offset for f in fields]
    assert got == want


def test_default_options():
    o = cp.cp_default_options()
    assert o.sigma_t == pytest.approx(0.3) and o.alpha == 1.0 and o.use_graph == 1
    assert o.form == cp.CP_FORM_DIRECT and o.input_memory == cp.CP_MEM_HOST


def test_status_strings():
    L = cp.lib()
    for s in range(7):
        assert L.cp_status_string(s)


@pytest.mark.parametrize("st,nm", [(0.6, 12), (0.3, 24), (0.15, 48), (0.1, 64)])
def test_bessel_coefficients_match_taylor_series(st, nm):
    a = cp.cp_bessel_coefficients(st, nm)
    b = np.array(taylor_harmonic_coefficients(st, nm))
    np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-15)
    tail = 1.0 - a.sum()                       # sum over all harmonics is the kernel peak, 1
    assert 0.0 <= tail < 2e-3
    assert np.all(np.diff(a[1:]) < 0)           # a_n = 2 e^-k I_n(k) decreases in n


def _plan_status(offsets, grid=None, **kw):
    n = int(offsets[-1])
    t = np.arange(max(n, 1), dtype=np.float64)
    m = np.zeros(max(n, 1), np.float32)
    e = np.ones(max(n, 1), np.float32)
    g = grid or cp.make_grid(0.01, 0.01, 10)
    try:
        cp.Plan(t, m, e, np.asarray(offsets, np.int64), g, **kw)
    except cp.CpError as err:
        return err.status
    return cp.CP_OK


def test_argument_validation_precedes_device_use():
    assert _plan_status([0, 1]) == cp.CP_EINVAL                       # N < 2
    assert _plan_status([1, 5]) == cp.CP_EINVAL                       # offsets[0] != 0
    assert _plan_status([0, 5, 4]) == cp.CP_EINVAL                    # decreasing
    assert _plan_status([0, cp.cp_max_points() + 1]) == cp.CP_EUNSUPPORTED
    assert _plan_status([0, 5], grid=cp.make_grid(0.01, 0.0, 10)) == cp.CP_EINVAL
    assert _plan_status([0, 5], grid=cp.make_grid(0.01, 0.01, 0)) == cp.CP_EINVAL
    assert _plan_status([0, 5], grid=cp.make_grid(0.01, 0.01, 10, True, 0.0, 3, 1e-3, 1e-2)) == cp.CP_EINVAL
    assert _plan_status([0, 5], grid=cp.make_grid(0.01, 0.01, 10, True, 0.05, 0, 1e-3, 1e-2)) == cp.CP_EINVAL
    assert _plan_status([0, 5], sigma_t=0.0) == cp.CP_EINVAL
    assert _plan_status([0, 5], alpha=-1.0) == cp.CP_EINVAL
    assert _plan_status([0, 5], sigma_t_mode=7) == cp.CP_EINVAL
    bands = dict(bands=True, n_bands=3, trials_per_band=150)
    assert _plan_status([0, 5], grid=cp.make_grid(0.01, 0.01, 10, **dict(bands, n_bands=0))) == cp.CP_EINVAL
    assert _plan_status([0, 5], grid=cp.make_grid(0.01, 0.01, 10, **dict(bands, n_bands=11))) == cp.CP_EINVAL
    assert _plan_status([0, 5], grid=cp.make_grid(0.01, 0.01, 10, **dict(bands, trials_per_band=0))) == cp.CP_EINVAL
    assert _plan_status([0, 5], grid=cp.make_grid(0.01, 0.01, 10, **dict(bands, trials_per_band=513))) == cp.CP_EINVAL
    g = cp.make_grid(0.01, 0.01, 10)
    g.hierarchical = 3
    assert _plan_status([0, 5], grid=g) == cp.CP_EINVAL
    good = {"buckets": [{"max_n": 256, "direct_fc": 16, "tensor": {"8": True, "16": True, "32": False}},
                        {"max_n": 4096, "direct_fc": 4, "tensor": {}}]}
    t = cp.tuning_from(good)
    assert t.n_buckets == 2 and list(t.tensor_classes[:2]) == [27, 31]   # bits: 8, 16, 32, 12, 48 harmonics
    bad_fc = cp.tuning_from(good); bad_fc.direct_fc[0] = 6
    assert _plan_status([0, 5], tuning=bad_fc) == cp.CP_EINVAL
    bad_order = cp.tuning_from(good); bad_order.bucket_max_n[1] = 100
    assert _plan_status([0, 5], tuning=bad_order) == cp.CP_EINVAL
    bad_mask = cp.tuning_from(good); bad_mask.tensor_classes[0] = 32
    assert _plan_status([0, 5], tuning=bad_mask) == cp.CP_EINVAL


def test_binding_constants_match_header():
    """Every CP_* enumerator of include/cp.h has the same value in the binding."""
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "cp.h")).read(), flags=re.S)
    found = 0
    for body in re.findall(r"enum\s*\{(.*?)\}", src, flags=re.S):
        for name, val in re.findall(r"\b(CP_[A-Z0-9_]+)\s*=\s*(-?\d+)", body):
            if hasattr(cp, name):
                assert getattr(cp, name) == int(val), name
                found += 1
    assert found >= 10 and cp.CP_DTYPE_BF16_SPLIT == 2


def test_tensor_operand_type_is_validated_before_device_use():
    tensor = dict(form=cp.CP_FORM_TENSOR)
    assert _plan_status([0, 5], dtype=3, **tensor) == cp.CP_EINVAL
    assert _plan_status([0, 5], dtype=-1, **tensor) == cp.CP_EINVAL
    # split Z has no 12-harmonic class
    assert _plan_status([0, 5], dtype=cp.CP_DTYPE_BF16_SPLIT, n_max=12, **tensor) == cp.CP_EINVAL
    assert _plan_status([0, 5], dtype=cp.CP_DTYPE_BF16_SPLIT, n_max=48, **tensor) == cp.CP_EINVAL
    assert _plan_status([0, 5], dtype=cp.CP_DTYPE_BF16, n_max=20, **tensor) == cp.CP_EINVAL


def test_exclusion_windows_are_validated_before_device_use():
    """Section 6.1 windows: at most CP_MAX_EXCLUDE, finite lo <= hi; the
    no-allocation entry point refuses them (it has no plan to hold them)."""
    assert _plan_status([0, 5], grid=cp.make_grid(0.01, 0.01, 10, exclude=[(0.3, 0.2)])) == cp.CP_EINVAL
    assert _plan_status([0, 5], grid=cp.make_grid(0.01, 0.01, 10, exclude=[(float("nan"), 0.2)])) == cp.CP_EINVAL
    assert _plan_status([0, 5], grid=cp.make_grid(0.01, 0.01, 10, exclude=[(0.1, float("inf"))])) == cp.CP_EINVAL
    many = [(0.1 + q, 0.2 + q) for q in range(cp.CP_MAX_EXCLUDE + 1)]
    assert _plan_status([0, 5], grid=cp.make_grid(0.01, 0.01, 10, exclude=many)) == cp.CP_EINVAL
    g = cp.make_grid(0.01, 0.01, 10)
    g.n_exclude = 2                       # count without an array
    assert _plan_status([0, 5], grid=g) == cp.CP_EINVAL
    off = np.array([0, 5], np.int64)
    dummy = np.zeros(8)
    st = cp.lib().cp_best_period_noalloc(dummy.ctypes.data, dummy.ctypes.data, dummy.ctypes.data, off.ctypes.data,
                                         1, ctypes.byref(cp.make_grid(0.01, 0.01, 10, exclude=[(0.1, 0.2)])),
                                         ctypes.c_float(0.3), None, None, None, None, None)
    assert st == cp.CP_EUNSUPPORTED


def test_no_device_is_an_error_not_a_fallback():
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    assert _plan_status([0, 5]) == cp.CP_ECUDA
