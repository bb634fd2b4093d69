"""cp_best_period_noalloc: the entry point for callers that cannot allocate
device memory when they need a result (hosts that reserve all device memory
for their own pools at start-up, latency-bounded pipelines that must not
enter the allocator, plug-ins whose host owns the allocator).  It keeps its
intermediates in a static device array instead of allocating; its results
must match the plan-based cp_best_period on the same inputs.

Collected last (file name) so that a failure here does not hide the others.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1412_1840_gb300 as cp  # noqa: E402

TOL = 1e-5   # the direct form's statistic tolerance used throughout the tests


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def via_noalloc(b, g, sigma_t):
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    n = b.n_curves
    idx = torch.full((n,), -7, dtype=torch.int64, device="cuda")
    f = torch.zeros(n, dtype=torch.float64, device="cuda")
    v = torch.zeros(n, dtype=torch.float32, device="cuda")
    per = torch.zeros(n, dtype=torch.uint8, device="cuda")
    cp.cp_best_period_noalloc(dev(b.times), dev(b.mags), dev(b.errs), b.offsets, cp.grid_from(g), sigma_t,
                              idx, f, v, per)
    return {"best_idx": idx.cpu().numpy(), "best_freq": f.cpu().numpy(), "best_stat": v.cpu().numpy(),
            "is_periodic": per.cpu().numpy().astype(bool)}


def via_plan(b, g, sigma_t):
    with cp.Plan(b.times, b.mags, b.errs, b.offsets, cp.grid_from(g), sigma_t=sigma_t) as p:
        return p.best_period()


def same(a, r):
    np.testing.assert_array_equal(a["best_idx"], r["best_idx"])
    np.testing.assert_allclose(a["best_freq"], r["best_freq"], rtol=0, atol=0)
    scale = np.maximum(np.abs(r["best_stat"]), 1e-30)
    assert np.all(np.abs(a["best_stat"] - r["best_stat"]) <= TOL * scale)
    np.testing.assert_array_equal(a["is_periodic"], r["is_periodic"])


def test_noalloc_matches_plan_on_two_calls_in_a_row():
    a = synth.ragged_batch(12, seed=41, n_lo=40, n_hi=420)
    b = synth.ragged_batch(7, seed=42, n_lo=200, n_hi=700)
    g = synth.Grid(0.01, 1e-3, 900)
    first = via_noalloc(a, g, 0.3)
    second = via_noalloc(b, g, 0.25)       # reuses the same scratch, other sizes
    same(first, via_plan(a, g, 0.3))
    same(second, via_plan(b, g, 0.25))


def test_noalloc_hierarchical_twice():
    b = synth.ragged_batch(9, seed=43, n_lo=60, n_hi=300, span=1500.0)
    g = synth.Grid(0.02, 1e-4, 19801, hierarchical=True, coarse_df=5e-3, top_k=5, fine_df=1e-4,
                   fine_halfwidth=3e-3)
    ref = via_plan(b, g, 0.4)
    same(via_noalloc(b, g, 0.4), ref)
    same(via_noalloc(b, g, 0.4), ref)


def test_noalloc_limits_are_reported():
    b = synth.ragged_batch(300, seed=44, n_lo=10, n_hi=12)
    g = synth.Grid(0.01, 1e-2, 10)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    with pytest.raises(cp.CpError) as e:
        cp.cp_best_period_noalloc(dev(b.times), dev(b.mags), dev(b.errs), b.offsets, cp.grid_from(g), 0.3)
    assert e.value.status == cp.CP_EUNSUPPORTED       # more than CP_NOALLOC_MAX_CURVES curves


def test_noalloc_does_not_shrink_a_plans_shared_memory():
    """A plan for long curves, then a no-allocation call on short ones, then
    the plan's first search: the plan's launches still get the shared
    memory they were planned with (the limit is process-wide per kernel)."""
    big = synth.ragged_batch(3, seed=45, n_lo=900, n_hi=1000)
    small = synth.ragged_batch(4, seed=46, n_lo=20, n_hi=60)
    g = synth.Grid(0.01, 1e-3, 300)
    p = cp.Plan(big.times, big.mags, big.errs, big.offsets, cp.grid_from(g), sigma_t=0.3)
    try:
        via_noalloc(small, g, 0.3)
        got = p.best_period()
    finally:
        p.close()
    same(got, via_plan(big, g, 0.3))


def test_noalloc_allocates_nothing():
    """After a first call, a second call changes neither the device's free
    memory nor what torch's allocator holds (the outputs are allocated by
    the caller beforehand)."""
    b = synth.ragged_batch(9, seed=47, n_lo=100, n_hi=500)
    g = synth.Grid(0.01, 1e-3, 700)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    t, m, e = dev(b.times), dev(b.mags), dev(b.errs)
    outs = (torch.empty(b.n_curves, dtype=torch.int64, device="cuda"),
            torch.empty(b.n_curves, dtype=torch.float64, device="cuda"),
            torch.empty(b.n_curves, dtype=torch.float32, device="cuda"),
            torch.empty(b.n_curves, dtype=torch.uint8, device="cuda"))
    cp.cp_best_period_noalloc(t, m, e, b.offsets, cp.grid_from(g), 0.3, *outs)
    torch.cuda.synchronize()
    free0, held0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    cp.cp_best_period_noalloc(t, m, e, b.offsets, cp.grid_from(g), 0.3, *outs)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == held0


def test_noalloc_rejects_bad_arguments_before_the_gpu():
    """Wrong dtypes, sizes and host pointers are refused before any kernel
    runs; so are grids whose refinement width overflows."""
    import ctypes
    b = synth.ragged_batch(3, seed=48, n_lo=30, n_hi=40)
    g = synth.Grid(0.01, 1e-3, 100)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    t, m, e = dev(b.times), dev(b.mags), dev(b.errs)
    with pytest.raises(ValueError):
        cp.cp_best_period_noalloc(t.float(), m, e, b.offsets, cp.grid_from(g), 0.3)
    with pytest.raises(ValueError):
        cp.cp_best_period_noalloc(t, m[:-1].contiguous(), e, b.offsets, cp.grid_from(g), 0.3)
    with pytest.raises(ValueError):
        cp.cp_best_period_noalloc(t, m, e, b.offsets, cp.grid_from(g), 0.3,
                                  best_stat=torch.empty(b.n_curves + 1, device="cuda"))
    L = cp.lib()
    off = np.ascontiguousarray(b.offsets, np.int64)
    grid = cp.grid_from(g)
    # host arrays through the C ABI: CP_EINVAL, nothing launched
    st = L.cp_best_period_noalloc(b.times.ctypes.data, b.mags.ctypes.data, b.errs.ctypes.data, off.ctypes.data,
                                  b.n_curves, ctypes.byref(grid), ctypes.c_float(0.3), None, None, None, None, None)
    assert st == cp.CP_EINVAL
    # a fine step so small that the refinement half-width overflows any integer type
    bad = cp.make_grid(0.01, 1e-3, 100, hierarchical=True, coarse_df=1e-2, top_k=3, fine_df=1e-300,
                       fine_halfwidth=1e-3)
    st = L.cp_best_period_noalloc(t.data_ptr(), m.data_ptr(), e.data_ptr(), off.ctypes.data, b.n_curves,
                                  ctypes.byref(bad), ctypes.c_float(0.3), None, None, None, None, None)
    assert st == cp.CP_EINVAL
    inf = cp.make_grid(0.01, 1e-3, 100, hierarchical=True, coarse_df=1e-2, top_k=3, fine_df=1e-4,
                       fine_halfwidth=float("inf"))
    st = L.cp_best_period_noalloc(t.data_ptr(), m.data_ptr(), e.data_ptr(), off.ctypes.data, b.n_curves,
                                  ctypes.byref(inf), ctypes.c_float(0.3), None, None, None, None, None)
    assert st == cp.CP_EINVAL
