"""Failure handling of the C ABI on a GPU, made on the host: an allocation
that the test makes fail (CP_FAIL_ALLOC) must give CP_ENOMEM, release what
the plan had allocated, and leave the next plan unaffected."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1412_1840_gb300 as cp  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_allocation_failure_reports_enomem_and_leaves_nothing(monkeypatch):
    b = synth.ragged_batch(256, seed=51, n_lo=900, n_hi=1000)    # ~0.5 GB of magnitude-kernel tiles
    g = synth.Grid(0.01, 1e-3, 64)
    grid = cp.grid_from(g)
    td = torch.from_numpy(b.times).cuda()
    md = torch.from_numpy(b.mags).cuda()
    ed = torch.from_numpy(b.errs).cuda()
    with cp.Plan(td, md, ed, b.offsets, grid, sigma_t=0.3) as p:
        want = p.best_period()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for k in (1, 2):                       # the device block, then the pinned host block
        monkeypatch.setenv("CP_FAIL_ALLOC", str(k))
        with pytest.raises(cp.CpError) as e:
            cp.Plan(td, md, ed, b.offsets, grid, sigma_t=0.3)
        assert e.value.status == cp.CP_ENOMEM
        torch.cuda.synchronize()
        assert abs(torch.cuda.mem_get_info()[0] - free0) < (64 << 20)
    monkeypatch.delenv("CP_FAIL_ALLOC")
    with cp.Plan(td, md, ed, b.offsets, grid, sigma_t=0.3) as p:
        got = p.best_period()
    for k in ("best_idx", "best_freq", "best_stat", "is_periodic"):
        np.testing.assert_array_equal(got[k], want[k])
