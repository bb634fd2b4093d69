"""Multi-process path on CPU (gloo, world_size 2): curve sharding and the
max-over-ranks timing reduction used by the multi-GPU benchmark."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

import synth
from paper_1412_1840_gb300.shard import curve_ranges, gather_results, local_csr, max_over_ranks


def test_curve_ranges_cover_and_balance():
    b = synth.ragged_batch(101, seed=3, n_lo=20, n_hi=400)
    for world in (1, 2, 3, 8):
        rs = curve_ranges(b.offsets, world)
        assert rs[0][0] == 0 and rs[-1][1] == b.n_curves
        assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
        n = b.sizes.astype(float)
        cost = [np.sum(n[a:c] * (n[a:c] - 1) / 2) for a, c in rs]
        assert max(cost) <= np.sum(n * (n - 1) / 2) / world + np.max(n * (n - 1) / 2)
    assert curve_ranges(np.array([0, 5, 9]), 4)[-1][1] == 2


def test_local_csr_rebases_offsets():
    b = synth.ragged_batch(9, seed=4, n_lo=3, n_hi=9)
    t, m, e, off = local_csr(b.times, b.mags, b.errs, b.offsets, (3, 7))
    assert off[0] == 0 and off[-1] == t.shape[0] == m.shape[0] == e.shape[0]
    np.testing.assert_array_equal(t, b.times[b.offsets[3]:b.offsets[7]])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = synth.ragged_batch(40, seed=5, n_lo=10, n_hi=60)
    a, c = curve_ranges(b.offsets, world)[rank]
    t, m, e, off = local_csr(b.times, b.mags, b.errs, b.offsets, (a, c))
    elapsed = 1.0 + rank                       # stand-in for a rank's measured step time
    dist.barrier()
    mx = max_over_ranks(elapsed)
    q.put((rank, a, c, int(off[-1]), mx))
    dist.destroy_process_group()


def test_two_ranks_shard_and_reduce_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    b = synth.ragged_batch(40, seed=5, n_lo=10, n_hi=60)
    assert res[0][1] == 0 and res[0][2] == res[1][1] and res[1][2] == b.n_curves
    assert res[0][3] + res[1][3] == b.offsets[-1]
    assert res[0][4] == res[1][4] == 2.0        # max over ranks


def _oracle_worker(rank, world, port, q):
    """One rank of a sharded search: the oracle stands in for the GPU on the
    rank's contiguous curve range; the results are gathered in curve order."""
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = synth.ragged_batch(11, seed=6, n_lo=8, n_hi=40, span=300.0)
    g = synth.Grid(0.02, 2e-3, 120)
    a, c = curve_ranges(b.offsets, world)[rank]
    t, m, e, off = local_csr(b.times, b.mags, b.errs, b.offsets, (a, c))
    sub = synth.Batch(t, m, e, off, b.period[a:c], b.periodic[a:c], b.kind[a:c])
    r = oracle.batch_best(sub, g, sigma_t=0.3) if c > a else {
        "best_idx": np.zeros(0, np.int64), "best_freq": np.zeros(0), "best_stat": np.zeros(0),
        "is_periodic": np.zeros(0, bool)}
    got = gather_results({k: r[k] for k in ("best_idx", "best_freq", "best_stat", "is_periodic")}, world)
    if rank == 0:
        q.put(got)
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_search_gathers_the_whole_batch_result():
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_oracle_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    b = synth.ragged_batch(11, seed=6, n_lo=8, n_hi=40, span=300.0)
    want = oracle.batch_best(b, synth.Grid(0.02, 2e-3, 120), sigma_t=0.3)
    for k in ("best_idx", "best_freq", "best_stat", "is_periodic"):
        np.testing.assert_array_equal(got[k], want[k])
