"""Slice-range ledger: checkpoint/resume and recovery of a lost worker's
slices (Sec. V), run as two gloo ranks on the CPU.  The per-range compute
here is the oracle (CPU); on a GPU the product passes Plan.contract_slices.
Failures are made on the host: a rank raises before publishing its ranges."""
import multiprocessing as mp
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2010_14962_gb300 import instances as I
from paper_2010_14962_gb300.ledger import SliceLedger, run_local, run_ranks, shard_range, sharded_amplitude

N, P = 20, 1
CUTS = [(0, 0), (3, 1), (5, 0), (7, 1), (9, 0)]


def problem():
    inst = I.qaoa_instance(N, P, 31)
    x = I.bitstrings(N, 1, 31)[0]
    return inst, x


def compute_fn(inst, x, log=None):
    def f(lo, hi):
        if log is not None:
            log.append((lo, hi))
        v = O.tn_amplitude(N, inst.edges, inst.gamma, inst.beta, x, cuts=CUTS, slices=(lo, hi)).value
        return v, 0j
    return f


def test_checkpoint_resume(tmp_path):
    inst, x = problem()
    full = O.tn_amplitude(N, inst.edges, inst.gamma, inst.beta, x, cuts=CUTS).value
    path = str(tmp_path / "ledger.json")
    led = SliceLedger(32, 5, path)
    f = compute_fn(inst, x)
    for r in led.ranges[:3]:  # a run that stopped after three ranges
        led.record(r, *f(*r))
    resumed = SliceLedger(32, 5, path)
    assert len(resumed.done) == 3
    log = []
    total = run_local(resumed, compute_fn(inst, x, log))
    assert log == resumed.ranges[3:]  # only the missing ranges ran
    assert abs(total - full) < 1e-14
    with pytest.raises(ValueError):
        SliceLedger(32, 4, path)  # a checkpoint of another slicing


def _rank_main(rank, world, port, fail_rank, result_q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    store = dist.distributed_c10d._get_default_store()
    inst, x = problem()
    led = SliceLedger(32, 4)
    f = compute_fn(inst, x)
    if rank == fail_rank:
        # the worker dies before reporting any of its ranges
        raise SystemExit(3)
    total = run_ranks(led, f, rank, world, store, deadline_s=5.0)
    if rank == 0:
        result_q.put((total, led.recomputed))
    dist.destroy_process_group()


@pytest.mark.parametrize("fail_rank", [None, 1])
def test_two_ranks_with_a_lost_worker(fail_rank):
    inst, x = problem()
    full = O.tn_amplitude(N, inst.edges, inst.gamma, inst.beta, x, cuts=CUTS).value
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000) + (7 if fail_rank else 0)
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, fail_rank, q)) for r in range(2)]
    for p in procs:
        p.start()
    total, recomputed = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert abs(total - full) < 1e-14
    led = SliceLedger(32, 4)
    lost = [r for i, r in enumerate(led.ranges) if i % 2 == 1] if fail_rank else []
    assert recomputed == lost


def test_shard_ranges_partition_the_slices():
    for S, G in ((32, 2), (65536, 8), (5, 3), (3, 4)):
        rs = [shard_range(S, g, G) for g in range(G)]
        assert rs[0][0] == 0 and rs[-1][1] == S
        assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
        assert max(hi - lo for lo, hi in rs) - min(hi - lo for lo, hi in rs) <= 1


def _shard_main(rank, world, port, fail_rank, result_q):
    import datetime

    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    inst, x = problem()

    def f(lo, hi):
        v = O.tn_amplitude(N, inst.edges, inst.gamma, inst.beta, x, cuts=CUTS, slices=(lo, hi)).value
        return v, 0j

    if rank == fail_rank:
        raise SystemExit(3)  # dies before the all-gather (made on the host)
    total, recomputed = sharded_amplitude(f, 32, rank, world, dist)
    if rank == 0:
        result_q.put((total, recomputed))
    try:
        dist.destroy_process_group()
    except Exception:
        pass


@pytest.mark.parametrize("fail_rank", [None, 1])
def test_sharded_amplitude_two_ranks(fail_rank):
    # One amplitude over two gloo ranks: contiguous slice ranges, one
    # all-gather of (sum, comp), fixed-order sum; a rank lost before the
    # collective is detected by the group's timeout and its range recomputed.
    inst, x = problem()
    full = O.tn_amplitude(N, inst.edges, inst.gamma, inst.beta, x, cuts=CUTS).value
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 31500 + (os.getpid() % 1000) + (11 if fail_rank else 0)
    procs = [ctx.Process(target=_shard_main, args=(r, 2, port, fail_rank, q)) for r in range(2)]
    for p in procs:
        p.start()
    total, recomputed = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert abs(total - full) < 1e-14
    assert recomputed == ([shard_range(32, 1, 2)] if fail_rank else [])
