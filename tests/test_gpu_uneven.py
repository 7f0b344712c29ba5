"""GPU parity of the multi-job launch (many independent circuits, each with its
own cut set and elimination order, Sec. III.A, in one launch sequence).

Every job's amplitude is compared with the oracle.  The oracle may take fewer
of the plan's cuts than the device (Eq. 2: the sum over slices does not depend
on which indices are cut), which is far cheaper for depth-1 jobs whose many
cuts leave tiny slices.
"""
import concurrent.futures as cf
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2010_14962_gb300 import instances as I
from paper_2010_14962_gb300 import qtn

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

U32 = 2.0 ** -24
THREADS = max(1, min(16, os.cpu_count() or 1))


def build_jobs(spec, x_seed):
    def one(jd):
        j, d = jd
        inst = I.qaoa_instance(d["n"], d["p"], d["seed"])
        net = qtn.Network(d["n"], inst.edges, inst.gamma, inst.beta)
        plan = qtn.plan_to_fit(net, d["k"])
        x = I.bitstrings(d["n"], 1, x_seed + j)[0]
        return inst, net, plan, x

    with cf.ThreadPoolExecutor(THREADS) as ex:
        return list(ex.map(one, enumerate(spec)))


def oracle_cuts(inst, plan, drop):
    names = plan.cut_names()
    return names[: max(0, len(names) - drop)] if inst.p == 1 else names


@pytest.fixture(scope="module")
def small_batch():
    # 24 jobs: n in 20..48, p in {1, 2}, 4..10 cuts requested.
    spec = I.uneven_jobs(jobs=24, n_range=(20, 48), k_range=(4, 10), seed=9, p2_n_max=32)
    jobs = build_jobs(spec, 500)
    refs = []
    for inst, net, plan, x in jobs:
        r = O.tn_amplitude(inst.n, inst.edges, inst.gamma, inst.beta, x, cuts=plan.cut_names(), per_slice=True,
                           threads=THREADS)
        refs.append((r.value, float(np.sum(np.abs(r.per_slice)))))
    return jobs, refs


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32x2", 1e-10)])
def test_small_batch_wide(gpu, small_batch, prec, tol):
    jobs, refs = small_batch
    got = qtn.contract_batch([j[2] for j in jobs], [j[3] for j in jobs], prec)
    errs = [abs(g - r) / abs(r) for g, (r, _) in zip(got, refs)]
    print(prec, "max rel err", max(errs))
    assert max(errs) < tol


def test_small_batch_fp32(gpu, small_batch):
    # Per job: |a - a*| <= 2 G u sum_s |a_s| (G = gate tensors + merges).
    jobs, refs = small_batch
    got = qtn.contract_batch([j[2] for j in jobs], [j[3] for j in jobs], "fp32")
    for g, (inst, net, plan, x), (r, l1) in zip(got, jobs, refs):
        G = len(inst.edges) * inst.p * 2
        assert abs(g - r) <= max(2 * G * U32 * l1, 1e-12 * abs(r)), (inst.n, inst.p)


def test_small_batch_repeat_and_order(gpu, small_batch):
    # The chunk partials are summed in a fixed order: repeated calls agree
    # bit for bit, and a job's value does not depend on its batch neighbours.
    jobs, _ = small_batch
    plans, xs = [j[2] for j in jobs], [j[3] for j in jobs]
    a = qtn.contract_batch(plans, xs, "fp64")
    b = qtn.contract_batch(plans, xs, "fp64")
    assert np.array_equal(a, b)
    rev = qtn.contract_batch(plans[::-1], xs[::-1], "fp64")[::-1]
    np.testing.assert_allclose(rev, a, rtol=1e-13, atol=0)
    one = qtn.contract_batch(plans[:1], xs[:1], "fp64")
    assert abs(one[0] - a[0]) <= 1e-13 * abs(a[0])


@pytest.fixture(scope="module")
def uneven64():
    spec = I.uneven_jobs(**{k: v for k, v in I.WORKLOADS["uneven64"].items() if k != "jobs"},
                         jobs=I.WORKLOADS["uneven64"]["jobs"])
    return spec, build_jobs(spec, 700)


def test_uneven64_vs_oracle(gpu, uneven64):
    # The full 64-job workload in one launch sequence, FP64 form, against the
    # oracle on every depth-1 job and on the depth-2 jobs of <= 2^31 flops.
    spec, jobs = uneven64
    got = qtn.contract_batch([j[2] for j in jobs], [j[3] for j in jobs], "fp64")
    checked = 0
    for g, (inst, net, plan, x) in zip(got, jobs):
        if inst.p == 2 and plan.cost()["log2_flops"] > 31:
            continue
        r = O.tn_amplitude(inst.n, inst.edges, inst.gamma, inst.beta, x, cuts=oracle_cuts(inst, plan, 8),
                           threads=THREADS).value
        assert abs(g - r) <= 1e-10 * abs(r), (inst.n, inst.p, plan.k)
        checked += 1
    print("checked", checked, "of", len(jobs))
    assert checked >= 40


def test_uneven64_vs_single_plan(gpu, uneven64):
    # Every job of the batch equals its single-plan contraction (FP64 form).
    spec, jobs = uneven64
    got = qtn.contract_batch([j[2] for j in jobs], [j[3] for j in jobs], "fp64")
    for g, (inst, net, plan, x) in zip(got, jobs):
        single = plan.contract_amplitude(x, "fp64")
        assert abs(g - single) <= 1e-11 * abs(single), (inst.n, inst.p, plan.k)


def test_uneven64_mixed_precision(gpu, uneven64):
    # FP32 merges, FP64 sums: relative error against the FP64 form.
    spec, jobs = uneven64
    plans, xs = [j[2] for j in jobs], [j[3] for j in jobs]
    ref = qtn.contract_batch(plans, xs, "fp64")
    for prec, tol in [("fp32x2", 1e-10), ("fp32", 1e-3)]:
        got = qtn.contract_batch(plans, xs, prec)
        err = np.abs(got - ref) / np.abs(ref)
        print(prec, "max rel err vs FP64", float(err.max()), "median", float(np.median(err)))
        assert float(err.max()) < tol


def test_batch_time_limit_and_cancel(gpu, uneven64):
    # Cooperative stop of the persistent executor (checked between chunks;
    # nothing waits on the device): a time limit, and a cancel from another
    # host thread.  A stopped call reports QTN_ERR_TIMEOUT; later calls work.
    import threading
    import time

    spec, jobs = uneven64
    plans, xs = [j[2] for j in jobs], [j[3] for j in jobs]
    t0 = time.perf_counter()
    full = qtn.contract_batch(plans, xs, "fp64")
    t_full = time.perf_counter() - t0
    qtn.batch_set_time_limit(0.001)
    try:
        with pytest.raises(qtn.QTNError) as e:
            qtn.contract_batch(plans, xs, "fp64")
        assert e.value.status == 5
    finally:
        qtn.batch_set_time_limit(0)
    if t_full > 0.1:
        timer = threading.Timer(t_full / 4, qtn.batch_cancel)
        timer.start()
        t0 = time.perf_counter()
        with pytest.raises(qtn.QTNError) as e:
            qtn.contract_batch(plans, xs, "fp64")
        assert e.value.status == 5 and time.perf_counter() - t0 < 0.9 * t_full
        timer.join()
    again = qtn.contract_batch(plans, xs, "fp64")
    assert np.array_equal(again, full)
    with pytest.raises(qtn.QTNError):
        qtn.batch_set_time_limit(-1)
