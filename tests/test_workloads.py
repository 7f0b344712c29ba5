"""Host-side helpers of the workloads: the uneven job list, fitting plans to
on-chip slices, and the batch's choice of program (no GPU)."""
import numpy as np
import pytest

from paper_2010_14962_gb300 import instances as I
from paper_2010_14962_gb300 import qtn


def test_uneven_jobs_recipe():
    a = I.uneven_jobs()
    b = I.uneven_jobs()
    assert a == b and len(a) == 64
    for d in a:
        assert d["n"] % 2 == 0 and 30 <= d["n"] <= 100 and 6 <= d["k"] <= 18 and d["p"] in (1, 2)
        if d["p"] == 2:
            assert d["n"] <= 40  # depth-2 jobs stay where 6-18 cuts reach on-chip slices
    assert {d["p"] for d in a} == {1, 2}
    small = I.uneven_jobs(jobs=8, n_range=(20, 30), k_range=(2, 3), seed=1, p2_n_max=24)
    assert all(20 <= d["n"] <= 30 and 2 <= d["k"] <= 3 for d in small)


def test_plan_to_fit():
    inst = I.qaoa_instance(36, 2, 11)
    net = qtn.Network(36, inst.edges, inst.gamma, inst.beta)
    plan = qtn.plan_to_fit(net, 6, slice_bytes=65536.0)
    c = plan.cost()
    assert c["k"] >= 6 and c["log2_peak_bytes"] <= 16.0 + 1e-9
    # The fewest cuts: one cut less does not fit (greedy prefixes).
    cuts, _, _ = qtn.search_cuts(net, 24)
    assert list(plan.cuts) == list(cuts[: c["k"]])
    if c["k"] > 6:
        with pytest.raises(qtn.QTNError):
            qtn.Plan(net, cuts=cuts[: c["k"] - 1], max_slice_bytes=65536.0)
    with pytest.raises(qtn.QTNError) as e:
        qtn.plan_to_fit(net, 1, k_max=2, slice_bytes=64.0)
    assert e.value.status == 3


def test_batch_program_is_least_work_level_program():
    inst = I.qaoa_instance(40, 2, 2)
    plan = qtn.Plan(qtn.Network(40, inst.edges, inst.gamma, inst.beta), k=10)
    progs = plan.describe()["programs"]
    for prec, other in (("fp32x2", "/fp32/"), ("fp32", "/fp64/")):
        name = qtn.batch_program(plan, prec)
        assert progs[name]["executor"] == "level" and other not in name
        work = lambda pr: (2 ** len(pr["outer_class"])) * pr["macs_per_item"]
        best = min(work(pr) for nm, pr in progs.items() if pr["executor"] == "level" and other not in nm)
        assert work(progs[name]) == best


def test_bench_step_classes_cover_the_program():
    # The benchmark's per-class breakdown: classes partition the steps and the
    # executed multiply-adds of the program.
    import os
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    inst = I.qaoa_instance(40, 2, 2)
    plan = qtn.Plan(qtn.Network(40, inst.edges, inst.gamma, inst.beta), k=10)
    for name, prog in plan.describe()["programs"].items():
        cls = bench.step_classes(prog, 16)
        assert sum(c["steps"] for c in cls) == len(prog["steps"]), name
        assert abs(sum(c["mac_share"] for c in cls) - 1.0) < 1e-12, name
        assert all(c["flop_per_byte"] > 0 for c in cls), name
