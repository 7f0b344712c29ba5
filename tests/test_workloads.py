"""Host-side helpers of the workloads: the uneven job list, fitting plans to
on-chip slices, the per-job choice of network form (no GPU)."""
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
    assert {d["p"] for d in a} == {1, 2}
    assert max(d["n"] for d in a if d["p"] == 2) > 90  # depth-2 jobs span the whole n range
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


def test_plan_job_picks_the_cheaper_network_form():
    # A depth-1 job stays on the paper's gate network; a deep job on many
    # qubits, whose gate network would need ~2^50 flops, takes the
    # graphical-model form of the same circuit (k cuts either way).
    inst = I.qaoa_instance(60, 1, 3)
    plan = qtn.plan_job(60, 1, inst.edges, inst.gamma, inst.beta, 8)
    assert plan.network.form == "gates" and plan.k == 8
    inst = I.qaoa_instance(74, 2, 4)
    plan = qtn.plan_job(74, 2, inst.edges, inst.gamma, inst.beta, 8)
    assert plan.network.form == "gm" and plan.k == 8
    gate = qtn.Network(74, inst.edges, inst.gamma, inst.beta)
    cuts, _, _ = qtn.search_cuts(gate, 8)
    assert qtn.surrogate_labels(gate, cuts)[0] > plan.cost()["log2_flops"] + 10


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
