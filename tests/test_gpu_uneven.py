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


def build_spec_jobs(spec, x_seed):
    # The workload as specified: every job plans its own k greedy cuts on the
    # gate network, or on the graphical-model form where the gate network
    # would need more than 2^36 flops (depth-2 jobs on many qubits).
    def one(jd):
        j, d = jd
        inst = I.qaoa_instance(d["n"], d["p"], d["seed"])
        plan = qtn.plan_job(d["n"], d["p"], inst.edges, inst.gamma, inst.beta, d["k"])
        x = I.bitstrings(d["n"], 1, x_seed + j)[0]
        return inst, plan.network, plan, x

    with cf.ThreadPoolExecutor(THREADS) as ex:
        return list(ex.map(one, enumerate(spec)))


@pytest.fixture(scope="module")
def uneven64():
    spec = I.uneven_jobs(**{k: v for k, v in I.WORKLOADS["uneven64"].items() if k != "jobs"},
                         jobs=I.WORKLOADS["uneven64"]["jobs"])
    jobs = build_spec_jobs(spec, 700)
    got = qtn.contract_batch([j[2] for j in jobs], [j[3] for j in jobs], "fp64")
    return spec, jobs, got


def oracle_feasible(inst):
    return inst.p == 1 or inst.n <= 40


def test_uneven64_as_specified(gpu, uneven64):
    # 64 jobs, n 30..100, p in {1, 2}, 6..18 cuts each, all in one call; the
    # deep jobs on many qubits run on the graphical-model form, several on the
    # wide executor.
    spec, jobs, got = uneven64
    assert [j[2].k for j in jobs] == [d["k"] for d in spec]
    assert max(d["n"] for d in spec if d["p"] == 2) > 90
    progs = qtn.batch_last_programs()
    assert len(progs) == len(jobs) and any(p.startswith("wide") for p in progs)
    assert all(np.isfinite(got))


def test_uneven64_vs_oracle(gpu, uneven64):
    # FP64 form against the oracle (its own cuts) on every job the oracle can
    # contract: all depth-1 jobs and the depth-2 jobs on at most 40 qubits.
    spec, jobs, got = uneven64
    checked = 0
    for g, (inst, net, plan, x) in zip(got, jobs):
        if not oracle_feasible(inst):
            continue
        cuts, _ = O.choose_cuts(inst.n, inst.edges, inst.p, 10 if inst.p == 2 else 8)
        r = O.tn_amplitude(inst.n, inst.edges, inst.gamma, inst.beta, x, cuts=cuts, threads=THREADS).value
        assert abs(g - r) <= 1e-10 * abs(r), (inst.n, inst.p, plan.k)
        checked += 1
    print("checked", checked, "of", len(jobs))
    assert checked >= 30


def test_uneven64_closed_forms_beyond_the_oracle(gpu, uneven64):
    # Depth-2 jobs beyond the oracle: the same plans at angles with closed
    # forms (any size): gamma = 0 gives a = e^{-i n (b1 + b2)} 2^{-n/2};
    # beta = 0 gives a = 2^{-n/2} e^{-i (g1 + g2) sum_E s_i s_j}, s = 1 - 2 x.
    spec, jobs, got = uneven64
    checked = 0
    for inst, net, plan, x in jobs:
        if oracle_feasible(inst):
            continue
        n = inst.n
        G = np.array([[0.0, 0.0], list(inst.gamma)])
        B = np.array([list(inst.beta), [0.0, 0.0]])
        d_x = torch.from_numpy(np.ascontiguousarray(np.stack([x, x]))).cuda()
        d_g = torch.from_numpy(np.ascontiguousarray(G)).cuda()
        d_b = torch.from_numpy(np.ascontiguousarray(B)).cuda()
        d_out = torch.zeros((2, 2), dtype=torch.float64, device="cuda")
        plan.contract_sweep_device(d_x, d_g, d_b, d_out, "fp32x2")
        torch.cuda.synchronize()
        o = d_out.cpu().numpy()
        a = o[:, 0] + 1j * o[:, 1]
        s = 1 - 2 * x.astype(np.int64)
        zz = int(np.sum(s[inst.edges[:, 0]] * s[inst.edges[:, 1]]))
        want = [np.exp(-1j * n * inst.beta.sum()) * 2.0 ** (-n / 2),
                np.exp(-1j * inst.gamma.sum() * zz) * 2.0 ** (-n / 2)]
        for got_i, want_i in zip(a, want):
            assert abs(got_i - want_i) <= 1e-10 * abs(want_i), (n, plan.k, got_i, want_i)
        checked += 1
    print("closed forms checked on", checked, "jobs")
    assert checked >= 10


def test_uneven64_vs_single_plan(gpu, uneven64):
    # Every job of the batch equals its single-plan contraction (FP64 form).
    spec, jobs, got = uneven64
    for g, (inst, net, plan, x) in zip(got, jobs):
        single = plan.contract_amplitude(x, "fp64")
        assert abs(g - single) <= 1e-11 * abs(single), (inst.n, inst.p, plan.k)
