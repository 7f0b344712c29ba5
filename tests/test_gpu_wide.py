"""GPU parity of the wide executor (intermediates in device memory, one
launch per merge) and of its tensor-core merge kernel, through the C ABI,
against the state vector and the oracle.

Deep circuits (p = 3) at n = 20 keep tensors of rank up to 23 with 2 cuts, so
the per-slice program itself is wide, and nearly all multiply-adds are in
dense merges (one side >= 128, the other >= 8, K >= 4) that the tcgen05
kernel takes.

Tolerances: complex128 and double-float: 1e-10 relative.  FP32-accumulated
forms (first order, per slice): each operand rounding contributes u (the
operand format's unit roundoff, per gate tensor, 2 G of them coherently) and
each merge's FP32 accumulation of K products at most (K - 1) u32 of the
magnitudes it adds; so |a - a*| <= (2 G u + sum_j K_j u32) * sum_s |a_s|,
with sum_s |a_s| from the oracle's per-slice values.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import oracle as O
from paper_2010_14962_gb300 import instances as I
from paper_2010_14962_gb300 import qtn

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

U32 = 2.0 ** -24
U_OPERAND = {"fp32": U32, "tf32x3": 2.0 ** -22, "tf32": 2.0 ** -11}


def amplitudes(plan, xs, prec):
    d_x = torch.from_numpy(np.ascontiguousarray(xs.astype(np.uint8))).cuda()
    d_out = torch.zeros((xs.shape[0], 2), dtype=torch.float64, device="cuda")
    plan.contract_amplitudes_device(d_x, d_out, prec)
    torch.cuda.synchronize()
    o = d_out.cpu().numpy()
    return o[:, 0] + 1j * o[:, 1]


@pytest.fixture(scope="module")
def deep20():
    n, p, k = 20, 3, 2
    inst = I.qaoa_instance(n, p, 11)
    plan = qtn.Plan(qtn.Network(n, inst.edges, inst.gamma, inst.beta), k=k)
    d = plan.describe()
    assert d["executor"] == "wide" and plan.cost()["width"] > 16
    sv = O.statevector(n, inst.edges, inst.gamma, inst.beta)
    xs = I.bitstrings(n, 4, 11)
    refs = np.array([sv[O.bits_to_int(x)] for x in xs])
    l1 = []
    for x in xs:
        r = O.tn_amplitude(n, inst.edges, inst.gamma, inst.beta, x, cuts=plan.cut_names(), per_slice=True,
                           threads=16)
        l1.append(np.sum(np.abs(r.per_slice)))
    ksum = sum(2 ** st["kb"] for st in d["programs"]["wide"]["steps"] + d["programs"]["wide"]["prologue"])
    return inst, plan, xs, refs, np.array(l1), ksum


def bound(inst, prec, l1, ksum):
    G = len(inst.edges) * inst.p
    return (2 * G * U_OPERAND[prec] + ksum * U32) * l1


@pytest.mark.parametrize("prec", ["fp64", "fp32x2", "fp32"])
def test_wide_executor_matches_statevector(gpu, deep20, prec):
    inst, plan, xs, refs, l1, ksum = deep20
    qtn.wide_set_kernel("auto")
    for name in ("wide/slices", "wide/classes"):
        plan.select_executor(name, prec, len(xs))
        got = amplitudes(plan, xs, prec)
        if prec == "fp32":
            assert np.all(np.abs(got - refs) <= bound(inst, prec, l1, ksum)), name
        else:
            assert np.max(np.abs(got - refs) / np.abs(refs)) < 1e-10, name


@pytest.mark.parametrize("prec", ["tf32x3", "tf32"])
def test_wide_tensor_core_merges(gpu, deep20, prec):
    # The tcgen05 kernel forced on every merge that allows it, then the SIMT
    # kernels (TF32 rounding emulated on the FP32 pipe) on the same plan:
    # both within the bound against the state vector.
    inst, plan, xs, refs, l1, ksum = deep20
    try:
        for mode in ("tcgen05", "simt"):
            qtn.wide_set_kernel(mode)
            plan.select_executor("wide/slices", prec, len(xs))
            got = amplitudes(plan, xs, prec)
            err = np.abs(got - refs)
            print(prec, mode, "max rel err", np.max(err / np.abs(refs)))
            assert np.all(err <= bound(inst, prec, l1, ksum)), mode
            states = [s for s in plan.describe()["programs"]["wide/slices"]["wide_states"]
                      if s["prec"] == qtn.PRECISIONS[prec] and s["nx"] == len(xs)]
            kinds = set(states[0]["step_kernels"])
            if mode == "tcgen05":
                assert "tcgen05" in kinds
            else:
                assert "tcgen05" not in kinds
    finally:
        qtn.wide_set_kernel("auto")


def test_wide_per_slice_values(gpu, deep20):
    # Slice ranges on the wide per-slice program: every slice value against
    # the oracle's, and the ranges add up to the amplitude (Eq. 2).
    inst, plan, xs, refs, l1, ksum = deep20
    x = xs[0]
    n = inst.n
    ref = O.tn_amplitude(n, inst.edges, inst.gamma, inst.beta, x, cuts=plan.cut_names(), per_slice=True, threads=16)
    total, comp, per = plan.contract_slices(x, 0, 4, "fp64", per_slice=True)
    scale = 2.0 ** (-n / 2)
    assert np.max(np.abs(per * scale - ref.per_slice)) < 1e-12 * np.max(np.abs(ref.per_slice))
    parts = [plan.contract_slices(x, lo, hi, "fp64") for lo, hi in ((0, 1), (1, 3), (3, 4))]
    assert abs(sum(s - c for s, c in parts) - (total - comp)) < 1e-13 * abs(total)


@pytest.mark.parametrize("n,p,k,seed", [(40, 2, 4, 2), (18, 3, 0, 11)])
def test_wide_executor_against_oracle(gpu, n, p, k, seed):
    # A plan that also fits on chip (n = 40, p = 2, 4 cuts: dense merges up
    # to M = 512, N = 64, K = 64) and an uncut one: the wide program in FP64
    # against the oracle's own plan; the uncut one also in TF32X3 on the
    # tensor cores (no slices: sum_s |a_s| = |a|, so the bound is relative).
    inst = I.qaoa_instance(n, p, seed)
    plan = qtn.Plan(qtn.Network(n, inst.edges, inst.gamma, inst.beta), k=k)
    xs = I.bitstrings(n, 2, seed)
    cuts, _ = O.choose_cuts(n, inst.edges, p, 10 if n >= 40 else 4)
    refs = np.array([O.tn_amplitude(n, inst.edges, inst.gamma, inst.beta, x, cuts=cuts, threads=16).value
                     for x in xs])
    name = "wide/classes"
    plan.select_executor(name, "fp64", len(xs))
    got = amplitudes(plan, xs, "fp64")
    assert np.max(np.abs(got - refs) / np.abs(refs)) < 1e-10
    if k:
        return
    d = plan.describe()
    ksum = sum(2 ** st["kb"] for st in d["programs"][name]["steps"] + d["programs"][name]["prologue"])
    try:
        qtn.wide_set_kernel("tcgen05")
        plan.select_executor(name, "tf32x3", len(xs))
        got = amplitudes(plan, xs, "tf32x3")
        rel = np.abs(got - refs) / np.abs(refs)
        print("tf32x3 on tensor cores: max rel err", rel.max())
        assert np.all(rel <= 2 * len(inst.edges) * p * U_OPERAND["tf32x3"] + ksum * U32)
    finally:
        qtn.wide_set_kernel("auto")


_CACHE_RUN = r"""
import json, sys
import numpy as np, torch
from paper_2010_14962_gb300 import instances as I, qtn
inst = I.qaoa_instance(20, 3, 11)
plan = qtn.Plan(qtn.Network(20, inst.edges, inst.gamma, inst.beta), k=2)
xs = I.bitstrings(20, 4, 11)
plan.select_executor("wide/slices", "fp32", len(xs))
d_x = torch.from_numpy(np.ascontiguousarray(xs)).cuda()
d_out = torch.zeros((len(xs), 2), dtype=torch.float64, device="cuda")
plan.contract_amplitudes_device(d_x, d_out, "fp32")
torch.cuda.synchronize()
st = [s for s in plan.describe()["programs"]["wide/slices"]["wide_states"] if s["nx"] == len(xs)][0]
o = d_out.cpu().numpy()
print(json.dumps({"kernels": st["step_kernels"], "re": o[:, 0].tolist(), "im": o[:, 1].tolist()}))
"""


def _cache_run(path):
    env = dict(os.environ, QTN_WIDE_TUNE_CACHE=str(path))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _CACHE_RUN], env=env, cwd=root, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return d["kernels"], np.array(d["re"]) + 1j * np.array(d["im"])


def test_wide_tune_cache_round_trip(gpu, deep20, tmp_path):
    # The per-shape winners file: a process that tunes writes one JSON line
    # per step shape (ma, nb, kb, bb, items, arithmetic -> kernel); a new
    # process reads it and runs the recorded kernels without timing.  Every
    # entry rewritten to the one-output SIMT kernel (not the winner of most
    # shapes) still gives the amplitudes within the FP32 bound.
    inst, plan, xs, refs, l1, ksum = deep20
    path = tmp_path / "wide_tune.jsonl"
    k1, a1 = _cache_run(path)
    lines = [json.loads(x) for x in path.read_text().splitlines()]
    assert lines and all({"ma", "nb", "kb", "bb", "items", "arith", "best"} <= set(e) for e in lines)
    assert np.all(np.abs(a1 - refs) <= bound(inst, "fp32", l1, ksum))
    path.write_text("".join(json.dumps(dict(e, best=0, kernel="simt"), separators=(",", ":")) + "\n" for e in lines))
    k2, a2 = _cache_run(path)
    assert set(k2) == {"simt"}, k2
    assert np.all(np.abs(a2 - refs) <= bound(inst, "fp32", l1, ksum))
