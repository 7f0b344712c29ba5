"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (relative error |a - a*| / |a*| unless stated):
  * complex128 path: 1e-10 (the FP64 form's bound).
  * complex64 path: the slice value is multilinear in the gate tensors, so
    to first order each rounding to FP32 (u = 2^-24) -- of a gate-tensor
    entry or of a merge's output -- perturbs it by at most u relative.  All
    gates share the same rounded cos/sin values, so these errors add
    coherently: per slice |da_s| <= 2 * G * u * |a_s| with G = #gates
    (leaves and merges).  The slices of Eq. 2 partly cancel, so the bound on
    the amplitude is absolute: |a - a*| <= 2 * G * u * sum_s |a_s|, with
    sum_s |a_s| from the oracle's per-slice values.  Where that sum is not
    computed, the relative bound stated at the test is used.
"""
import ctypes
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2010_14962_gb300 import instances as I
from paper_2010_14962_gb300 import qtn

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


U32 = 2.0 ** -24


def rel(a, b):
    return abs(a - b) / abs(b)


def fp32_bound(n_gates, per_slice):
    return 2 * n_gates * U32 * np.sum(np.abs(per_slice))


def device_amplitudes(plan, xs, prec):
    d_x = torch.from_numpy(np.ascontiguousarray(xs.astype(np.uint8))).cuda()
    d_out = torch.zeros((xs.shape[0], 2), dtype=torch.float64, device="cuda")
    plan.contract_amplitudes_device(d_x, d_out, prec)
    torch.cuda.synchronize()
    o = d_out.cpu().numpy()
    return o[:, 0] + 1j * o[:, 1]


@pytest.fixture(scope="module")
def config16():
    n, p, k = 16, 1, 2
    inst = I.qaoa_instance(n, p, 1)
    net = qtn.Network(n, inst.edges, inst.gamma, inst.beta)
    plan = qtn.Plan(net, k=k)
    sv = O.statevector(n, inst.edges, inst.gamma, inst.beta)
    return inst, net, plan, sv


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_every_amplitude_n16(gpu, config16, prec, tol):
    # All 2^16 amplitudes of the n = 16, p = 1, 2-cut workload against the
    # state vector; and the total probability.
    inst, net, plan, sv = config16
    n = 16
    xs = ((np.arange(1 << n)[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8)
    got = device_amplitudes(plan, xs, prec)
    err = np.abs(got - sv)
    scale = 2.0 ** (-n / 2)
    big = np.abs(sv) > 1e-2 * scale
    assert np.max(err[big] / np.abs(sv[big])) < tol
    assert np.max(err) < tol * scale
    assert abs(np.sum(np.abs(got) ** 2) - 1.0) < (1e-12 if prec == "fp64" else 1e-5)


def test_host_and_device_entry_points_agree(gpu, config16):
    inst, net, plan, sv = config16
    for x in I.bitstrings(16, 3, 9):
        a = plan.contract_amplitude(x, "fp64")
        b = device_amplitudes(plan, x[None, :], "fp64")[0]
        assert a == b
        assert rel(a, sv[O.bits_to_int(x)]) < 1e-10


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n,p,k,seed", [(24, 1, 6, 2), (20, 2, 5, 4)])
def test_per_slice_values(gpu, prec, n, p, k, seed):
    # Every slice scalar (Sec. III.A, Eq. 2) against the oracle's, with the
    # same cut edges and slice numbering.
    inst = I.qaoa_instance(n, p, seed)
    net = qtn.Network(n, inst.edges, inst.gamma, inst.beta)
    plan = qtn.Plan(net, k=k)
    x = I.bitstrings(n, 1, seed)[0]
    ref = O.tn_amplitude(n, inst.edges, inst.gamma, inst.beta, x, cuts=plan.cut_names(), per_slice=True)
    s, c, per = plan.contract_slices(x, 0, 1 << k, prec, per_slice=True)
    scale = 2.0 ** (-n / 2)
    per = per * scale
    if prec == "fp64":
        tol = 1e-12
    else:
        tol = 2 * p * len(inst.edges) * U32
    zero = ref.per_slice == 0  # structurally zero slices (a diagonal gate with both wire legs cut)
    assert np.all(per[zero] == 0)
    assert np.max(np.abs(per[~zero] - ref.per_slice[~zero]) / np.abs(ref.per_slice[~zero])) < tol
    assert abs((s - c) * scale - ref.value) < tol * np.sum(np.abs(ref.per_slice))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_block_executor_n40_p2(gpu, prec):
    # n = 40, p = 2 with 10 greedy cuts (1024 slices): tensors of rank > 5 run
    # on the block executor.
    n, p, k = 40, 2, 10
    inst = I.qaoa_instance(n, p, 2)
    net = qtn.Network(n, inst.edges, inst.gamma, inst.beta)
    plan = qtn.Plan(net, k=k)
    assert plan.executor == "block"
    xs = I.bitstrings(n, 2, 2)
    got = device_amplitudes(plan, xs, prec)
    for x, g in zip(xs, got):
        ref = O.tn_amplitude(n, inst.edges, inst.gamma, inst.beta, x, cuts=plan.cut_names()[:3], threads=4)
        assert rel(g, ref.value) < (1e-10 if prec == "fp64" else 1e-5)


@pytest.fixture(scope="module")
def config80():
    n, p, k = 80, 1, 16
    inst = I.qaoa_instance(n, p, 3)
    net = qtn.Network(n, inst.edges, inst.gamma, inst.beta)
    plan = qtn.Plan(net, k=k)
    xs = I.bitstrings(n, 8, 3)
    refs = [O.tn_amplitude(n, inst.edges, inst.gamma, inst.beta, x, threads=4).value for x in xs]
    return inst, plan, xs, np.array(refs)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 2e-5)])
def test_n80_eight_bitstrings(gpu, config80, prec, tol):
    # The 80-qubit, 16-cut (65536-slice) workload in the launch configuration
    # the benchmark times (8 bit strings, one graph).  complex64: relative
    # bound 2e-5 (see the module docstring; test_n80_fp32_error_bound checks
    # the absolute bound on one bit string).
    inst, plan, xs, refs = config80
    got = device_amplitudes(plan, xs, prec)
    errs = np.abs(got - refs) / np.abs(refs)
    print(prec, "max rel err", errs.max())
    assert errs.max() < tol


def test_n80_fp32_error_bound(gpu, config80):
    inst, plan, xs, refs = config80
    x = xs[0]
    ref = O.tn_amplitude(80, inst.edges, inst.gamma, inst.beta, x, cuts=plan.cut_names(), per_slice=True, threads=16)
    got = device_amplitudes(plan, x[None, :], "fp32")[0]
    l1 = np.sum(np.abs(ref.per_slice))
    print("n80 cancellation ratio", l1 / abs(ref.value), "fp32 abs err / l1", abs(got - ref.value) / l1)
    assert abs(got - ref.value) <= fp32_bound(len(inst.edges), ref.per_slice)


def test_n80_sampled_slices(gpu, config80):
    inst, plan, xs, refs = config80
    x = xs[0]
    n = 80
    _, _, per = plan.contract_slices(x, 0, 1 << 16, "fp64", per_slice=True)
    scale = 2.0 ** (-n / 2)
    for s in (0, 1, 31, 32, 4097, 40000, 65535):
        ref = O.tn_amplitude(n, inst.edges, inst.gamma, inst.beta, x, cuts=plan.cut_names(), slices=(s, s + 1))
        assert abs(per[s] * scale - ref.value) <= 1e-12 * abs(ref.value) + 1e-300


def test_slice_ranges_add_up(gpu, config80):
    # Sec. V: a lost range of slices can be recomputed alone; ranges add up.
    inst, plan, xs, refs = config80
    x = xs[1]
    full, cf = plan.contract_slices(x, 0, 1 << 16, "fp64")
    parts = [plan.contract_slices(x, lo, hi, "fp64") for lo, hi in [(0, 1000), (1000, 1001), (1001, 65536)]]
    tot = sum(s - c for s, c in parts)
    assert abs(tot - (full - cf)) < 1e-13 * abs(full)
    empty = plan.contract_slices(x, 5, 5, "fp64")
    assert empty == (0j, 0j)


@pytest.mark.parametrize("which", ["gamma0", "beta0", "beta_pi2"])
def test_closed_forms_n120(gpu, which):
    n, p, k = 120, 1, 12
    inst = I.qaoa_instance(n, p, 5)
    g, b = inst.gamma.copy(), inst.beta.copy()
    if which == "gamma0":
        g[:] = 0
    elif which == "beta0":
        b[:] = 0
    else:
        b[:] = math.pi / 2
    net = qtn.Network(n, inst.edges, g, b)
    plan = qtn.Plan(net, k=k)
    x = I.bitstrings(n, 1, 5)[0]
    s = 1 - 2 * x.astype(np.int64)
    C = int(sum(s[a] * s[bb] for a, bb in inst.edges))
    h = 2.0 ** (-n / 2)
    want = {"gamma0": np.exp(-1j * n * b[0]) * h, "beta0": h * np.exp(-1j * g[0] * C),
            "beta_pi2": (-1j) ** n * h * np.exp(-1j * g[0] * C)}[which]
    assert rel(plan.contract_amplitude(x, "fp64"), want) < 1e-10
    ref = O.tn_amplitude(n, inst.edges, g, b, x, cuts=plan.cut_names(), per_slice=True, threads=16)
    assert rel(ref.value, want) < 1e-12
    assert abs(plan.contract_amplitude(x, "fp32") - want) <= fp32_bound(len(inst.edges), ref.per_slice)


def test_edge_cases(gpu):
    # a single gate (no merge at all), no cuts, a disconnected graph, an
    # unsupported precision.
    e = np.array([[0, 1]], np.int32)
    net = qtn.Network(2, e, [0.37], [1.1])
    sv = O.statevector(2, e, [0.37], [1.1])
    plan = qtn.Plan(net, cuts=[])
    for xi in range(4):
        x = [(xi >> q) & 1 for q in range(2)]
        assert rel(plan.contract_amplitude(x, "fp64"), sv[xi]) < 1e-13
    e2 = np.array([[0, 1], [1, 2], [0, 2], [3, 4], [4, 5], [3, 5]], np.int32)  # two triangles
    net2 = qtn.Network(6, e2, [0.3, 0.9], [0.4, 1.7])
    sv2 = O.statevector(6, e2, [0.3, 0.9], [0.4, 1.7])
    for k in (0, 3):
        plan2 = qtn.Plan(net2, k=k)
        for xi in (0, 17, 63):
            x = [(xi >> q) & 1 for q in range(6)]
            assert rel(plan2.contract_amplitude(x, "fp64"), sv2[xi]) < 1e-12
    L = qtn.lib()
    xb = np.zeros(2, np.uint8)
    out = np.zeros(2)
    st = L.qtn_contract_amplitude(plan.handle, xb.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), 99,
                                  ctypes.c_void_p(0), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    assert st == 6  # unknown precision
    with pytest.raises(qtn.QTNError):
        plan.contract_amplitude([0, 2], "fp64")


def test_deterministic(gpu, config80):
    inst, plan, xs, refs = config80
    a = device_amplitudes(plan, xs, "fp32")
    b = device_amplitudes(plan, xs, "fp32")
    assert np.array_equal(a, b)


def test_batch_of_plans(gpu):
    jobs = []
    for j, (n, p, k) in enumerate([(20, 1, 4), (24, 2, 6), (20, 1, 4)]):
        inst = I.qaoa_instance(n, p, 50 + j)
        net = qtn.Network(n, inst.edges, inst.gamma, inst.beta)
        jobs.append((inst, qtn.Plan(net, k=k)))
    plans = [jobs[0][1], jobs[1][1], jobs[2][1], jobs[0][1]]
    insts = [jobs[0][0], jobs[1][0], jobs[2][0], jobs[0][0]]
    xs = [I.bitstrings(pl.n, 1, 60 + i)[0] for i, pl in enumerate(plans)]
    got = qtn.contract_batch(plans, xs, "fp64")
    for g, inst, pl, x in zip(got, insts, plans, xs):
        ref = O.tn_amplitude(inst.n, inst.edges, inst.gamma, inst.beta, x).value
        assert rel(g, ref) < 1e-10


# Unit roundoff of each arithmetic's products (first order): TF32 keeps 10
# fraction bits (u = 2^-11); a 2-piece split drops the lo*lo product
# (2^-16 for BF16, 2^-22 for TF32); the 3-piece BF16 split and FP32 keep
# FP32 accuracy (2^-24); the double-float pair carries ~2^-44.
PREC_U = {"fp32": 2.0 ** -24, "tf32": 2.0 ** -11, "bf16x3": 2.0 ** -16, "tf32x3": 2.0 ** -22,
          "bf16x6": 2.0 ** -24, "fp32x2": 2.0 ** -44}


@pytest.fixture(scope="module")
def config80_l1(config80):
    inst, plan, xs, refs = config80
    ref = O.tn_amplitude(80, inst.edges, inst.gamma, inst.beta, xs[0], cuts=plan.cut_names(), per_slice=True,
                         threads=16)
    return ref.value, np.sum(np.abs(ref.per_slice))


@pytest.mark.parametrize("prec", sorted(PREC_U))
def test_precision_sweep_n80(gpu, config80, config80_l1, prec):
    # Sec. III.A slices summed in FP64; merges in each arithmetic.  Bound:
    # |a - a*| <= 2 G u sum_s |a_s| (G gates, coherent first-order rounding).
    inst, plan, xs, refs = config80
    ref, l1 = config80_l1
    got = device_amplitudes(plan, xs[:1], prec)[0]
    bound = 2 * len(inst.edges) * PREC_U[prec] * l1
    print(prec, "rel err", abs(got - ref) / abs(ref), "bound/|a|", bound / abs(ref))
    assert abs(got - ref) <= max(bound, 1e-12 * abs(ref))


def test_fp32x2_meets_fp64_accuracy(gpu, config80):
    # The double-float form is the mixed-precision variant that meets the
    # 1e-10 bound of the complex128 path on all 8 bit strings.
    inst, plan, xs, refs = config80
    got = device_amplitudes(plan, xs, "fp32x2")
    assert np.max(np.abs(got - refs) / np.abs(refs)) < 1e-10


@pytest.fixture(scope="module")
def draws80(config80):
    # The n = 80 graph and 16-cut plan under four seeded (gamma, beta) draws
    # (the workload's own first), 8 bit strings each; references from the
    # oracle with its own 8-cut plan.
    inst, plan, xs, refs = config80
    draws = [(inst.gamma, inst.beta)] + [I.angles(1, 7000 + d) for d in range(1, 4)]
    cuts, _ = O.choose_cuts(80, inst.edges, 1, 8)
    ref = np.array([O.tn_amplitude(80, inst.edges, g, b, x, cuts=cuts, threads=16).value for g, b in draws for x in xs])
    G = np.repeat(np.stack([g for g, _ in draws]), len(xs), axis=0)
    B = np.repeat(np.stack([b for _, b in draws]), len(xs), axis=0)
    return np.tile(xs, (len(draws), 1)), G, B, ref


@pytest.mark.parametrize("prec", ["fp64", "fp32x2"])
def test_precision_draws_n80(gpu, config80, draws80, prec):
    # The precision choice over several angle draws: the complex128 form and
    # the double-float form stay within 1e-10 of the oracle on every draw and
    # bit string (element by element); plain FP32 is reported beside them.
    inst, plan, xs, refs = config80
    X, G, B, ref = draws80
    got = _sweep(plan, X, G, B, prec)
    errs = np.abs(got - ref) / np.abs(ref)
    f32 = np.abs(_sweep(plan, X, G, B, "fp32") - ref) / np.abs(ref)
    print(prec, "max rel err per draw", errs.reshape(4, -1).max(axis=1), "fp32:", f32.reshape(4, -1).max(axis=1))
    assert errs.max() < 1e-10


@pytest.mark.parametrize("base,prec", [("level/fp64/192KiB/t1024", "fp32x2"), ("level/fp64/192KiB/t1024", "fp64"),
                                       ("level/fp32/48KiB", "fp32")])
def test_specialised_level_executor_n80(gpu, config80, base, prec):
    # The kernel generated for this plan's level program (merges as straight
    # code) against the oracle on the benchmark's 8 bit strings, and against
    # the interpreted level executor of the same program.
    # Both schedules: single-phase, and two-phase (small merges over more
    # items, their results parked in device scratch and reloaded).
    inst, plan, xs, refs = config80
    plan.select_executor(base, prec, len(xs))
    interp = device_amplitudes(plan, xs, prec)
    for form in ("jit", "jit2"):
        plan.select_executor(base + "/" + form, prec, len(xs))
        got = device_amplitudes(plan, xs, prec)
        d = plan.describe()["programs"][base + "/" + form + "-" + prec]
        assert d["executor"] == "level-jit"
        assert (d["jit"]["split_level"] > 0) == (form == "jit2")
        tol = 2e-5 if prec == "fp32" else 1e-10
        assert np.max(np.abs(got - refs) / np.abs(refs)) < tol, form
        assert np.max(np.abs(got - interp) / np.abs(interp)) < (1e-5 if prec == "fp32" else 1e-12), form


@pytest.mark.parametrize("n,p,k,seed", [(40, 2, 10, 2), (30, 1, 8, 5)])
def test_specialised_level_executor_small(gpu, n, p, k, seed):
    # Generated kernels of every level program of smaller plans (ragged item
    # counts, several levels per merge shape) against the oracle.
    inst = I.qaoa_instance(n, p, seed)
    plan = qtn.Plan(qtn.Network(n, inst.edges, inst.gamma, inst.beta), k=k)
    xs = I.bitstrings(n, 3, seed)
    refs = [O.tn_amplitude(n, inst.edges, inst.gamma, inst.beta, x, cuts=plan.cut_names(), threads=8).value
            for x in xs]
    names = [nm for nm, pr in plan.describe()["programs"].items() if pr["executor"] == "level"]
    checked = {"jit": 0, "jit2": 0}
    for nm in names:
        for prec in _executor_precisions(nm):
            for form in ("jit", "jit2"):
                try:
                    plan.select_executor(nm + "/" + form, prec, len(xs))
                except qtn.QTNError:
                    continue
                got = device_amplitudes(plan, xs, prec)
                tol = 2e-5 if prec == "fp32" else 1e-10
                assert np.max(np.abs(got - refs) / np.abs(refs)) < tol, (nm, form, prec)
                checked[form] += 1
    # n = 30 programs already run 32 items per pass: no two-phase schedule.
    assert checked["jit"] >= 3 and checked["jit2"] >= (1 if n == 40 else 0), checked


def _executor_precisions(name):
    for form in ("/jit-", "/jit2-"):  # a generated kernel runs the one arithmetic it was made for
        if form in name:
            return [name.rsplit(form, 1)[1]]
    if "/fp64/" in name:
        return ["fp64", "fp32x2"]
    if "/fp32/" in name:
        return ["fp32"]
    if name.startswith("lane"):
        return ["fp64", "fp32"]
    return ["fp64", "fp32x2", "fp32"]


@pytest.mark.parametrize("n,p,k,seed,nx", [(16, 1, 2, 1, 3), (40, 2, 10, 2, 2), (80, 1, 16, 3, 1)])
def test_every_executor_matches_oracle(gpu, n, p, k, seed, nx):
    # Every compiled program on its executor (lane, block, warp, level), forced
    # through qtn_plan_select_executor, in every arithmetic it is compiled for.
    inst = I.qaoa_instance(n, p, seed)
    net = qtn.Network(n, inst.edges, inst.gamma, inst.beta)
    plan = qtn.Plan(net, k=k)
    xs = I.bitstrings(n, nx, seed + 40)
    refs, l1s = [], []
    for x in xs:
        r = O.tn_amplitude(n, inst.edges, inst.gamma, inst.beta, x, cuts=plan.cut_names(), per_slice=True,
                           threads=16)
        refs.append(r.value)
        l1s.append(np.sum(np.abs(r.per_slice)))
    d = plan.describe()
    checked = []
    for name in d["programs"]:
        if name == d["executor"]:
            continue  # the per-slice program: slice ranges, tested by the slice tests
        for prec in _executor_precisions(name):
            plan.select_executor(name, prec, nx)
            try:
                got = device_amplitudes(plan, xs, prec)
            except qtn.QTNError as e:  # a program whose working set exceeds shared memory at this width
                assert e.status == 6 and "shared memory" in str(e), (name, prec, str(e))
                continue
            for g, r, l1 in zip(got, refs, l1s):
                if prec == "fp32":
                    assert abs(g - r) <= fp32_bound(len(inst.edges) * p, [l1]), (name, prec)
                else:
                    assert abs(g - r) <= 1e-10 * abs(r), (name, prec, abs(g - r) / abs(r))
            checked.append((name, prec))
    print(len(checked), "program/arithmetic pairs:", checked)
    assert any(nm.startswith("level") for nm, _ in checked)
    assert {pr for _, pr in checked} >= {"fp64", "fp32x2", "fp32"}


def _sweep(plan, xs, G, B, prec):
    d_x = torch.from_numpy(np.ascontiguousarray(xs.astype(np.uint8))).cuda()
    d_g = torch.from_numpy(np.ascontiguousarray(G)).cuda()
    d_b = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    d_out = torch.zeros((xs.shape[0], 2), dtype=torch.float64, device="cuda")
    plan.contract_sweep_device(d_x, d_g, d_b, d_out, prec)
    torch.cuda.synchronize()
    o = d_out.cpu().numpy()
    return o[:, 0] + 1j * o[:, 1]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32x2", 1e-10)])
def test_parameter_sweep_matches_statevector(gpu, prec, tol):
    # One plan serves a QAOA parameter scan (Sec. II.A: only the gate tensors
    # depend on gamma, beta): every (bit string, angle set) pair against the
    # state vector of its own angles.
    n, p, nx = 16, 2, 6
    inst = I.qaoa_instance(n, p, 21)
    net = qtn.Network(n, inst.edges, inst.gamma, inst.beta)
    plan = qtn.Plan(net, k=3)
    rng = np.random.default_rng(4)
    G, B = rng.uniform(0, np.pi, (nx, p)), rng.uniform(0, np.pi, (nx, p))
    xs = I.bitstrings(n, nx, 21)
    got = _sweep(plan, xs, G, B, prec)
    for i in range(nx):
        sv = O.statevector(n, inst.edges, G[i], B[i])
        assert rel(got[i], sv[O.bits_to_int(xs[i])]) < tol, i


def test_parameter_sweep_n80_and_shared_angles(gpu, config80):
    # n = 80 sweep against the oracle (FP64 form), and a sweep whose angle sets
    # all equal the network's reproduces the fixed-angle launch bit for bit.
    inst, plan, xs, refs = config80
    rng = np.random.default_rng(9)
    G, B = rng.uniform(0, np.pi, (3, 1)), rng.uniform(0, np.pi, (3, 1))
    got = _sweep(plan, xs[:3], G, B, "fp64")
    for i in range(3):
        ref = O.tn_amplitude(80, inst.edges, G[i], B[i], xs[i], cuts=plan.cut_names(), threads=16).value
        assert rel(got[i], ref) < 1e-10, i
    same = _sweep(plan, xs, np.tile(inst.gamma, (8, 1)), np.tile(inst.beta, (8, 1)), "fp64")
    fixed = device_amplitudes(plan, xs, "fp64")
    assert np.array_equal(same, fixed)


@pytest.mark.parametrize("n,p,k,seed", [(16, 1, 2, 1), (12, 2, 6, 4)])
def test_density_form_every_executor(gpu, n, p, k, seed):
    # The density form (dimension-4 edges, 4^k slices) on every executor:
    # <x| rho |x> = |a(x)|^2 from the state vector.
    inst = I.qaoa_instance(n, p, seed)
    net = qtn.Network(n, inst.edges, inst.gamma, inst.beta)
    plan = qtn.Plan(net, k=k)
    dplan = qtn.density_plan(plan, net.density())
    sv = O.statevector(n, inst.edges, inst.gamma, inst.beta)
    xs = I.bitstrings(n, 2, seed + 7)
    probs = np.array([abs(sv[O.bits_to_int(x)]) ** 2 for x in xs])
    d = dplan.describe()
    checked = 0
    for name in d["programs"]:
        if name == d["executor"]:
            continue
        for prec in _executor_precisions(name):
            if prec == "fp32":
                continue
            dplan.select_executor(name, prec, 2)
            try:
                got = device_amplitudes(dplan, xs, prec)
            except qtn.QTNError as e:
                assert e.status == 6 and "shared memory" in str(e), (name, prec, str(e))
                continue
            assert np.max(np.abs(got - probs) / probs) < 1e-10, (name, prec)
            checked += 1
    for x, pr in zip(xs, probs):  # host entry point, per-slice program
        assert abs(dplan.contract_amplitude(x, "fp64") - pr) < 1e-10 * pr
    assert checked >= 4


@pytest.mark.parametrize("n,p,k,seed,nx", [(16, 1, 2, 1, 3), (40, 2, 8, 2, 2)])
def test_graphical_model_every_executor(gpu, n, p, k, seed, nx):
    # Graphical-model form (one index per qubit and layer, shared by the
    # diagonal gates) on every executor: the same amplitudes as the oracle.
    # complex64: relative bound 1e-4 (its per-slice sums are not computed).
    inst = I.qaoa_instance(n, p, seed)
    net = qtn.Network(n, inst.edges, inst.gamma, inst.beta, form="gm")
    plan = qtn.Plan(net, k=k)
    gates = qtn.Plan(qtn.Network(n, inst.edges, inst.gamma, inst.beta), k=10 if n >= 40 else k)
    xs = I.bitstrings(n, nx, seed + 40)
    refs = [O.tn_amplitude(n, inst.edges, inst.gamma, inst.beta, x, cuts=gates.cut_names(), threads=16).value
            for x in xs]
    d = plan.describe()
    checked = set()
    for name in d["programs"]:
        if name == d["executor"]:
            continue
        for prec in _executor_precisions(name):
            plan.select_executor(name, prec, nx)
            try:
                got = device_amplitudes(plan, xs, prec)
            except qtn.QTNError as e:
                assert e.status == 6 and "shared memory" in str(e), (name, prec, str(e))
                continue
            tol = 1e-4 if prec == "fp32" else 1e-10
            for g, r in zip(got, refs):
                assert rel(g, r) < tol, (name, prec, rel(g, r))
            checked.add((name, prec))
    for x, r in zip(xs, refs):  # per-slice program through the host entry point
        assert rel(plan.contract_amplitude(x, "fp64"), r) < 1e-10
    assert any(nm.startswith("level") for nm, _ in checked)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32x2", 1e-10)])
def test_graphical_model_n80(gpu, config80, prec, tol):
    # The n = 80 workload in graphical-model form (8 cuts): the benchmark's
    # eight amplitudes.
    inst, plan, xs, refs = config80
    gm = qtn.Plan(qtn.Network(80, inst.edges, inst.gamma, inst.beta, form="gm"), k=8)
    got = device_amplitudes(gm, xs, prec)
    assert np.max(np.abs(got - refs) / np.abs(refs)) < tol


def test_n120_k22_sampled_slices(gpu):
    # The n = 120, 22-cut workload (4 M slices): slice values over three
    # sampled ranges against the oracle's own slices (FP64 form).
    n, p, k = 120, 1, 22
    inst = I.qaoa_instance(n, p, 5)
    net = qtn.Network(n, inst.edges, inst.gamma, inst.beta)
    plan = qtn.Plan(net, k=k)
    x = I.bitstrings(n, 1, 5)[0]
    S = 1 << k
    for lo in (0, S // 2 + 4096, S - 128):
        hi = lo + 128
        total, comp, vals = plan.contract_slices(x, lo, hi, "fp64", per_slice=True)
        ref = O.tn_amplitude(n, inst.edges, inst.gamma, inst.beta, x, cuts=plan.cut_names(), slices=(lo, hi),
                             per_slice=True, threads=16)
        scale = 2.0 ** (-n / 2)
        mag = np.max(np.abs(ref.per_slice))
        assert mag > 0
        assert np.max(np.abs(vals * scale - ref.per_slice)) <= 1e-12 * mag, lo
        assert np.array_equal(vals == 0, ref.per_slice == 0), lo  # structurally zero slices on both sides
        assert abs((total - comp) * scale - ref.value) <= 1e-12 * np.sum(np.abs(ref.per_slice)), lo
