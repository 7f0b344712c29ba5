"""Host-side logic of the library (no GPU needed): the C ABI loads and
exports every declared symbol, the network build, the planner (tree
decomposition conditions of Sec. II.B, exact cost counter), the cut searches
(greedy; Algorithm 1), and the compiled step programs, emulated on the CPU
against the oracle slice by slice (Sec. III.A, Eq. 2)."""
import ctypes
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from paper_2010_14962_gb300 import instances as I
from paper_2010_14962_gb300 import qtn

from . import program_emulator as E


def test_library_exports_every_declared_symbol():
    L = ctypes.CDLL(qtn.LIB_PATH)
    names = qtn.declared_symbols()
    assert "qtn_contract_amplitude" in names and "qtn_plan" in names
    for name in names:
        assert hasattr(L, name), name


def test_network_counts_and_names():
    for n, p in [(16, 1), (40, 2), (80, 1)]:
        inst = I.qaoa_instance(n, p, 3)
        net = qtn.Network(n, inst.edges, inst.gamma, inst.beta)
        nt, ni = net.info()
        assert nt == p * len(inst.edges) == p * 3 * n // 2
        assert ni == n * (3 * p - 1)
        zz = O.zz_per_qubit(n, inst.edges, p)
        seen = set()
        for i in range(ni):
            q, pos, ta, tb = net.index(i)
            assert 0 <= pos < zz[q] - 1 and ta < tb
            seen.add((q, pos))
        assert len(seen) == ni


@pytest.mark.parametrize("edges", [[[0, 0]], [[0, 1], [1, 0]], [[0, 5]], [[0, 1]]])
def test_network_rejects_bad_graphs(edges):
    n = 3 if edges != [[0, 1]] else 3  # the last graph leaves qubit 2 without a gate
    with pytest.raises(qtn.QTNError) as ei:
        qtn.Network(n, edges, [0.1], [0.2])
    assert ei.value.status == 1


def test_plan_rejects_bad_cuts_and_orders():
    inst = I.qaoa_instance(12, 1, 1)
    net = qtn.Network(12, inst.edges, inst.gamma, inst.beta)
    _, ni = net.info()
    for cuts in ([0, 0], [ni], [-1]):
        with pytest.raises(qtn.QTNError):
            qtn.Plan(net, cuts=cuts)
    with pytest.raises(qtn.QTNError):
        qtn.Plan(net, cuts=[0], order=list(range(ni)))  # contains the cut index
    with pytest.raises(qtn.QTNError):
        qtn.Plan(net, cuts=[], order=list(range(ni - 1)))  # not every index


def bags(desc):
    T = desc["tensors"]
    return [sorted(set(T[a]) | set(T[b])) for a, b, _ in desc["merges"]]


@pytest.mark.parametrize("n,p,k", [(16, 1, 2), (24, 2, 4), (40, 1, 6)])
def test_plan_is_a_tree_decomposition(n, p, k):
    # Sec. II.B: the bags {A u B} of the merges, arranged as the contraction
    # tree, satisfy conditions (1)-(3) for the graph whose vertices are the
    # non-cut indices and whose edges join indices of a common gate tensor.
    inst = I.qaoa_instance(n, p, 5)
    net = qtn.Network(n, inst.edges, inst.gamma, inst.beta)
    plan = qtn.Plan(net, k=k)
    d = plan.describe()
    B = bags(d)
    T = d["tensors"]
    L = d["n_leaves"]
    cuts = set(d["cuts"])
    _, ni = net.info()
    live = [i for i in range(ni) if i not in cuts]
    # (1) every vertex is in a bag
    assert set(live) <= set(itertools.chain.from_iterable(B))
    # (2) every edge is inside a bag: indices of one leaf
    for t in range(L):
        pairs = itertools.combinations(T[t], 2)
        for u, v in pairs:
            assert any(u in b and v in b for b in B)
    # (3) the bags holding an index are connected in the contraction tree
    parent = {}
    prod = {c: j for j, (_, _, c) in enumerate(d["merges"])}
    for j, (a, b, c) in enumerate(d["merges"]):
        for child in (a, b):
            if child in prod:
                parent[prod[child]] = j
    for u in live:
        holders = [j for j, b in enumerate(B) if u in b]
        tops = [j for j in holders if parent.get(j) not in holders]
        assert len(tops) == 1, (u, holders)
    # width and exact MAC count agree with the counter
    assert max(len(b) for b in B) == plan.cost()["width"]
    assert sum(2 ** len(b) for b in B) == plan.cost()["macs_per_slice"]


def treewidth_dp(vertices, adj):
    """Exact treewidth by dynamic programming over vertex subsets."""
    vs = list(vertices)
    idx = {v: i for i, v in enumerate(vs)}
    N = len(vs)
    nbr = [0] * N
    for v in vs:
        for u in adj[v]:
            nbr[idx[v]] |= 1 << idx[u]

    def q_size(S, v):
        # vertices outside S u {v} reachable from v through S
        seen = 1 << v
        stack = [v]
        out = 0
        while stack:
            w = stack.pop()
            m = nbr[w] & ~seen
            while m:
                b = m & -m
                m ^= b
                u = b.bit_length() - 1
                seen |= b
                if S >> u & 1:
                    stack.append(u)
                else:
                    out += 1
        return out

    TW = {0: -1}
    for size in range(1, N + 1):
        for combo in itertools.combinations(range(N), size):
            S = sum(1 << c for c in combo)
            best = N
            for v in combo:
                rest = S & ~(1 << v)
                best = min(best, max(TW[rest], q_size(rest, v)))
            TW[S] = best
    return TW[(1 << N) - 1]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_min_fill_width_bounds_exact_treewidth(seed):
    n = 6
    inst = I.qaoa_instance(n, 1, seed)
    net = qtn.Network(n, inst.edges, inst.gamma, inst.beta)
    plan = qtn.Plan(net, cuts=[])
    d = plan.describe()
    _, ni = net.info()
    adj = {i: set() for i in range(ni)}
    for t in d["tensors"][: d["n_leaves"]]:
        for u, v in itertools.combinations(t, 2):
            adj[u].add(v)
            adj[v].add(u)
    tw = treewidth_dp(range(ni), adj)
    assert plan.cost()["width"] - 1 >= tw


def test_greedy_cuts_lower_width():
    n = 40
    inst = I.qaoa_instance(n, 1, 7)
    net = qtn.Network(n, inst.edges, inst.gamma, inst.beta)
    cuts, trace, _ = qtn.search_cuts(net, 8, "greedy")
    assert len(set(cuts.tolist())) == 8
    widths = [int(t) for t in trace]
    assert widths[-1] < qtn.Plan(net, cuts=[]).cost()["width"]
    assert all(b <= a for a, b in zip(widths, widths[1:]))


def test_genetic_search_is_deterministic_and_elitist():
    # Algorithm 1: the best individual is never crossed or mutated, so the
    # best fitness per generation never rises; T = 4 runs the body 5 times
    # (t = 0..4) plus the final evaluation of Step 5.
    n = 40
    inst = I.qaoa_instance(n, 1, 8)
    net = qtn.Network(n, inst.edges, inst.gamma, inst.beta)
    c1, tr1, ev1 = qtn.search_cuts(net, 6, "ga", seed=3)
    c2, tr2, ev2 = qtn.search_cuts(net, 6, "ga", seed=3)
    assert list(c1) == list(c2) and np.array_equal(tr1, tr2)
    assert len(tr1) == 6 and ev1 == 6 * 11
    assert all(b <= a + 1e-12 for a, b in zip(tr1, tr1[1:]))
    greedy, gtr, _ = qtn.search_cuts(net, 6, "greedy")
    assert tr1[-1] <= gtr[-1] + 1e-12  # seeded with the greedy set


def oracle_cuts(plan):
    return plan.cut_names()


@pytest.mark.parametrize("n,p,k,seed", [(12, 1, 3, 1), (16, 1, 2, 1), (14, 2, 4, 6), (24, 1, 8, 2), (40, 2, 6, 2)])
def test_emulated_programs_match_oracle_per_slice(n, p, k, seed):
    # Every compiled program of the plan (the per-slice one and the
    # throughput ones: cut classes, batched inner classes) reproduces the
    # oracle's slice values; slices a program skips are exactly zero.
    inst = I.qaoa_instance(n, p, seed)
    net = qtn.Network(n, inst.edges, inst.gamma, inst.beta)
    plan = qtn.Plan(net, k=k)
    d = plan.describe()
    x = I.bitstrings(n, 1, seed)[0]
    ref = O.tn_amplitude(n, inst.edges, inst.gamma, inst.beta, x, cuts=plan.cut_names(), per_slice=True,
                         threads=4)
    scale = 2.0 ** (-n / 2)
    mag = np.max(np.abs(ref.per_slice))
    for name in d["programs"]:
        vals = E.run_program(d, name, inst.gamma, inst.beta, x)
        got = np.zeros(1 << k, dtype=complex)
        for s_id, v in vals.items():
            got[s_id] = v * scale
        assert np.max(np.abs(got - ref.per_slice)) < 1e-13 * mag, name
        skipped = np.ones(1 << k, bool)
        skipped[list(vals)] = False
        assert np.all(ref.per_slice[skipped] == 0), name
        assert abs(got.sum() - ref.value) < 1e-13 * np.sum(np.abs(ref.per_slice)), name


@pytest.mark.parametrize("n,p,k,seed", [(10, 1, 2, 1), (12, 2, 3, 4)])
def test_density_form_slices_are_ket_bra_products(n, p, k, seed):
    # The density form (Sec. II.A, dimension-4 edges): cutting k edges gives
    # 4^k slices (Sec. III.A); slice (s, t) -- ket cut bits s, bra cut bits
    # t -- is a_s * conj(a_t) with a_s the amplitude network's slice s, so
    # the sum is |a|^2.  Every compiled program of the density plan, emulated.
    inst = I.qaoa_instance(n, p, seed)
    net = qtn.Network(n, inst.edges, inst.gamma, inst.beta)
    plan = qtn.Plan(net, k=k)
    dnet = net.density()
    _, ni = net.info()
    _, dni = dnet.info()
    assert dni == 2 * ni
    dplan = qtn.density_plan(plan, dnet)
    assert dplan.cost()["k"] == 2 * k
    d = dplan.describe()
    assert d["density"] is True
    x = I.bitstrings(n, 1, seed)[0]
    ref = O.tn_amplitude(n, inst.edges, inst.gamma, inst.beta, x, cuts=plan.cut_names(), per_slice=True)
    a_s = ref.per_slice  # scaled by 2^{-n/2}
    want = np.array([a_s[i % (1 << k)] * np.conj(a_s[i >> k]) for i in range(1 << 2 * k)])
    sv = O.statevector(n, inst.edges, inst.gamma, inst.beta)
    prob = abs(sv[O.bits_to_int(x)]) ** 2
    assert abs(want.sum() - prob) < 1e-12 * prob
    scale = 2.0 ** (-n)
    for name in d["programs"]:
        vals = E.run_program(d, name, inst.gamma, inst.beta, x)
        got = np.zeros(1 << 2 * k, dtype=complex)
        for s_id, v in vals.items():
            got[s_id] = v * scale
        assert np.max(np.abs(got - want)) < 1e-13 * np.max(np.abs(want)), name
        assert abs(got.sum() - prob) < 1e-12 * prob, name


@pytest.mark.parametrize("n,p,k,seed", [(16, 1, 2, 1), (40, 2, 10, 2), (80, 1, 16, 3)])
def test_level_programs_are_race_free(n, p, k, seed):
    # Level-ordered programs: the merges of a level run at the same time, so
    # within a level no result may overlap another result or any operand the
    # level reads; the level table must tile the steps and their output units.
    inst = I.qaoa_instance(n, p, seed)
    net = qtn.Network(n, inst.edges, inst.gamma, inst.beta)
    d = qtn.Plan(net, k=k).describe()
    level_progs = {k_: v for k_, v in d["programs"].items() if v["executor"] == "level"}
    assert "level/classes" in level_progs
    for name, prog in level_progs.items():
        steps, levels, out_start = prog["steps"], prog["levels"], prog["out_start"]
        assert levels and levels[0][0] == 0 and len(out_start) == 2 * len(steps), name
        nxt = 0
        for li, (first, count, units1, units) in enumerate(levels):
            assert first == nxt and count >= 1, name
            nxt = first + count
            acc = acc1 = 0
            reads, writes = [], []
            for j in range(first, first + count):
                st = steps[j]
                ma, nb, kb, bb = st["ma"], st["nb"], st["kb"], st["bb"]
                assert out_start[2 * j] == acc1 and out_start[2 * j + 1] == acc, name
                rc = ma + nb + bb
                split = min(kb, 2) if st["flags"] & 4 else 0  # four-output table: root k sum in <= 4 parts
                acc1 += 1 << rc
                acc += 1 << max(0, rc + split - 2)  # units of 4 outputs (all, if fewer)
                if not st["flags"] & 1:
                    reads.append((st["a"], st["a"] + (1 << (ma + kb + bb))))
                if not st["flags"] & 2:
                    reads.append((st["b"], st["b"] + (1 << (kb + nb + bb))))
                if st["flags"] & 4:
                    assert li == len(levels) - 1, name  # the root is in the last level
                else:
                    writes.append((st["c"], st["c"] + (1 << (ma + nb + bb))))
            assert acc == units and acc1 == units1, name
            for lo, hi in reads + writes:
                assert 0 <= lo < hi <= prog["arena_elems"], name
            for i, (lo, hi) in enumerate(writes):
                for lo2, hi2 in writes[i + 1:] + reads:
                    assert hi <= lo2 or hi2 <= lo, (name, li)
        assert nxt == len(steps), name


def test_emulated_program_n80_sampled_slices():
    n, p = 80, 1
    inst = I.qaoa_instance(n, p, 3)
    net = qtn.Network(n, inst.edges, inst.gamma, inst.beta)
    plan = qtn.Plan(net, k=16)
    d = plan.describe()
    x = I.bitstrings(n, 1, 3)[0]
    prog = d["programs"][d["executor"]]
    lt = E.leaf_table(d, prog, inst.gamma, inst.beta, x)
    E.run_prologue(prog, lt)
    scale = 2.0 ** (-n / 2)
    for s in (0, 1, 12345, 65535):
        ref = O.tn_amplitude(n, inst.edges, inst.gamma, inst.beta, x, cuts=plan.cut_names(), slices=(s, s + 1))
        got = E.run_item(prog, lt, s)[0] * scale
        assert abs(got - ref.value) < 1e-12 * abs(ref.value) + 1e-30


def test_cut_classes_and_batched_programs_n80():
    # The 16 greedy cuts of the n = 80 workload contain one diagonal pair:
    # 15 classes, so half of the 65536 slices are never enumerated; the
    # batched program carries some classes as batch bits.
    inst = I.qaoa_instance(80, 1, 3)
    net = qtn.Network(80, inst.edges, inst.gamma, inst.beta)
    d = qtn.Plan(net, k=16).describe()
    assert max(d["cut_class"]) + 1 == 15
    batched = [v for k, v in d["programs"].items() if k.startswith("batched")]
    assert batched and all(len(v["inner_class"]) >= 1 for v in batched)
    per_slice = d["programs"][d["executor"]]["macs_per_item"]
    for v in batched:
        assert v["macs_per_item"] / 2 ** len(v["inner_class"]) < per_slice


def test_plan_cost_matches_counter_and_cap():
    inst = I.qaoa_instance(40, 2, 2)
    net = qtn.Network(40, inst.edges, inst.gamma, inst.beta)
    plan = qtn.Plan(net, k=10)
    c = plan.cost()
    assert c["k"] == 10
    assert abs(c["log2_flops"] - (10 + np.log2(8 * c["macs_per_slice"]))) < 1e-9
    with pytest.raises(qtn.QTNError) as ei:
        qtn.Plan(net, cuts=plan.cuts, max_slice_bytes=1024)
    assert ei.value.status == 3


def _gm_restricted_path_sum(n, edges, gamma, beta, x, fixed):
    """Brute force over z (p = 1): 2^{-n/2} sum_z prod_E exp(-i g s_i s_j)
    prod_q <x_q|RX(2b)|z_q>, with the variables in `fixed` held."""
    g, b = gamma[0], beta[0]
    total = 0j
    for z in range(1 << n):
        if any(((z >> q) & 1) != v for q, v in fixed.items()):
            continue
        s = [1 - 2 * ((z >> q) & 1) for q in range(n)]
        ph = sum(s[i] * s[j] for i, j in edges)
        t = np.exp(-1j * g * ph)
        for q in range(n):
            t *= np.cos(b) if ((z >> q) & 1) == int(x[q]) else -1j * np.sin(b)
        total += t
    return total * 2.0 ** (-n / 2)


def test_graphical_model_slices_brute_force():
    # Graphical-model form (diagonal gates share one index per qubit and
    # layer): a slice fixes the cut variables; its value is the path sum
    # restricted to them (brute force), and the slices add up to a(x).
    n, p, k = 8, 1, 3
    inst = I.qaoa_instance(n, p, 2)
    net = qtn.Network(n, inst.edges, inst.gamma, inst.beta, form="gm")
    plan = qtn.Plan(net, k=k)
    d = plan.describe()
    assert d["gm"] is True and len(d["cuts"]) == k
    x = I.bitstrings(n, 1, 2)[0]
    cut_q = [net.index(int(c))[0] for c in d["cuts"]]
    want = np.array([_gm_restricted_path_sum(n, inst.edges, inst.gamma, inst.beta, x,
                                             {q: (s >> j) & 1 for j, q in enumerate(cut_q)})
                     for s in range(1 << k)])
    sv = O.statevector(n, inst.edges, inst.gamma, inst.beta)
    assert abs(want.sum() - sv[O.bits_to_int(x)]) < 1e-12
    scale = 2.0 ** (-n / 2)
    for name in d["programs"]:
        vals = E.run_program(d, name, inst.gamma, inst.beta, x)
        got = np.zeros(1 << k, dtype=complex)
        for s_id, v in vals.items():
            got[s_id] = v * scale
        assert np.max(np.abs(got - want)) < 1e-13, name


@pytest.mark.parametrize("n,p,k,seed", [(12, 2, 4, 6), (16, 1, 2, 1), (40, 2, 8, 2)])
def test_graphical_model_programs_match_oracle(n, p, k, seed):
    # Every compiled program of a graphical-model plan (hyperedge merges keep
    # a shared index as a batch bit until its last holder) gives the
    # oracle's amplitude; its width is below the gate network's.
    inst = I.qaoa_instance(n, p, seed)
    gm = qtn.Network(n, inst.edges, inst.gamma, inst.beta, form="gm")
    gates = qtn.Network(n, inst.edges, inst.gamma, inst.beta)
    plan = qtn.Plan(gm, k=k)
    gplan = qtn.Plan(gates, k=max(k, 10) if p == 2 and n >= 40 else k)
    assert plan.cost()["width"] < gplan.cost()["width"] or plan.cost()["log2_flops"] < gplan.cost()["log2_flops"]
    x = I.bitstrings(n, 1, seed)[0]
    ref = O.tn_amplitude(n, inst.edges, inst.gamma, inst.beta, x, cuts=gplan.cut_names(), threads=8).value
    d = plan.describe()
    scale = 2.0 ** (-n / 2)
    for name in d["programs"]:
        vals = E.run_program(d, name, inst.gamma, inst.beta, x)
        got = sum(vals.values()) * scale
        assert abs(got - ref) < 1e-12 * abs(ref), name


def test_nonzero_slice_search():
    # Algorithm 1 with the flops of the structurally non-zero slices as the
    # fitness (cut classes, width capped at the greedy set's): seeded with the
    # greedy set and elitist, so never worse than it on that fitness.
    inst = I.qaoa_instance(40, 1, 3)
    net = qtn.Network(40, inst.edges, inst.gamma, inst.beta)
    greedy = qtn.Plan(net, k=8)
    cuts, trace, ev = qtn.search_cuts(net, 8, "ga_nonzero", seed=3, ga_T=6, ga_N=11)
    again, _, _ = qtn.search_cuts(net, 8, "ga_nonzero", seed=3, ga_T=6, ga_N=11)
    assert np.array_equal(cuts, again) and ev > 0
    assert all(b <= a + 1e-12 for a, b in zip(trace, trace[1:]))

    def fitness(plan):
        d, c = plan.describe(), plan.cost()
        return np.log2(8 * c["macs_per_slice"]) + (max(d["cut_class"]) + 1) + 8 * max(0, c["width"] - greedy.cost()["width"])

    assert fitness(qtn.Plan(net, cuts=cuts)) <= fitness(greedy) + 1e-9


def test_contract_batch_checks_bit_strings_before_the_library():
    # Marshalling of contract_batch: a length mismatch or a bit string of the
    # wrong size is refused on the host, for the list and the 2-D forms.
    inst = I.qaoa_instance(16, 1, 1)
    plan = qtn.Plan(qtn.Network(16, inst.edges, inst.gamma, inst.beta), k=2)
    xs = I.bitstrings(16, 3, 1)
    with pytest.raises(ValueError):
        qtn.contract_batch([plan] * 2, xs, "fp64")
    with pytest.raises(ValueError):
        qtn.contract_batch([plan] * 3, xs[:, :15], "fp64")
    with pytest.raises(ValueError):
        qtn.contract_batch([plan] * 3, [xs[0], xs[1][:15], xs[2]], "fp64")
