"""Test-only CPU emulation of a compiled step program (complex128).

Reads the JSON of ``qtn_plan_describe`` and runs the same program the device
executors run -- leaf tables, canonical [m|k|b] x [k|n|b] merges, permuted
stores, leaf sub-blocks selected by the outer slice classes, batch bits for
the inner classes -- so the host-side compiler (layouts, bit weights, arena
offsets, leaf layouts, cut classes) can be checked against the oracle
without a GPU.  The gate-tensor values are written here from the circuit
definition (ZZ phase exp(-i g s0 s1), RX(2b) = [[cos b, -i sin b],
[-i sin b, cos b]], H|0> = (1, 1)), independently of the CUDA leaf kernel.
"""
import math

import numpy as np

OUT_PLAIN, OUT_RX, OUT_FINAL = 0, 1, 2


def gate_entry(gate, gamma, beta, x, v):
    """Value of a gate tensor at leg values v[slot] (slot 0/1 in, 2/3 out)."""
    l = gate["layer"]
    g, b = gamma[l], beta[l]
    total = 0j
    for u0 in (0, 1):
        for u1 in (0, 1):
            u = (u0, u1)
            s = (1 - 2 * u0) * (1 - 2 * u1)
            t = complex(math.cos(g), -s * math.sin(g))
            for w in (0, 1):
                if not gate["in_h"][w] and v[w] != u[w]:
                    t = 0
                kind = gate["out_kind"][w]
                if kind == OUT_PLAIN:
                    if v[2 + w] != u[w]:
                        t = 0
                else:
                    row = v[2 + w] if kind == OUT_RX else int(x[gate["q"][w]])
                    t *= math.cos(b) if row == u[w] else -1j * math.sin(b)
            total += t
    return total


def gm_factor_entry(gate, gamma, beta, x, v):
    """Graphical-model factors: the ZZ phase exp(-i g s0 s1) on z_i, z_j, or
    <z_out|RX(2b)|z_in> with z_out = x_q in the last layer."""
    l = gate["layer"]
    if gate["kind"] == 1:
        s = (1 - 2 * v[0]) * (1 - 2 * v[1])
        return complex(math.cos(gamma[l]), -s * math.sin(gamma[l]))
    out = v[1] if v[1] >= 0 else int(x[gate["q"][0]])
    return math.cos(beta[l]) if out == v[0] else -1j * math.sin(beta[l])


def leaf_value(desc, gate, gamma, beta, x, v):
    """A leaf's entry: the gate at ket legs v[0..3]; in the density form
    (dimension-4 edges) times the conjugate gate at the bra legs v[4..7]."""
    if gate.get("kind", 0) != 0:
        return gm_factor_entry(gate, gamma, beta, x, v)
    val = gate_entry(gate, gamma, beta, x, v[:4])
    if desc.get("density"):
        val *= np.conj(gate_entry(gate, gamma, beta, x, v[4:]))
    return val


def leaf_table(desc, prog, gamma, beta, x):
    lt = np.zeros(max(prog["leaf_elems"], 1), dtype=complex)
    for L in prog["leaves"]:
        if L["gate"] == -2:  # pseudo-leaf: written by the prologue
            continue
        r = L["rank_nc"] + len(L["cut_bit"])
        for e in range(1 << r):
            if L["gate"] < 0:
                val = 1.0
            else:
                v = [-1] * 8
                for bit, mask in enumerate(L["slot_mask"]):
                    for sl in range(8):
                        if (mask >> sl) & 1:
                            v[sl] = (e >> bit) & 1
                val = leaf_value(desc, desc["gates"][L["gate"]], gamma, beta, x, v)
            lt[L["base"] + e] = val
    return lt


def positions(w, rc):
    """Store offset of every canonical output o = m + (n << ma) + (b << (ma +
    nb)), in o order: sum of the weights of o's set bits."""
    o = np.arange(1 << rc, dtype=np.int64)
    pos = np.zeros(1 << rc, dtype=np.int64)
    for j in range(rc):
        pos += ((o >> j) & 1) * int(w[j])
    return pos


def run_prologue(prog, lt):
    """Hoisted merges, once per bit string; exported results become
    pseudo-leaves of the leaf table (in place)."""
    leaves = prog["leaves"]
    arena = np.zeros(max(prog["pro_arena_elems"], 1) + 64, dtype=complex)
    for st in prog["prologue"]:
        ma, nb, kb, bb = st["ma"], st["nb"], st["kb"], st["bb"]
        rc = ma + nb + bb
        A = (lt[leaves[st["a"]]["base"]:] if st["flags"] & 1 else arena[st["a"]:])[: 1 << (ma + kb + bb)].copy()
        B = (lt[leaves[st["b"]]["base"]:] if st["flags"] & 2 else arena[st["b"]:])[: 1 << (kb + nb + bb)].copy()
        C = np.einsum("bkm,bnk->bnm", A.reshape(1 << bb, 1 << kb, 1 << ma), B.reshape(1 << bb, 1 << nb, 1 << kb))
        pos = positions(st["w"], rc)
        if st["flags"] & 8:
            lt[leaves[st["c"]]["base"] + pos] = C.reshape(-1)
        else:
            arena[st["c"] + pos] = C.reshape(-1)


def run_item(prog, lt, item):
    """Root outputs of one work item (a slice, or an outer-class assignment
    whose root holds one scalar per inner assignment), unnormalised."""
    leaves = prog["leaves"]
    lane = prog["executor"] == "lane"
    arena = np.zeros(max(prog["arena_elems"], 1) + 64, dtype=complex)

    def leaf_off(ref):
        L = leaves[ref]
        off = L["base"]
        for j, cb in enumerate(L["cut_bit"]):
            off += ((item >> cb) & 1) << (L["rank_nc"] + j)
        return off

    root = None
    for st in prog["steps"]:
        ma, nb, kb, bb = st["ma"], st["nb"], st["kb"], st["bb"]
        rc = ma + nb + bb
        na, nbe = 1 << (ma + kb + bb), 1 << (kb + nb + bb)
        src_a = lt if st["flags"] & 1 else arena
        src_b = lt if st["flags"] & 2 else arena
        a0 = leaf_off(st["a"]) if st["flags"] & 1 else st["a"]
        b0 = leaf_off(st["b"]) if st["flags"] & 2 else st["b"]
        A = src_a[a0:a0 + na].copy()
        out = np.zeros(1 << rc, dtype=complex)
        is_root = st["flags"] & 4

        def store(o, v):
            if is_root:
                out[o] = v
            else:
                pos = sum(st["w"][j] for j in range(rc) if (o >> j) & 1)
                arena[st["c"] + pos] = v

        if lane:
            # The lane executor reads A whole, then per column n reads B's
            # column and stores C's column (so a store that clobbers unread
            # B data shows up here).
            assert bb == 0
            Am = A.reshape(1 << kb, 1 << ma).T
            for n in range(1 << nb):
                col = src_b[b0 + (n << kb): b0 + ((n + 1) << kb)].copy()
                Ccol = Am @ col
                for m in range(1 << ma):
                    store(m + (n << ma), Ccol[m])
        else:
            B = src_b[b0:b0 + nbe].copy()
            Ab = A.reshape(1 << bb, 1 << kb, 1 << ma)     # [b, k, m]
            Bb = B.reshape(1 << bb, 1 << nb, 1 << kb)     # [b, n, k]
            C = np.einsum("bkm,bnk->bnm", Ab, Bb)          # [b, n, m], flat = canonical o
            if is_root:
                out[:] = C.reshape(-1)
            else:
                arena[st["c"] + positions(st["w"], rc)] = C.reshape(-1)
        if is_root:
            root = out
    return root


def slice_of(prog, cut_class, item, o):
    """Slice id (cut j <- bit j) of root output o of work item `item`."""
    cls_val = {}
    for pos, c in enumerate(prog["outer_class"]):
        cls_val[c] = (item >> pos) & 1
    for bit, c in enumerate(prog["root_class"]):
        cls_val[c] = (o >> bit) & 1
    s = 0
    for j, c in enumerate(cut_class):
        s |= cls_val[c] << j
    return s


def run_program(desc, name, gamma, beta, x):
    """{slice id: unnormalised value} over the slices the program enumerates."""
    prog = desc["programs"][name]
    lt = leaf_table(desc, prog, gamma, beta, x)
    run_prologue(prog, lt)
    trivial = list(range(len(desc["cuts"])))
    cut_class = trivial if name == desc["executor"] else desc["cut_class"]
    vals = {}
    for item in range(1 << len(prog["outer_class"])):
        out = run_item(prog, lt, item)
        for o, v in enumerate(out):
            vals[slice_of(prog, cut_class, item, o)] = v
    return vals
