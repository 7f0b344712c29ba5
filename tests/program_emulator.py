"""Test-only CPU emulation of a compiled step program (complex128).

Reads the JSON of ``qtn_plan_describe`` and runs the same program the device
executors run -- leaf tables, canonical [m|k] x [k|n] merges, permuted
stores, sliced leaf sub-blocks -- so the host-side compiler (layouts, bit
weights, arena offsets, leaf layouts) can be checked against the oracle
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


def leaf_table(desc, which, gamma, beta, x):
    pg = desc["programs"][which]
    lt = np.zeros(max(pg["leaf_elems"], 1), dtype=complex)
    for L in pg["leaves"]:
        r = L["rank_nc"] + len(L["cut_bit"])
        for e in range(1 << r):
            if L["gate"] < 0:
                val = 1.0
            else:
                v = [-1] * 4
                for bit, slot in enumerate(L["slot_of_bit"]):
                    v[slot] = (e >> bit) & 1
                val = gate_entry(desc["gates"][L["gate"]], gamma, beta, x, v)
            lt[L["base"] + e] = val
    return lt


def run_slice(desc, which, lt, s):
    """Unnormalised scalar of slice s."""
    pg = desc["programs"][which]
    leaves = pg["leaves"]
    arena = np.zeros(max(pg["arena_elems"], 1) + 64, dtype=complex)
    res = None

    def operand(is_leaf, ref, size):
        if is_leaf:
            L = leaves[ref]
            off = L["base"]
            for j, cb in enumerate(L["cut_bit"]):
                off += ((s >> cb) & 1) << (L["rank_nc"] + j)
            return lt[off:off + size].copy()
        return arena[ref:ref + size].copy()

    for st in pg["steps"]:
        ma, nb, kb = st["ma"], st["nb"], st["kb"]
        rc = ma + nb
        # Same read/write order as the lane executor: A is read whole, then
        # for each column n the k entries of B are read and the column of C
        # is stored (so a store that clobbers unread B data shows up here).
        A = operand(st["flags"] & 1, st["a"], 1 << (ma + kb))
        Am = A.reshape(1 << kb, 1 << ma).T      # A[m + (k << ma)] -> Am[m, k]
        for n in range(1 << nb):
            if st["flags"] & 2:
                L = leaves[st["b"]]
                off = L["base"]
                for j, cb in enumerate(L["cut_bit"]):
                    off += ((s >> cb) & 1) << (L["rank_nc"] + j)
                col = lt[off + (n << kb): off + ((n + 1) << kb)].copy()
            else:
                col = arena[st["b"] + (n << kb): st["b"] + ((n + 1) << kb)].copy()
            Ccol = Am @ col                      # C[m, n] for this n
            if st["flags"] & 4:
                res = Ccol[0]
                continue
            for m in range(1 << ma):
                o = m + (n << ma)
                pos = sum(st["w"][j] for j in range(rc) if (o >> j) & 1)
                arena[st["c"] + pos] = Ccol[m]
    return res
