"""Host logic of the kernel generator's two-phase schedule (no GPU needed).

A two-phase kernel runs the levels below a split level over more work items
per pass in arenas that hold only what those levels write (the forest
extent), parks the tensors the later levels read, and reloads them into
full arenas for the remaining levels.  Emulated here on the CPU with the
program emulator, with every arena element that the schedule does not carry
across the split set to NaN: the root outputs must equal the plain program's
for every level program of several plans, so the parked set is complete and
the early levels stay inside the forest extent (Eq. 1 merges, Eq. 2 slices).
"""
import numpy as np
import pytest

from paper_2010_14962_gb300 import instances as I
from paper_2010_14962_gb300 import qtn

from . import program_emulator as E


def _run_steps(prog, lt, item, arena, j_lo, j_hi, limit):
    """Steps [j_lo, j_hi) of one work item on `arena` (elements >= limit may
    not be touched); the root's outputs if the root is among them."""
    leaves = prog["leaves"]

    def leaf_off(ref):
        L = leaves[ref]
        off = L["base"]
        for j, cb in enumerate(L["cut_bit"]):
            off += ((item >> cb) & 1) << (L["rank_nc"] + j)
        return off

    root = None
    for st in prog["steps"][j_lo:j_hi]:
        ma, nb, kb, bb = st["ma"], st["nb"], st["kb"], st["bb"]
        rc = ma + nb + bb
        na, nbe = 1 << (ma + kb + bb), 1 << (kb + nb + bb)
        if st["flags"] & 1:
            A = lt[leaf_off(st["a"]):][:na]
        else:
            assert st["a"] + na <= limit
            A = arena[st["a"]:st["a"] + na]
        if st["flags"] & 2:
            B = lt[leaf_off(st["b"]):][:nbe]
        else:
            assert st["b"] + nbe <= limit
            B = arena[st["b"]:st["b"] + nbe]
        C = np.einsum("bkm,bnk->bnm", A.reshape(1 << bb, 1 << kb, 1 << ma), B.reshape(1 << bb, 1 << nb, 1 << kb))
        if st["flags"] & 4:
            root = C.reshape(-1)
        else:
            assert st["c"] + (1 << rc) <= limit
            arena[st["c"] + E.positions(st["w"], rc)] = C.reshape(-1)
    return root


@pytest.mark.parametrize("n,p,k,seed,form", [(40, 2, 10, 2, "gates"), (56, 1, 10, 8, "gates"),
                                             (80, 1, 16, 3, "gates"), (24, 2, 6, 7, "gates"),
                                             (40, 2, 6, 4, "gm")])
def test_two_phase_schedule_parks_what_later_levels_read(n, p, k, seed, form):
    inst = I.qaoa_instance(n, p, seed)
    plan = qtn.Plan(qtn.Network(n, inst.edges, inst.gamma, inst.beta, form=form), k=k)
    desc = plan.describe()
    x = I.bitstrings(n, 1, seed)[0]
    checked = 0
    for name, prog in desc["programs"].items():
        if prog["executor"] != "level":
            continue
        for prec in (["fp32x2"] if "/fp64/" in name else ["fp32"] if "/fp32/" in name else ["fp32x2", "fp32"]):
            try:
                sch = plan.jit_schedule(name, prec, two_phase=True)
            except qtn.QTNError:
                continue  # no two-phase schedule fits this program
            split = sch["split_level"]
            assert 0 < split < len(prog["levels"])
            assert sch["forest_stride"] == sch["forest_extent"] | 1
            assert sch["cross_elems"] == sum(c[1] for c in sch["crossings"])
            first_spine = prog["levels"][split][0]
            lt = E.leaf_table(desc, prog, inst.gamma, inst.beta, x)
            E.run_prologue(prog, lt)
            n_items = 1 << len(prog["outer_class"])
            for item in sorted({0, n_items // 2, n_items - 1}):
                plain = _run_steps(prog, lt, item, np.zeros(prog["arena_elems"] + 64, complex), 0,
                                   len(prog["steps"]), prog["arena_elems"])
                forest = np.full(sch["forest_extent"], np.nan + 1j * np.nan)
                assert _run_steps(prog, lt, item, forest, 0, first_spine, sch["forest_extent"]) is None
                spine = np.full(prog["arena_elems"] + 64, np.nan + 1j * np.nan)
                for off, size, _ in sch["crossings"]:
                    spine[off:off + size] = forest[off:off + size]
                got = _run_steps(prog, lt, item, spine, first_spine, len(prog["steps"]), prog["arena_elems"])
                assert got is not None and np.array_equal(got, plain), (name, prec, item)
            checked += 1
    assert checked >= 1
