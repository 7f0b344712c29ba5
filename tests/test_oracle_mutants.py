"""Planted mistakes: each compiles a copy of the oracle with one plausible
error (a sign, a dropped term, a wrong index) on the CPU, and checks that the
pins of test_oracle.py reject it.  The unmodified source must pass the same
checks, so the pins are shown to be able to tell right from wrong."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2010_14962_gb300 import instances as I

from .test_oracle import closed_forms, dense_reference

MUTANTS = {
    "rx_offdiag_sign": ("return row == col ? cos(b) + 0.0 * I : -I * sin(b);",
                        "return row == col ? cos(b) + 0.0 * I : I * sin(b);"),
    "zz_phase_sign": ("return cexp(-I * g * (double)s);", "return cexp(I * g * (double)s);"),
    "hadamard_sign": ("H.data[1] = h;  /* out 1, in 0 */", "H.data[1] = -h;  /* out 1, in 0 */"),
    "contract_wrong_index": ("for (int j = 0; j < e->rank; ++j) ie |= ((v >> pe[j]) & 1) << j;",
                             "for (int j = 0; j < e->rank; ++j) ie |= ((v >> pe[0]) & 1) << j;"),
    "fix_wrong_stride": ("size_t src = low | ((size_t)value << pos) | (high << (pos + 1));",
                         "size_t src = low | ((size_t)value << pos) | (high << pos);"),
    "sv_dropped_term": ("psi[z] = rx_entry(beta[l], 0, 0) * a0 + rx_entry(beta[l], 0, 1) * a1;",
                        "psi[z] = rx_entry(beta[l], 0, 0) * a0;"),
    "sv_wrong_qubit": ("ph *= zz_phase(gamma[l], (int)((z >> a) & 1), (int)((z >> b) & 1));",
                       "ph *= zz_phase(gamma[l], (int)((z >> a) & 1), (int)((z >> a) & 1));"),
    "pathsum_dropped_edge": ("      for (int e = 0; e < m; ++e) {\n        int a = edges[2 * e], b = edges[2 * e + 1];\n"
                             "        ising +=",
                             "      for (int e = 0; e < m - 1; ++e) {\n        int a = edges[2 * e], b = edges[2 * e + 1];\n"
                             "        ising +="),
}


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def pins_hold(lib) -> bool:
    try:
        # two-qubit closed form
        g, b = 0.37, 1.1
        same = 0.5 * (np.exp(-1j * g) * math.cos(2 * b) - 1j * math.sin(2 * b) * np.exp(1j * g))
        diff = 0.5 * (np.exp(1j * g) * math.cos(2 * b) - 1j * math.sin(2 * b) * np.exp(-1j * g))
        e = np.array([[0, 1]], np.int32)
        want = [same, diff, diff, same]
        if not np.allclose(O.statevector(2, e, [g], [b], lib=lib), want, atol=1e-14, rtol=0):
            return False
        for xi, w in enumerate(want):
            x = [(xi >> q) & 1 for q in range(2)]
            if rel(O.pathsum(2, e, [g], [b], xi, lib=lib), w) > 1e-12:
                return False
            if rel(O.tn_amplitude(2, e, [g], [b], x, lib=lib).value, w) > 1e-12:
                return False
        # dense expm, n = 6, p = 2, with cuts in the network oracle
        inst = I.qaoa_instance(6, 2, 2)
        ref = dense_reference(6, inst.edges, inst.gamma, inst.beta)
        if np.max(np.abs(O.statevector(6, inst.edges, inst.gamma, inst.beta, lib=lib) - ref)) > 1e-12:
            return False
        for x in I.bitstrings(6, 3, 2):
            xi = O.bits_to_int(x)
            if rel(O.pathsum(6, inst.edges, inst.gamma, inst.beta, x, lib=lib), ref[xi]) > 1e-12:
                return False
            r = O.tn_amplitude(6, inst.edges, inst.gamma, inst.beta, x, cuts=[(0, 1), (3, 2)], lib=lib)
            if rel(r.value, ref[xi]) > 1e-12:
                return False
        # closed form beta = 0 at n = 12 (network, with cuts)
        inst = I.qaoa_instance(12, 1, 11)
        bz = np.zeros(1)
        for x in I.bitstrings(12, 2, 3):
            w = closed_forms(12, inst.edges, inst.gamma, bz, x, "beta0")
            if rel(O.tn_amplitude(12, inst.edges, inst.gamma, bz, x, cuts=[(1, 0)], lib=lib).value, w) > 1e-12:
                return False
        return True
    except (ValueError, ZeroDivisionError, OverflowError):
        return False


def test_unmodified_oracle_passes(tmp_path):
    lib = O.load_variant(O.source(), str(tmp_path))
    assert pins_hold(lib)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = O.source()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    lib = O.load_variant(src.replace(old, new), str(tmp_path))
    assert not pins_hold(lib), f"planted mistake {name} was not caught by the pins"
