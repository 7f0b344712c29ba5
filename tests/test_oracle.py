"""Pins of the CPU oracle against facts that do not come from the oracle.

* Closed forms derived by hand from the circuit definition (two qubits; the
  gamma = 0, beta = 0 and beta = pi/2 special cases at any n).
* Dense matrix exponentials from scipy for n <= 8 (a library routine).
* Normalisation sum |a|^2 = 1 (unitarity).
* The three oracle evaluations against one another (state vector, explicit
  path sum, tensor-network contraction).
* Eq. 2 of the paper (Sec. III.A): the sum over all slices of a cut network
  equals the uncut contraction, for arbitrary cut sets.
"""
import cmath
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import oracle as O
from paper_2010_14962_gb300 import instances as I


def ising(edges, x):
    s = 1 - 2 * np.asarray(x, dtype=np.int64)
    return int(sum(s[a] * s[b] for a, b in edges))


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


# ----------------------------------------------------------- closed forms --

@pytest.mark.parametrize("g,b", [(0.37, 1.1), (2.9, 0.05), (1.3, 2.2)])
def test_two_qubit_closed_form(g, b):
    # One edge, p = 1.  Summing the four basis paths by hand:
    #   a(00) = a(11) = (e^{-ig} cos 2b - i sin 2b e^{ig}) / 2
    #   a(10) = a(01) = (e^{ig} cos 2b - i sin 2b e^{-ig}) / 2
    same = 0.5 * (cmath.exp(-1j * g) * math.cos(2 * b) - 1j * math.sin(2 * b) * cmath.exp(1j * g))
    diff = 0.5 * (cmath.exp(1j * g) * math.cos(2 * b) - 1j * math.sin(2 * b) * cmath.exp(-1j * g))
    e = np.array([[0, 1]], np.int32)
    sv = O.statevector(2, e, [g], [b])
    assert np.allclose(sv, [same, diff, diff, same], atol=1e-15, rtol=0)
    for x, want in [((0, 0), same), ((1, 0), diff), ((0, 1), diff), ((1, 1), same)]:
        assert rel(O.pathsum(2, e, [g], [b], x), want) < 1e-14
        assert rel(O.tn_amplitude(2, e, [g], [b], x).value, want) < 1e-14


def closed_forms(n, edges, gammas, betas, x, which):
    """gamma = 0:  a = e^{-i n sum(beta)} 2^{-n/2};
    beta = 0:      a = 2^{-n/2} e^{-i sum(gamma) C(x)},  C(x) = sum_E s_i s_j;
    beta = pi/2 (p = 1): a = (-i)^n 2^{-n/2} e^{-i gamma C(x)}."""
    h = 2.0 ** (-n / 2)
    if which == "gamma0":
        return cmath.exp(-1j * n * sum(betas)) * h
    if which == "beta0":
        return h * cmath.exp(-1j * sum(gammas) * ising(edges, x))
    if which == "beta_pi2":
        return (-1j) ** n * h * cmath.exp(-1j * gammas[0] * ising(edges, x))
    raise ValueError(which)


@pytest.mark.parametrize("which,p", [("gamma0", 1), ("gamma0", 2), ("beta0", 1), ("beta0", 2), ("beta_pi2", 1)])
def test_closed_forms_small(which, p):
    n = 12
    inst = I.qaoa_instance(n, p, 11)
    g, b = inst.gamma.copy(), inst.beta.copy()
    if which == "gamma0":
        g[:] = 0
    elif which == "beta0":
        b[:] = 0
    else:
        b[:] = math.pi / 2
    sv = O.statevector(n, inst.edges, g, b)
    for x in I.bitstrings(n, 4, 3):
        want = closed_forms(n, inst.edges, g, b, x, which)
        assert rel(sv[O.bits_to_int(x)], want) < 1e-12
        assert rel(O.tn_amplitude(n, inst.edges, g, b, x, cuts=[(1, 0), (4, 1)]).value, want) < 1e-12
        if n * p <= 16:
            assert rel(O.pathsum(n, inst.edges, g, b, x), want) < 1e-12


@pytest.mark.parametrize("which", ["gamma0", "beta0", "beta_pi2"])
def test_closed_forms_n80_network(which):
    # Large n, where no state vector fits: the network oracle alone.
    n = 80
    inst = I.qaoa_instance(n, 1, 3)
    g, b = inst.gamma.copy(), inst.beta.copy()
    if which == "gamma0":
        g[:] = 0
    elif which == "beta0":
        b[:] = 0
    else:
        b[:] = math.pi / 2
    x = I.bitstrings(n, 1, 7)[0]
    want = closed_forms(n, inst.edges, g, b, x, which)
    got = O.tn_amplitude(n, inst.edges, g, b, x, cuts=[(0, 0), (17, 1)], threads=2).value
    assert rel(got, want) < 1e-12


# --------------------------------------------------------- library pins --

def dense_reference(n, edges, gammas, betas):
    """psi = U_B(b_p) U_C(g_p) ... H^n |0> with scipy's expm on 2^n x 2^n."""
    I2 = np.eye(2)
    X = np.array([[0, 1], [1, 0]], dtype=complex)
    Z = np.diag([1.0, -1.0]).astype(complex)
    Hd = np.array([[1, 1], [1, -1]], dtype=complex) / math.sqrt(2)

    def on(q, P):  # operator on qubit q, qubit q = bit q of the index
        out = np.array([[1.0 + 0j]])
        for j in reversed(range(n)):
            out = np.kron(out, P if j == q else I2)
        return out

    HC = sum(on(a, Z) @ on(b, Z) for a, b in edges)
    HB = sum(on(q, X) for q in range(n))
    psi = np.zeros(1 << n, dtype=complex)
    psi[0] = 1
    Hn = np.array([[1.0 + 0j]])
    for _ in range(n):
        Hn = np.kron(Hn, Hd)
    psi = Hn @ psi
    for g, b in zip(gammas, betas):
        psi = scipy.linalg.expm(-1j * g * HC) @ psi
        psi = scipy.linalg.expm(-1j * b * HB) @ psi
    return psi


@pytest.mark.parametrize("n,p,seed", [(4, 1, 1), (6, 2, 2), (8, 1, 3)])
def test_against_dense_expm(n, p, seed):
    inst = I.qaoa_instance(n, p, seed)
    ref = dense_reference(n, inst.edges, inst.gamma, inst.beta)
    sv = O.statevector(n, inst.edges, inst.gamma, inst.beta)
    assert np.max(np.abs(sv - ref)) < 1e-13
    for x in I.bitstrings(n, 3, seed):
        idx = O.bits_to_int(x)
        assert rel(O.tn_amplitude(n, inst.edges, inst.gamma, inst.beta, x).value, ref[idx]) < 1e-12
        assert rel(O.pathsum(n, inst.edges, inst.gamma, inst.beta, x), ref[idx]) < 1e-12


# ----------------------------------------------------------- invariants --

@pytest.mark.parametrize("n,p", [(12, 1), (10, 2)])
def test_normalisation(n, p):
    inst = I.qaoa_instance(n, p, 21)
    sv = O.statevector(n, inst.edges, inst.gamma, inst.beta)
    assert abs(np.sum(np.abs(sv) ** 2) - 1.0) < 1e-12


@pytest.mark.parametrize("n,p", [(8, 1), (6, 2)])
def test_statevector_equals_pathsum_every_amplitude(n, p):
    inst = I.qaoa_instance(n, p, 5)
    sv = O.statevector(n, inst.edges, inst.gamma, inst.beta)
    for xi in range(1 << n):
        assert abs(O.pathsum(n, inst.edges, inst.gamma, inst.beta, xi) - sv[xi]) < 1e-13


@pytest.mark.parametrize("n,p,seed", [(16, 1, 1), (14, 2, 6)])
def test_network_equals_statevector(n, p, seed):
    inst = I.qaoa_instance(n, p, seed)
    sv = O.statevector(n, inst.edges, inst.gamma, inst.beta)
    zz = O.zz_per_qubit(n, inst.edges, p)
    rng = np.random.default_rng(seed)
    for x in I.bitstrings(n, 6, seed):
        q = rng.choice(n, size=3, replace=False)
        cuts = [(int(a), int(rng.integers(0, zz[a] - 1))) for a in q]
        r = O.tn_amplitude(n, inst.edges, inst.gamma, inst.beta, x, cuts=cuts)
        assert rel(r.value, sv[O.bits_to_int(x)]) < 1e-12


@pytest.mark.parametrize("k", [1, 3, 6])
def test_eq2_sliced_sum_equals_unsliced(k):
    # Sec. III.A, Eq. 2: fixing a cut edge to each value and adding the
    # subnetwork results reproduces the contraction of the whole network.
    n, p = 24, 1
    inst = I.qaoa_instance(n, p, 40 + k)
    x = I.bitstrings(n, 1, k)[0]
    zz = O.zz_per_qubit(n, inst.edges, p)
    rng = np.random.default_rng(k)
    pairs = [(q, t) for q in range(n) for t in range(zz[q] - 1)]
    pick = rng.choice(len(pairs), size=k, replace=False)
    cuts = [pairs[i] for i in pick]
    full = O.tn_amplitude(n, inst.edges, inst.gamma, inst.beta, x).value
    sliced = O.tn_amplitude(n, inst.edges, inst.gamma, inst.beta, x, cuts=cuts, per_slice=True, threads=2)
    assert rel(sliced.value, full) < 1e-13
    assert abs(np.sum(sliced.per_slice) - sliced.value) < 1e-15 * (1 + np.sum(np.abs(sliced.per_slice)))
    # the slice range split used by the worker threads adds up the same way
    lo = O.tn_amplitude(n, inst.edges, inst.gamma, inst.beta, x, cuts=cuts, slices=(0, 1 << (k - 1))).value
    hi = O.tn_amplitude(n, inst.edges, inst.gamma, inst.beta, x, cuts=cuts, slices=(1 << (k - 1), 1 << k)).value
    assert rel(lo + hi, full) < 1e-13


def test_cutting_lowers_width():
    # Sec. III.A: the cut subnetworks have smaller width (and cost per slice).
    n = 40
    inst = I.qaoa_instance(n, 1, 9)
    x = I.bitstrings(n, 1, 9)[0]
    full = O.tn_amplitude(n, inst.edges, inst.gamma, inst.beta, x)
    zz = O.zz_per_qubit(n, inst.edges, 1)
    cuts = [(q, 0) for q in range(0, n, 3) if zz[q] > 1][:8]
    one = O.tn_amplitude(n, inst.edges, inst.gamma, inst.beta, x, cuts=cuts, slices=(0, 1))
    assert one.width <= full.width
    assert one.macs < full.macs


def test_invalid_cut_rejected():
    inst = I.qaoa_instance(8, 1, 1)
    x = np.zeros(8, np.uint8)
    with pytest.raises(ValueError):
        O.tn_amplitude(8, inst.edges, inst.gamma, inst.beta, x, cuts=[(0, 2)])  # 3 ZZ gates: pos <= 1
    with pytest.raises(ValueError):
        O.tn_amplitude(8, inst.edges, inst.gamma, inst.beta, x, cuts=[(0, 0), (0, 0)])


def test_oracle_own_cuts_are_valid_and_exact():
    # The oracle's own cut chooser (used by the benchmark's CPU arm and for
    # reference values): k distinct segments that oracle_tn accepts, and the
    # sliced sum (Eq. 2) over them equals the state vector's amplitude.
    n, p = 14, 2
    inst = I.qaoa_instance(n, p, 6)
    sv = O.statevector(n, inst.edges, inst.gamma, inst.beta)
    x = I.bitstrings(n, 1, 6)[0]
    for k in (1, 3, 5):
        cuts, width = O.choose_cuts(n, inst.edges, p, k)
        assert len(set(cuts)) == k
        r = O.tn_amplitude(n, inst.edges, inst.gamma, inst.beta, x, cuts=cuts)
        assert r.width == width
        assert abs(r.value - sv[O.bits_to_int(x)]) < 1e-12 * abs(sv[O.bits_to_int(x)])


def test_oracle_own_cuts_lower_the_width():
    # Sec. III.A: cutting edges lowers the width of the subnetworks.
    inst = I.qaoa_instance(80, 1, 3)
    widths = [O.choose_cuts(80, inst.edges, 1, k)[1] for k in (0, 4, 8, 16)]
    assert widths == sorted(widths, reverse=True) and widths[-1] < widths[0] - 8, widths
