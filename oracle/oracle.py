"""Python access to the CPU oracle (``qtn_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use this module; the product library never
imports it.  The C source is compiled here with gcc into ``oracle/_build``.

Functions return complex128 values of the QAOA amplitude
a(x) = <x| U_B(beta_p) U_C(gamma_p) ... U_B(beta_1) U_C(gamma_1) H^n |0^n>
(qubit q <-> bit q of a basis index):

* ``statevector``: all 2^n amplitudes (the definition on a state vector).
* ``pathsum``: one amplitude as an explicit sum over basis paths (tiny n*p).
* ``choose_cuts``: the oracle's own cut set (greedy on its own min-fill
  order), so that its timings and reference values need no product plan.
* ``tn_amplitude``: the paper's method -- circuit as a tensor network with
  gates/inputs/measurements as vertices and wire segments as edges
  (Sec. II.A), cut edges fixed to every value (Sec. III.A, Eq. 2), pairwise
  contraction (Eq. 1) along a min-fill order (Sec. II.B), Kahan-summed
  slices.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qtn_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library; returns its path."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.run(
            ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"],
            check=True,
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(lib):
    i32p = ctypes.POINTER(ctypes.c_int32)
    f64p = ctypes.POINTER(ctypes.c_double)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    lib.oracle_statevector.argtypes = [ctypes.c_int, ctypes.c_int, i32p, ctypes.c_int, f64p, f64p, f64p, f64p]
    lib.oracle_pathsum.argtypes = [ctypes.c_int, ctypes.c_int, i32p, ctypes.c_int, f64p, f64p,
                                   ctypes.c_uint64, f64p]
    lib.oracle_tn.argtypes = [ctypes.c_int, ctypes.c_int, i32p, ctypes.c_int, f64p, f64p, u8p, i32p, i32p,
                              ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, f64p, f64p,
                              f64p, ctypes.POINTER(ctypes.c_int)]
    lib.oracle_zz_per_qubit.argtypes = [ctypes.c_int, ctypes.c_int, i32p, ctypes.c_int, i32p]
    lib.oracle_choose_cuts.argtypes = [ctypes.c_int, ctypes.c_int, i32p, ctypes.c_int, ctypes.c_int, i32p, i32p,
                                       ctypes.POINTER(ctypes.c_int)]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


def load_variant(c_source: str, workdir: str):
    """Compile a variant of the oracle source (used by the planted-mistake
    tests) and return its bound library; pass it as ``lib=`` below."""
    src = os.path.join(workdir, "variant.c")
    so = os.path.join(workdir, "libvariant.so")
    with open(src, "w") as f:
        f.write(c_source)
    subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", so, src, "-lm", "-lpthread"], check=True)
    return _bind(ctypes.CDLL(so))


def source() -> str:
    with open(_SRC) as f:
        return f.read()


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _prep(edges, gamma, beta):
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    g = np.ascontiguousarray(np.atleast_1d(np.asarray(gamma, dtype=np.float64)))
    b = np.ascontiguousarray(np.atleast_1d(np.asarray(beta, dtype=np.float64)))
    assert g.shape == b.shape
    return e, g, b


def statevector(n, edges, gamma, beta, lib=None) -> np.ndarray:
    """All 2^n amplitudes as complex128 (index bit q = qubit q)."""
    lib = lib or _load()
    e, g, b = _prep(edges, gamma, beta)
    re = np.empty(1 << n)
    im = np.empty(1 << n)
    rc = lib.oracle_statevector(n, len(g), _ptr(e, ctypes.c_int32), len(e), _ptr(g, ctypes.c_double),
                                _ptr(b, ctypes.c_double), _ptr(re, ctypes.c_double), _ptr(im, ctypes.c_double))
    if rc != 0:
        raise ValueError(f"oracle_statevector failed ({rc})")
    return re + 1j * im


def pathsum(n, edges, gamma, beta, x, lib=None) -> complex:
    """One amplitude by the explicit path sum; x is an int or a bit array."""
    lib = lib or _load()
    e, g, b = _prep(edges, gamma, beta)
    xi = bits_to_int(x) if not isinstance(x, (int, np.integer)) else int(x)
    out = np.zeros(2)
    rc = lib.oracle_pathsum(n, len(g), _ptr(e, ctypes.c_int32), len(e), _ptr(g, ctypes.c_double),
                            _ptr(b, ctypes.c_double), ctypes.c_uint64(xi), _ptr(out, ctypes.c_double))
    if rc != 0:
        raise ValueError(f"oracle_pathsum failed ({rc})")
    return complex(out[0], out[1])


def bits_to_int(x) -> int:
    x = np.asarray(x, dtype=np.uint8)
    return int(sum(int(v) << i for i, v in enumerate(x)))


def zz_per_qubit(n, edges, p, lib=None) -> np.ndarray:
    lib = lib or _load()
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    out = np.zeros(n, dtype=np.int32)
    lib.oracle_zz_per_qubit(n, p, _ptr(e, ctypes.c_int32), len(e), _ptr(out, ctypes.c_int32))
    return out


def choose_cuts(n, edges, p, k, lib=None):
    """The oracle's own k cut segments as (qubit, pos) pairs, and the width
    they leave: repeatedly cut the segment found in the most widest merges of
    the current min-fill order (independent of the product's planner)."""
    lib = lib or _load()
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    cq = np.zeros(max(k, 1), dtype=np.int32)
    cp = np.zeros(max(k, 1), dtype=np.int32)
    width = ctypes.c_int(0)
    rc = lib.oracle_choose_cuts(n, int(p), _ptr(e, ctypes.c_int32), len(e), int(k), _ptr(cq, ctypes.c_int32),
                                _ptr(cp, ctypes.c_int32), ctypes.byref(width))
    if rc != 0:
        raise ValueError(f"oracle_choose_cuts failed ({rc})")
    return [(int(cq[j]), int(cp[j])) for j in range(k)], int(width.value)


class TNResult:
    def __init__(self, value, per_slice, macs, width):
        self.value = value
        self.per_slice = per_slice
        self.macs = macs
        self.width = width


def tn_amplitude(n, edges, gamma, beta, x, cuts=(), slices=None, threads=1, per_slice=False, lib=None) -> TNResult:
    """The paper's method on the host.

    ``cuts`` is a sequence of (qubit, pos) pairs: the wire segment that enters
    the (pos+1)-th ZZ gate acting on ``qubit`` is cut.  Slice s fixes cut j to
    bit j of s.  ``slices`` = (lo, hi) restricts the sum to a slice range.
    """
    lib = lib or _load()
    e, g, b = _prep(edges, gamma, beta)
    xb = np.ascontiguousarray(np.asarray(x, dtype=np.uint8).reshape(-1))
    assert xb.size == n
    cq = np.ascontiguousarray(np.array([c[0] for c in cuts], dtype=np.int32))
    cp = np.ascontiguousarray(np.array([c[1] for c in cuts], dtype=np.int32))
    k = len(cuts)
    lo, hi = (0, 1 << k) if slices is None else slices
    out = np.zeros(2)
    ps = np.zeros(2 * (hi - lo)) if per_slice else None
    macs = np.zeros(1)
    width = ctypes.c_int(0)
    rc = lib.oracle_tn(n, len(g), _ptr(e, ctypes.c_int32), len(e), _ptr(g, ctypes.c_double),
                       _ptr(b, ctypes.c_double), _ptr(xb, ctypes.c_uint8),
                       _ptr(cq, ctypes.c_int32) if k else None, _ptr(cp, ctypes.c_int32) if k else None, k,
                       ctypes.c_uint64(lo), ctypes.c_uint64(hi), int(threads), _ptr(out, ctypes.c_double),
                       _ptr(ps, ctypes.c_double) if per_slice else None, _ptr(macs, ctypes.c_double),
                       ctypes.byref(width))
    if rc != 0:
        raise ValueError(f"oracle_tn failed ({rc})")
    psv = ps[0::2] + 1j * ps[1::2] if per_slice else None
    return TNResult(complex(out[0], out[1]), psv, float(macs[0]), int(width.value))
