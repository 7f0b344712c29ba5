"""Python binding of the qtn C ABI (``include/qtn.h``).

Argument marshalling only: every step of the contraction runs in the CUDA
library ``_build/libqtn.so``.  Loading fails loudly when the library has not
been built (``python -c "import __graft_entry__ as g; g.build()"``); there is
no CPU fallback.  PyTorch is used only to hand device buffers and streams to
the library.
"""
from __future__ import annotations

import ctypes
import itertools
import json
import os
import re
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libqtn.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "qtn.h")

PRECISIONS = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16x3": 3, "tf32x3": 4, "bf16x6": 5, "fp32x2": 6}
SEARCHES = {"greedy": 0, "ga": 1, "ga_flops": 2, "ga_nonzero": 3}
SURROGATE_FEATURES = 48
SURROGATE_TARGETS = 2


class QTNError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"qtn status {status}: {message}")
        self.status = status


class _PlanOpts(ctypes.Structure):
    _fields_ = [("search", ctypes.c_int), ("k", ctypes.c_int), ("seed", ctypes.c_uint64), ("ga_T", ctypes.c_int),
                ("ga_N", ctypes.c_int), ("max_slice_bytes", ctypes.c_double), ("ga_seed_greedy", ctypes.c_int),
                ("time_budget_s", ctypes.c_double)]


_lock = threading.Lock()
_lib = None


def declared_symbols() -> list[str]:
    """Every function declared in include/qtn.h."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qtn_[a-z0-9_]+)\s*\(", text)))


def lib():
    """The loaded library (raises if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"qtn CUDA library not built: {LIB_PATH} is missing; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER
        i32p, f64p, u8p, vp = P(ctypes.c_int32), P(ctypes.c_double), P(ctypes.c_uint8), ctypes.c_void_p
        sig = {
            "qtn_build_network": [ctypes.c_int, ctypes.c_int, i32p, ctypes.c_int, f64p, f64p, P(vp)],
            "qtn_network_destroy": [vp],
            "qtn_network_density": [vp, P(vp)],
            "qtn_build_network_gm": [ctypes.c_int, ctypes.c_int, i32p, ctypes.c_int, f64p, f64p, P(vp)],
            "qtn_network_info": [vp, P(ctypes.c_int), P(ctypes.c_int)],
            "qtn_network_index": [vp, ctypes.c_int, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int),
                                  P(ctypes.c_int)],
            "qtn_plan_opts_default": [P(_PlanOpts)],
            "qtn_plan": [vp, i32p, ctypes.c_int, i32p, ctypes.c_int, P(_PlanOpts), P(vp)],
            "qtn_plan_destroy": [vp],
            "qtn_plan_cost": [vp, f64p, f64p, P(ctypes.c_int), P(ctypes.c_int)],
            "qtn_plan_cuts": [vp, i32p],
            "qtn_plan_macs_per_slice": [vp, f64p],
            "qtn_contract_amplitude": [vp, u8p, ctypes.c_int, vp, f64p],
            "qtn_contract_amplitudes_device": [vp, vp, ctypes.c_int, ctypes.c_int, vp, vp],
            "qtn_contract_amplitudes_noalloc": [vp, vp, ctypes.c_int, ctypes.c_int, vp, vp],
            "qtn_contract_slices": [vp, u8p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, vp, f64p, vp],
            "qtn_contract_sweep_device": [vp, vp, vp, vp, ctypes.c_int, ctypes.c_int, vp, vp],
            "qtn_contract_batch": [P(vp), vp, ctypes.c_int, ctypes.c_int, vp, vp],
            "qtn_plan_executor": [vp, P(ctypes.c_char_p)],
            "qtn_plan_describe": [vp, ctypes.c_char_p, ctypes.c_size_t, P(ctypes.c_size_t)],
            "qtn_plan_jit_schedule": [vp, ctypes.c_char_p, ctypes.c_int, ctypes.c_int, ctypes.c_size_t,
                                      ctypes.c_char_p, ctypes.c_size_t, P(ctypes.c_size_t)],
            "qtn_plan_jit_source": [vp, ctypes.c_char_p, ctypes.c_int, ctypes.c_int, ctypes.c_size_t,
                                    ctypes.c_char_p, ctypes.c_size_t, P(ctypes.c_size_t)],
            "qtn_plan_set_kernel_timing": [vp, ctypes.c_int],
            "qtn_plan_select_executor": [vp, ctypes.c_int, ctypes.c_int, ctypes.c_char_p],
            "qtn_plan_kernel_ms": [vp, P(ctypes.c_float)],
            "qtn_batch_last_ms": [P(ctypes.c_float), P(ctypes.c_int)],
            "qtn_batch_last_programs": [ctypes.c_char_p, ctypes.c_size_t, P(ctypes.c_size_t)],
            "qtn_batch_cancel": [],
            "qtn_batch_set_time_limit": [ctypes.c_double],
            "qtn_search_cuts": [vp, P(_PlanOpts), i32p, f64p, ctypes.c_int, P(ctypes.c_int), P(ctypes.c_int)],
            "qtn_surrogate_features": [vp, i32p, ctypes.c_int, P(ctypes.c_float)],
            "qtn_surrogate_labels": [vp, i32p, ctypes.c_int, P(ctypes.c_float)],
            "qtn_surrogate_dataset": [ctypes.c_int] * 7 + [ctypes.c_uint64, ctypes.c_int, P(ctypes.c_float),
                                                           P(ctypes.c_float)],
            "qtn_mlp_create": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, P(vp)],
            "qtn_mlp_destroy": [vp],
            "qtn_mlp_num_params": [vp, P(ctypes.c_size_t)],
            "qtn_mlp_params": [vp, P(ctypes.c_float), ctypes.c_int],
            "qtn_mlp_normalisation": [vp] + [P(ctypes.c_float)] * 4 + [ctypes.c_int],
            "qtn_mlp_gradients": [vp, P(ctypes.c_float), P(ctypes.c_float), ctypes.c_int, P(ctypes.c_float),
                                  P(ctypes.c_float)],
            "qtn_mlp_fit": [vp, P(ctypes.c_float), P(ctypes.c_float), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                            ctypes.c_float, ctypes.c_uint64, P(ctypes.c_float)],
            "qtn_mlp_predict": [vp, P(ctypes.c_float), ctypes.c_int, P(ctypes.c_float)],
            "qtn_search_cuts_surrogate": [vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_uint64, ctypes.c_int, i32p, f64p, P(ctypes.c_int),
                                          P(ctypes.c_int), f64p, ctypes.c_int, P(ctypes.c_int)],
            "qtn_pipe_peaks": [ctypes.c_int, f64p, f64p],
            "qtn_pipe_peak_fp32x2": [ctypes.c_int, f64p],
            "qtn_arith_check": [f64p, f64p, ctypes.c_int, ctypes.c_int, f64p, f64p, P(ctypes.c_int)],
            "qtn_wide_set_kernel": [ctypes.c_char_p],
            "qtn_status_string": [ctypes.c_int],
            "qtn_last_error": [],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.qtn_plan_opts_default.restype = None
        L.qtn_network_destroy.restype = None
        L.qtn_plan_destroy.restype = None
        L.qtn_mlp_destroy.restype = None
        L.qtn_status_string.restype = ctypes.c_char_p
        L.qtn_last_error.restype = ctypes.c_char_p
        _lib = L
        return L


def _check(status: int):
    if status != 0:
        raise QTNError(status, lib().qtn_last_error().decode())


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _stream_handle(stream):
    if stream is None:
        try:
            import torch

            if torch.cuda.is_initialized():  # (implies a device; cheaper than is_available)
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return ctypes.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


class Network:
    """qtn_build_network: the ZZ-gate tensor network of a p-layer QAOA circuit."""

    def __init__(self, n: int, edges, gamma, beta, form: str = "gates"):
        """form: "gates" (ZZ gates as vertices, wire segments as indices) or
        "gm" (graphical model: one index per qubit and layer, shared by the
        diagonal gates; qtn_build_network_gm)."""
        e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
        g = np.ascontiguousarray(np.atleast_1d(np.asarray(gamma, dtype=np.float64)))
        b = np.ascontiguousarray(np.atleast_1d(np.asarray(beta, dtype=np.float64)))
        if g.shape != b.shape:
            raise ValueError("gamma and beta need the same length p")
        if form not in ("gates", "gm"):
            raise ValueError("form must be 'gates' or 'gm'")
        self.n, self.p = int(n), int(g.size)
        self.form = form
        build = lib().qtn_build_network if form == "gates" else lib().qtn_build_network_gm
        h = ctypes.c_void_p()
        _check(build(self.n, self.p, _ptr(e, ctypes.c_int32), len(e), _ptr(g, ctypes.c_double),
                     _ptr(b, ctypes.c_double), ctypes.byref(h)))
        self._h = h

    def density(self) -> "Network":
        """qtn_network_density: the dimension-4 (density) form of this network."""
        h = ctypes.c_void_p()
        _check(lib().qtn_network_density(self._h, ctypes.byref(h)))
        d = Network.__new__(Network)
        d.n, d.p, d._h, d.form = self.n, self.p, h, self.form
        d.is_density = True
        return d

    is_density = False

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.qtn_network_destroy(self._h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def info(self):
        nt, ni = ctypes.c_int(), ctypes.c_int()
        _check(lib().qtn_network_info(self._h, ctypes.byref(nt), ctypes.byref(ni)))
        return nt.value, ni.value

    def index(self, i: int):
        """(qubit, pos, tensor_a, tensor_b) of index i."""
        q, p, a, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().qtn_network_index(self._h, int(i), ctypes.byref(q), ctypes.byref(p), ctypes.byref(a),
                                       ctypes.byref(b)))
        return q.value, p.value, a.value, b.value


def search_cuts(network: Network, k: int, search: str = "greedy", seed: int = 1, ga_T: int = 4, ga_N: int = 11,
                seed_greedy: bool = True, time_budget_s: float = 0.0):
    """qtn_search_cuts: (cuts, fitness trace, fitness evaluations)."""
    opts = _PlanOpts()
    lib().qtn_plan_opts_default(ctypes.byref(opts))
    opts.search, opts.k, opts.seed, opts.ga_T, opts.ga_N = SEARCHES[search], int(k), int(seed), int(ga_T), int(ga_N)
    opts.ga_seed_greedy = int(bool(seed_greedy))
    opts.time_budget_s = float(time_budget_s)
    cuts = np.zeros(max(k, 1), dtype=np.int32)
    trace = np.zeros(256)
    tl, ev = ctypes.c_int(), ctypes.c_int()
    _check(lib().qtn_search_cuts(network.handle, ctypes.byref(opts), _ptr(cuts, ctypes.c_int32),
                                 _ptr(trace, ctypes.c_double), len(trace), ctypes.byref(tl), ctypes.byref(ev)))
    return cuts[:k], trace[: tl.value], ev.value


def plan_to_fit(network: "Network", k_min: int, k_max: int = 24, slice_bytes: float = 65536.0) -> "Plan":
    """Plan with the fewest greedy cuts in [k_min, k_max] whose per-slice
    working set (complex64, planner's count) is at most ``slice_bytes``.

    Greedy cuts are chosen one at a time (each given the earlier ones), so the
    first j cuts of a k_max search are the j-cut greedy set: one search serves
    every j.  Raises QTNError(PLAN_EXCEEDS_CAP) when no j fits.
    """
    cuts, _, _ = search_cuts(network, k_max)
    last = None
    for k in range(k_min, k_max + 1):
        try:
            pl = Plan(network, cuts=cuts[:k], max_slice_bytes=slice_bytes)
            return pl
        except QTNError as e:
            last = e
    raise QTNError(3, f"no greedy cut set of {k_min}..{k_max} cuts fits {slice_bytes:g} bytes per slice ({last})")


def density_plan(amplitude_plan: "Plan", density_net: "Network", **kw) -> "Plan":
    """Plan of the density form that cuts the same edges as ``amplitude_plan``:
    each cut edge is both its ket index c and its bra index c + I, so k cut
    edges give 4^k slices (ket cut bits first, then the bra bits)."""
    _, n_idx = amplitude_plan.network.info()
    c = [int(x) for x in amplitude_plan.cuts]
    return Plan(density_net, cuts=c + [x + n_idx for x in c], **kw)


class Plan:
    """qtn_plan: cut set + elimination order + compiled step program."""

    def __init__(self, network: Network, cuts=None, k: int = 0, order=None, search: str = "greedy", seed: int = 1,
                 ga_T: int = 4, ga_N: int = 11, max_slice_bytes: float = 0.0):
        self.network = network
        opts = _PlanOpts()
        lib().qtn_plan_opts_default(ctypes.byref(opts))
        opts.search = SEARCHES[search]
        opts.k = int(k)
        opts.seed = int(seed)
        opts.ga_T = int(ga_T)
        opts.ga_N = int(ga_N)
        opts.max_slice_bytes = float(max_slice_bytes)
        c = None if cuts is None else np.ascontiguousarray(np.asarray(cuts, dtype=np.int32))
        o = None if order is None else np.ascontiguousarray(np.asarray(order, dtype=np.int32))
        h = ctypes.c_void_p()
        _check(lib().qtn_plan(network.handle, None if c is None else _ptr(c, ctypes.c_int32),
                              0 if c is None else len(c), None if o is None else _ptr(o, ctypes.c_int32),
                              0 if o is None else len(o), ctypes.byref(opts), ctypes.byref(h)))
        self._h = h
        self.n = network.n

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.qtn_plan_destroy(self._h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def cost(self) -> dict:
        f, m, w, k = ctypes.c_double(), ctypes.c_double(), ctypes.c_int(), ctypes.c_int()
        _check(lib().qtn_plan_cost(self._h, ctypes.byref(f), ctypes.byref(m), ctypes.byref(w), ctypes.byref(k)))
        macs = ctypes.c_double()
        _check(lib().qtn_plan_macs_per_slice(self._h, ctypes.byref(macs)))
        return dict(log2_flops=f.value, log2_peak_bytes=m.value, width=w.value, k=k.value, macs_per_slice=macs.value)

    @property
    def k(self) -> int:
        return self.cost()["k"]

    @property
    def cuts(self) -> np.ndarray:
        out = np.zeros(max(self.k, 1), dtype=np.int32)
        _check(lib().qtn_plan_cuts(self._h, _ptr(out, ctypes.c_int32)))
        return out[: self.k]

    @property
    def executor(self) -> str:
        s = ctypes.c_char_p()
        _check(lib().qtn_plan_executor(self._h, ctypes.byref(s)))
        return s.value.decode()

    def describe(self) -> dict:
        need = ctypes.c_size_t()
        _check(lib().qtn_plan_describe(self._h, None, 0, ctypes.byref(need)))
        buf = ctypes.create_string_buffer(need.value)
        _check(lib().qtn_plan_describe(self._h, buf, need.value, ctypes.byref(need)))
        return json.loads(buf.value.decode())

    def jit_schedule(self, program: str, precision: str = "fp32x2", two_phase: bool = True,
                     smem_cap: int = 232448) -> dict:
        """qtn_plan_jit_schedule: the generated kernel's schedule for a level
        program (host only; smem_cap defaults to a GB300 block's opt-in)."""
        need = ctypes.c_size_t()
        args = (self._h, program.encode(), PRECISIONS[precision], int(bool(two_phase)), ctypes.c_size_t(smem_cap))
        _check(lib().qtn_plan_jit_schedule(*args, None, 0, ctypes.byref(need)))
        buf = ctypes.create_string_buffer(need.value)
        _check(lib().qtn_plan_jit_schedule(*args, buf, need.value, ctypes.byref(need)))
        return json.loads(buf.value.decode())

    def jit_source(self, program: str, precision: str = "fp32x2", two_phase: bool = True,
                   smem_cap: int = 232448) -> str:
        """qtn_plan_jit_source: the CUDA source generated for a level program."""
        need = ctypes.c_size_t()
        args = (self._h, program.encode(), PRECISIONS[precision], int(bool(two_phase)), ctypes.c_size_t(smem_cap))
        _check(lib().qtn_plan_jit_source(*args, None, 0, ctypes.byref(need)))
        buf = ctypes.create_string_buffer(need.value)
        _check(lib().qtn_plan_jit_source(*args, buf, need.value, ctypes.byref(need)))
        return buf.value.decode()

    def select_executor(self, name: str, precision: str = "fp32", nx: int = 1):
        """Override the autotuner for (precision, nx)."""
        _check(lib().qtn_plan_select_executor(self._h, PRECISIONS[precision], int(nx), name.encode()))

    def set_kernel_timing(self, on: bool = True):
        _check(lib().qtn_plan_set_kernel_timing(self._h, int(bool(on))))

    def kernel_ms(self) -> float:
        """Executor kernel duration of the latest (synchronised) call."""
        ms = ctypes.c_float()
        _check(lib().qtn_plan_kernel_ms(self._h, ctypes.byref(ms)))
        return float(ms.value)

    def cut_names(self):
        """The cuts as (qubit, pos) wire-segment names."""
        return [self.network.index(int(c))[:2] for c in self.cuts]

    def contract_amplitude(self, x, precision: str = "fp32", stream=None) -> complex:
        xb = np.ascontiguousarray(np.asarray(x, dtype=np.uint8).reshape(-1))
        if xb.size != self.n:
            raise ValueError("x must have n entries")
        out = np.zeros(2)
        _check(lib().qtn_contract_amplitude(self._h, _ptr(xb, ctypes.c_uint8), PRECISIONS[precision],
                                            _stream_handle(stream), _ptr(out, ctypes.c_double)))
        return complex(out[0], out[1])

    def contract_amplitudes_device(self, d_x, d_out, precision: str = "fp32", stream=None):
        """d_x: CUDA uint8 tensor (nx, n); d_out: CUDA float64 tensor (nx, 2).
        Asynchronous on `stream` (default: torch's current stream)."""
        if not (d_x.is_cuda and d_out.is_cuda) or d_x.dtype.itemsize != 1 or d_out.element_size() != 8:
            raise ValueError("d_x must be a CUDA uint8 tensor and d_out a CUDA float64 tensor")
        nx = int(d_x.shape[0])
        if d_x.numel() != nx * self.n or d_out.numel() != 2 * nx or not d_x.is_contiguous() or not d_out.is_contiguous():
            raise ValueError("shapes must be (nx, n) and (nx, 2), contiguous")
        _check(lib().qtn_contract_amplitudes_device(self._h, ctypes.c_void_p(d_x.data_ptr()), nx,
                                                    PRECISIONS[precision], _stream_handle(stream),
                                                    ctypes.c_void_p(d_out.data_ptr())))

    def contract_sweep_device(self, d_x, d_gamma, d_beta, d_out, precision: str = "fp32", stream=None):
        """Amplitudes of (bit string i, angles i): d_x CUDA uint8 (nx, n);
        d_gamma, d_beta CUDA float64 (nx, p); d_out CUDA float64 (nx, 2)."""
        for t in (d_x, d_gamma, d_beta, d_out):
            if not t.is_cuda or not t.is_contiguous():
                raise ValueError("every buffer must be a contiguous CUDA tensor")
        nx = int(d_x.shape[0])
        p = self.network.p
        if (d_x.dtype.itemsize != 1 or d_x.numel() != nx * self.n or d_gamma.element_size() != 8
                or d_beta.element_size() != 8 or d_gamma.numel() != nx * p or d_beta.numel() != nx * p
                or d_out.element_size() != 8 or d_out.numel() != 2 * nx):
            raise ValueError("shapes must be (nx, n) uint8, (nx, p) float64 twice and (nx, 2) float64")
        _check(lib().qtn_contract_sweep_device(self._h, ctypes.c_void_p(d_x.data_ptr()),
                                               ctypes.c_void_p(d_gamma.data_ptr()),
                                               ctypes.c_void_p(d_beta.data_ptr()), nx, PRECISIONS[precision],
                                               _stream_handle(stream), ctypes.c_void_p(d_out.data_ptr())))

    def contract_amplitudes_noalloc(self, d_x, d_out, precision: str = "fp32", stream=None):
        """Like contract_amplitudes_device, but the library allocates no device
        memory (a fixed in-library scratch array; see include/qtn.h)."""
        if not (d_x.is_cuda and d_out.is_cuda) or d_x.dtype.itemsize != 1 or d_out.element_size() != 8:
            raise ValueError("d_x must be a CUDA uint8 tensor and d_out a CUDA float64 tensor")
        nx = int(d_x.shape[0])
        if d_x.numel() != nx * self.n or d_out.numel() != 2 * nx or not d_x.is_contiguous() or not d_out.is_contiguous():
            raise ValueError("shapes must be (nx, n) and (nx, 2), contiguous")
        _check(lib().qtn_contract_amplitudes_noalloc(self._h, ctypes.c_void_p(d_x.data_ptr()), nx,
                                                     PRECISIONS[precision], _stream_handle(stream),
                                                     ctypes.c_void_p(d_out.data_ptr())))

    def contract_slices(self, x, lo: int, hi: int, precision: str = "fp32", per_slice: bool = False, stream=None):
        """Kahan sum (and compensation) of slices [lo, hi), unscaled; optionally
        every slice's value (unscaled, as a complex128 numpy array)."""
        xb = np.ascontiguousarray(np.asarray(x, dtype=np.uint8).reshape(-1))
        out = np.zeros(4)
        dev = None
        if per_slice:
            import torch

            dev = torch.empty((max(hi - lo, 1), 2), dtype=torch.float64, device="cuda")
        _check(lib().qtn_contract_slices(self._h, _ptr(xb, ctypes.c_uint8), int(lo), int(hi), PRECISIONS[precision],
                                         _stream_handle(stream), _ptr(out, ctypes.c_double),
                                         None if dev is None else ctypes.c_void_p(dev.data_ptr())))
        total = complex(out[0], out[1])
        comp = complex(out[2], out[3])
        if per_slice:
            v = dev[: hi - lo].cpu().numpy()
            return total, comp, v[:, 0] + 1j * v[:, 1]
        return total, comp


def contract_batch(plans, xs, precision: str = "fp32", stream=None) -> np.ndarray:
    """Amplitudes of independent (plan, x) jobs.  ``xs``: one bit string per
    job (a sequence), or a 2-D array with one row per job (all of one n)."""
    n = len(plans)
    if len(xs) != n:
        raise ValueError("plans and xs must have the same length")
    # All bit strings in one contiguous host buffer; the row pointers are
    # addresses in it (cheaper to marshal than one ctypes pointer per array).
    if isinstance(xs, np.ndarray) and xs.ndim == 2:
        flat = np.ascontiguousarray(xs, dtype=np.uint8)
        sizes = [flat.shape[1]] * n
    else:
        parts = [np.asarray(x, dtype=np.uint8).reshape(-1) for x in xs]
        sizes = [a.size for a in parts]
        flat = np.concatenate(parts) if parts else np.zeros(1, np.uint8)
    for p, m in zip(plans, sizes):
        if m != p.n:
            raise ValueError("every x must have its plan's n entries")
    base = flat.ctypes.data
    starts = list(itertools.accumulate(sizes[:-1], initial=0))[:n]
    xp = (ctypes.c_void_p * n)(*[base + o for o in starts])
    hp = (ctypes.c_void_p * n)(*[p.handle for p in plans])
    out = np.empty(2 * max(n, 1))
    _check(lib().qtn_contract_batch(hp, xp, n, PRECISIONS[precision], _stream_handle(stream),
                                    out.ctypes.data))
    return out.view(np.complex128)[:n]


def pipe_peaks(reps: int = 3) -> dict:
    """qtn_pipe_peaks: measured FP32 and FP64 multiply-add peaks (TFLOP/s) of
    the current device."""
    f32, f64 = ctypes.c_double(), ctypes.c_double()
    _check(lib().qtn_pipe_peaks(int(reps), ctypes.byref(f32), ctypes.byref(f64)))
    return {"fp32_tflops": f32.value, "fp64_tflops": f64.value}


def arith_check(a: np.ndarray, b: np.ndarray):
    """qtn_arith_check: complex dot products over the last axis of a and b
    (count x K complex128) in double-float arithmetic on the device, by the
    scalar sequence and by the merge loops' form.  (scalar, merge, packed)."""
    a = np.ascontiguousarray(a, dtype=np.complex128)
    b = np.ascontiguousarray(b, dtype=np.complex128)
    if a.shape != b.shape or a.ndim != 2:
        raise ValueError("a and b must be count x K arrays of one shape")
    count, K = a.shape
    s = np.zeros(count, dtype=np.complex128)
    m = np.zeros(count, dtype=np.complex128)
    packed = ctypes.c_int()
    _check(lib().qtn_arith_check(_ptr(a.view(np.float64), ctypes.c_double), _ptr(b.view(np.float64), ctypes.c_double),
                                 count, K, _ptr(s.view(np.float64), ctypes.c_double),
                                 _ptr(m.view(np.float64), ctypes.c_double), ctypes.byref(packed)))
    return s, m, bool(packed.value)


def pipe_peak_fp32x2(reps: int = 3) -> float:
    """qtn_pipe_peak_fp32x2: measured packed-FP32-pair multiply-add peak
    (TFLOP/s) of the current device."""
    t = ctypes.c_double()
    _check(lib().qtn_pipe_peak_fp32x2(int(reps), ctypes.byref(t)))
    return t.value


def wide_set_kernel(name: str = "auto"):
    """qtn_wide_set_kernel: force the wide executor's per-step kernel
    ("auto", "simt", "simt4", "tcgen05")."""
    _check(lib().qtn_wide_set_kernel(name.encode()))


def batch_cancel():
    """Stop the multi-plan contract_batch in progress (any thread)."""
    _check(lib().qtn_batch_cancel())


def batch_set_time_limit(ms: float):
    """Executor time limit per multi-plan contract_batch call (0: none)."""
    _check(lib().qtn_batch_set_time_limit(float(ms)))


def batch_last_ms():
    """(device ms, kernels launched) of the latest multi-plan contract_batch."""
    ms, k = ctypes.c_float(), ctypes.c_int()
    _check(lib().qtn_batch_last_ms(ctypes.byref(ms), ctypes.byref(k)))
    return float(ms.value), int(k.value)


def batch_last_programs() -> list:
    """qtn_batch_last_programs: the program each job of the latest
    contract_batch ran (names as in Plan.describe()["programs"])."""
    need = ctypes.c_size_t()
    _check(lib().qtn_batch_last_programs(None, 0, ctypes.byref(need)))
    buf = ctypes.create_string_buffer(need.value)
    _check(lib().qtn_batch_last_programs(buf, need.value, ctypes.byref(need)))
    return json.loads(buf.value.decode())


def plan_job(n: int, p: int, edges, gamma, beta, k: int, gate_log2_flops_max: float = 36.0) -> "Plan":
    """Plan of one job with k greedy cuts on the paper's gate network, or, if
    that needs more than 2^gate_log2_flops_max flops per amplitude (deep
    circuits on many qubits), on the graphical-model form of the same circuit
    when it is cheaper (the same amplitude; qtn_build_network_gm).  Costs come
    from the exact counter (surrogate_labels) before anything is compiled."""
    net = Network(n, edges, gamma, beta)
    cuts, _, _ = search_cuts(net, k)
    f_gate = float(surrogate_labels(net, cuts)[0])
    if f_gate <= gate_log2_flops_max:
        return Plan(net, cuts=cuts)
    gm = Network(n, edges, gamma, beta, form="gm")
    gcuts, _, _ = search_cuts(gm, k)
    f_gm = float(surrogate_labels(gm, gcuts)[0])
    return Plan(gm, cuts=gcuts) if f_gm < f_gate else Plan(net, cuts=cuts)


# ------------------------------------------------------- learned surrogate --

def _f32(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    return a if shape is None else a.reshape(shape)


def surrogate_features(network: Network, cuts) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(cuts, dtype=np.int32))
    out = np.zeros(SURROGATE_FEATURES, dtype=np.float32)
    _check(lib().qtn_surrogate_features(network.handle, _ptr(c, ctypes.c_int32), len(c), _ptr(out, ctypes.c_float)))
    return out


def surrogate_labels(network: Network, cuts) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(cuts, dtype=np.int32))
    out = np.zeros(SURROGATE_TARGETS, dtype=np.float32)
    _check(lib().qtn_surrogate_labels(network.handle, _ptr(c, ctypes.c_int32), len(c), _ptr(out, ctypes.c_float)))
    return out


def surrogate_dataset(count, n_lo, n_hi, p_lo, p_hi, k_lo, k_hi, seed=0, threads=8):
    """(X, Y): features and exact labels of `count` random (graph, cut set) samples."""
    X = np.zeros((count, SURROGATE_FEATURES), dtype=np.float32)
    Y = np.zeros((count, SURROGATE_TARGETS), dtype=np.float32)
    _check(lib().qtn_surrogate_dataset(count, n_lo, n_hi, p_lo, p_hi, k_lo, k_hi, ctypes.c_uint64(seed), threads,
                                       _ptr(X, ctypes.c_float), _ptr(Y, ctypes.c_float)))
    return X, Y


class MLP:
    """The cost surrogate (qtn_mlp_*): trained and evaluated on the device."""

    def __init__(self, n_in=SURROGATE_FEATURES, hidden=256, n_out=SURROGATE_TARGETS, seed=0):
        h = ctypes.c_void_p()
        _check(lib().qtn_mlp_create(n_in, hidden, n_out, ctypes.c_uint64(seed), ctypes.byref(h)))
        self._h = h
        self.n_in, self.hidden, self.n_out = n_in, hidden, n_out
        n = ctypes.c_size_t()
        _check(lib().qtn_mlp_num_params(h, ctypes.byref(n)))
        self.num_params = n.value

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.qtn_mlp_destroy(self._h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def params(self) -> np.ndarray:
        out = np.zeros(self.num_params, dtype=np.float32)
        _check(lib().qtn_mlp_params(self._h, _ptr(out, ctypes.c_float), 0))
        return out

    def set_params(self, p):
        p = _f32(p)
        assert p.size == self.num_params
        _check(lib().qtn_mlp_params(self._h, _ptr(p, ctypes.c_float), 1))

    def set_normalisation(self, x_mean, x_std, y_mean, y_std):
        a, b, c, d = _f32(x_mean), _f32(x_std), _f32(y_mean), _f32(y_std)
        _check(lib().qtn_mlp_normalisation(self._h, _ptr(a, ctypes.c_float), _ptr(b, ctypes.c_float),
                                           _ptr(c, ctypes.c_float), _ptr(d, ctypes.c_float), 1))

    def gradients(self, X, Y):
        X, Y = _f32(X), _f32(Y)
        g = np.zeros(self.num_params, dtype=np.float32)
        loss = ctypes.c_float()
        _check(lib().qtn_mlp_gradients(self._h, _ptr(X, ctypes.c_float), _ptr(Y, ctypes.c_float), X.shape[0],
                                       _ptr(g, ctypes.c_float), ctypes.byref(loss)))
        return g, float(loss.value)

    def fit(self, X, Y, epochs=20, batch=256, lr=1e-3, seed=0):
        X, Y = _f32(X), _f32(Y)
        losses = np.zeros(max(epochs, 1), dtype=np.float32)
        _check(lib().qtn_mlp_fit(self._h, _ptr(X, ctypes.c_float), _ptr(Y, ctypes.c_float), X.shape[0], epochs,
                                 batch, ctypes.c_float(lr), ctypes.c_uint64(seed), _ptr(losses, ctypes.c_float)))
        return losses[:epochs]

    def predict(self, X) -> np.ndarray:
        X = _f32(X)
        Y = np.zeros((X.shape[0], self.n_out), dtype=np.float32)
        _check(lib().qtn_mlp_predict(self._h, _ptr(X, ctypes.c_float), X.shape[0], _ptr(Y, ctypes.c_float)))
        return Y


def search_cuts_surrogate(network: Network, k: int, mlp: MLP, T=8, N=256, top=4, seed=0, seed_greedy=True):
    """(cuts, best exact log2 flops, exact evaluations, surrogate evaluations, trace)."""
    cuts = np.zeros(k, dtype=np.int32)
    best = ctypes.c_double()
    ne, ns, tl = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    trace = np.zeros(256)
    _check(lib().qtn_search_cuts_surrogate(network.handle, k, mlp.handle, T, N, top, ctypes.c_uint64(seed),
                                           int(bool(seed_greedy)), _ptr(cuts, ctypes.c_int32), ctypes.byref(best), ctypes.byref(ne),
                                           ctypes.byref(ns), _ptr(trace, ctypes.c_double), len(trace),
                                           ctypes.byref(tl)))
    return cuts, best.value, ne.value, ns.value, trace[: tl.value]
