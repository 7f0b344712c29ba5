"""The kernel generator's CUDA source compiles for sm_103a (no GPU needed:
the run-time compiler runs on the host) for level programs of several plan
shapes and network forms, in both double- and single-word arithmetic and
both schedules; programs with hoisted merges also get the generated
prologue kernel."""
import ctypes
import os

import pytest

from paper_2010_14962_gb300 import instances as I
from paper_2010_14962_gb300 import qtn


def _nvrtc():
    for name in ("libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                 "/usr/local/cuda/lib64/libnvrtc.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("libnvrtc not available")


def _compile(nv, src):
    prog = ctypes.c_void_p()
    assert nv.nvrtcCreateProgram(ctypes.byref(prog), src.encode(), b"gen.cu", 0, None, None) == 0
    opts = (ctypes.c_char_p * 3)(b"-arch=sm_103a", b"-std=c++17", b"-default-device")
    rc = nv.nvrtcCompileProgram(prog, 3, opts)
    size = ctypes.c_size_t()
    nv.nvrtcGetProgramLogSize(prog, ctypes.byref(size))
    log = ctypes.create_string_buffer(size.value)
    nv.nvrtcGetProgramLog(prog, log)
    nv.nvrtcDestroyProgram(ctypes.byref(prog))
    return rc, log.value.decode(errors="replace")


@pytest.mark.parametrize("n,p,k,seed,form", [(40, 2, 10, 2, "gates"), (40, 2, 6, 4, "gm"), (56, 1, 10, 8, "gates")])
def test_generated_source_compiles(n, p, k, seed, form):
    nv = _nvrtc()
    inst = I.qaoa_instance(n, p, seed)
    plan = qtn.Plan(qtn.Network(n, inst.edges, inst.gamma, inst.beta, form=form), k=k)
    progs = [(name, pr) for name, pr in plan.describe()["programs"].items() if pr["executor"] == "level"]
    # the largest double-word program (most levels and merges) in both schedules, and the largest single-word
    # program in the schedule with the fewer estimated steps
    compiled = 0
    for tag, precs, forms in (("/fp64/", ["fp32x2"], (False, True)), ("/fp32/", ["fp32"], (True,))):
        group = sorted((pr["macs_per_item"], name) for name, pr in progs if tag in name)
        if not group:
            continue
        name = group[-1][1]
        pr = dict(progs)[name]
        for prec in precs:
            for two in forms:
                try:
                    src = plan.jit_source(name, prec, two_phase=two)
                except qtn.QTNError:
                    continue  # no schedule of this form fits
                assert ("qtn_prologue_jit" in src) == bool(pr["prologue"]), name
                rc, log = _compile(nv, src)
                assert rc == 0, (name, prec, two, log[:2000])
                compiled += 1
    assert compiled >= 1
