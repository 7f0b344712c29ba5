"""The allocation-free entry point, qtn_contract_amplitudes_noalloc.

It serves callers that cannot let the library call cudaMalloc (a framework
that already holds the device memory in its own pool, or code where an
allocation is not allowed).  Checked through the C ABI against
qtn_contract_amplitudes_device on two calls in a row (and that path against
the oracle), within the tolerances of the parity tests (complex128: 1e-10
relative; complex64: 2e-5 relative),
and the second call must leave the device's free memory unchanged.  The
first call on a device may reserve the 64 MiB array (CUDA loads the library
part that holds it lazily, at that call) and nothing more.  This file
is collected last so that a run stopping at the first failure has run every
other test already; it builds everything it needs itself.
"""
import ctypes

import numpy as np
import pytest

from oracle import oracle as O
from paper_2010_14962_gb300 import instances as I
from paper_2010_14962_gb300 import qtn

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {"fp64": 1e-10, "fp32": 2e-5}
SCRATCH = 64 << 20
PAGE_SLACK = 4 << 20  # module code and allocation granularity


def call_noalloc(plan, d_x, d_out, prec):
    L = qtn.lib()
    st = L.qtn_contract_amplitudes_noalloc(plan.handle, ctypes.c_void_p(d_x.data_ptr()), int(d_x.shape[0]),
                                           qtn.PRECISIONS[prec],
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                           ctypes.c_void_p(d_out.data_ptr()))
    assert st == 0, L.qtn_last_error().decode()


def call_wrapper(plan, d_x, d_out, prec):
    plan.contract_amplitudes_noalloc(d_x, d_out, prec)


@pytest.mark.parametrize("call", [call_noalloc, call_wrapper], ids=["c_abi", "python_wrapper"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n,p,k,nx", [(40, 1, 8, 4), (24, 2, 6, 3)])
def test_noalloc_matches_device_path(gpu, prec, n, p, k, nx, call):
    inst = I.qaoa_instance(n, p, 77)
    net = qtn.Network(n, inst.edges, inst.gamma, inst.beta)
    plan = qtn.Plan(net, k=k)
    xs = I.bitstrings(n, nx, 78)
    d_x = torch.from_numpy(np.ascontiguousarray(xs)).cuda()
    ref = torch.zeros((nx, 2), dtype=torch.float64, device="cuda")
    plan.contract_amplitudes_device(d_x, ref, prec)
    torch.cuda.synchronize()
    want = ref[:, 0].cpu().numpy() + 1j * ref[:, 1].cpu().numpy()
    outs = [torch.full((nx, 2), float("nan"), dtype=torch.float64, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    call(plan, d_x, outs[0], prec)  # first call on the device: set-up (may load the array)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    call(plan, d_x, outs[1], prec)
    torch.cuda.synchronize()
    free2, _ = torch.cuda.mem_get_info()
    assert free0 - free1 <= SCRATCH + PAGE_SLACK, free0 - free1
    assert free2 == free1
    for o in outs:
        got = o[:, 0].cpu().numpy() + 1j * o[:, 1].cpu().numpy()
        assert np.all(np.abs(got - want) <= TOL[prec] * np.abs(want))
    # and both against the oracle on the same cut set
    oracle = np.array([O.tn_amplitude(n, inst.edges, inst.gamma, inst.beta, x, cuts=plan.cut_names(), threads=8).value
                       for x in xs])
    assert np.all(np.abs(want - oracle) <= TOL[prec] * np.abs(oracle))


def test_noalloc_rejects_double_float(gpu):
    # The allocation-free path runs the FP64 and FP32 executors only.
    inst = I.qaoa_instance(24, 1, 5)
    plan = qtn.Plan(qtn.Network(24, inst.edges, inst.gamma, inst.beta), k=4)
    d_x = torch.zeros((1, 24), dtype=torch.uint8, device="cuda")
    d_out = torch.zeros((1, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(qtn.QTNError) as e:
        plan.contract_amplitudes_noalloc(d_x, d_out, "fp32x2")
    assert e.value.status == 6  # QTN_ERR_UNSUPPORTED


def test_noalloc_rejects_oversized_request(gpu):
    n, p, k = 40, 2, 10
    inst = I.qaoa_instance(n, p, 2)
    net = qtn.Network(n, inst.edges, inst.gamma, inst.beta)
    plan = qtn.Plan(net, k=k)
    nx = 4096  # the gate tensors of 4096 bit strings exceed the 64 MiB scratch
    d_x = torch.zeros((nx, n), dtype=torch.uint8, device="cuda")
    d_out = torch.zeros((nx, 2), dtype=torch.float64, device="cuda")
    L = qtn.lib()
    st = L.qtn_contract_amplitudes_noalloc(plan.handle, ctypes.c_void_p(d_x.data_ptr()), nx, qtn.PRECISIONS["fp64"],
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                           ctypes.c_void_p(d_out.data_ptr()))
    assert st == 1
    assert "scratch" in L.qtn_last_error().decode()
