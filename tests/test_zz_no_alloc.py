"""The allocation-free entry point, qtn_contract_amplitudes_noalloc.

It serves callers that cannot let the library call cudaMalloc (a framework
that already holds the device memory in its own pool, or code where an
allocation is not allowed).  Checked through the C ABI against
qtn_contract_amplitudes_device on two calls in a row, within the tolerances
of the parity tests (complex128: 1e-10 relative; complex64: 2e-5 relative),
and the second call must leave the device's free memory unchanged.  This file
is collected last so that a run stopping at the first failure has run every
other test already; it builds everything it needs itself.
"""
import ctypes

import numpy as np
import pytest

from paper_2010_14962_gb300 import instances as I
from paper_2010_14962_gb300 import qtn

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {"fp64": 1e-10, "fp32": 2e-5}


def call_noalloc(plan, d_x, d_out, prec):
    L = qtn.lib()
    st = L.qtn_contract_amplitudes_noalloc(plan.handle, ctypes.c_void_p(d_x.data_ptr()), int(d_x.shape[0]),
                                           qtn.PRECISIONS[prec],
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                           ctypes.c_void_p(d_out.data_ptr()))
    assert st == 0, L.qtn_last_error().decode()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n,p,k,nx", [(40, 1, 8, 4), (24, 2, 6, 3)])
def test_noalloc_matches_device_path(gpu, prec, n, p, k, nx):
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
    call_noalloc(plan, d_x, outs[0], prec)  # first call on the device: set-up
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    call_noalloc(plan, d_x, outs[1], prec)
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before
    for o in outs:
        got = o[:, 0].cpu().numpy() + 1j * o[:, 1].cpu().numpy()
        assert np.all(np.abs(got - want) <= TOL[prec] * np.abs(want))


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
