"""The stored amplitudes of tests/golden/ against the oracle (CPU) and the
device path (GPU).

The fixtures freeze the oracle's state-vector amplitudes of three seeded
random 3-regular QAOA instances (p = 1, 2, 3; Sec. IV workload, Sec. II
circuit).  On the CPU the instance generator, the state vector, the explicit
path sum and the tensor-network contraction must reproduce them; on the GPU
the sliced contraction (Eq. 1, Eq. 2) through the C ABI must.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2010_14962_gb300 import instances as I
from paper_2010_14962_gb300 import qtn

from .golden_fixtures import all_fixtures

FIXTURES = all_fixtures()
SEEDS = {"qaoa16_p1_seed1.txt": 1, "qaoa14_p2_seed4.txt": 4, "qaoa12_p3_seed7.txt": 7}


def test_fixtures_present():
    assert sorted(f.name for f in FIXTURES) == sorted(SEEDS)
    for f in FIXTURES:
        assert len(f.xs) == len(f.amps) == 32 and f.xs.shape[1] == f.n
        assert abs(f.norm - 1.0) < 1e-12


@pytest.mark.parametrize("fx", FIXTURES, ids=lambda f: f.name)
def test_generator_reproduces_fixture_instance(fx):
    inst = I.qaoa_instance(fx.n, fx.p, SEEDS[fx.name])
    assert np.array_equal(np.asarray(inst.edges), fx.edges)
    assert np.allclose(inst.gamma, fx.gamma, rtol=0, atol=0) and np.allclose(inst.beta, fx.beta, rtol=0, atol=0)


@pytest.mark.parametrize("fx", FIXTURES, ids=lambda f: f.name)
def test_oracle_reproduces_fixture(fx):
    sv = O.statevector(fx.n, fx.edges, fx.gamma, fx.beta)
    got = np.array([sv[O.bits_to_int(x)] for x in fx.xs])
    assert np.max(np.abs(got - fx.amps) / np.abs(fx.amps)) < 1e-12
    for x, a in list(zip(fx.xs, fx.amps))[:4]:
        r = O.tn_amplitude(fx.n, fx.edges, fx.gamma, fx.beta, x, cuts=((0, 0), (3, 1))).value
        assert abs(r - a) <= 1e-12 * abs(a)
        if fx.p == 1:
            assert abs(O.pathsum(fx.n, fx.edges, fx.gamma, fx.beta, x) - a) <= 1e-12 * abs(a)


@pytest.mark.gpu
@pytest.mark.parametrize("fx", FIXTURES, ids=lambda f: f.name)
def test_device_reproduces_fixture(gpu, fx):
    # Sliced contraction of the stored instance (3 cuts) through the host and
    # device entry points, FP64 and double-float forms.
    net = qtn.Network(fx.n, fx.edges, fx.gamma, fx.beta)
    plan = qtn.Plan(net, k=3)
    for prec in ("fp64", "fp32x2"):
        got = qtn.contract_batch([plan] * len(fx.xs), fx.xs, prec)
        err = np.abs(got - fx.amps) / np.abs(fx.amps)
        assert float(err.max()) < 1e-10, (prec, float(err.max()))
    import torch

    d_x = torch.from_numpy(np.ascontiguousarray(fx.xs)).cuda()
    d_out = torch.zeros((len(fx.xs), 2), dtype=torch.float64, device="cuda")
    plan.contract_amplitudes_device(d_x, d_out, "fp64")
    torch.cuda.synchronize()
    got = d_out[:, 0].cpu().numpy() + 1j * d_out[:, 1].cpu().numpy()
    assert float(np.max(np.abs(got - fx.amps) / np.abs(fx.amps))) < 1e-10
