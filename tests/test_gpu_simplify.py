"""Simplified networks (Sec. 3.7 structure simplifications on the host) on
the GPU: the same value as the FP64 oracle on the original network."""
import math

import numpy as np
import pytest

from oracle import tree
from paper_2002_01935_gb300 import inputs, planner, simplify

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_01935_gb300 import build
    build.build()
    return _t


def _gpu_value(torch, net, mode):
    from paper_2002_01935_gb300 import binding
    cplx = net.is_complex
    dt = torch.complex64 if cplx else torch.float32
    ts = [torch.from_numpy(np.array(t, order="C")).to(dt).cuda() for t in net.tensors]
    tnw = binding.TensorNetwork(net.labels, net.dims, net.open, ts, complex_=cplx)
    try:
        pairs = planner.greedy_tree(net.labels, net.dims, net.open)
        m, e = tnw.contract(pairs, [], mode)
        torch.cuda.synchronize()
        return m.cpu().numpy(), int(e.cpu())
    finally:
        tnw.close()


@pytest.mark.parametrize("mode", ["fp32", "tf32_split"])
def test_simplified_circuit_amplitude(torch, mode):
    net = inputs.circuit_network(inputs.random_circuit(4, 4, 8, seed=0),
                                 inputs.random_bitstrings(16, 1, seed=1000)[0])
    s, _ = simplify.simplify(net)
    m, e = _gpu_value(torch, s, mode)
    mo, eo = tree.contract_net(net, planner.greedy_tree(net.labels, net.dims, net.open))
    got, ref = complex(m) * 2.0 ** e, complex(mo) * 2.0 ** eo
    assert abs(got - ref) <= 1e-5 * abs(ref)


def test_simplified_ising(torch):
    net = inputs.random_ising(60, seed=4)
    s, _ = simplify.simplify(net)
    m, e = _gpu_value(torch, s, "fp32")
    mo, eo = tree.contract_net(net, planner.greedy_tree(net.labels, net.dims, net.open))
    lz = math.log(float(m)) + e * math.log(2)
    assert abs(math.expm1(lz - (math.log(float(mo)) + eo * math.log(2)))) <= 1e-5
