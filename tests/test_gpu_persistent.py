"""The persistent launch (tn_options.persistent): every node of every slice
of a call in one dataflow launch, small or narrow nodes as chunks of
outputs and large ones as 64 x 64 tile items, then one fold of the slices'
roots in slice order (Sec. 4.7.1: the slices are independent contractions
summed at the end).  Against the FP64 oracle on the leaf values the GPU
reads, and against the per-step launch sequence."""
import math

import numpy as np
import pytest

from oracle import tree
from paper_2002_01935_gb300 import inputs, planner

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_01935_gb300 import build
    build.build()
    return _t


def handle(torch, net):
    from paper_2002_01935_gb300 import binding
    dt = torch.complex64 if net.is_complex else torch.float32
    ts = [torch.from_numpy(np.array(t, order="C")).to(dt).contiguous().cuda() for t in net.tensors]
    return binding.TensorNetwork(net.labels, net.dims, net.open, ts, complex_=net.is_complex), ts


@pytest.mark.parametrize("target", [18.0, 16.0])
def test_cfg1_ising_sliced_in_one_launch(torch, target):
    net = inputs.random_ising(100, seed=0)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    sliced = planner.slice_greedy(net.labels, net.dims, pairs, net.open, target)
    info = planner.tree_info(net.labels, net.dims, pairs, net.open, sliced)
    assert info.W <= target and info.d_sliced >= 8
    mo, eo = tree.contract_net(net.as_stored(), pairs, sliced)
    ref = math.log(float(mo)) + eo * math.log(2)
    tnw, keep = handle(torch, net)
    try:
        for mode in ("fp32", "tf32_split"):  # every node on the CUDA cores either way
            for call in range(2):
                m, e = tnw.contract(pairs, sliced, mode, persistent=True)
                torch.cuda.synchronize()
                got = math.log(float(m.cpu())) + int(e.cpu()) * math.log(2)
                assert abs(math.expm1(got - ref)) <= 1e-5, (mode, call, got, ref)
        m2, e2 = tnw.contract(pairs, sliced, "fp32")
        torch.cuda.synchronize()
        step = math.log(float(m2.cpu())) + int(e2.cpu()) * math.log(2)
        assert abs(math.expm1(got - step)) <= 1e-5
    finally:
        tnw.close()


@pytest.mark.parametrize("seed", range(6))
def test_random_networks_open_and_sliced(torch, seed):
    net = inputs.random_network(9 + seed % 3, 14 + seed % 4, 900 + seed, n_open=seed % 3,
                                complex_=seed % 2 == 0, max_dim=2)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    summed = [l for l in sorted(net.dims) if l not in net.open]
    sliced = summed[:2] if seed >= 2 else []
    mo, eo = tree.contract_net(net.as_stored(), pairs, sliced)
    ref = mo * 2.0 ** eo
    scale = tree.value([np.abs(t) for t in net.as_stored().tensors], net.labels, net.dims, net.open, pairs)
    tnw, keep = handle(torch, net)
    try:
        m, e = tnw.contract(pairs, sliced, "fp32", persistent=True)
        torch.cuda.synchronize()
        got = m.cpu().numpy() * 2.0 ** int(e.cpu())
    finally:
        tnw.close()
    assert np.all(np.abs(got - ref) <= 1e-5 * np.abs(scale) + 1e-30)


def test_circuit_amplitude_and_open_tensor(torch):
    circ = inputs.random_circuit(4, 4, 8, seed=0)
    for net in (inputs.circuit_network(circ, inputs.random_bitstrings(16, 1, seed=1000)[0]),
                inputs.circuit_network(circ, open_qubits=[3, 7, 11, 15, 0, 5])):
        pairs = planner.greedy_tree(net.labels, net.dims, net.open)
        sliced = planner.slice_greedy(net.labels, net.dims, pairs, net.open, 9)
        mo, eo = tree.contract_net(net.as_stored(), pairs, sliced)
        ref = mo * 2.0 ** eo
        tnw, keep = handle(torch, net)
        try:
            m, e = tnw.contract(pairs, sliced, "fp32", persistent=True)
            torch.cuda.synchronize()
            got = m.cpu().numpy() * 2.0 ** int(e.cpu())
        finally:
            tnw.close()
        assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)
