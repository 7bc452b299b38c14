"""Instances: several copies of one plan per launch.

Slice-parallel execution (consecutive slices side by side, folded into the
FP64 sum in slice order) and independent copies (many output bitstrings of
one circuit in one launch sequence), against the FP64 oracle and the
state vector.
"""
import math

import numpy as np
import pytest

from oracle import brute, statevector, tree
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
    ts = [torch.from_numpy(np.array(t, order="C")).to(dt).cuda() for t in net.tensors]
    return binding.TensorNetwork(net.labels, net.dims, net.open, ts, complex_=net.is_complex)


@pytest.mark.parametrize("batch", [1, 4, 7, 64])
def test_slice_parallel_ising(torch, batch):
    net = inputs.random_ising(100, seed=0)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    sl = planner.slice_greedy(net.labels, net.dims, pairs, net.open, 16)
    tnw = handle(torch, net)
    try:
        m, e = tnw.contract(pairs, sl, "fp32", slice_batch=batch)
        m1, e1 = tnw.contract(pairs, sl, "fp32", slice_batch=1)
        torch.cuda.synchronize()
        lz = math.log(float(m.cpu())) + int(e.cpu()) * math.log(2)
        lz1 = math.log(float(m1.cpu())) + int(e1.cpu()) * math.log(2)
    finally:
        tnw.close()
    mo, eo = tree.contract_net(net, pairs)
    lz_ref = math.log(float(mo)) + eo * math.log(2)
    assert abs(math.expm1(lz - lz_ref)) <= 1e-5
    assert abs(lz - lz1) <= 1e-12 * abs(lz1)


@pytest.mark.parametrize("seed", range(4))
def test_slice_parallel_open_outputs(torch, seed):
    net = inputs.random_network(9, 14, 950 + seed, n_open=1 + seed % 2, complex_=seed % 2 == 0,
                                max_dim=2)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    summed = [l for l in sorted(net.dims) if l not in net.open]
    sl = summed[:3]
    tnw = handle(torch, net)
    try:
        m, e = tnw.contract(pairs, sl, "fp32", slice_batch=3)
        torch.cuda.synchronize()
        got = m.cpu().numpy() * 2.0 ** int(e.cpu())
    finally:
        tnw.close()
    ref = brute.nested_sum(net.tensors, net.labels, net.dims, net.open)
    scale = brute.nested_sum([np.abs(t) for t in net.tensors], net.labels, net.dims, net.open)
    assert np.all(np.abs(got - ref) <= 1e-5 * np.abs(scale) + 1e-30)


@pytest.mark.parametrize("mode", ["fp32", "tf32_split"])
def test_slice_parallel_circuit_tensor_cores(torch, mode):
    circ = inputs.random_circuit(5, 5, 10, seed=0)
    net = inputs.circuit_network(circ, inputs.random_bitstrings(25, 1, seed=1000)[0])
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    sl = planner.slice_greedy(net.labels, net.dims, pairs, net.open, 20)
    tnw = handle(torch, net)
    try:
        info = tnw.plan_info(pairs, sl, mode)
        m, e = tnw.contract(pairs, sl, mode, slice_batch=5)
        torch.cuda.synchronize()
        got = complex(m.cpu()) * 2.0 ** int(e.cpu())
    finally:
        tnw.close()
    if mode != "fp32":
        assert info["n_tensor_core"] >= 1
    mo, eo = tree.contract_net(net, pairs)
    ref = complex(mo) * 2.0 ** eo
    assert abs(got - ref) <= 1e-4 * abs(ref)


def test_independent_instances_many_bitstrings(torch):
    """32 output bitstrings of one circuit: the output leaves differ per
    copy (strided), the gates are shared (stride 0)."""
    from paper_2002_01935_gb300 import binding
    R, C, T = 3, 4, 8
    circ = inputs.random_circuit(R, C, T, seed=6)
    bits = inputs.random_bitstrings(R * C, 32, seed=77)
    nets = [inputs.circuit_network(circ, b) for b in bits]
    base = nets[0]
    pairs = planner.greedy_tree(base.labels, base.dims, base.open)
    n_leaves = base.n_tensors
    first_out = n_leaves - R * C  # output states are the last leaves
    leaves, strides = [], []
    for v in range(n_leaves):
        if v >= first_out:
            stack = np.stack([np.array(nt.tensors[v]) for nt in nets])
            leaves.append(torch.from_numpy(stack).to(torch.complex64).cuda())
            strides.append(int(np.prod(stack.shape[1:])))
        else:
            leaves.append(torch.from_numpy(np.array(base.tensors[v], order="C")).to(torch.complex64).cuda())
            strides.append(0)
    tnw = binding.TensorNetwork(base.labels, base.dims, base.open, None, complex_=True)
    tnw._keep = leaves
    for v, t in enumerate(leaves):
        binding.tn_set_tensor(tnw.h, v, t.data_ptr(), binding.TN_MEM_DEVICE)
    try:
        for mode in ("fp32", "tf32_split"):
            out, ex = tnw.contract_instances(pairs, mode, len(bits), strides)
            torch.cuda.synchronize()
            out, ex = out.cpu().numpy(), ex.cpu().numpy()
            psi = statevector.final_state(R * C, circ.gates)
            for i, b in enumerate(bits):
                got = complex(out[i, 0], out[i, 1]) * 2.0 ** int(ex[i])
                ref = complex(psi[tuple(b)])
                # rounding bound: the same network on |T| (no cancellation)
                scale = float(tree.value([np.abs(t) for t in nets[i].tensors], base.labels,
                                         base.dims, base.open, pairs))
                assert abs(got - ref) <= 1e-5 * scale, (mode, i)
    finally:
        tnw.close()
