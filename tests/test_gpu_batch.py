"""Batches of independent networks in one captured launch sequence.

Complex circuit amplitudes and real Ising partition functions, each with
its own greedy tree, mixed in one batch; every result against the FP64
oracle (relative 1e-5), and the per-network completion times are sane.
"""
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


def make_nets(n_amp, n_ising, circuit=(4, 4, 8)):
    R, C, T = circuit
    circ = inputs.random_circuit(R, C, T, seed=3)
    bits = inputs.random_bitstrings(R * C, n_amp, seed=1234)
    nets = [inputs.circuit_network(circ, b) for b in bits]
    rng = np.random.default_rng(5)
    for j in range(n_ising):
        n = int(rng.choice(np.arange(12, 61, 2)))
        nets.append(inputs.random_ising(n, seed=500 + j))
    return nets


@pytest.mark.parametrize("mode", ["fp32", "tf32_split"])
def test_mixed_batch_matches_oracle(torch, mode):
    from paper_2002_01935_gb300 import binding
    nets = make_nets(24, 12)
    handles, trees, keep = [], [], []
    for net in nets:
        dt = torch.complex64 if net.is_complex else torch.float32
        ts = [torch.from_numpy(np.array(t, order="C")).to(dt).cuda() for t in net.tensors]
        keep.append(ts)
        handles.append(binding.TensorNetwork(net.labels, net.dims, net.open, ts, complex_=net.is_complex))
        trees.append(planner.greedy_tree(net.labels, net.dims, net.open))
    batch = binding.Batch(handles, trees, mode)
    try:
        for call in range(2):  # graph capture, then replay
            out, ex, lat = batch.contract()
            torch.cuda.synchronize()
            out, ex, lat = out.cpu().numpy(), ex.cpu().numpy(), lat.cpu().numpy()
            for i, net in enumerate(nets):
                mo, eo = tree.contract_net(net, trees[i])
                if net.is_complex:
                    got = complex(out[i, 0], out[i, 1]) * 2.0 ** (int(ex[i]) - eo)
                    ref = complex(mo)
                    assert abs(got - ref) <= 1e-5 * abs(ref), (call, i)
                else:
                    d = math.log(out[i, 0]) + (int(ex[i]) - eo) * math.log(2) - math.log(float(mo))
                    assert abs(math.expm1(d)) <= 1e-5, (call, i)
            assert np.all(lat > 0) and np.all(lat < 10**9)
    finally:
        batch.close()
        for h in handles:
            h.close()


@pytest.mark.parametrize("mode", ["fp32", "fp16_split"])
def test_mixed_batch_with_sliced_members(torch, mode):
    """Circuit amplitudes and Ising networks of N in [12, 60] in the merged
    forest, plus Ising networks sliced to a width cap as members that run
    their own slice loops: an N = 152 network (greedy width 24, sliced to
    W_s <= 22) and an N = 100 one (width 21, sliced to W_s <= 16).  Every
    value against the oracle's contraction of the same sliced tree (on the
    leaf values the GPU reads); the sliced members complete after the forest."""
    from paper_2002_01935_gb300 import binding
    nets = make_nets(6, 6)
    trees = [planner.greedy_tree(n.labels, n.dims, n.open) for n in nets]
    sliced = [[] for _ in nets]
    for n_v, seed, cap in ((152, 15, 22.0), (100, 0, 16.0)):
        net = inputs.random_ising(n_v, seed=seed)
        pairs = planner.greedy_tree(net.labels, net.dims, net.open)
        sl = planner.slice_greedy(net.labels, net.dims, pairs, net.open, cap)
        assert sl
        nets.append(net)
        trees.append(pairs)
        sliced.append(sl)
    handles, keep = [], []
    for net in nets:
        dt = torch.complex64 if net.is_complex else torch.float32
        ts = [torch.from_numpy(np.array(t, order="C")).to(dt).cuda() for t in net.tensors]
        keep.append(ts)
        handles.append(binding.TensorNetwork(net.labels, net.dims, net.open, ts, complex_=net.is_complex))
    refs = [tree.contract_net(net.as_stored(), trees[i], sliced[i]) for i, net in enumerate(nets)]
    batch = binding.Batch(handles, trees, mode, sliced=sliced)
    tol = 1e-5
    try:
        for call in range(2):
            out, ex, lat = batch.contract()
            torch.cuda.synchronize()
            out, ex, lat = out.cpu().numpy(), ex.cpu().numpy(), lat.cpu().numpy()
            for i, net in enumerate(nets):
                mo, eo = refs[i]
                if net.is_complex:
                    got = complex(out[i, 0], out[i, 1]) * 2.0 ** (int(ex[i]) - eo)
                    ref = complex(mo)
                    assert abs(got - ref) <= tol * abs(ref), (call, i)
                else:
                    assert out[i, 1] == 0.0
                    d = math.log(out[i, 0]) + (int(ex[i]) - eo) * math.log(2) - math.log(float(mo))
                    assert abs(math.expm1(d)) <= tol, (call, i, d)
            assert np.all(lat > 0) and np.all(lat < 60 * 10**9)
            # the sliced members run after the forest, the second after the first
            assert lat[-2] >= lat[:-2].max() and lat[-1] >= lat[-2]
    finally:
        batch.close()
        for h in handles:
            h.close()
