"""The per-node kernel autotuner: every candidate it may keep computes the
same contraction, so results after tuning match the FP64 oracle within the
mode's tolerance, are stable across calls (the captured graph is rebuilt),
and the choices are valid."""
import math

import numpy as np
import pytest

from oracle import tree
from paper_2002_01935_gb300 import inputs, planner

pytestmark = pytest.mark.gpu

VALID = {0, 1, 2, 3, 4, 6, 8, 9, 10}


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


@pytest.mark.parametrize("mode", ["fp32", "tf32_split", "fp16_split", "bf16_split"])
def test_ising_after_autotune(torch, mode):
    net = inputs.random_ising(100, seed=0)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    tnw = handle(torch, net)
    try:
        choice = tnw.autotune(pairs, [], mode, reps=2)
        vals = []
        for _ in range(2):
            m, e = tnw.contract(pairs, [], mode)
            torch.cuda.synchronize()
            vals.append(math.log(float(m.cpu())) + int(e.cpu()) * math.log(2))
    finally:
        tnw.close()
    assert set(choice) <= VALID and len(choice) == len(pairs)
    assert any(c != 0 for c in choice)
    if mode == "fp32":
        assert not {8, 9, 10} & set(choice)
    mo, eo = tree.contract_net(net.as_stored(), pairs)
    ref = math.log(float(mo)) + eo * math.log(2)
    assert abs(math.expm1(vals[0] - ref)) <= (1e-4 if mode == "bf16_split" else 1e-5)
    assert vals[0] == vals[1]


@pytest.mark.parametrize("mode", ["tf32_split", "fp16_split", "bf16_split"])
def test_circuit_sliced_after_autotune(torch, mode):
    circ = inputs.random_circuit(5, 5, 10, seed=0)
    net = inputs.circuit_network(circ, inputs.random_bitstrings(25, 1, seed=1000)[0])
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    sl = planner.slice_greedy(net.labels, net.dims, pairs, net.open, 20)
    tnw = handle(torch, net)
    try:
        before, eb = tnw.contract(pairs, sl, mode)
        choice = tnw.autotune(pairs, sl, mode, reps=2)
        after, ea = tnw.contract(pairs, sl, mode)
        torch.cuda.synchronize()
        got_b = complex(before.cpu()) * 2.0 ** int(eb.cpu())
        got_a = complex(after.cpu()) * 2.0 ** int(ea.cpu())
    finally:
        tnw.close()
    assert set(choice) <= VALID
    # the oracle on the leaf values the GPU reads (complex64), at the mode's bound
    mo, eo = tree.contract_net(net.as_stored(), pairs, sl)
    ref = complex(mo) * 2.0 ** eo
    tol = {"tf32_split": 1e-5, "fp16_split": 1e-5, "bf16_split": 1e-4}[mode]
    assert abs(got_a - ref) <= tol * abs(ref)
    assert abs(got_a - got_b) <= tol * abs(ref)


def test_autotune_open_outputs_random_networks(torch):
    from oracle import brute
    for seed in range(4):
        net = inputs.random_network(8, 12, 700 + seed, n_open=2, complex_=True, max_dim=2)
        pairs = planner.greedy_tree(net.labels, net.dims, net.open)
        tnw = handle(torch, net)
        try:
            tnw.autotune(pairs, [], "fp32", reps=1)
            m, e = tnw.contract(pairs, [], "fp32")
            torch.cuda.synchronize()
            got = m.cpu().numpy() * 2.0 ** int(e.cpu())
        finally:
            tnw.close()
        ref = brute.nested_sum(net.tensors, net.labels, net.dims, net.open)
        scale = brute.nested_sum([np.abs(t) for t in net.tensors], net.labels, net.dims, net.open)
        assert np.all(np.abs(got - ref) <= 1e-5 * np.abs(scale) + 1e-30)
