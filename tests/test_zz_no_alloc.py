"""tn_contract_noalloc: the contraction for callers that cannot allocate
device memory (hosts that forbid device allocation after start-up, and
processes whose device memory is owned by another allocator's pool).  Its
results must match tn_contract's and the FP64 oracle's (run on the leaf
values the GPU reads), on consecutive calls that reuse the shared fixed
scratch -- including the first call on a fresh handle, a single-leaf network
and a sliced tree with open outputs -- and trees too large for the scratch
must be refused with a clear error.
Collected last so a stop-at-first-failure run has executed every other test.
"""
import numpy as np
import pytest

from oracle import tree
from paper_2002_01935_gb300 import inputs, planner

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_01935_gb300 import build
    build.build()
    from paper_2002_01935_gb300 import binding
    return torch, binding


def _leaves(torch, net):
    dt = torch.complex64 if net.is_complex else torch.float32
    return [torch.from_numpy(np.array(t, order="C")).to(dt).contiguous().cuda() for t in net.tensors]


def _oracle(net, pairs, sliced=()):
    m, e = tree.contract_net(net.as_stored(), pairs, sliced)
    return m * 2.0 ** e


def _noalloc_device(torch, binding, tnw, pairs, sliced, cplx):
    odt = torch.complex128 if cplx else torch.float64
    out = torch.full(tnw.out_shape, 7.0, dtype=odt, device="cuda")
    oe = torch.full((), 99, dtype=torch.int64, device="cuda")
    binding.tn_contract_noalloc(tnw.h, pairs, sliced, out.data_ptr(), binding.TN_MEM_DEVICE,
                                oe.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy() * 2.0 ** int(oe.cpu())


def test_noalloc_matches_tn_contract_on_two_calls(env):
    torch, binding = env
    circ = inputs.random_circuit(4, 4, 8, seed=0)
    net = inputs.circuit_network(circ, inputs.random_bitstrings(16, 1, seed=1000)[0])
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    sliced = planner.slice_greedy(net.labels, net.dims, pairs, net.open, 10)
    oref = complex(_oracle(net, pairs, sliced))
    ts = _leaves(torch, net)
    tnw = binding.TensorNetwork(net.labels, net.dims, net.open, ts, complex_=True)
    try:
        m, e = tnw.contract(pairs, sliced, "fp32")
        torch.cuda.synchronize()
        ref = complex(m.cpu()) * 2.0 ** int(e.cpu())
        stream = torch.cuda.current_stream().cuda_stream
        for call in range(2):
            out = torch.full((), complex(7, 7), dtype=torch.complex128, device="cuda")
            oe = torch.full((), 99, dtype=torch.int64, device="cuda")
            binding.tn_contract_noalloc(tnw.h, pairs, sliced, out.data_ptr(),
                                        binding.TN_MEM_DEVICE, oe.data_ptr(), stream)
            torch.cuda.synchronize()
            got = complex(out.cpu()) * 2.0 ** int(oe.cpu())
            assert abs(got - ref) <= TOL * abs(ref), (call, got, ref)
            assert abs(got - oref) <= TOL * abs(oref), (call, got, oref)
    finally:
        tnw.close()


def test_noalloc_open_outputs_to_host(env):
    torch, binding = env
    circ = inputs.random_circuit(3, 3, 5, seed=2)
    net = inputs.circuit_network(circ, open_qubits=[2, 0, 1, 3, 4, 5, 6, 7, 8])
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    oref = _oracle(net, pairs)
    ts = _leaves(torch, net)
    tnw = binding.TensorNetwork(net.labels, net.dims, net.open, ts, complex_=True)
    try:
        m, e = tnw.contract(pairs, [], "fp32")
        torch.cuda.synchronize()
        ref = m.cpu().numpy() * 2.0 ** int(e.cpu())
        for call in range(2):
            out = torch.zeros(tnw.out_shape, dtype=torch.complex128).pin_memory()
            oe = torch.zeros((), dtype=torch.int64).pin_memory()
            binding.tn_contract_noalloc(tnw.h, pairs, [], out.data_ptr(), binding.TN_MEM_HOST,
                                        oe.data_ptr(), torch.cuda.current_stream().cuda_stream)
            got = out.numpy() * 2.0 ** int(oe)
            assert np.linalg.norm(got - ref) <= TOL * np.linalg.norm(ref)
            assert np.linalg.norm(got - oref) <= TOL * np.linalg.norm(oref)
    finally:
        tnw.close()


def test_noalloc_refuses_trees_beyond_the_scratch(env):
    torch, binding = env
    net = inputs.random_ising(100, seed=0)  # ~19.6 MB of workspace > 8 MiB
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    ts = _leaves(torch, net)
    tnw = binding.TensorNetwork(net.labels, net.dims, net.open, ts, complex_=False)
    try:
        out = torch.zeros((), dtype=torch.float64, device="cuda")
        oe = torch.zeros((), dtype=torch.int64, device="cuda")
        with pytest.raises(binding.TNError) as err:
            binding.tn_contract_noalloc(tnw.h, pairs, [], out.data_ptr(), binding.TN_MEM_DEVICE,
                                        oe.data_ptr(), torch.cuda.current_stream().cuda_stream)
        assert err.value.status == binding.TN_EUNSUPPORTED
        assert "8 MiB" in str(err.value)
    finally:
        tnw.close()


def test_noalloc_first_call_on_fresh_handle_sliced_open_outputs(env):
    """No tn_contract before: the handle's plan has never been run, so the
    call cannot lean on a workspace or device state tn_contract made."""
    torch, binding = env
    circ = inputs.random_circuit(3, 3, 6, seed=4)
    net = inputs.circuit_network(circ, inputs.random_bitstrings(9, 1, seed=1004)[0],
                                 open_qubits=[4, 1, 7])
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    sliced = planner.slice_greedy(net.labels, net.dims, pairs, net.open, 6)
    assert sliced
    ref = _oracle(net, pairs, sliced)
    tnw = binding.TensorNetwork(net.labels, net.dims, net.open, _leaves(torch, net), complex_=True)
    try:
        for call in range(2):
            got = _noalloc_device(torch, binding, tnw, pairs, sliced, True)
            assert np.linalg.norm(got - ref) <= TOL * np.linalg.norm(ref), call
        m, e = tnw.contract(pairs, sliced, "fp32")
        torch.cuda.synchronize()
        again = m.cpu().numpy() * 2.0 ** int(e.cpu())
        assert np.linalg.norm(again - got) <= TOL * np.linalg.norm(ref)
    finally:
        tnw.close()


@pytest.mark.parametrize("open_labels", [[0, 2], []])
def test_noalloc_single_leaf(env, open_labels):
    """One tensor and no pairs: its summed label is contracted against the
    scratch's own unit scalar."""
    torch, binding = env
    rng = np.random.default_rng(9)
    t = rng.standard_normal((2, 4, 2)) + 1j * rng.standard_normal((2, 4, 2))
    net = inputs.Network([t], [[0, 1, 2]], {0: 2, 1: 4, 2: 2}, list(open_labels))
    ref = _oracle(net, [])
    tnw = binding.TensorNetwork(net.labels, net.dims, net.open, _leaves(torch, net), complex_=True)
    try:
        for call in range(2):
            got = _noalloc_device(torch, binding, tnw, [], [], True)
            assert np.linalg.norm(got - ref) <= TOL * np.linalg.norm(ref), call
    finally:
        tnw.close()


def test_noalloc_real_network_against_oracle(env):
    torch, binding = env
    net = inputs.random_ising(16, seed=3)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    sliced = planner.slice_greedy(net.labels, net.dims, pairs, net.open, 3)
    assert sliced
    ref = float(_oracle(net, pairs, sliced))
    tnw = binding.TensorNetwork(net.labels, net.dims, net.open, _leaves(torch, net), complex_=False)
    try:
        for call in range(2):
            got = float(_noalloc_device(torch, binding, tnw, pairs, sliced, False))
            assert abs(got - ref) <= TOL * abs(ref), (call, got, ref)
    finally:
        tnw.close()


def test_noalloc_host_outputs_refused_while_capturing(env):
    """Host outputs make the call wait for its stream; on a stream that is
    capturing a graph the call refuses them before it launches anything."""
    torch, binding = env
    net = inputs.random_ising(12, seed=5)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    tnw = binding.TensorNetwork(net.labels, net.dims, net.open, _leaves(torch, net), complex_=False)
    try:
        ref = float(_oracle(net, pairs))
        got = float(_noalloc_device(torch, binding, tnw, pairs, [], False))  # set-up call
        assert abs(got - ref) <= TOL * abs(ref)
        out = torch.zeros((), dtype=torch.float64).pin_memory()
        oe = torch.zeros((), dtype=torch.int64).pin_memory()
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with pytest.raises(binding.TNError) as err:
            with torch.cuda.graph(g, stream=s):
                binding.tn_contract_noalloc(tnw.h, pairs, [], out.data_ptr(), binding.TN_MEM_HOST,
                                            oe.data_ptr(), s.cuda_stream)
        assert err.value.status == binding.TN_EUNSUPPORTED
        torch.cuda.synchronize()
        again = float(_noalloc_device(torch, binding, tnw, pairs, [], False))
        assert abs(again - ref) <= TOL * abs(ref)
    finally:
        tnw.close()
