"""tn_contract_noalloc: the contraction for callers that cannot allocate
device memory (graph-capturing code, allocation-free hosts, processes whose
device memory belongs to another allocator).  Its results must match
tn_contract's, on consecutive calls that reuse the shared fixed scratch,
and trees too large for the scratch must be refused with a clear error.
Collected last so a stop-at-first-failure run has executed every other test.
"""
import numpy as np
import pytest

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


def test_noalloc_matches_tn_contract_on_two_calls(env):
    torch, binding = env
    circ = inputs.random_circuit(4, 4, 8, seed=0)
    net = inputs.circuit_network(circ, inputs.random_bitstrings(16, 1, seed=1000)[0])
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    sliced = planner.slice_greedy(net.labels, net.dims, pairs, net.open, 10)
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
    finally:
        tnw.close()


def test_noalloc_open_outputs_to_host(env):
    torch, binding = env
    circ = inputs.random_circuit(3, 3, 5, seed=2)
    net = inputs.circuit_network(circ, open_qubits=[2, 0, 1, 3, 4, 5, 6, 7, 8])
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
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
