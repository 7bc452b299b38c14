"""GPU parity: the CUDA executor (through the C-ABI) against the FP64 oracle.

Element-by-element on seeded inputs.  Tolerances (FP32 arithmetic inside
each contraction, FP64 across slices): relative 1e-5 for amplitudes and
open tensors, |exp(lnZ - lnZ_ref) - 1| <= 1e-5 for partition functions,
and for random networks |x - x_ref| <= 1e-5 * (the same network evaluated
on |T|), the cancellation-free scale of the rounding error.
"""
import math

import numpy as np
import pytest

from oracle import brute, statevector, tree
from paper_2002_01935_gb300 import inputs, planner

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_01935_gb300 import build
    build.build()
    return _t


def gpu_contract(torch, net, pairs, sliced=(), mode="fp32", host=False, **kw):
    from paper_2002_01935_gb300 import binding
    cplx = net.is_complex
    dt = torch.complex64 if cplx else torch.float32
    ts = [torch.from_numpy(np.array(t, order="C")).to(dt).contiguous() for t in net.tensors]
    if host:
        ts = [t.pin_memory() for t in ts]
    else:
        ts = [t.cuda() for t in ts]
    tnw = binding.TensorNetwork(net.labels, net.dims, net.open, ts, complex_=cplx)
    try:
        if host:
            odt = torch.complex128 if cplx else torch.float64
            out = torch.empty(tnw.out_shape, dtype=odt).pin_memory()
            oe = torch.empty((), dtype=torch.int64).pin_memory()
            m, e = tnw.contract(pairs, sliced, mode, out=out, out_exp=oe, **kw)
        else:
            m, e = tnw.contract(pairs, sliced, mode, **kw)
        torch.cuda.synchronize()
        return m.cpu().numpy(), int(e.cpu())
    finally:
        tnw.close()


def oracle(net, pairs, sliced=(), **kw):
    """The FP64 oracle on the leaf values the GPU reads (complex64 / float32)."""
    return tree.contract_net(net.as_stored(), pairs, sliced, **kw)


def assert_close_scaled(got, ref, scale, tol=TOL):
    got = np.asarray(got)
    assert got.shape == np.asarray(ref).shape
    assert np.all(np.abs(got - ref) <= tol * np.abs(scale) + 1e-30), (
        float(np.max(np.abs(got - ref) / (np.abs(scale) + 1e-30))))


def rel_err(got, ref):
    return float(np.linalg.norm(np.ravel(got - ref)) / max(np.linalg.norm(np.ravel(ref)), 1e-300))


# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(16))
def test_random_networks(torch, seed):
    """Hyperedges, summed-only labels, open labels, outer products, sizes 1..3."""
    net = inputs.random_network(7 + seed % 4, 12 + seed % 5, 900 + seed, n_open=seed % 3,
                                complex_=seed % 2 == 0)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    m, e = gpu_contract(torch, net, pairs)
    ref = brute.nested_sum(net.tensors, net.labels, net.dims, net.open)
    scale = brute.nested_sum([np.abs(t) for t in net.tensors], net.labels, net.dims, net.open)
    assert_close_scaled(m * 2.0 ** e, ref, scale)


@pytest.mark.parametrize("seed", range(6))
def test_random_networks_sliced(torch, seed):
    net = inputs.random_network(9, 14, 950 + seed, n_open=seed % 2, complex_=seed % 2 == 0)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    summed = [l for l in sorted(net.dims) if l not in net.open]
    rng = np.random.default_rng(seed)
    sl = [int(x) for x in rng.choice(summed, size=min(3, len(summed)), replace=False)]
    m, e = gpu_contract(torch, net, pairs, sl)
    ref = brute.nested_sum(net.tensors, net.labels, net.dims, net.open)
    scale = brute.nested_sum([np.abs(t) for t in net.tensors], net.labels, net.dims, net.open)
    assert_close_scaled(m * 2.0 ** e, ref, scale)
    # slice ranges partition the sum: each single slice against the oracle's slice
    d = int(np.prod([net.dims[l] for l in sl]))
    for s in range(d):
        ms, es = gpu_contract(torch, net, pairs, sl, slice_begin=s, slice_count=1)
        mo, eo = oracle(net, pairs, sl, slice_begin=s, slice_count=1)
        assert_close_scaled(ms * 2.0 ** es, mo * 2.0 ** eo, scale)


def test_cfg0_circuit_amplitude(torch):
    """4x4 grid, 8 cycles, greedy tree, no slicing: complex64 vs complex128."""
    circ = inputs.random_circuit(4, 4, 8, seed=0)
    bs = inputs.random_bitstrings(16, 1, seed=1000)[0]
    net = inputs.circuit_network(circ, bs)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    m, e = gpu_contract(torch, net, pairs)
    mo, eo = oracle(net, pairs)
    got, ref = complex(m) * 2.0 ** e, complex(mo) * 2.0 ** eo
    assert abs(got - ref) <= TOL * abs(ref)
    # the oracle on the complex128 leaves is the state vector's amplitude
    mw, ew = tree.contract_net(net, pairs)
    wide = complex(mw) * 2.0 ** ew
    assert abs(wide - statevector.amplitude(16, circ.gates, bs)) <= 1e-12 * abs(wide)


def test_cfg0_tree_independence(torch):
    circ = inputs.random_circuit(4, 4, 8, seed=0)
    bs = inputs.random_bitstrings(16, 1, seed=1000)[0]
    net = inputs.circuit_network(circ, bs)
    mo, eo = oracle(net, planner.greedy_tree(net.labels, net.dims, net.open))
    ref = complex(mo) * 2.0 ** eo
    for pairs in (planner.greedy_tree(net.labels, net.dims, net.open, alpha=0.0),
                  planner.greedy_tree(net.labels, net.dims, net.open, tau=0.3, seed=4),
                  planner.left_deep_tree(net.n_tensors)):
        m, e = gpu_contract(torch, net, pairs)
        assert abs(complex(m) * 2.0 ** e - ref) <= TOL * abs(ref)


def test_cfg0_sliced(torch):
    circ = inputs.random_circuit(4, 4, 8, seed=0)
    bs = inputs.random_bitstrings(16, 1, seed=1000)[0]
    net = inputs.circuit_network(circ, bs)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    sl = planner.slice_greedy(net.labels, net.dims, pairs, net.open, 8)
    m, e = gpu_contract(torch, net, pairs, sl)
    mo, eo = oracle(net, pairs)
    ref = complex(mo) * 2.0 ** eo
    assert abs(complex(m) * 2.0 ** e - ref) <= TOL * abs(ref)
    # graph replay and direct launches agree bit for bit
    m2, e2 = gpu_contract(torch, net, pairs, sl, no_graph=True)
    assert e2 == e and complex(m2) == complex(m)


def test_cfg1_ising_partition_function(torch):
    """N=100 random 3-regular Ising, beta=0.3, J=+-1: ln Z in fp32 vs FP64."""
    net = inputs.random_ising(100, seed=0)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    info = planner.tree_info(net.labels, net.dims, pairs, net.open)
    sl = planner.slice_greedy(net.labels, net.dims, pairs, net.open, 24) if info.W > 24 else []
    m, e = gpu_contract(torch, net, pairs, sl)
    mo, eo = oracle(net, pairs)
    lz = math.log(float(m)) + e * math.log(2)
    lz_ref = math.log(float(mo)) + eo * math.log(2)
    assert abs(math.expm1(lz - lz_ref)) <= TOL


def test_cfg1_sliced_to_width_18(torch):
    """The same network sliced harder (2^k slices in one call)."""
    net = inputs.random_ising(100, seed=0)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    sl = planner.slice_greedy(net.labels, net.dims, pairs, net.open, 18)
    assert len(sl) >= 2
    m, e = gpu_contract(torch, net, pairs, sl)
    mo, eo = oracle(net, pairs)
    lz = math.log(float(m)) + e * math.log(2)
    lz_ref = math.log(float(mo)) + eo * math.log(2)
    assert abs(math.expm1(lz - lz_ref)) <= TOL


def test_renormalisation_beyond_float_range(torch):
    """Edge matrices scaled by 2^100: Z grows by 2^(100|E|), far outside
    FP32 and FP64; the exponent bookkeeping must carry it exactly."""
    net = inputs.random_ising(40, seed=9)
    n_e = len(net.meta["edges"])
    scaled = net.with_tensors([t if i < 40 else t * 2.0 ** 100 for i, t in enumerate(net.tensors)])
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    m0, e0 = gpu_contract(torch, net, pairs)
    m1, e1 = gpu_contract(torch, scaled, pairs)
    d = (math.log2(float(m1)) + e1) - (math.log2(float(m0)) + e0)
    assert abs(d - 100 * n_e) < 1e-4


def test_open_outputs_all_amplitudes(torch):
    """All 2^9 amplitudes of a 3x3 circuit as one open tensor."""
    circ = inputs.random_circuit(3, 3, 6, seed=2)
    net = inputs.circuit_network(circ, open_qubits=[4, 0, 8, 1, 2, 3, 5, 6, 7])
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    m, e = gpu_contract(torch, net, pairs)
    amp = m * 2.0 ** e
    psi = statevector.final_state(9, circ.gates).transpose(4, 0, 8, 1, 2, 3, 5, 6, 7)
    assert rel_err(amp, psi) <= TOL
    assert abs(np.sum(np.abs(amp) ** 2) - 1) <= 1e-5


def test_host_buffers(torch):
    """Host leaves and host outputs (copies inside the call)."""
    circ = inputs.random_circuit(3, 3, 6, seed=5)
    bs = inputs.random_bitstrings(9, 1, seed=6)[0]
    net = inputs.circuit_network(circ, bs)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    m, e = gpu_contract(torch, net, pairs, host=True)
    ref = statevector.amplitude(9, circ.gates, bs)
    assert abs(complex(m) * 2.0 ** e - ref) <= TOL * abs(ref)


def test_degenerate_networks(torch):
    rng = np.random.default_rng(0)
    a = rng.standard_normal((2, 3)).astype(np.complex128)
    # a lone tensor: sum one label, keep the other
    net = inputs.Network([a], [[0, 1]], {0: 2, 1: 3}, [1])
    m, e = gpu_contract(torch, net, [])
    assert np.allclose(m * 2.0 ** e, a.sum(axis=0), rtol=1e-6)
    # a lone tensor summed to a scalar
    net = inputs.Network([a], [[0, 1]], {0: 2, 1: 3}, [])
    m, e = gpu_contract(torch, net, [])
    assert abs(complex(m) * 2.0 ** e - a.sum()) <= 1e-6 * abs(a).sum()
    # rank-0 leaves and a size-1 label
    s = np.array(3.0 + 1j)
    b = rng.standard_normal((1, 3)).astype(np.complex128)
    net = inputs.Network([s, b, a], [[], [2, 1], [0, 1]], {0: 2, 1: 3, 2: 1}, [0])
    m, e = gpu_contract(torch, net, [(0, 1), (3, 2)])
    ref = s * np.einsum("ki,ji->j", b, a)
    assert np.allclose(m * 2.0 ** e, ref, rtol=1e-6)
    # an all-zero leaf: exact zero with exponent 0
    z = np.zeros((2, 3), dtype=np.complex128)
    net = inputs.Network([z, b], [[0, 1], [2, 1]], {0: 2, 1: 3, 2: 1}, [])
    m, e = gpu_contract(torch, net, [(0, 1)])
    assert complex(m) == 0 and e == 0


def test_cfg3_amplitudes_20_qubits(torch):
    """5x4 grid, 12 cycles (the differentiation workload's forward)."""
    circ = inputs.random_circuit(5, 4, 12, seed=0)
    psi = statevector.final_state(20, circ.gates)
    for bs in inputs.random_bitstrings(20, 2, seed=1000):
        net = inputs.circuit_network(circ, bs)
        pairs = planner.greedy_tree(net.labels, net.dims, net.open)
        m, e = gpu_contract(torch, net, pairs)
        ref = complex(psi[tuple(bs)])
        assert abs(complex(m) * 2.0 ** e - ref) <= TOL * abs(ref)


def test_cfg2_variant_5x5_10_cycles(torch):
    """The 5x5 / 10-cycle variant of the 7x7 workload, in full, unsliced and
    sliced to W_s <= 20, against the oracle."""
    circ = inputs.random_circuit(5, 5, 10, seed=0)
    bs = inputs.random_bitstrings(25, 1, seed=1000)[0]
    net = inputs.circuit_network(circ, bs)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    mo, eo = oracle(net, pairs)
    ref = complex(mo) * 2.0 ** eo
    m, e = gpu_contract(torch, net, pairs)
    assert abs(complex(m) * 2.0 ** e - ref) <= TOL * abs(ref)
    sl = planner.slice_greedy(net.labels, net.dims, pairs, net.open, 20)
    m, e = gpu_contract(torch, net, pairs, sl)
    assert abs(complex(m) * 2.0 ** e - ref) <= TOL * abs(ref)


def test_dataflow_waves_match_level_launches(torch, monkeypatch):
    """The same contraction with the small nodes of consecutive tree levels
    in one dataflow launch and with one launch per level: identical bits."""
    from paper_2002_01935_gb300 import binding
    res = []
    for flow in ("0", "1"):
        monkeypatch.setenv("TN_NO_FLOW", flow)
        for net in (inputs.random_ising(100, seed=0),
                    inputs.circuit_network(inputs.random_circuit(4, 4, 8, seed=0),
                                           inputs.random_bitstrings(16, 1, seed=1000)[0])):
            pairs = planner.greedy_tree(net.labels, net.dims, net.open)
            dt = torch.complex64 if net.is_complex else torch.float32
            ts = [torch.from_numpy(np.array(t, order="C")).to(dt).cuda() for t in net.tensors]
            h = binding.TensorNetwork(net.labels, net.dims, net.open, ts, complex_=net.is_complex)
            try:
                steps = h.plan_steps(pairs, [], "fp32")
                m, e = h.contract(pairs, [], "fp32")
                torch.cuda.synchronize()
                res.append((len(steps), m.cpu().numpy().tobytes(), int(e.cpu())))
            finally:
                h.close()
    (s0a, m0a, e0a), (s0b, m0b, e0b), (s1a, m1a, e1a), (s1b, m1b, e1b) = res
    assert s0a < s1a and s0b < s1b  # fewer launch steps with the dataflow
    assert (m0a, e0a) == (m1a, e1a) and (m0b, e0b) == (m1b, e1b)
