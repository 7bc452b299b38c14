"""Precision modes on the tensor cores against the FP64 oracle.

Large nodes run on tcgen05 tensor cores in the reduced-precision modes:
TF32 single pass, TF32 hi+lo split and BF16 hi+lo split (three products,
FP32 accumulation) and FP16 hi+lo split.  Single nodes: tolerances
relative to the cancellation-free scale of each entry (the same contraction
on |A|, |B|): 1e-5 for the TF32 and FP16 splits, 1e-4 for the BF16 split,
2e-3 for a single TF32 pass (10-bit mantissa).  Whole networks: relative
error of the value against the oracle run on the leaf values the GPU reads
(complex64 / float32), at the mode's bound (1e-2 for the single pass).
"""
import math

import numpy as np
import pytest

from oracle import brute, tree
from paper_2002_01935_gb300 import inputs, planner

pytestmark = pytest.mark.gpu

TOL = {"tf32_split": 1e-5, "fp16_split": 1e-5, "bf16_split": 1e-4, "tf32_3m": 2e-3, "fp32": 1e-5}
NET_TOL = dict(TOL, tf32_3m=1e-2)


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_01935_gb300 import build
    build.build()
    return _t


def run(torch, net, pairs, sliced=(), mode="fp32"):
    from paper_2002_01935_gb300 import binding
    cplx = net.is_complex
    dt = torch.complex64 if cplx else torch.float32
    ts = [torch.from_numpy(np.array(t, order="C")).to(dt).contiguous().cuda() for t in net.tensors]
    tnw = binding.TensorNetwork(net.labels, net.dims, net.open, ts, complex_=cplx)
    try:
        info = tnw.plan_info(pairs, sliced, mode)
        m, e = tnw.contract(pairs, sliced, mode)
        torch.cuda.synchronize()
        return m.cpu().numpy(), int(e.cpu()), info
    finally:
        tnw.close()


def gemm_net(mb, nb, kb, batch=0, cplx=True, seed=0, interleave=True):
    """C[b,m,n] = sum_k A[b,m,k] B[b,k,n] with all labels of size 2; the K
    labels interleave with M and N labels in the operand layouts."""
    rng = np.random.default_rng(seed)
    lab = 0
    bl = list(range(lab, lab + batch)); lab += batch
    ml = list(range(lab, lab + mb)); lab += mb
    nl = list(range(lab, lab + nb)); lab += nb
    kl = list(range(lab, lab + kb)); lab += kb
    dims = {l: 2 for l in range(lab)}
    if interleave:
        la = bl + kl[::2] + ml + kl[1::2]
        lb = nl[:2] + kl + bl + nl[2:]
    else:
        la = bl + ml + kl
        lb = bl + kl + nl
    def t(shape):
        x = rng.standard_normal(shape)
        return x + 1j * rng.standard_normal(shape) if cplx else x
    ta, tb = t([2] * len(la)), t([2] * len(lb))
    return inputs.Network([ta, tb], [la, lb], dims, bl + ml + nl)


@pytest.mark.parametrize("mode", ["tf32_split", "fp16_split", "bf16_split", "tf32_3m"])
@pytest.mark.parametrize("shape", [(8, 8, 8, 0, True), (7, 9, 6, 0, False), (9, 7, 10, 0, True),
                                   (7, 7, 4, 1, True), (8, 8, 7, 0, False), (7, 8, 3, 0, True),
                                   (6, 9, 5, 0, True), (6, 10, 6, 1, True), (10, 6, 5, 0, True),
                                   (7, 6, 9, 0, True), (7, 7, 10, 0, False), (6, 7, 9, 1, True),
                                   # narrow complex nodes (32 complex columns in a padded tile),
                                   # swapped or not, batch labels, K splits, K = 16; narrow real
                                   # nodes stay on the CUDA cores
                                   (5, 8, 6, 0, True), (8, 5, 6, 1, True), (5, 8, 10, 0, True),
                                   (9, 5, 4, 1, True), (8, 6, 6, 0, False), (7, 6, 9, 1, False)])
def test_single_gemm_node(torch, mode, shape):
    mb, nb, kb, batch, cplx = shape
    net = gemm_net(mb, nb, kb, batch, cplx, seed=sum(shape))
    pairs = [(0, 1)]
    m, e, info = run(torch, net, pairs, mode=mode)
    got = m * 2.0 ** e
    ref = brute.nested_sum(net.tensors, net.labels, net.dims, net.open) if mb + nb + kb + batch <= 22 \
        else tree.value(net.tensors, net.labels, net.dims, net.open, pairs)
    scale = tree.value([np.abs(x) for x in net.tensors], net.labels, net.dims, net.open, pairs)
    # tensor cores: K >= 16, >= 128 accumulator rows and >= 128 real columns
    # (a complex node puts its larger operand on the rows; its 32 complex
    # columns expand to 64 real ones in a padded tile)
    fits = max(mb, nb) >= 7 and min(mb, nb) >= 5 if cplx else min(mb, nb) >= 7
    if kb >= 4 and fits:
        assert info["n_tensor_core"] == 1
    err = float(np.max(np.abs(got - ref) / scale))
    assert err <= TOL[mode], err


@pytest.mark.parametrize("mode", ["tf32_split", "fp16_split", "bf16_split", "tf32_3m"])
def test_cfg1_ising_modes(torch, mode):
    net = inputs.random_ising(100, seed=0)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    m, e, info = run(torch, net, pairs, mode=mode)
    assert info["n_tensor_core"] >= 1
    mo, eo = tree.contract_net(net.as_stored(), pairs)
    d = math.log(float(m)) + e * math.log(2) - (math.log(float(mo)) + eo * math.log(2))
    assert abs(math.expm1(d)) <= NET_TOL[mode], d


@pytest.mark.parametrize("mode", ["fp32", "tf32_split", "fp16_split", "bf16_split", "tf32_3m"])
def test_circuit_5x5_modes(torch, mode):
    """Complex 4M on the tensor cores over a whole circuit network; the
    amplitude's error against the FP64 oracle (run on the complex64 leaf
    values the GPU reads) is within the mode's bound."""
    circ = inputs.random_circuit(5, 5, 10, seed=0)
    net = inputs.circuit_network(circ, inputs.random_bitstrings(25, 1, seed=1000)[0])
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    m, e, info = run(torch, net, pairs, mode=mode)
    assert (info["n_tensor_core"] >= 1) == (mode != "fp32")
    mo, eo = tree.contract_net(net.as_stored(), pairs)
    ref = complex(mo) * 2.0 ** eo
    err = abs(complex(m) * 2.0 ** e - ref) / abs(ref)
    assert err <= NET_TOL[mode], err


@pytest.mark.parametrize("mode", ["tf32_split", "fp16_split", "bf16_split"])
@pytest.mark.parametrize("shape", [(8, 8, 8, 0, True), (9, 7, 10, 0, True), (7, 7, 4, 1, True),
                                   (7, 9, 6, 1, True), (10, 7, 5, 0, True)])
def test_single_gemm_node_planar_layout(torch, mode, shape, monkeypatch):
    """The planar complex layout (Re and Im planes, negated Im x Im product)
    on single complex nodes, incl. batch labels, the swapped orientation and
    K shorter than one 64-byte row (K = 16)."""
    monkeypatch.setenv("TN_PLANAR", "1")
    mb, nb, kb, batch, cplx = shape
    net = gemm_net(mb, nb, kb, batch, cplx, seed=100 + sum(shape))
    pairs = [(0, 1)]
    m, e, info = run(torch, net, pairs, mode=mode)
    assert info["n_tensor_core"] == 1
    got = m * 2.0 ** e
    ref = tree.value(net.tensors, net.labels, net.dims, net.open, pairs)
    scale = tree.value([np.abs(x) for x in net.tensors], net.labels, net.dims, net.open, pairs)
    err = float(np.max(np.abs(got - ref) / scale))
    assert err <= TOL[mode], err


@pytest.mark.parametrize("mode", ["tf32_split", "fp16_split"])
def test_circuit_5x5_planar_layout(torch, mode, monkeypatch):
    monkeypatch.setenv("TN_PLANAR", "1")
    circ = inputs.random_circuit(5, 5, 10, seed=0)
    net = inputs.circuit_network(circ, inputs.random_bitstrings(25, 1, seed=1000)[0])
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    m, e, info = run(torch, net, pairs, mode=mode)
    mo, eo = tree.contract_net(net.as_stored(), pairs)
    ref = complex(mo) * 2.0 ** eo
    err = abs(complex(m) * 2.0 ** e - ref) / abs(ref)
    assert err <= NET_TOL[mode], err
