"""Parity at the size of the 7x7-qubit, 14-cycle circuit amplitude whose
Hyper-Greedy tree is sliced to W_s <= 28 (Sec. 4.7.1 slicing; the paper's
single-amplitude task of Sec. 4.7.2), in every precision mode, through the
C-ABI.

1. The tree's largest node alone (M 2^15 x K 2^10 times K 2^10 x N 2^13,
   complex): 256 sampled output entries, each against the oracle contracting
   the K-only network that is left when the entry's M and N labels are fixed.
2. Sub-slices of the real tree with its slicing refined to W_s <= 20 (a
   W_s <= 28 slice takes the oracle hours): a seeded sample, each
   sub-slice's value against the oracle's value of that sub-slice.
3. Whole W_s <= 28 slices in the configuration the benchmark times (same
   tree, same slicing, autotuned plan) on a network of the same structure
   whose gates are product-form stand-ins (a two-qubit gate is the tensor
   product of two single-qubit matrices; entries share one phase per gate,
   so nothing cancels).  The value of a slice is then known exactly: the
   network rewired with every two-qubit gate split into its two factors has
   the same sum of products (Sec. 2), and the oracle contracts the rewired
   network -- 49 independent qubit wires -- in milliseconds.

References are computed on the leaf values the GPU reads (complex64 widened
to complex128), so each comparison measures the executor's arithmetic.
"""
import os
import sys

import numpy as np
import pytest

from oracle import tree
from paper_2002_01935_gb300 import inputs, planner

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MODES = ["fp32", "tf32_split", "fp16_split", "bf16_split", "tf32_3m"]
# relative error bound of each mode (the FP64 oracle on the same leaf values)
TOL = {"fp32": 1e-5, "tf32_split": 1e-5, "fp16_split": 1e-5, "bf16_split": 1e-4, "tf32_3m": 1e-2}


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_01935_gb300 import build
    build.build()
    return _t


@pytest.fixture(scope="module")
def workload():
    """The benchmark's 7x7x14 workload: circuit, bitstring, tree, slicing."""
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    w = bench.wl_circuit7x7(0, 2)
    assert w["info"].W <= 28 and w["info"].d_sliced >= 2 ** 20
    return w


def _device_leaves(torch, net):
    return [torch.from_numpy(np.array(t, order="C")).to(torch.complex64).contiguous().cuda()
            for t in net.tensors]


def _largest_node(w):
    """(M, N, K) label bits of the largest contraction of the sliced tree."""
    net, pairs, sliced = w["net"], w["pairs"], w["sliced"]
    sets = planner.node_labels(net.labels, pairs, net.open, removed=sliced)
    n = net.n_tensors
    best = None
    for k, (a, b) in enumerate(pairs):
        sa, sb = sets[a], sets[b]
        kk = len(sa & sb - sets[n + k])
        mm, nn = len(sa - sb), len(sb - sa)
        if best is None or mm + nn + kk > sum(best):
            best = (max(mm, nn), min(mm, nn), kk)
    return best


def test_largest_node_sampled_outputs_every_mode(torch, workload):
    from paper_2002_01935_gb300 import binding
    mb, nb, kb = _largest_node(workload)
    assert (mb, nb, kb) == (15, 13, 10)
    rng = np.random.default_rng(11)
    ml = list(range(mb))
    nl = list(range(mb, mb + nb))
    kl = list(range(mb + nb, mb + nb + kb))
    dims = {l: 2 for l in ml + nl + kl}
    # K labels interleaved with the M and N labels, as in a contraction tree
    la = kl[::2] + ml + kl[1::2]
    lb = nl[:3] + kl + nl[3:]
    f = lambda s: (rng.standard_normal(s) + 1j * rng.standard_normal(s)).astype(np.complex64)
    ta, tb = f([2] * len(la)), f([2] * len(lb))
    net = inputs.Network([ta, tb], [la, lb], dims, ml + nl)
    ii = rng.integers(0, 2 ** mb, 256)
    jj = rng.integers(0, 2 ** nb, 256)
    # the oracle, one entry at a time: fix the M and N labels, contract over K
    A = ta.astype(np.complex128)
    B = tb.astype(np.complex128)
    la_k = [l for l in la if l in kl]
    lb_k = [l for l in lb if l in kl]
    ref = np.empty(256, dtype=np.complex128)
    for s, (i, j) in enumerate(zip(ii, jj)):
        mv = {l: (int(i) >> (mb - 1 - p)) & 1 for p, l in enumerate(ml)}
        nv = {l: (int(j) >> (nb - 1 - p)) & 1 for p, l in enumerate(nl)}
        ai = A[tuple(mv[l] if l in mv else slice(None) for l in la)]
        bj = B[tuple(nv[l] if l in nv else slice(None) for l in lb)]
        m, e = tree.contract([ai, bj], [la_k, lb_k], {l: 2 for l in kl}, [], [(0, 1)])
        ref[s] = complex(m) * 2.0 ** e
    leaves = [torch.from_numpy(t).cuda() for t in (ta, tb)]
    tnw = binding.TensorNetwork(net.labels, net.dims, net.open, leaves, complex_=True)
    try:
        flat = torch.from_numpy(ii * 2 ** nb + jj).cuda()
        for mode in MODES:
            info = tnw.plan_info([(0, 1)], [], mode)
            if mode != "fp32":
                assert info["n_tensor_core"] == 1, mode
            m, e = tnw.contract([(0, 1)], [], mode)
            got = m.reshape(-1)[flat].cpu().numpy() * 2.0 ** int(e.cpu())
            del m
            err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert err <= TOL[mode], (mode, err)
    finally:
        tnw.close()
        torch.cuda.empty_cache()


def test_refined_subslices_every_mode(torch, workload):
    from paper_2002_01935_gb300 import binding
    net, pairs = workload["net"], workload["pairs"]
    sl2 = planner.slice_greedy(net.labels, net.dims, pairs, net.open, 20.0)
    i2 = planner.tree_info(net.labels, net.dims, pairs, net.open, sl2)
    assert i2.W <= 20
    stored = net.as_stored()
    ids = sorted(int(x) for x in np.random.default_rng(5).integers(0, int(i2.d_sliced), 4))
    refs = []
    for s in ids:
        m, e = tree.contract_net(stored, pairs, sl2, slice_begin=s, slice_count=1)
        refs.append(complex(m) * 2.0 ** e)
    tnw = binding.TensorNetwork(net.labels, net.dims, net.open, _device_leaves(torch, net),
                                complex_=True)
    try:
        for mode in MODES:
            if mode != "fp32":
                assert tnw.plan_info(pairs, sl2, mode)["n_tensor_core"] >= 1, mode
            for s, ref in zip(ids, refs):
                m, e = tnw.contract(pairs, sl2, mode, slice_begin=s, slice_count=1)
                got = complex(m.cpu()) * 2.0 ** int(e.cpu())
                err = abs(got - ref) / abs(ref)
                assert err <= TOL[mode], (mode, s, err)
    finally:
        tnw.close()
        torch.cuda.empty_cache()


def _product_form_circuit(seed):
    """The 7x7x14 circuit's network with every gate replaced by a
    product-form stand-in of the same shape: single-qubit gates
    e^{i phi} P and two-qubit gates e^{i phi} (P_a (x) P_b), P with random
    entries in [0.5, 1].  All terms of the network's sum then share their
    phase, so no value results from cancellation, and the network is a
    product over qubit wires.  Returns the network and its rewired twin in
    which every two-qubit leaf G[oa, ob, ia, ib] = P_a[oa, ia] P_b[ob, ib]
    is split into its two factors (same labels, same sum of products)."""
    rng = np.random.default_rng(seed)
    circ = inputs.random_circuit(7, 7, 14, seed=0)
    bits = inputs.random_bitstrings(49, 1, seed=1000)[0]
    over, factors = {}, {}
    for gi, g in enumerate(circ.gates):
        ph = np.exp(1j * rng.uniform(0, 2 * np.pi))
        if len(g.qubits) == 1:
            over[gi] = ph * rng.uniform(0.5, 1.0, (2, 2))
        else:
            pa, pb = rng.uniform(0.5, 1.0, (2, 2)), rng.uniform(0.5, 1.0, (2, 2))
            over[gi] = ph * np.kron(pa, pb)
            factors[gi] = (ph * pa, pb)
    net = inputs.circuit_network(circ, bits, gate_overrides=over).as_stored()
    leaf_of = {net.meta["gate_leaf"][gi]: gi for gi in factors}
    tensors, labels = [], []
    for v, (t, ls) in enumerate(zip(net.tensors, net.labels)):
        if v in leaf_of:
            oa, ob, ia, ib = ls
            fa, fb = factors[leaf_of[v]]
            tensors += [fa, fb]
            labels += [[oa, ia], [ob, ib]]
        else:
            tensors.append(t)
            labels.append(list(ls))
    split = inputs.Network(tensors, labels, dict(net.dims), list(net.open)).as_stored()
    return net, split


def test_full_size_slices_product_form_every_mode(torch, workload):
    """Whole W_s <= 28 slices, benchmark plan (autotuned), exact reference."""
    from paper_2002_01935_gb300 import binding
    net0, pairs, sliced = workload["net"], workload["pairs"], workload["sliced"]
    net, split = _product_form_circuit(21)
    assert net.labels == net0.labels  # same structure: the same tree and slicing apply
    split_tree = planner.greedy_tree(split.labels, split.dims, split.open)
    d = int(workload["info"].d_sliced)
    ids = [0, d - 1] + [int(x) for x in np.random.default_rng(4).integers(0, d, 2)]
    vals = {}
    for s in ids:
        m, e = tree.contract_net(split, split_tree, sliced, slice_begin=s, slice_count=1)
        vals[s] = complex(m) * 2.0 ** e
    tnw = binding.TensorNetwork(net.labels, net.dims, net.open, _device_leaves(torch, net),
                                complex_=True)
    try:
        for mode in MODES:
            if mode in ("tf32_split", "fp16_split"):
                tnw.autotune(pairs, sliced, mode, reps=2)
            if mode != "fp32":
                assert tnw.plan_info(pairs, sliced, mode)["n_tensor_core"] >= 4, mode
            for s in ids:
                m, e = tnw.contract(pairs, sliced, mode, slice_begin=s, slice_count=1)
                got = complex(m.cpu()) * 2.0 ** int(e.cpu())
                err = abs(got - vals[s]) / abs(vals[s])
                assert err <= TOL[mode], (mode, s, err)
    finally:
        tnw.close()
        torch.cuda.empty_cache()
