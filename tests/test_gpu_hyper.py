"""Hyperedge-form networks on the GPU: the Ising partition function with
one label per spin shared by the matrices of its three edges (Sec. 3.5), so
every intermediate contraction carries batch labels.  Compared with the
FP64 oracle (which is pinned to enumeration and to the COPY form)."""
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


@pytest.mark.parametrize("n,target,mode", [(100, 24.0, "fp32"), (100, 24.0, "tf32_split"),
                                           (100, 12.0, "fp32"), (60, 24.0, "bf16_split")])
def test_hyperedge_ising_ln_z(torch, n, target, mode):
    from paper_2002_01935_gb300 import binding
    net = inputs.random_ising_hyper(n, seed=0)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    info = planner.tree_info(net.labels, net.dims, pairs, net.open)
    sliced = planner.slice_greedy(net.labels, net.dims, pairs, net.open, target) if info.W > target else []
    ts = [torch.from_numpy(np.array(t, order="C")).float().cuda() for t in net.tensors]
    tnw = binding.TensorNetwork(net.labels, net.dims, net.open, ts, complex_=False)
    try:
        m, e = tnw.contract(pairs, sliced, mode)
        torch.cuda.synchronize()
        lz = math.log(float(m.cpu())) + int(e.cpu()) * math.log(2)
    finally:
        tnw.close()
    mo, eo = tree.contract_net(net, pairs, sliced)
    ref = math.log(float(mo)) + eo * math.log(2)
    tol = 1e-4 if mode == "bf16_split" else 1e-5
    assert abs(math.expm1(lz - ref)) <= tol, (lz, ref)
