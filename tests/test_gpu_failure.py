"""Failure detection without a GPU fault: a bounded device wait is made to
run out (a completion counter that nothing raises), the kernel records
TN_ETIMEOUT and returns, the host reads the status, and the CUDA context
stays usable for the next contraction."""
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


def test_dataflow_wait_times_out_and_context_survives(torch):
    from paper_2002_01935_gb300 import binding
    s = torch.cuda.current_stream().cuda_stream
    assert binding.tn_selftest_flow_timeout(s) == binding.TN_ETIMEOUT
    # the context still runs contractions correctly
    net = inputs.random_ising(30, seed=5)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    ts = [torch.from_numpy(np.array(t, order="C")).float().cuda() for t in net.tensors]
    tnw = binding.TensorNetwork(net.labels, net.dims, net.open, ts, complex_=False)
    try:
        m, e = tnw.contract(pairs, [], "fp32")
        torch.cuda.synchronize()
        lz = math.log(float(m.cpu())) + int(e.cpu()) * math.log(2)
    finally:
        tnw.close()
    mo, eo = tree.contract_net(net, pairs)
    assert abs(math.expm1(lz - (math.log(float(mo)) + eo * math.log(2)))) <= 1e-5
