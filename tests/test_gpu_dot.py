"""Inner-product nodes (few outputs, long K) on the dot kernel against the
FP64 oracle: K from 2^9 (one short tile) to 2^13, one to 64 outputs, complex
and real, batch labels, and a sliced K label (the slice offset enters the
tile bases).  The K tiles are copied asynchronously into a stage ring, so a
mis-ordered wait, a wrong stage or a wrong tile base would show here.
"""
import numpy as np
import pytest

from oracle import tree
from paper_2002_01935_gb300 import inputs

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


def dot_net(mb, nb, kb, batch, cplx, seed):
    """C[b,m,n] = sum_k A[b,m,k] B[b,k,n], K labels spread through both
    operands' layouts in different orders."""
    rng = np.random.default_rng(seed)
    lab = 0
    bl = list(range(lab, lab + batch)); lab += batch
    ml = list(range(lab, lab + mb)); lab += mb
    nl = list(range(lab, lab + nb)); lab += nb
    kl = list(range(lab, lab + kb)); lab += kb
    dims = {l: 2 for l in range(lab)}
    la = kl[1::2] + ml + bl + kl[::2]
    lb = nl + kl[::-1] + bl
    def t(shape):
        x = rng.standard_normal(shape)
        return x + 1j * rng.standard_normal(shape) if cplx else x
    return inputs.Network([t([2] * len(la)), t([2] * len(lb))], [la, lb], dims, bl + ml + nl), kl


SHAPES = [(0, 0, 9, 0, True), (0, 0, 10, 0, True), (0, 0, 13, 0, True), (1, 1, 10, 0, True),
          (3, 3, 12, 0, True), (2, 4, 11, 1, True), (0, 0, 13, 0, False), (2, 3, 12, 1, False)]


# (0, 0, 9) sliced would leave K = 256, below the dot kernel's range
@pytest.mark.parametrize("shape,sliced", [(sh, False) for sh in SHAPES] + [(sh, True) for sh in SHAPES[1:]])
def test_dot_nodes(torch, shape, sliced):
    from paper_2002_01935_gb300 import binding
    mb, nb, kb, batch, cplx = shape
    net, kl = dot_net(mb, nb, kb, batch, cplx, seed=7 + sum(shape) + sliced)
    pairs = [(0, 1)]
    sl = [kl[3]] if sliced else []
    dt = torch.complex64 if cplx else torch.float32
    ts = [torch.from_numpy(np.array(x, order="C")).to(dt).contiguous().cuda() for x in net.tensors]
    tnw = binding.TensorNetwork(net.labels, net.dims, net.open, ts, complex_=cplx)
    try:
        steps = tnw.plan_steps(pairs, sl, "fp32")
        assert [s["cfg"] for s in steps] == [5]  # the dot kernel
        m, e = tnw.contract(pairs, sl, "fp32")
        torch.cuda.synchronize()
        got = m.cpu().numpy() * 2.0 ** int(e.cpu())
    finally:
        tnw.close()
    stored = net.as_stored()
    ref = tree.value(stored.tensors, stored.labels, stored.dims, stored.open, pairs)
    scale = tree.value([np.abs(x) for x in stored.tensors], stored.labels, stored.dims, stored.open, pairs)
    err = float(np.max(np.abs(np.asarray(got) - ref) / scale))
    assert err <= TOL, err
