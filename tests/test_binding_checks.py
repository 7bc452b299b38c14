"""The binding's argument checks (no GPU needed: every case is refused
before any device call).

The library sees plain pointers, so the extents it reads and writes are
checked in the binding: caller gradient buffers, leaves read by several
copies, output buffers.  Undersized or malformed buffers raise TNError
(TN_EINVAL) or TypeError instead of being accessed out of bounds.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2002_01935_gb300 import binding, inputs, planner  # noqa: E402


@pytest.fixture()
def tnw():
    net = inputs.random_network(5, 7, 3, n_open=1, max_dim=2)
    ts = [torch.from_numpy(np.array(t, order="C")).to(torch.complex64) for t in net.tensors]
    h = binding.TensorNetwork(net.labels, net.dims, net.open, ts, complex_=True)
    h.test_pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    h.test_leaves = ts
    yield h
    h.close()


def _einval(fn):
    with pytest.raises(binding.TNError) as e:
        fn()
    assert e.value.status == binding.TN_EINVAL


def test_gradient_buffers_are_checked(tnw):
    ts = tnw.test_leaves
    _einval(lambda: tnw._check_grads([None] * (len(ts) - 1)))  # one entry per leaf
    _einval(lambda: tnw._check_grads([torch.empty_like(t) for t in ts]))  # host memory
    with pytest.raises(TypeError):
        tnw._check_grads([torch.empty(t.shape, dtype=torch.complex128) for t in ts])
    tnw._check_grads([None] * len(ts))  # all skipped: nothing to check


def test_instance_extents_are_checked(tnw):
    ts = tnw.test_leaves
    n = len(ts)
    tnw._check_strides(4, [0] * n)  # shared leaves: one copy's extent
    tnw._check_strides(1, [ts[0].numel()] + [0] * (n - 1))  # one copy reads one leaf
    _einval(lambda: tnw._check_strides(2, [ts[0].numel()] + [0] * (n - 1)))  # second copy past the end
    _einval(lambda: tnw._check_strides(2, [-1] + [0] * (n - 1)))
    _einval(lambda: tnw._check_strides(2, [0] * (n - 1)))
    # a stacked leaf holds exactly what its copies read
    stacked = list(ts)
    stacked[0] = torch.stack([ts[0]] * 3)
    tnw.set_tensors(stacked)
    tnw._check_strides(3, [ts[0].numel()] + [0] * (n - 1))
    _einval(lambda: tnw._check_strides(4, [ts[0].numel()] + [0] * (n - 1)))
    # instance gradients: varying leaves need every copy's extent
    with pytest.raises(binding.TNError):
        tnw.grad_instances(tnw.test_pairs, [], "fp32", 4, [ts[0].numel()] + [0] * (n - 1),
                           np.zeros((4,) + tnw.out_shape, dtype=np.complex128))


def test_output_buffers_are_checked(tnw):
    pairs = tnw.test_pairs
    ex = torch.empty((), dtype=torch.int64)
    n_out = int(np.prod(tnw.out_shape))
    _einval(lambda: tnw.contract(pairs, [], "fp32", out=torch.empty(n_out + 2, dtype=torch.complex128),
                                 out_exp=ex))
    with pytest.raises(TypeError):
        tnw.contract(pairs, [], "fp32", out=torch.empty(tnw.out_shape, dtype=torch.complex64), out_exp=ex)
    with pytest.raises(TypeError):
        tnw.contract(pairs, [], "fp32", out=torch.empty(tnw.out_shape, dtype=torch.complex128),
                     out_exp=torch.empty((), dtype=torch.int32))
    _einval(lambda: tnw.contract(pairs, [], "fp32", out=torch.empty(tnw.out_shape, dtype=torch.complex128),
                                 out_exp=torch.empty(2, dtype=torch.int64)))


def test_flattened_trees_follow_the_pair_list():
    """The flattened tree is reused only for an equal pair list: replacing
    a pair, lists of lists and non-list inputs all give the current pairs."""
    pairs = [(0, 1), (2, 3), (4, 5)]
    a = binding._tree(pairs)
    assert a.tolist() == [0, 1, 2, 3, 4, 5]
    assert binding._tree(pairs) is a  # unchanged: reused
    pairs[1] = (3, 2)
    assert binding._tree(pairs).tolist() == [0, 1, 3, 2, 4, 5]
    lol = [[0, 1], [2, 3]]
    b = binding._tree(lol)
    assert b.tolist() == [0, 1, 2, 3]
    assert binding._tree(lol) is b  # a list of lists is reused too
    lol[0][1] = 9
    assert binding._tree(lol).tolist() == [0, 9, 2, 3]
    assert binding._tree(np.array([[1, 0]])).tolist() == [1, 0]
    rows = list(np.array([[0, 1], [2, 3]]))  # a list of numpy rows
    assert binding._tree(rows).tolist() == [0, 1, 2, 3]
    rows[0] = np.array([1, 0])
    assert binding._tree(rows).tolist() == [1, 0, 2, 3]
    assert binding._tree([]).tolist() == [0]


def test_pair_lists_of_the_wrong_length_are_refused():
    """The library reads n_tensors - 1 pairs: shorter or longer lists are
    refused by the binding (a short one would be read past its end)."""
    h = binding.tn_create(binding.TN_C64, [[0], [0, 1], [1]], {0: 2, 1: 2}, [])
    try:
        for pairs in ([(0, 1)], [(0, 1), (2, 3), (4, 0)], []):
            _einval(lambda: binding.tn_plan_info(h, pairs, []))
        assert binding.tn_plan_info(h, [(0, 1), (2, 3)], [])["C"] > 0
    finally:
        binding.tn_destroy(h)
    one = binding.tn_create(binding.TN_C64, [[0]], {0: 2}, [0])
    try:
        _einval(lambda: binding.tn_plan_info(one, [(0, 0)], []))
        binding.tn_plan_info(one, [], [])
    finally:
        binding.tn_destroy(one)


def test_undersized_or_surplus_leaves_are_refused(tnw):
    ts = tnw.test_leaves
    v = max(range(len(ts)), key=lambda i: ts[i].numel())
    short = list(ts)
    short[v] = ts[v].reshape(-1)[:-1].contiguous()
    _einval(lambda: tnw.set_tensors(short))
    _einval(lambda: tnw.set_tensors(list(ts) + [ts[0]]))
    tnw.set_tensors(ts)  # the full leaves still attach
