"""Structure simplifications (Sec. 3.7) on the host: every rule keeps the
network's value (FP64 oracle) and its output axes, and does what the paper
describes on small hand-made cases."""
import numpy as np
import pytest

from oracle import tree
from paper_2002_01935_gb300 import inputs, planner, simplify


def _value(net):
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    m, e = tree.contract_net(net, pairs)
    return np.asarray(m) * 2.0 ** e


@pytest.mark.parametrize("case", ["circuit", "circuit_open", "ising", "random", "random_open"])
def test_simplification_keeps_the_value(case):
    if case == "circuit":
        net = inputs.circuit_network(inputs.random_circuit(3, 3, 6, seed=3),
                                     inputs.random_bitstrings(9, 1, seed=4)[0])
    elif case == "circuit_open":
        net = inputs.circuit_network(inputs.random_circuit(3, 3, 5, seed=5), [0] * 9, open_qubits=[7, 2])
    elif case == "ising":
        net = inputs.random_ising(24, seed=6)
    elif case == "random":
        net = inputs.random_network(9, 14, 31, n_open=0)
    else:
        net = inputs.random_network(9, 14, 32, n_open=2)
    s, done = simplify.simplify(net)
    assert s.open == net.open
    assert s.n_tensors <= net.n_tensors
    a, b = _value(net), _value(s)
    assert np.shape(a) == np.shape(b)
    assert np.max(np.abs(a - b)) <= 1e-12 * max(np.max(np.abs(a)), 1e-300)


def test_circuit_shrinks_and_ising_becomes_hyperedge_form():
    c = inputs.circuit_network(inputs.random_circuit(4, 4, 8, seed=0), inputs.random_bitstrings(16, 1, seed=1000)[0])
    s, done = simplify.simplify(c)
    assert s.n_tensors < c.n_tensors // 2 and done["rank"] > 0 and done["column"] > 0
    ising = inputs.random_ising(20, seed=1)
    s2, done2 = simplify.simplify(ising)
    # every COPY tensor reduced to its diagonal: each spin is one label in three edge matrices
    assert done2["diagonal"] == 2 * 20 and s2.n_tensors == 30
    assert all(len(ls) == 2 for ls in s2.labels)


def test_column_reduction_projects_the_label():
    t = np.array([[1.0, 0.0], [2.0, 0.0]])          # vanishes unless b == 0
    u = np.array([[3.0, 4.0], [5.0, 6.0]])           # labels (b, c)
    net = inputs.Network([t, u, np.array([1.0, 1.0]), np.array([1.0, 2.0])],
                         [[0, 1], [1, 2], [0], [2]], {0: 2, 1: 2, 2: 2}, [])
    w = simplify._Net(net, ())
    assert w.column(1e-12)
    assert 1 not in w.dims and w.l[1] == [2] and np.allclose(w.t[1], [3.0, 4.0])


def test_diagonal_reduction_makes_a_hyperedge():
    d = np.diag([2.0, -1.0])                          # labels (a, b): zero off the diagonal
    net = inputs.Network([d, np.array([1.0, 3.0]), np.array([5.0, 7.0])], [[0, 1], [0], [1]],
                         {0: 2, 1: 2}, [])
    w = simplify._Net(net, ())
    assert w.diagonal(1e-12)
    assert 1 not in w.dims and w.l == [[0], [0], [0]]
    s, _ = simplify.simplify(net)
    assert np.isclose(float(_value(s)), 2.0 * 1 * 5 - 1.0 * 3 * 7)


def test_antidiagonal_gauging_then_diagonal():
    x = np.array([[0.0, 2.0], [3.0, 0.0]])           # vanishes unless a == 1 - b
    net = inputs.Network([x, np.array([1.0, 4.0]), np.array([2.0, 5.0])], [[0, 1], [0], [1]],
                         {0: 2, 1: 2}, [])
    w = simplify._Net(net, ())
    assert w.antidiagonal(1e-12) and w.diagonal(1e-12)
    s, done = simplify.simplify(net)
    assert np.isclose(float(_value(s)), float(_value(net)))


def test_frozen_leaves_are_kept_first_and_untouched():
    circ = inputs.random_circuit(3, 3, 4, seed=9)
    net = inputs.circuit_network(circ, [1, 0, 1, 1, 0, 0, 1, 0, 1])
    out_leaves = list(range(net.n_tensors - 9, net.n_tensors))
    s, _ = simplify.simplify(net, frozen=out_leaves)
    for i, v in enumerate(out_leaves):
        assert np.array_equal(s.tensors[i], net.tensors[v]) and s.labels[i] == net.labels[v]
    assert np.max(np.abs(_value(s) - _value(net))) <= 1e-12 * np.max(np.abs(_value(net)))


def test_split_simplification_factors_a_low_rank_tensor():
    rng = np.random.default_rng(5)
    a, b = rng.standard_normal((2, 2)), rng.standard_normal((2, 2, 2))
    t = np.einsum("ij,klm->ijklm", a, b)             # rank 1 across {i, j} | {k, l, m}
    others = [rng.standard_normal(2) for _ in range(5)]
    net = inputs.Network([t] + others, [[0, 1, 2, 3, 4], [0], [1], [2], [3], [4]],
                         {l: 2 for l in range(5)}, [])
    w = simplify._Net(net, ())
    assert w.split(1e-12)
    assert sorted(len(x) for x in w.l[:1] + w.l[-1:]) == [3, 4]  # {i, j, new} and {new, k, l, m}
    s, done = simplify.simplify(net, frozen=[1, 2, 3, 4, 5])  # the vectors stay, t is split
    assert done["split"] >= 1 and s.n_tensors == net.n_tensors + 1
    assert np.isclose(float(_value(s)), float(_value(net)), rtol=1e-12)


def test_simplify_terminates_with_split_on_random_networks():
    for seed in range(5):
        net = inputs.random_network(8, 12, 200 + seed, n_open=1)
        s, done = simplify.simplify(net, max_rounds=200)
        a, b = _value(net), _value(s)
        assert np.max(np.abs(a - b)) <= 1e-11 * np.max(np.abs(a))


def _planted(seed):
    """A random network (hyperedges, open labels, sizes 1..3) whose tensors
    carry planted structure for every rule: diagonal or antidiagonal pairs
    of axes, an axis supported on one value, low rank across a split."""
    rng = np.random.default_rng(seed)
    net = inputs.random_network(8, 12, 700 + seed, n_open=int(seed % 3), max_dim=3)
    tensors = [np.array(t, dtype=complex) for t in net.tensors]
    for v, t in enumerate(tensors):
        ls = net.labels[v]
        kind = rng.integers(0, 5)
        if kind in (0, 1) and len(ls) >= 2:
            pairs = [(x, y) for x in range(len(ls)) for y in range(x + 1, len(ls))
                     if net.dims[ls[x]] == net.dims[ls[y]] > 1]
            if pairs:
                x, y = pairs[rng.integers(len(pairs))]
                d = net.dims[ls[x]]
                i = np.arange(d)
                keep = (i[:, None] == i[None, :]) if kind == 0 else (i[:, None] == d - 1 - i[None, :])
                shape = [d if a in (x, y) else 1 for a in range(t.ndim)]
                tensors[v] = t * keep.reshape(shape)
        elif kind == 2 and len(ls) >= 1:
            x = int(rng.integers(len(ls)))
            d = net.dims[ls[x]]
            if d > 1:
                mask = np.zeros(d)
                mask[rng.integers(d)] = 1.0
                shape = [d if a == x else 1 for a in range(t.ndim)]
                tensors[v] = t * mask.reshape(shape)
        elif kind == 3 and len(ls) >= 3:
            k = len(ls) // 2
            left = [net.dims[l] for l in ls[:k]]
            right = [net.dims[l] for l in ls[k:]]
            r = 1 + int(rng.integers(2))
            u = rng.standard_normal((int(np.prod(left)), r)) + 1j * rng.standard_normal((int(np.prod(left)), r))
            w = rng.standard_normal((r, int(np.prod(right)))) + 1j * rng.standard_normal((r, int(np.prod(right))))
            tensors[v] = (u @ w).reshape(left + right)
    return inputs.Network(tensors, net.labels, net.dims, net.open)


def _error_scale(net):
    """Rounding scale of the network's value: its value on |T|, or, for a
    structurally zero network (that value 0), the bound prod_v max|T_v| times
    the number of summed assignments."""
    absnet = inputs.Network([np.abs(t) for t in net.tensors], net.labels, net.dims, net.open)
    scale = float(np.max(np.abs(_value(absnet))))
    if scale > 0:
        return scale
    bound = float(np.prod([np.max(np.abs(t)) if np.size(t) else 0.0 for t in net.tensors]))
    summed = [l for l in net.dims if l not in net.open]
    return bound * float(np.prod([net.dims[l] for l in summed]))


@pytest.mark.parametrize("seed", range(48))
def test_planted_structure_is_simplified_without_changing_the_value(seed):
    """Odd seeds freeze a random subset of the leaves: they come first in the
    result, unchanged, and the value still holds."""
    net = _planted(seed)
    frozen = []
    if seed % 2:
        rng = np.random.default_rng(seed + 5)
        frozen = sorted(int(x) for x in rng.choice(net.n_tensors, size=int(rng.integers(1, net.n_tensors)),
                                                   replace=False))
    s, done = simplify.simplify(net, frozen=frozen)
    assert s.open == net.open
    for i, v in enumerate(frozen):
        assert s.labels[i] == list(net.labels[v]) and np.array_equal(s.tensors[i], net.tensors[v])
    assert all(len(set(ls)) == len(ls) for ls in s.labels)  # no label twice in a tensor
    a, b = _value(net), _value(s)
    assert np.shape(a) == np.shape(b)
    assert np.max(np.abs(a - b)) <= 1e-11 * max(_error_scale(net), 1e-300), done
