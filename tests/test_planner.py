"""Host planner and cost model against the paper's definitions and numbers."""
import math
import os

import numpy as np
import pytest

from paper_2002_01935_gb300 import inputs, planner

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_table_benchmark_flop_convention():
    """Tab. benchmark: efficiency = 8 C_s / time / 3.031 TFLOP/s, i.e. a
    complex contraction costs 8 C FLOPs (Sec. 2).  Every printed row must
    reproduce through the cost model's FLOP count."""
    rows = []
    with open(os.path.join(GOLDEN, "tab_benchmark.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, t, cs, dlog, eff = [x.strip() for x in line.split("|")]
            rows.append((name, float(t), float(cs), int(dlog), float(eff)))
    assert len(rows) == 16
    for name, t, cs, dlog, eff in rows:
        info = planner.TreeInfo(0, [], [], 0.0, cs / 2 ** dlog, 2 ** dlog, ())
        got = info.flops(is_complex=True) / t / 3.031e12 * 100
        assert abs(got - eff) <= 0.01 * eff + 0.05, name
        assert info.flops(is_complex=False) == pytest.approx(info.flops(True) / 4)


def test_matrix_chain_width_and_cost():
    """A(i,j) B(j,k) C(k,l) with dims 2,4,8,16: Eqs. edgecon and vertexcon."""
    labels = [[0, 1], [1, 2], [2, 3]]
    dims = {0: 2, 1: 4, 2: 8, 3: 16}
    opn = [0, 3]
    info = planner.tree_info(labels, dims, [(0, 1), (3, 2)], opn)
    # (AB): union {i,j,k} -> 2*4*8 = 64 ; ((AB)C): union {i,k,l} -> 2*8*16 = 256
    assert info.C == 64 + 256
    # widths: leaves 8, 32, 128; AB -> {i,k} 16; root {i,l} 32
    assert info.W == math.log2(128)
    info2 = planner.tree_info(labels, dims, [(1, 2), (0, 3)], opn)
    # (BC): {j,k,l} -> 512 ; A(BC): {i,j,l} -> 128
    assert info2.C == 512 + 128


def test_incidence_is_symmetric_difference_on_graphs():
    """Without open labels or hyperedges, the generalised incidence is
    s_l (+) s_r of Eq. incidence."""
    net = inputs.random_ising(30, seed=1)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    sets = planner.node_labels(net.labels, pairs)
    for k, (a, b) in enumerate(pairs):
        assert sets[net.n_tensors + k] == sets[a] ^ sets[b]


def test_incidence_keeps_hyperedges_and_open_labels():
    # label 0 shared by three tensors, label 5 open
    labels = [[0, 1], [0, 2], [0, 5], [1, 2]]
    sets = planner.node_labels(labels, [(0, 1), (4, 2), (5, 3)], open_labels=[5])
    assert sets[4] == {0, 1, 2}        # hyperedge 0 still used by tensor 2
    assert sets[5] == {1, 2, 5}        # 0 fully contracted, 5 open
    assert sets[6] == {5}


def test_greedy_tree_valid_and_deterministic():
    net = inputs.circuit_network(inputs.random_circuit(3, 3, 6, 0))
    p1 = planner.greedy_tree(net.labels, net.dims, net.open)
    p2 = planner.greedy_tree(net.labels, net.dims, net.open)
    assert p1 == p2
    planner.validate_tree(net.n_tensors, p1)
    # disconnected network: outer products join the components
    p = planner.greedy_tree([[0], [0], [1], [1]], {0: 2, 1: 2})
    planner.validate_tree(4, p)


def test_greedy_first_step_minimises_memory_change():
    """alpha = 1: the first pair chosen minimises size(k) - size(i) - size(j)."""
    labels = [[0, 1, 2], [2, 3], [3, 4], [0, 1, 4, 5]]
    dims = {l: 2 for l in range(6)}
    pairs = planner.greedy_tree(labels, dims, open_labels=[5])
    # candidate costs: (0,1): 16-8-4=4 ; (1,2): 4-4-4=-4 ; (0,3): 8-8-16=-16 ; (2,3): 16-4-16=-4
    assert pairs[0] == (0, 3)


def test_validate_tree_rejects_bad_trees():
    with pytest.raises(ValueError):
        planner.validate_tree(3, [(0, 1)])
    with pytest.raises(ValueError):
        planner.validate_tree(3, [(0, 1), (1, 3)])
    with pytest.raises(ValueError):
        planner.validate_tree(3, [(0, 4), (1, 2)])


def test_slicing_reaches_target_and_raises_cost():
    """Sec. 4.7.1: W_s <= target, and C_s = d_sliced C_sliced >= C."""
    circ = inputs.random_circuit(4, 4, 8, 0)
    net = inputs.circuit_network(circ)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    base = planner.tree_info(net.labels, net.dims, pairs, net.open)
    for target in (base.W - 1, base.W - 3):
        sl = planner.slice_greedy(net.labels, net.dims, pairs, net.open, target)
        info = planner.tree_info(net.labels, net.dims, pairs, net.open, sl)
        assert info.W <= target
        assert info.d_sliced == 2 ** len(sl)
        assert info.C_s >= base.C * (1 - 1e-12)
        assert not set(sl) & set(net.open)


def test_sliced_cost_formula():
    """Removing label e divides 2^vc by w(e) at every node whose s_l u s_r
    holds e (Eq. vertexcon); C_s multiplies back by d_sliced."""
    net = inputs.random_ising(20, seed=3)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    base = planner.tree_info(net.labels, net.dims, pairs, net.open)
    e = net.labels[0][0]
    info = planner.tree_info(net.labels, net.dims, pairs, net.open, [e])
    expect = 0.0
    for k, (a, b) in enumerate(pairs):
        u = base.sets[a] | base.sets[b]
        expect += 2.0 ** base.vc[k] / (2.0 if e in u else 1.0)
    assert info.C == pytest.approx(expect)
    assert info.C_s == pytest.approx(2 * expect)


def test_hyper_greedy_is_seeded_valid_and_no_worse_than_greedy():
    """Hyper-Greedy (Sec. 3.4): the same seed gives the same tree; the tree
    is valid, never costlier than the plain greedy tree it starts from, and
    gives the network's value (tree independence, oracle)."""
    from oracle import tree
    circ = inputs.random_circuit(3, 3, 6, seed=2)
    net = inputs.circuit_network(circ, inputs.random_bitstrings(9, 1, seed=7)[0])
    p1, s1, i1 = planner.hyper_greedy(net.labels, net.dims, net.open, trials=8, seed=5)
    p2, s2, i2 = planner.hyper_greedy(net.labels, net.dims, net.open, trials=8, seed=5)
    assert p1 == p2 and s1 == s2 and s1 == []
    planner.validate_tree(net.n_tensors, p1)
    g = planner.greedy_tree(net.labels, net.dims, net.open)
    assert i1.C <= planner.tree_info(net.labels, net.dims, g, net.open).C
    v_h = complex(tree.value(net.tensors, net.labels, net.dims, net.open, p1))
    v_g = complex(tree.value(net.tensors, net.labels, net.dims, net.open, g))
    assert abs(v_h - v_g) <= 1e-12 * abs(v_g)


def test_hyper_greedy_with_slicing_meets_the_width_target():
    net = inputs.random_ising(60, seed=3)
    g = planner.greedy_tree(net.labels, net.dims, net.open)
    target = planner.tree_info(net.labels, net.dims, g, net.open).W - 4
    pairs, sliced, info = planner.hyper_greedy(net.labels, net.dims, net.open, trials=6, seed=1,
                                               target_width=target)
    assert info.W <= target + 1e-9 and len(sliced) > 0
    # the reported cost is the sliced cost of that tree and slicing
    again = planner.tree_info(net.labels, net.dims, pairs, net.open, sliced)
    assert again.C_s == info.C_s and again.d_sliced == info.d_sliced


def test_randomised_slicer_repeats_never_worse_and_seeded():
    net = inputs.random_ising(60, seed=8)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    target = planner.tree_info(net.labels, net.dims, pairs, net.open).W - 5
    g = planner.slice_greedy(net.labels, net.dims, pairs, net.open, target)
    r1 = planner.slice_repeats(net.labels, net.dims, pairs, net.open, target, repeats=6, seed=3)
    r2 = planner.slice_repeats(net.labels, net.dims, pairs, net.open, target, repeats=6, seed=3)
    assert r1 == r2
    i_g = planner.tree_info(net.labels, net.dims, pairs, net.open, g)
    i_r = planner.tree_info(net.labels, net.dims, pairs, net.open, r1)
    assert i_r.W <= target + 1e-9 and i_r.C_s <= i_g.C_s
    # slicing never changes the value (oracle), whichever labels were chosen
    from oracle import tree
    m1, e1 = tree.contract_net(net, pairs, g)
    m2, e2 = tree.contract_net(net, pairs, r1)
    assert abs(math.log(float(m1)) + e1 * math.log(2) - math.log(float(m2)) - e2 * math.log(2)) < 1e-12
    p3, s3, i3 = planner.hyper_greedy(net.labels, net.dims, net.open, trials=3, seed=2,
                                      target_width=target, slicer_repeats=3)
    assert i3.W <= target + 1e-9


def test_tree_files_round_trip_and_refuse_other_structures(tmp_path):
    """A saved tree loads back unchanged for a network of the same structure
    (other tensor entries: another bitstring), and is refused for another
    structure, a broken tree or bad sliced labels."""
    import json
    circ = inputs.random_circuit(3, 3, 6, seed=3)
    a = inputs.circuit_network(circ, [0] * 9)
    b = inputs.circuit_network(circ, [1] * 9)  # same structure, other entries
    pairs = planner.greedy_tree(a.labels, a.dims, a.open)
    info = planner.tree_info(a.labels, a.dims, pairs, a.open)
    sliced = planner.slice_greedy(a.labels, a.dims, pairs, a.open, info.W - 1)
    path = str(tmp_path / "tree.json")
    planner.save_tree(path, a.labels, a.dims, a.open, pairs, sliced)
    got_pairs, got_sliced = planner.load_tree(path, b.labels, b.dims, b.open)
    assert got_pairs == [tuple(p) for p in pairs] and got_sliced == list(sliced)
    doc = json.load(open(path))
    ref = planner.tree_info(a.labels, a.dims, pairs, a.open, sliced)
    assert doc["W_s"] == ref.W and doc["C_s"] == ref.C_s and doc["d_sliced"] == ref.d_sliced
    other = inputs.circuit_network(inputs.random_circuit(3, 3, 7, seed=3), [0] * 9)
    with pytest.raises(ValueError):
        planner.load_tree(path, other.labels, other.dims, other.open)
    with pytest.raises(ValueError):  # the same leaves with an open label is another structure
        planner.load_tree(path, a.labels, a.dims, [a.labels[-1][0]])
    for key, bad in (("pairs", doc["pairs"][:-1]), ("sliced", [doc["sliced"][0]] * 2 if doc["sliced"] else [10 ** 9]),
                     ("format", 99)):
        broken = dict(doc, **{key: bad})
        json.dump(broken, open(path, "w"))
        with pytest.raises(ValueError):
            planner.load_tree(path, a.labels, a.dims, a.open)


@pytest.mark.parametrize("seed", range(30))
def test_slicing_never_widens_and_never_saves_work(seed):
    """Sec. 4.7.1 on random networks, trees and sliced label sets: W_s <= W
    and C_s = d_sliced * C(sliced tree) >= C, with equality of the costs
    exactly when every contraction's label union holds every sliced label
    of size > 1."""
    rng = np.random.default_rng(seed)
    net = inputs.random_network(int(rng.integers(2, 9)), int(rng.integers(2, 14)), 31000 + seed,
                                n_open=int(rng.integers(0, 3)), max_dim=3)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    base = planner.tree_info(net.labels, net.dims, pairs, net.open)
    summed = [l for l in sorted(net.dims) if l not in net.open]
    if not summed:
        pytest.skip("no summed label")
    k = int(rng.integers(1, min(3, len(summed)) + 1))
    sliced = [int(x) for x in rng.choice(summed, size=k, replace=False)]
    s = planner.tree_info(net.labels, net.dims, pairs, net.open, sliced)
    assert s.W <= base.W + 1e-12
    assert s.C_s >= base.C * (1 - 1e-12)
    n = net.n_tensors
    sets = planner.node_labels(net.labels, pairs, net.open)
    unions = []
    for a, b in pairs:
        unions.append(set(sets[a]) | set(sets[b]))
    every = all(l in u or net.dims[l] == 1 for u in unions for l in sliced)  # size-1 labels change nothing
    assert (abs(s.C_s - base.C) <= 1e-9 * base.C) == every
