"""The C-ABI library loads, exports every declared symbol, and its host-side
planning (validation, Eqs. edgecon/vertexcon) agrees with the planner.
No device work: these run without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2002_01935_gb300 import build
    build.build()
    from paper_2002_01935_gb300 import binding
    return binding


def declared_functions():
    src = open(os.path.join(ROOT, "include", "tn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tn_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "tn_contract" in names and "tn_create" in names and "tn_contract_grad" in names
    so = ctypes.CDLL(lib.LIB_PATH)
    for name in names:
        assert hasattr(so, name), name
    assert set(names) <= set(lib.EXPORTS)


def test_version(lib):
    assert "sm_103a" in lib.tn_version()


@pytest.mark.parametrize("case", ["repeat", "unknown", "open_missing", "dim0", "unused"])
def test_create_rejects_malformed_networks(lib, case):
    dims = {0: 2, 1: 2}
    labels = [[0, 1], [1]]
    opn = []
    if case == "repeat":
        labels = [[0, 0]]
        dims = {0: 2}
    elif case == "unknown":
        labels = [[0, 7]]
    elif case == "open_missing":
        dims = {0: 2, 1: 2, 5: 2}
        labels = [[0, 1], [1, 5]]
        opn = [9]
    elif case == "dim0":
        dims = {0: 0, 1: 2}
    elif case == "unused":
        dims = {0: 2, 1: 2, 3: 2}
    with pytest.raises(lib.TNError) as e:
        lib.tn_create(lib.TN_C64, labels, dims, opn)
    assert e.value.status == lib.TN_EINVAL
    assert lib.tn_last_error()


def test_tensors_beyond_the_size_limit_are_refused(lib):
    """Entry counts are formed in int64: a leaf or an intermediate of more
    than 2^40 entries is refused on the host (TN_EUNSUPPORTED) instead of
    overflowing; a leaf of exactly 2^40 entries is accepted."""
    big = {i: 2 for i in range(41)}
    with pytest.raises(lib.TNError) as e:
        lib.tn_create(lib.TN_C64, [list(range(41))], big, [])
    assert e.value.status == lib.TN_EUNSUPPORTED
    wide = {i: 4 for i in range(21)}  # 4^21 = 2^42
    with pytest.raises(lib.TNError) as e:
        lib.tn_create(lib.TN_C64, [list(range(21))], wide, [])
    assert e.value.status == lib.TN_EUNSUPPORTED
    h = lib.tn_create(lib.TN_C64, [list(range(40))], {i: 2 for i in range(40)}, [])
    lib.tn_destroy(h)
    # two leaves of 2^21 entries whose outer product (all labels open) has 2^42
    dims = {i: 2 for i in range(42)}
    h = lib.tn_create(lib.TN_C64, [list(range(21)), list(range(21, 42))], dims, list(range(42)))
    try:
        with pytest.raises(lib.TNError) as e:
            lib.tn_plan_info(h, [(0, 1)], [])
        assert e.value.status == lib.TN_EUNSUPPORTED
        assert "2^40" in lib.tn_last_error()
        # sliced down to 2^40 it plans
        h2 = lib.tn_create(lib.TN_C64, [list(range(21)), list(range(21, 42)), [0], [21]], dims,
                           list(range(1, 21)) + list(range(22, 42)))
        try:
            info = lib.tn_plan_info(h2, [(0, 2), (1, 3), (4, 5)], [0, 21])
            assert info["W"] == 40
        finally:
            lib.tn_destroy(h2)
    finally:
        lib.tn_destroy(h)


@pytest.mark.parametrize("pairs", [[(0, 1)], [(0, 1), (1, 3)], [(0, 4), (1, 2)], [(0, 0), (1, 2)]])
def test_malformed_trees_are_rejected(lib, pairs):
    h = lib.tn_create(lib.TN_C64, [[0], [0, 1], [1]], {0: 2, 1: 2}, [])
    try:
        with pytest.raises(lib.TNError) as e:
            lib.tn_plan_info(h, pairs, [])
        assert e.value.status == lib.TN_EINVAL
    finally:
        lib.tn_destroy(h)


def test_sliced_open_label_is_rejected(lib):
    h = lib.tn_create(lib.TN_C64, [[0, 1], [1]], {0: 2, 1: 2}, [0])
    try:
        with pytest.raises(lib.TNError):
            lib.tn_plan_info(h, [(0, 1)], [0])
        with pytest.raises(lib.TNError):
            lib.tn_plan_info(h, [(0, 1)], [42])
    finally:
        lib.tn_destroy(h)


@pytest.mark.parametrize("which", ["circuit", "ising", "random"])
def test_plan_costs_match_planner(lib, which):
    """W_s, C and FLOPs of the library's node plan equal the Python cost
    model (Eqs. edgecon, vertexcon; FLOPs 8C/2C) for the same tree."""
    from paper_2002_01935_gb300 import inputs, planner
    if which == "circuit":
        net = inputs.circuit_network(inputs.random_circuit(4, 4, 8, 0),
                                     inputs.random_bitstrings(16, 1, 1000)[0])
    elif which == "ising":
        net = inputs.random_ising(60, 2)
    else:
        net = inputs.random_network(9, 14, 3, n_open=2, max_dim=3)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    for target in (None, 0):
        sliced = []
        if target is not None:
            base = planner.tree_info(net.labels, net.dims, pairs, net.open)
            sliced = planner.slice_greedy(net.labels, net.dims, pairs, net.open, base.W - 2)
        ref = planner.tree_info(net.labels, net.dims, pairs, net.open, sliced)
        h = lib.tn_create(lib.TN_C64 if net.is_complex else lib.TN_R32, net.labels, net.dims,
                          net.open)
        try:
            info = lib.tn_plan_info(h, pairs, sliced)
        finally:
            lib.tn_destroy(h)
        assert info["W"] == pytest.approx(ref.W)
        assert info["C"] == pytest.approx(ref.C, rel=1e-12)
        assert info["d_sliced"] == ref.d_sliced
        assert info["flops"] == pytest.approx(ref.flops(net.is_complex), rel=1e-12)
        assert info["ws_bytes"] > 0


def _steps(lib, net, pairs, sliced=(), mode="fp32"):
    h = lib.TensorNetwork(net.labels, net.dims, net.open, None, complex_=net.is_complex)
    try:
        return h.plan_steps(pairs, sliced, mode), h.plan_info(pairs, sliced, mode)
    finally:
        h.close()


def test_launch_schedule_covers_every_node_once_in_dependency_order(lib):
    """Host plan only: every tree node is in exactly one launch step, and a
    node's children run in an earlier step or earlier in the same (dataflow)
    step; consecutive wave levels are merged into one dataflow step."""
    from paper_2002_01935_gb300 import inputs, planner
    for net in (inputs.random_ising(60, seed=2),
                inputs.circuit_network(inputs.random_circuit(4, 4, 8, seed=0),
                                       inputs.random_bitstrings(16, 1, seed=1000)[0])):
        pairs = planner.greedy_tree(net.labels, net.dims, net.open)
        steps, info = _steps(lib, net, pairs)
        n = net.n_tensors
        seen = {}
        for s, st in enumerate(steps):
            for pos, k in enumerate(st["nodes"]):
                assert k not in seen
                seen[k] = (s, pos)
        assert sorted(seen) == list(range(len(pairs)))
        for k, (a, b) in enumerate(pairs):
            for c in (a, b):
                if c >= n:
                    assert seen[c - n] < seen[k], (k, c - n)
        # no two wave steps in a row: they would have been merged
        for s0, s1 in zip(steps, steps[1:]):
            assert not (s0["wave"] and s1["wave"])
        assert sum(s["launches"] for s in steps) >= len(steps)


def test_wave_steps_hold_only_small_nodes(lib):
    """Host plan only: a node runs inside a wave launch only when it is small
    (at most 2^16 outputs, 2^22 multiply-adds, 2^14 summed entries per
    output); the largest nodes of these trees run alone."""
    from paper_2002_01935_gb300 import inputs, planner
    for net in (inputs.random_ising(100, seed=0),
                inputs.circuit_network(inputs.random_circuit(5, 4, 12, seed=0),
                                       inputs.random_bitstrings(20, 1, seed=1000)[0])):
        pairs = planner.greedy_tree(net.labels, net.dims, net.open)
        info = planner.tree_info(net.labels, net.dims, pairs, net.open)
        steps, _ = _steps(lib, net, pairs)
        n = net.n_tensors
        in_wave = {k for st in steps if st["wave"] for k in st["nodes"]}
        for k in in_wave:
            size = len(info.sets[n + k])          # log2 of the outputs (all dims 2)
            vc = info.vc[k]                       # log2 of the multiply-adds
            assert size <= 16 and vc <= 22 and vc - size <= 14, (k, size, vc)
        biggest = max(range(len(pairs)), key=lambda k: info.vc[k])
        assert biggest not in in_wave


def _gemm_node(mb, nb, kb, cplx):
    from paper_2002_01935_gb300 import inputs
    lab = 0
    ml = list(range(lab, lab + mb)); lab += mb
    nl = list(range(lab, lab + nb)); lab += nb
    kl = list(range(lab, lab + kb)); lab += kb
    dims = {l: 2 for l in range(lab)}
    la, lb = kl[::2] + ml + kl[1::2], nl + kl
    z = lambda labels: np.zeros([2] * len(labels), dtype=np.complex128 if cplx else np.float64)
    return inputs.Network([z(la), z(lb)], [la, lb], dims, ml + nl)


@pytest.mark.parametrize("mb,nb,kb,cplx,tc", [
    (8, 8, 6, True, True), (5, 8, 6, True, True), (8, 5, 6, True, True),   # 32 complex columns: padded tile
    (4, 8, 6, True, False), (8, 4, 6, True, False),                        # 16 complex columns: CUDA cores
    (6, 6, 6, True, False),                                                # no side with 128 rows
    (5, 8, 3, True, False),                                                # K = 8 < 16
    (8, 7, 6, False, True), (8, 6, 6, False, False), (6, 8, 6, False, False)])  # real: 128 x 128 needed
def test_tensor_core_choice(lib, mb, nb, kb, cplx, tc):
    """Host plan only: a single GEMM node goes to the tensor cores in a
    reduced-precision mode exactly when it has K >= 16, >= 128 accumulator
    rows on its larger side and >= 128 real columns (a complex node's 32
    complex columns expand to 64 real ones, which fill half of a padded
    128-column tile); never in the FP32 mode."""
    net = _gemm_node(mb, nb, kb, cplx)
    for mode in ("fp16_split", "tf32_split", "bf16_split", "tf32_3m"):
        steps, info = _steps(lib, net, [(0, 1)], (), mode)
        assert [s["kind"] for s in steps] == [2 if tc else 1], (mode, steps)
        assert info["n_tensor_core"] == (1 if tc else 0)
    steps, info = _steps(lib, net, [(0, 1)], (), "fp32")
    assert [s["kind"] for s in steps] == [1] and info["n_tensor_core"] == 0


def _random_tree(n, rng):
    """A uniformly shuffled valid SSA tree: any two live ids are joined (so
    outer products of unconnected parts occur too)."""
    live = list(range(n))
    pairs = []
    for k in range(n - 1):
        i, j = sorted(rng.choice(len(live), size=2, replace=False))
        a, b = live[i], live[j]
        pairs.append((int(a), int(b)))
        live = [x for x in live if x not in (a, b)] + [n + k]
    return pairs


@pytest.mark.parametrize("seed", range(60))
def test_random_plans_match_the_cost_model_and_schedule_every_node(lib, seed):
    """Host plan only, on random networks (hyperedges, open and summed-only
    labels, sizes 1..4, real and complex), random trees and random sliced
    labels, in every mode: the library's W_s, C, d_sliced and FLOPs equal
    the Python cost model's, and the launch steps hold every node once, each
    after its children."""
    from paper_2002_01935_gb300 import inputs, planner
    rng = np.random.default_rng(seed)
    net = inputs.random_network(int(rng.integers(1, 10)), int(rng.integers(1, 16)), 4000 + seed,
                                n_open=int(rng.integers(0, 3)), max_dim=4)
    cplx = bool(seed % 2)
    tensors, labels = list(net.tensors), [list(l) for l in net.labels]
    if not cplx:
        tensors = [np.real(t) for t in tensors]
    if seed % 5 == 4:  # a scalar leaf
        tensors.append(np.array(1.5))
        labels.append([])
    net = inputs.Network(tensors, labels, net.dims, net.open)
    pairs = _random_tree(net.n_tensors, rng) if seed % 3 else planner.greedy_tree(net.labels, net.dims, net.open)
    summed = [l for l in sorted(net.dims) if l not in net.open]
    k = int(rng.integers(0, min(3, len(summed)) + 1))
    sliced = [int(x) for x in rng.choice(summed, size=k, replace=False)] if k else []
    ref = planner.tree_info(net.labels, net.dims, pairs, net.open, sliced)
    n = net.n_tensors
    for mode in ("fp32", "tf32_split", "tf32_3m", "bf16_split"):
        steps, info = _steps(lib, net, pairs, sliced, mode)
        assert info["W"] == pytest.approx(ref.W)
        assert info["C"] == pytest.approx(ref.C, rel=1e-12)
        assert info["d_sliced"] == ref.d_sliced
        assert info["flops"] == pytest.approx(ref.flops(cplx), rel=1e-12)
        seen = {}
        for s, st in enumerate(steps):
            for pos, node in enumerate(st["nodes"]):
                assert node not in seen
                seen[node] = (s, pos)
        assert sorted(seen) == list(range(max(n - 1, 1)))  # one leaf: one reduction node
        for node, (a, b) in enumerate(pairs):
            for c in (a, b):
                if c >= n:
                    assert seen[c - n] < seen[node]
