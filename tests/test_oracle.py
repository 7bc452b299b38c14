"""Pins of the CPU FP64 oracle against values fixed by the mathematics.

Each check is independent of the tree executor's own code: the literal
nested sum of products (Sec. 4.7.1), dense state-vector simulation
(Eq. trans-amp), Ising enumeration and closed forms, and the invariants the
paper states (tree independence and slice sums, Sec. 4.7.1).
"""
import itertools
import math

import numpy as np
import pytest

from oracle import brute, gradient, ising, statevector, tree
from paper_2002_01935_gb300 import inputs, planner

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def random_tree(n, seed):
    rng = np.random.default_rng(seed)
    ids = list(range(n))
    pairs = []
    nxt = n
    while len(ids) > 1:
        i, j = sorted(rng.choice(len(ids), size=2, replace=False))
        a, b = ids[i], ids[j]
        pairs.append((a, b))
        ids = [x for k, x in enumerate(ids) if k not in (i, j)] + [nxt]
        nxt += 1
    return pairs


# --------------------------------------------------------------------------
# nested sum of products (Sec. 4.7.1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(24))
def test_tree_matches_nested_sum(seed):
    """Hyperedges, dangling (summed-only) labels, open labels, dims 1..3."""
    net = inputs.random_network(6 + seed % 4, 11 + seed % 5, seed, n_open=seed % 3,
                                complex_=seed % 2 == 0)
    ref = brute.nested_sum(net.tensors, net.labels, net.dims, net.open)
    # rounding bound: a few ulps of the sum of |products| (cancellation-free scale)
    scale = brute.nested_sum([np.abs(t) for t in net.tensors], net.labels, net.dims, net.open)
    for pairs in (planner.greedy_tree(net.labels, net.dims, net.open),
                  random_tree(net.n_tensors, seed)):
        got = tree.value(net.tensors, net.labels, net.dims, net.open, pairs)
        assert got.shape == ref.shape
        assert np.all(np.abs(got - ref) <= 1e-13 * np.abs(scale) + 1e-300)


def test_outer_product_and_single_tensor():
    rng = np.random.default_rng(5)
    a = rng.standard_normal((2, 3)) + 1j * rng.standard_normal((2, 3))
    b = rng.standard_normal(4) + 1j * rng.standard_normal(4)
    dims = {0: 2, 1: 3, 2: 4}
    got = tree.value([a, b], [[0, 1], [2]], dims, [2, 0, 1], [(0, 1)])
    assert rel(got, np.einsum("ij,k->kij", a, b)) < 1e-15
    # disconnected components joined by an outer product, then summed
    got = tree.value([a, b], [[0, 1], [2]], dims, [], [(1, 0)])
    assert rel(got, a.sum() * b.sum()) < 1e-14
    # a lone tensor with a summed label and an open one
    got = tree.value([a], [[0, 1]], dims, [1], [])
    assert rel(got, a.sum(axis=0)) < 1e-15


def test_open_label_order_is_respected():
    rng = np.random.default_rng(1)
    a = rng.standard_normal((2, 3, 4))
    b = rng.standard_normal((4, 5))
    dims = {0: 2, 1: 3, 2: 4, 3: 5}
    got = tree.value([a, b], [[0, 1, 2], [2, 3]], dims, [3, 0, 1], [(0, 1)])
    assert rel(got, np.einsum("ijk,kl->lij", a, b)) < 1e-14


@pytest.mark.parametrize("seed", range(8))
def test_slice_sum_equals_unsliced(seed):
    """Any subset of summed labels, including hyperedges (Sec. 4.7.1)."""
    net = inputs.random_network(8, 13, 100 + seed, n_open=seed % 2)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    full_m, full_e = tree.contract_net(net, pairs)
    full = full_m * 2.0 ** full_e
    summed = [l for l in sorted(net.dims) if l not in net.open]
    rng = np.random.default_rng(seed)
    sl = list(rng.choice(summed, size=min(3, len(summed)), replace=False))
    scale = brute.nested_sum([np.abs(t) for t in net.tensors], net.labels, net.dims, net.open)
    tol = 1e-13 * np.abs(scale) + 1e-300
    got = tree.value(net.tensors, net.labels, net.dims, net.open, pairs, sl)
    assert np.all(np.abs(got - full) <= tol)
    # the slice ids partition the sum
    d = int(np.prod([net.dims[l] for l in sl]))
    parts = sum(tree.value(net.tensors, net.labels, net.dims, net.open, pairs, sl,
                           slice_begin=s, slice_count=1) for s in range(d))
    assert np.all(np.abs(parts - full) <= tol)


def test_slice_selects_fixed_label_values():
    """Slice id s fixes the sliced labels to the mixed-radix digits of s."""
    rng = np.random.default_rng(3)
    a = rng.standard_normal((2, 3))
    b = rng.standard_normal((3, 2))
    dims = {0: 2, 1: 3, 2: 2}
    for s in range(3):
        got = tree.value([a, b], [[0, 1], [1, 2]], dims, [0, 2], [(0, 1)], [1],
                         slice_begin=s, slice_count=1)
        assert rel(got, np.outer(a[:, s], b[s, :])) < 1e-15


# --------------------------------------------------------------------------
# random circuits (Eq. trans-amp) against a dense state vector
# --------------------------------------------------------------------------

def test_gate_definitions():
    for name, g in (("sqrt_x", "X"), ("sqrt_y", "Y"), ("sqrt_w", "W")):
        m = inputs.gate_matrix(name)
        p = inputs._PAULI[g]
        assert np.allclose(m @ m, -1j * p, atol=1e-15)
        assert np.allclose(m.conj().T @ m, np.eye(2), atol=1e-15)
    f = inputs.fsim(math.pi / 2, 0.0)
    ket01 = np.zeros(4)
    ket01[1] = 1
    assert np.allclose(f @ ket01, -1j * np.eye(4)[2], atol=1e-15)
    f = inputs.fsim(0.3, 1.1)
    assert np.allclose(f.conj().T @ f, np.eye(4), atol=1e-15)


@pytest.mark.parametrize("shape", [(2, 2, 4), (3, 3, 6), (2, 4, 5)])
def test_circuit_amplitude_matches_state_vector(shape):
    r, c, t = shape
    circ = inputs.random_circuit(r, c, t, seed=7)
    psi = statevector.final_state(r * c, circ.gates)
    for bs in inputs.random_bitstrings(r * c, 3, seed=11):
        net = inputs.circuit_network(circ, bs)
        pairs = planner.greedy_tree(net.labels, net.dims, net.open)
        got = complex(tree.value(net.tensors, net.labels, net.dims, net.open, pairs))
        ref = complex(psi[tuple(bs)])
        assert abs(got - ref) <= 1e-12 * abs(ref)


def test_cfg0_amplitude_matches_state_vector():
    """4x4 grid, 8 cycles: the plain-method circuit workload."""
    circ = inputs.random_circuit(4, 4, 8, seed=0)
    bs = inputs.random_bitstrings(16, 1, seed=1000)[0]
    net = inputs.circuit_network(circ, bs)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    m, e = tree.contract_net(net, pairs)
    ref = statevector.amplitude(16, circ.gates, bs)
    assert abs(complex(m) * 2.0 ** e - ref) <= 1e-12 * abs(ref)


def test_open_outputs_give_normalised_state():
    """All 2^N amplitudes as one open tensor: sum |c_x|^2 = 1 and they equal
    the state vector entry by entry."""
    circ = inputs.random_circuit(3, 3, 5, seed=2)
    n = 9
    net = inputs.circuit_network(circ, open_qubits=list(range(n)))
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    amp = tree.value(net.tensors, net.labels, net.dims, net.open, pairs)
    assert amp.shape == (2,) * n
    assert abs(np.sum(np.abs(amp) ** 2) - 1.0) < 1e-13
    psi = statevector.final_state(n, circ.gates)
    assert rel(amp, psi) < 1e-13


def test_partially_open_outputs():
    circ = inputs.random_circuit(2, 3, 6, seed=4)
    bs = inputs.random_bitstrings(6, 1, seed=5)[0]
    opn = [4, 1]
    net = inputs.circuit_network(circ, bs, open_qubits=opn)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    amp = tree.value(net.tensors, net.labels, net.dims, net.open, pairs)
    psi = statevector.final_state(6, circ.gates)
    for x4, x1 in itertools.product(range(2), range(2)):
        idx = list(bs)
        idx[4], idx[1] = x4, x1
        assert abs(amp[x4, x1] - psi[tuple(idx)]) < 1e-13


def test_identity_fsim_factorises():
    """theta = phi = 0 makes fSim the identity: c_x is a product over qubits
    of <x_q| g_T ... g_1 |0>."""
    circ = inputs.random_circuit(2, 3, 6, seed=9)
    for g in circ.gates:
        if g.name == "fsim":
            g.matrix = inputs.fsim(0.0, 0.0)
    bs = inputs.random_bitstrings(6, 1, seed=3)[0]
    ref = 1.0 + 0j
    for q in range(6):
        v = np.array([1.0, 0.0], dtype=complex)
        for g in circ.gates:
            if g.qubits == (q,):
                v = g.matrix @ v
        ref *= v[bs[q]]
    net = inputs.circuit_network(circ, bs)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    got = complex(tree.value(net.tensors, net.labels, net.dims, net.open, pairs))
    assert abs(got - ref) < 1e-14


def test_tree_independence_circuit():
    circ = inputs.random_circuit(3, 3, 6, seed=1)
    bs = inputs.random_bitstrings(9, 1, seed=2)[0]
    net = inputs.circuit_network(circ, bs)
    vals = []
    for pairs in (planner.greedy_tree(net.labels, net.dims, net.open),
                  planner.greedy_tree(net.labels, net.dims, net.open, alpha=0.0),
                  planner.greedy_tree(net.labels, net.dims, net.open, tau=0.5, seed=3),
                  planner.left_deep_tree(net.n_tensors)):
        vals.append(complex(tree.value(net.tensors, net.labels, net.dims, net.open, pairs)))
    for v in vals[1:]:
        assert abs(v - vals[0]) <= 1e-12 * abs(vals[0])


# --------------------------------------------------------------------------
# Ising partition functions
# --------------------------------------------------------------------------

def log_z(net, pairs, sliced=()):
    m, e = tree.contract_net(net, pairs, sliced)
    return math.log(abs(float(m))) + e * math.log(2.0)


@pytest.mark.parametrize("n,seed", [(8, 0), (12, 1), (16, 2), (20, 3)])
def test_ising_matches_enumeration(n, seed):
    net = inputs.random_ising(n, seed)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    ref = ising.log_z_enumerate(n, net.meta["edges"], net.meta["J"], net.meta["beta"])
    assert abs(log_z(net, pairs) - ref) < 1e-12


@pytest.mark.parametrize("n,seed", [(8, 0), (12, 4), (16, 9)])
def test_ising_hyperedge_form_matches_enumeration(n, seed):
    """The hyperedge form (one label per spin, shared by the matrices of its
    three edges) gives the same Z as the enumeration and as the COPY form."""
    net = inputs.random_ising_hyper(n, seed)
    edges, J = net.meta["edges"], net.meta["J"]
    assert all(sum(l in ls for ls in net.labels) == 3 for l in net.dims)  # degree-3 hyperedges
    lz = log_z(net, planner.greedy_tree(net.labels, net.dims, net.open))
    assert abs(lz - ising.log_z_enumerate(n, edges, J, 0.3)) < 1e-12
    copy_form = inputs.random_ising(n, seed)
    assert abs(lz - log_z(copy_form, planner.greedy_tree(copy_form.labels, copy_form.dims,
                                                         copy_form.open))) < 1e-12


def _copy(rank):
    t = np.zeros((2,) * rank)
    t[(0,) * rank] = t[(1,) * rank] = 1.0
    return t


@pytest.mark.parametrize("n,seed", [(10, 5), (14, 6)])
def test_ising_copy_tensors_rewired(n, seed):
    """Sec. 3.5: a COPY tensor may be replaced by any connected network of
    COPY tensors over the same open labels without changing the value.
    Every vertex's rank-3 COPY tensor becomes a random connected COPY
    subgraph (a chain through two new labels, or a rank-3 tensor joined to a
    rank-2 one); Z stays that of the enumeration."""
    net = inputs.random_ising(n, seed)
    rng = np.random.default_rng(seed)
    tensors, labels = list(net.tensors[n:]), [list(l) for l in net.labels[n:]]
    nxt = max(net.dims) + 1
    for v in range(n):
        a, b, c = [net.labels[v][i] for i in rng.permutation(3)]
        if rng.random() < 0.5:  # chain a - x - b - y - c
            x, y = nxt, nxt + 1
            nxt += 2
            tensors += [_copy(2), _copy(3), _copy(2)]
            labels += [[a, x], [x, b, y], [y, c]]
        else:  # (a, b, x) joined to (x, c)
            x = nxt
            nxt += 1
            tensors += [_copy(3), _copy(2)]
            labels += [[a, b, x], [x, c]]
    dims = {l: 2 for ls in labels for l in ls}
    rewired = inputs.Network(tensors, labels, dims, [])
    rewired.validate()
    lz = log_z(rewired, planner.greedy_tree(labels, dims, []))
    assert abs(lz - ising.log_z_enumerate(n, net.meta["edges"], net.meta["J"], net.meta["beta"])) < 1e-12


def test_ising_closed_forms():
    # beta = 0: Z = 2^N exactly
    edges = inputs.random_regular_graph(40, 3, seed=4)
    net = inputs.ising_network(40, edges, np.ones(len(edges)), 0.0)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    m, e = tree.contract_net(net, pairs)
    assert float(m) * 2.0 ** (e - 40) == 1.0
    # ring: transfer-matrix closed form
    n = 30
    ring = [(i, (i + 1) % n) for i in range(n)]
    J = inputs.ising_couplings(n, seed=5)
    net = inputs.ising_network(n, [tuple(sorted(e)) for e in ring], J, 0.7)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    assert abs(log_z(net, pairs) - ising.log_z_ring(J, 0.7)) < 1e-12
    # tree graph: 2 prod 2cosh
    rng = np.random.default_rng(6)
    tedges = [(int(rng.integers(0, v)), v) for v in range(1, 25)]
    J = inputs.ising_couplings(len(tedges), seed=7)
    net = inputs.ising_network(25, tedges, J, 0.45)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    assert abs(log_z(net, pairs) - ising.log_z_tree(25, J, 0.45)) < 1e-12


def test_ising_gauge_invariance():
    """Flipping J on all edges at one vertex is s_v -> -s_v: Z unchanged."""
    net = inputs.random_ising(60, seed=8)
    edges, J = net.meta["edges"], np.array(net.meta["J"])
    J2 = J.copy()
    for k, (u, v) in enumerate(edges):
        if 7 in (u, v):
            J2[k] = -J2[k]
    net2 = inputs.ising_network(60, edges, J2, net.meta["beta"])
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    assert abs(log_z(net, pairs) - log_z(net2, pairs)) < 1e-12


def test_renormalisation_tracks_huge_values():
    """Scaling every edge matrix by 2^600 multiplies Z by 2^(600|E|), far
    beyond the double range; the exponent bookkeeping must be exact."""
    net = inputs.random_ising(40, seed=9)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    n_edges = len(net.meta["edges"])
    scaled = [t if i < 40 else t * 2.0 ** 600 for i, t in enumerate(net.tensors)]
    m0, e0 = tree.contract_net(net, pairs)
    m1, e1 = tree.contract(scaled, net.labels, net.dims, net.open, pairs)
    lz0 = math.log2(float(m0)) + e0
    lz1 = math.log2(float(m1)) + e1
    assert abs((lz1 - lz0) - 600 * n_edges) < 1e-9


def test_cfg1_ising_slices():
    """N=100 random 3-regular Ising: slicing 3 labels leaves ln Z unchanged."""
    net = inputs.random_ising(100, seed=0)
    pairs = planner.greedy_tree(net.labels, net.dims, net.open)
    sl = planner.slice_greedy(net.labels, net.dims, pairs, net.open, 18)
    assert len(sl) >= 1
    assert abs(log_z(net, pairs) - log_z(net, pairs, sl)) < 1e-12


# --------------------------------------------------------------------------
# gradients as environments
# --------------------------------------------------------------------------

def test_environment_gradient_matches_finite_differences():
    """d c_x / d theta of one fSim gate: chain rule through the environment
    against a central difference of the state-vector amplitude."""
    circ = inputs.random_circuit(2, 3, 5, seed=12)
    bs = inputs.random_bitstrings(6, 1, seed=13)[0]
    net = inputs.circuit_network(circ, bs)
    tf = lambda l, d, o: planner.greedy_tree(l, d, o)
    for gi in circ.fsim_gates()[:3]:
        v = net.meta["gate_leaf"][gi]
        env = gradient.environment(net.tensors, net.labels, net.dims, v, tf)
        th, ph = circ.gates[gi].params
        h = 1e-3
        for which in (0, 1):
            p = [th, ph]
            dG = np.zeros((4, 4), dtype=complex)
            for sgn in (1, -1):
                q = list(p)
                q[which] += sgn * h
                dG += sgn * inputs.fsim(*q) / (2 * h)
            analytic = np.sum(env * dG.reshape(2, 2, 2, 2))
            amps = []
            for sgn in (1, -1):
                q = list(p)
                q[which] += sgn * h
                g2 = [inputs.Gate(g.name, g.qubits, g.matrix, g.params) for g in circ.gates]
                g2[gi] = inputs.Gate("fsim", g2[gi].qubits, inputs.fsim(*q), tuple(q))
                amps.append(statevector.amplitude(6, g2, bs))
            fd = (amps[0] - amps[1]) / (2 * h)
            assert abs(analytic - fd) <= 1e-6 * max(abs(fd), 1e-3)


def test_environment_of_plain_product():
    """c = a . b: dc/da = b exactly."""
    rng = np.random.default_rng(2)
    a = rng.standard_normal(3) + 1j * rng.standard_normal(3)
    b = rng.standard_normal(3) + 1j * rng.standard_normal(3)
    env = gradient.environment([a, b], [[0], [0]], {0: 3}, 0,
                               lambda l, d, o: planner.greedy_tree(l, d, o))
    assert rel(env, b) < 1e-15


def _random_ssa_tree(n, rng):
    live, pairs = list(range(n)), []
    for k in range(n - 1):
        i, j = sorted(rng.choice(len(live), size=2, replace=False))
        a, b = live[i], live[j]
        pairs.append((int(a), int(b)))
        live = [x for x in live if x not in (a, b)] + [n + k]
    return pairs


@pytest.mark.parametrize("seed", range(60))
def test_random_trees_scalars_and_slice_ranges_match_nested_sum(seed):
    """Brute force on tiny random networks with any tree (outer products of
    unconnected parts included), a scalar leaf now and then, random sliced
    labels, and the slice range cut in two: the two partial sums add up to
    the nested sum of products."""
    rng = np.random.default_rng(seed)
    net = inputs.random_network(int(rng.integers(1, 7)), int(rng.integers(1, 9)), 12000 + seed,
                                n_open=int(rng.integers(0, 3)), max_dim=int(rng.integers(1, 4)))
    tensors, labels = list(net.tensors), [list(l) for l in net.labels]
    if rng.random() < 0.3:
        tensors.append(np.array(rng.standard_normal() + 1j * rng.standard_normal()))
        labels.append([])
    n = len(tensors)
    pairs = _random_ssa_tree(n, rng) if n > 1 else []
    summed = [l for l in sorted(net.dims) if l not in net.open]
    k = int(rng.integers(0, min(2, len(summed)) + 1))
    sliced = [int(x) for x in rng.choice(summed, size=k, replace=False)] if k else []
    ref = brute.nested_sum(tensors, labels, net.dims, net.open)
    scale = np.abs(brute.nested_sum([np.abs(t) for t in tensors], labels, net.dims, net.open))
    m, e = tree.contract(tensors, labels, net.dims, net.open, pairs, sliced)
    assert np.all(np.abs(np.asarray(m) * 2.0 ** e - ref) <= 1e-12 * scale + 1e-300)
    d = int(np.prod([net.dims[l] for l in sliced])) if sliced else 1
    cut = int(rng.integers(0, d + 1))
    total = 0
    for b, c in ((0, cut), (cut, d - cut)):
        if c:
            mm, ee = tree.contract(tensors, labels, net.dims, net.open, pairs, sliced, slice_begin=b, slice_count=c)
            total = total + np.asarray(mm) * 2.0 ** ee
    assert np.all(np.abs(total - ref) <= 1e-12 * scale + 1e-300)


@pytest.mark.parametrize("n,seed", [(10, 2), (14, 3)])
def test_environments_give_the_ising_energy(n, seed):
    """d ln Z / d beta from the edge matrices' environments (chain rule
    through M_e = exp(beta J_e s s')) equals the central difference of the
    enumerated ln Z: a pin of the gradient oracle on a real network."""
    beta = 0.3
    net = inputs.random_ising(n, seed, beta=beta)
    edges, J = net.meta["edges"], net.meta["J"]
    tf = lambda l, d, o: planner.greedy_tree(l, d, o)
    z = float(np.real(tree.value(net.tensors, net.labels, net.dims, net.open, tf(net.labels, net.dims, net.open))))
    spin = np.array([1.0, -1.0])
    dz = 0.0
    for e in range(len(edges)):
        v = n + e  # edge matrices follow the COPY tensors
        env = gradient.environment(net.tensors, net.labels, net.dims, v, tf)
        dm = J[e] * np.outer(spin, spin) * net.tensors[v]
        dz += float(np.real(np.sum(env * dm)))
    h = 1e-4
    fd = (ising.log_z_enumerate(n, edges, J, beta + h) - ising.log_z_enumerate(n, edges, J, beta - h)) / (2 * h)
    assert abs(dz / z - fd) <= 1e-6 * max(abs(fd), 1.0)


# --------------------------------------------------------------------------
# loss gradient of the differentiation workload (state-vector adjoint)
# --------------------------------------------------------------------------

def test_fsim_derivatives_match_finite_differences():
    h = 1e-6
    for theta, phi in [(0.3, 1.1), (1.2, 2.9), (0.0, 0.0)]:
        dt, dp = statevector.fsim_derivatives(theta, phi)
        fd_t = (inputs.fsim(theta + h, phi) - inputs.fsim(theta - h, phi)) / (2 * h)
        fd_p = (inputs.fsim(theta, phi + h) - inputs.fsim(theta, phi - h)) / (2 * h)
        assert np.max(np.abs(dt - fd_t)) < 1e-9
        assert np.max(np.abs(dp - fd_p)) < 1e-9


def test_mean_log_prob_grad_matches_finite_differences():
    """Every fSim (theta, phi) of a 3x3, 5-cycle circuit: the adjoint-state
    gradient of L = mean ln|c_x|^2 against central differences of L computed
    by plain forward simulation."""
    circ = inputs.random_circuit(3, 3, 5, seed=6)
    bits = inputs.random_bitstrings(9, 5, seed=1006)
    fs = circ.fsim_gates()
    dg = {g: list(statevector.fsim_derivatives(*circ.gates[g].params)) for g in fs}
    L, grads = statevector.mean_log_prob_grad(9, circ.gates, bits, dg)

    def loss(gates):
        psi = statevector.final_state(9, gates)
        return float(np.mean([math.log(abs(psi[tuple(int(b) for b in x)]) ** 2) for x in bits]))

    assert abs(L - loss(circ.gates)) < 1e-12
    h = 1e-5
    for g in fs:
        th, ph = circ.gates[g].params
        for which in (0, 1):
            vals = []
            for sgn in (1, -1):
                p = [th, ph]
                p[which] += sgn * h
                gates = list(circ.gates)
                gates[g] = inputs.Gate("fsim", gates[g].qubits, inputs.fsim(*p), tuple(p))
                vals.append(loss(gates))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(grads[g][which] - fd) <= 1e-6 * max(1.0, abs(fd)), (g, which, grads[g][which], fd)
