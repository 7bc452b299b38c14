"""The pins of the oracle's Python modules catch plausible mistakes.

Each case plants one mistake in a copy of ``oracle/statevector.py`` (its
state vector, or its adjoint gradient of the mean log-probability) or
``oracle/gradient.py`` (a gate read transposed, qubits swapped on output, a
bitstring read backwards, environment axes in the wrong order, the exponent
of a renormalised environment dropped, dangling labels not closed), loads the
copy as a module of the ``oracle`` package, and checks that a pin rejects it.
The pins are independent of the module under test: the state vector against
the tree executor (itself pinned by brute-force nested sums), the
environments against brute-force derivatives (the network value with the
leaf replaced by a unit tensor, summed by ``oracle.brute``).  The oracle
itself is never modified.
"""
import importlib.util
import itertools
import os

import numpy as np
import pytest

from oracle import brute, tree
from paper_2002_01935_gb300 import inputs, planner

ORACLE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")

SV_MUTANTS = [
    ("one-qubit gate read transposed", "axes=([1], [q])", "axes=([0], [q])"),
    ("two-qubit gate outputs swapped", "np.moveaxis(psi, [0, 1], [a, b])", "np.moveaxis(psi, [0, 1], [b, a])"),
    ("bitstring read backwards", "psi[tuple(int(b) for b in bitstring)]",
     "psi[tuple(int(b) for b in bitstring)[::-1]]"),
]

GRAD_MUTANTS = [
    ("environment axes reversed", "open_l = list(labels[v])", "open_l = list(labels[v])[::-1]"),
    ("renormalisation exponent dropped", "return m * (2.0 ** e)", "return m"),
    ("dangling labels left unclosed", "for l in missing:", "for l in missing[:0]:"),
]


LOSS_GRAD_MUTANTS = [
    ("adjoint carried by G instead of its conjugate transpose",
     "lam = _apply(lam, np.conj(m).T, gate.qubits)", "lam = _apply(lam, m, gate.qubits)"),
    ("adjoint state not conjugated", "lam[idx] += np.conj(1.0 / c) / B", "lam[idx] += (1.0 / c) / B"),
    ("imaginary part taken for the real part", "2.0 * float(np.real(np.sum(M * d)))",
     "2.0 * float(np.imag(np.sum(M * d)))"),
    ("state taken after the gate instead of before",
     "        if g in dgates:\n            before[g] = psi\n"
     "        psi = _apply(psi, np.asarray(gate.matrix, dtype=np.complex128), gate.qubits)\n",
     "        psi = _apply(psi, np.asarray(gate.matrix, dtype=np.complex128), gate.qubits)\n"
     "        if g in dgates:\n            before[g] = psi\n"),
    ("fSim theta derivative sign", "dt[1, 1] = dt[2, 2] = -np.sin(theta)", "dt[1, 1] = dt[2, 2] = np.sin(theta)"),
]


def _load(fname: str, src: str, tag: str):
    """``src`` as module ``oracle.<tag>`` (relative imports resolve in the
    oracle package)."""
    path = os.path.join(ORACLE, fname)
    spec = importlib.util.spec_from_file_location(f"oracle.{tag}", path)
    mod = importlib.util.module_from_spec(spec)
    exec(compile(src, path, "exec"), mod.__dict__)
    return mod


def _sv_pins_pass(sv) -> bool:
    """All amplitudes of two small circuits, from the module's state vector
    and from its amplitude reader, against the tree executor."""
    try:
        for (r, c, t), seed in (((2, 3, 5), 21), ((3, 2, 6), 22)):
            n = r * c
            circ = inputs.random_circuit(r, c, t, seed=seed)
            net = inputs.circuit_network(circ, open_qubits=list(range(n)))
            pairs = planner.greedy_tree(net.labels, net.dims, net.open)
            ref = tree.value(net.tensors, net.labels, net.dims, net.open, pairs)
            psi = sv.final_state(n, circ.gates)
            if not np.max(np.abs(psi - ref)) < 1e-12:
                return False
            for bs in inputs.random_bitstrings(n, 4, seed=seed + 100):
                if not abs(sv.amplitude(n, circ.gates, bs) - ref[tuple(bs)]) < 1e-12:
                    return False
    except (ValueError, IndexError):
        return False
    return True


def _brute_derivative(tensors, labels, dims, v):
    """dc/dT_v entry by entry: the value with T_v replaced by unit tensors."""
    shape = tensors[v].shape
    out = np.zeros(shape, dtype=complex)
    for idx in itertools.product(*(range(s) for s in shape)):
        unit = np.zeros(shape, dtype=complex)
        unit[idx] = 1.0
        ts = list(tensors)
        ts[v] = unit
        out[idx] = brute.nested_sum(ts, labels, dims, [])
    return out


def _grad_pins_pass(g) -> bool:
    """Environments of every leaf of small closed networks (hyperedges,
    labels of different sizes, labels carried by one leaf only, values
    scaled so that the tree renormalises) against brute-force derivatives."""
    tf = lambda l, d, o: planner.greedy_tree(l, d, o)
    cases = []
    for seed in range(3):
        net = inputs.random_network(5, 7, 900 + seed, n_open=0, max_dim=3)
        cases.append((list(net.tensors), net.labels, net.dims))
    # a label held by one leaf only, and entries far from 1
    rng = np.random.default_rng(5)
    a = (rng.standard_normal((2, 3)) + 1j * rng.standard_normal((2, 3))) * 2.0 ** 40
    b = rng.standard_normal((3, 4)) + 1j * rng.standard_normal((3, 4))
    c = rng.standard_normal((4,)) * 2.0 ** -30
    cases.append(([a, b, c], [[0, 1], [1, 2], [2]], {0: 2, 1: 3, 2: 4}))
    try:
        for tensors, labels, dims in cases:
            for v in range(len(tensors)):
                env = np.asarray(g.environment(tensors, labels, dims, v, tf))
                ref = _brute_derivative(tensors, labels, dims, v)
                if env.shape != ref.shape:
                    return False
                scale = np.max(np.abs(ref)) if ref.size else 0.0
                if not np.all(np.abs(env - ref) <= 1e-12 * scale + 1e-300):
                    return False
    except (ValueError, KeyError, IndexError):
        return False
    return True


def test_unmodified_python_oracle_passes_pins():
    from oracle import gradient, statevector
    assert _sv_pins_pass(statevector)
    assert _grad_pins_pass(gradient)


@pytest.mark.parametrize("name,orig,mutated", SV_MUTANTS, ids=[m[0] for m in SV_MUTANTS])
def test_planted_state_vector_mistake_is_caught(name, orig, mutated):
    src = open(os.path.join(ORACLE, "statevector.py")).read()
    assert src.count(orig) == 1, f"mutation anchor not found: {name}"
    mod = _load("statevector.py", src.replace(orig, mutated), "statevector_mutant")
    assert not _sv_pins_pass(mod), f"pins did not catch: {name}"


@pytest.mark.parametrize("name,orig,mutated", GRAD_MUTANTS, ids=[m[0] for m in GRAD_MUTANTS])
def test_planted_gradient_mistake_is_caught(name, orig, mutated):
    src = open(os.path.join(ORACLE, "gradient.py")).read()
    assert src.count(orig) == 1, f"mutation anchor not found: {name}"
    mod = _load("gradient.py", src.replace(orig, mutated), "gradient_mutant")
    assert not _grad_pins_pass(mod), f"pins did not catch: {name}"


def _loss_grad_pins_pass(sv) -> bool:
    """Every fSim (theta, phi) of a small circuit: the module's adjoint loss
    gradient against central differences of the loss from forward
    simulation (the unmutated final_state of the oracle)."""
    from oracle import statevector as ref_sv
    circ = inputs.random_circuit(2, 3, 5, seed=31)
    bits = inputs.random_bitstrings(6, 3, seed=1031)
    fs = circ.fsim_gates()
    try:
        dg = {g: list(sv.fsim_derivatives(*circ.gates[g].params)) for g in fs}
        _, grads = sv.mean_log_prob_grad(6, circ.gates, bits, dg)

        def loss(gates):
            psi = ref_sv.final_state(6, gates)
            return float(np.mean([np.log(abs(psi[tuple(int(b) for b in x)]) ** 2) for x in bits]))

        h = 1e-5
        for g in fs:
            for which in (0, 1):
                vals = []
                for sgn in (1, -1):
                    p = list(circ.gates[g].params)
                    p[which] += sgn * h
                    gates = list(circ.gates)
                    gates[g] = inputs.Gate("fsim", gates[g].qubits, inputs.fsim(*p), tuple(p))
                    vals.append(loss(gates))
                fd = (vals[0] - vals[1]) / (2 * h)
                if not abs(grads[g][which] - fd) <= 1e-6 * max(1.0, abs(fd)):
                    return False
    except (ValueError, IndexError):
        return False
    return True


def test_unmodified_loss_gradient_passes_pins():
    from oracle import statevector
    assert _loss_grad_pins_pass(statevector)


@pytest.mark.parametrize("name,orig,mutated", LOSS_GRAD_MUTANTS, ids=[m[0] for m in LOSS_GRAD_MUTANTS])
def test_planted_loss_gradient_mistake_is_caught(name, orig, mutated):
    src = open(os.path.join(ORACLE, "statevector.py")).read()
    assert src.count(orig) == 1, f"mutation anchor not found: {name}"
    mod = _load("statevector.py", src.replace(orig, mutated), "statevector_grad_mutant")
    assert not _loss_grad_pins_pass(mod), f"pins did not catch: {name}"
