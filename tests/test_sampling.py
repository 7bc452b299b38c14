"""The fidelity-mixture sampler over open-output contractions (the sampling
procedure of Sec. 5's runtime estimate), checked with oracle amplitudes:
the sampler's x_f follows |<x_u x_f|psi>|^2 / Z, its fixed qubits are
uniform, and the share of samples from psi is the fidelity (f / g when psi
has fidelity g)."""
import numpy as np
import pytest

from oracle import statevector, tree
from paper_2002_01935_gb300 import inputs, planner, sampling


def _oracle_provider(circ, open_qubits):
    fixed = [q for q in range(circ.n_qubits) if q not in set(open_qubits)]
    cache = {}

    def amps(x_u):
        key = tuple(int(b) for b in x_u)
        if key not in cache:
            cache[key] = _amps(key)
        return cache[key]

    def _amps(x_u):
        bits = [0] * circ.n_qubits
        for q, b in zip(fixed, x_u):
            bits[q] = b
        net = inputs.circuit_network(circ, bits, open_qubits=open_qubits)
        pairs = planner.greedy_tree(net.labels, net.dims, net.open)
        m, e = tree.contract_net(net, pairs)
        return np.asarray(m) * 2.0 ** e
    return amps


def test_open_amplitudes_are_the_state_vector_slice():
    circ = inputs.random_circuit(2, 3, 5, seed=3)
    psi = statevector.final_state(6, circ.gates)
    open_q = [4, 1, 5]
    amps = _oracle_provider(circ, open_q)
    x_u = [1, 0, 1]  # qubits 0, 2, 3
    got = amps(x_u)
    idx = [slice(None)] * 6
    for q, b in zip([0, 2, 3], x_u):
        idx[q] = b
    ref = np.moveaxis(psi[tuple(idx)], [0, 1, 2], [1, 0, 2])  # remaining axes 1, 4, 5 -> order 4, 1, 5
    assert np.allclose(got, ref, atol=1e-12)


def test_samples_follow_the_conditional_distribution():
    circ = inputs.random_circuit(2, 2, 6, seed=1)
    open_q = [0, 1, 2, 3]  # N_u = 0: the sampler draws from |psi|^2 itself
    psi = statevector.final_state(4, circ.gates)
    p = (np.abs(psi) ** 2).reshape(-1)
    s = sampling.sample(4, open_q, _oracle_provider(circ, open_q), 20000, seed=7)
    assert all(from_psi for _, from_psi in s)
    counts = np.zeros(16)
    for bits, _ in s:
        counts[int("".join(map(str, bits)), 2)] += 1
    chi2 = float(np.sum((counts - 20000 * p) ** 2 / (20000 * p)))
    assert chi2 < 45.0  # 15 degrees of freedom; p-value ~ 1e-4 at this bound


def test_fixed_qubits_are_uniform_and_open_ones_conditional():
    circ = inputs.random_circuit(2, 3, 5, seed=4)
    open_q = [5, 2]
    amps = _oracle_provider(circ, open_q)
    s = sampling.sample(6, open_q, amps, 3000, seed=11)
    fixed = [0, 1, 3, 4]
    for q in fixed:
        share = np.mean([bits[q] for bits, _ in s])
        assert abs(share - 0.5) < 0.05, q
    # every drawn x_f has nonzero conditional probability
    for bits, _ in s[:50]:
        a = amps([bits[q] for q in fixed])
        assert abs(a[bits[5], bits[2]]) > 0


@pytest.mark.parametrize("f,g,share", [(0.3, 1.0, 0.3), (0.2, 0.5, 0.4), (0.8, 0.5, 1.0)])
def test_fidelity_mixture_share(f, g, share):
    circ = inputs.random_circuit(2, 2, 4, seed=2)
    open_q = [1, 3]
    s = sampling.sample(4, open_q, _oracle_provider(circ, open_q), 4000, fidelity=f, psi_fidelity=g,
                        seed=5)
    got = np.mean([fp for _, fp in s])
    assert abs(got - share) < 4 * np.sqrt(share * (1 - share) / 4000) + 1e-12


def test_bad_fidelities_are_refused():
    for f, g in [(-0.1, 1.0), (1.1, 1.0), (0.5, 0.0)]:
        with pytest.raises(ValueError):
            sampling.sample(2, [0], lambda x: np.ones(2), 1, fidelity=f, psi_fidelity=g)
