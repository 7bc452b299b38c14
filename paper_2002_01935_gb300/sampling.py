"""Approximately unbiased bitstring samples of a random circuit at a chosen
fidelity, from open-output contractions (the sampling procedure of the
paper's runtime estimate for Sycamore, Sec. 5).

For a chaotic circuit the marginal over N_u of the qubits is close to
uniform once the other N_f qubits are traced out.  A sample therefore fixes
the N_u qubits to a uniformly drawn x_u, computes the 2^N_f amplitudes
<x_u x_f|psi> over the remaining qubits in one contraction (the network of
Eq. trans-amp with N_f output labels left open), and draws x_f with
probability |<x_u x_f|psi>|^2 / Z.  Fidelity f is simulated by the mixture
(1 - f) 1/2^N + f |psi><psi|: with probability f the sample comes from psi,
otherwise it is uniform; when psi itself only has fidelity g, f is replaced
by f / g (at most 1).

``OpenAmplitudes`` computes the amplitude tensors on the GPU through the
library (one tree, planned once; only the output-state leaves change from
one x_u to the next); ``sample`` takes any amplitude provider with the same
call signature.
"""
from __future__ import annotations

from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np

from . import inputs, planner


class OpenAmplitudes:
    """x_u (bits of the fixed qubits, in increasing qubit order) ->
    complex128 array of shape (2,) * N_f: <x_u x_f|psi> with the axes of x_f
    in ``open_qubits`` order.  One contraction on the GPU per call."""

    def __init__(self, circuit: inputs.Circuit, open_qubits: Sequence[int], mode: str = "tf32_split",
                 pairs=None, sliced=()):
        import torch
        from . import binding

        self.circuit = circuit
        self.open_qubits = [int(q) for q in open_qubits]
        self.fixed = [q for q in range(circuit.n_qubits) if q not in set(self.open_qubits)]
        self.mode = mode
        net = inputs.circuit_network(circuit, [0] * circuit.n_qubits, open_qubits=self.open_qubits)
        self.pairs = pairs if pairs is not None else planner.greedy_tree(net.labels, net.dims, net.open)
        self.sliced = list(sliced)
        # the output-state leaves are the last ones, one per fixed qubit
        self.first_out = net.n_tensors - len(self.fixed)
        self._leaves = [torch.from_numpy(np.array(t, order="C")).to(torch.complex64).cuda()
                        for t in net.tensors]
        self._basis = torch.eye(2, dtype=torch.complex64, device="cuda")
        self.tnw = binding.TensorNetwork(net.labels, net.dims, net.open, self._leaves, complex_=True)

    def __call__(self, x_u: Sequence[int]) -> np.ndarray:
        if len(x_u) != len(self.fixed):
            raise ValueError(f"x_u needs {len(self.fixed)} bits")
        leaves = list(self._leaves)
        for i, b in enumerate(x_u):
            leaves[self.first_out + i] = self._basis[int(b)]
        self.tnw.set_tensors(leaves)
        m, e = self.tnw.contract(self.pairs, self.sliced, self.mode)
        return m.cpu().numpy() * 2.0 ** int(e.cpu())

    def close(self) -> None:
        self.tnw.close()


def sample(n_qubits: int, open_qubits: Sequence[int], amplitudes: Callable[[Sequence[int]], np.ndarray],
           n_samples: int, fidelity: float = 1.0, psi_fidelity: float = 1.0,
           seed: int = 0) -> List[Tuple[Tuple[int, ...], bool]]:
    """``n_samples`` bitstrings (tuples of N bits, qubit order) and, for each,
    whether it was drawn from psi (True) or uniformly (False)."""
    if not 0.0 <= fidelity <= 1.0 or not 0.0 < psi_fidelity <= 1.0:
        raise ValueError("need 0 <= fidelity <= 1 and 0 < psi_fidelity <= 1")
    f = min(1.0, fidelity / psi_fidelity)
    open_qubits = [int(q) for q in open_qubits]
    fixed = [q for q in range(n_qubits) if q not in set(open_qubits)]
    rng = np.random.Generator(np.random.PCG64(seed))
    out: List[Tuple[Tuple[int, ...], bool]] = []
    for _ in range(n_samples):
        bits = [0] * n_qubits
        if rng.random() < f:
            x_u = [int(b) for b in rng.integers(0, 2, size=len(fixed))]
            amp = np.asarray(amplitudes(x_u)).reshape(-1)
            p = np.abs(amp) ** 2
            z = float(p.sum())
            if not z > 0.0:
                raise ValueError("all amplitudes of this x_u are zero")
            k = int(rng.choice(p.size, p=p / z))
            x_f = [(k >> (len(open_qubits) - 1 - j)) & 1 for j in range(len(open_qubits))]
            for q, b in zip(fixed, x_u):
                bits[q] = b
            for q, b in zip(open_qubits, x_f):
                bits[q] = b
            out.append((tuple(bits), True))
        else:
            out.append((tuple(int(b) for b in rng.integers(0, 2, size=n_qubits)), False))
    return out
