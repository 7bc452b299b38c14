"""Dense state-vector simulation of a circuit (Eq. trans-amp).

c_x = <x| U_d ... U_1 |0^N>: start from |0...0>, apply every gate of the
circuit in order to a 2^N complex128 vector, read entry x.  Qubit q is axis
q of the (2,)*N state array.  Independent of the tensor-network encoding:
it reads only the gate list (matrices [out, in], first qubit most
significant for two-qubit gates).

Test infrastructure only.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np


def final_state(n_qubits: int, gates) -> np.ndarray:
    psi = np.zeros((2,) * n_qubits, dtype=np.complex128)
    psi[(0,) * n_qubits] = 1.0
    for g in gates:
        m = np.asarray(g.matrix, dtype=np.complex128)
        if len(g.qubits) == 1:
            (q,) = g.qubits
            psi = np.tensordot(m, psi, axes=([1], [q]))
            psi = np.moveaxis(psi, 0, q)
        else:
            a, b = g.qubits
            m4 = m.reshape(2, 2, 2, 2)
            psi = np.tensordot(m4, psi, axes=([2, 3], [a, b]))
            psi = np.moveaxis(psi, [0, 1], [a, b])
    return psi


def amplitude(n_qubits: int, gates, bitstring: Sequence[int]) -> complex:
    psi = final_state(n_qubits, gates)
    return complex(psi[tuple(int(b) for b in bitstring)])
