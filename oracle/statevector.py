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


def _apply(psi: np.ndarray, m: np.ndarray, qubits) -> np.ndarray:
    """Gate matrix m [out, in] applied to the state array on ``qubits``."""
    k = len(qubits)
    # contract the gate's input axes with the state's qubit axes, then put
    # the gate's output axes where those qubits were
    out = np.tensordot(m.reshape((2,) * (2 * k)), psi, axes=(tuple(range(k, 2 * k)), tuple(qubits)))
    return np.moveaxis(out, tuple(range(k)), tuple(qubits))


def fsim_derivatives(theta: float, phi: float):
    """d fSim / d theta and d fSim / d phi, from the fSim matrix in the basis
    |00>, |01>, |10>, |11> (first qubit most significant):
    [[1, 0, 0, 0], [0, cos t, -i sin t, 0], [0, -i sin t, cos t, 0],
    [0, 0, 0, exp(-i p)]]."""
    dt = np.zeros((4, 4), dtype=np.complex128)
    dt[1, 1] = dt[2, 2] = -np.sin(theta)
    dt[1, 2] = dt[2, 1] = -1j * np.cos(theta)
    dp = np.zeros((4, 4), dtype=np.complex128)
    dp[3, 3] = -1j * np.exp(-1j * phi)
    return dt, dp


def mean_log_prob_grad(n_qubits: int, gates, bitstrings, dgates):
    """L = (1/B) sum_x ln|c_x|^2 over the B bitstrings, c_x = <x|U|0^N>, and
    dL/dp for the gate parameters named in ``dgates`` ({gate index: [dG/dp,
    ...]}, matrices [out, in] like the gate's).  Adjoint state method:
    with lambda = (1/B) sum_x conj(1/c_x) |x>, L's derivative is
    2 Re <lambda| U_after (dG/dp) U_before |0>, evaluated for every gate
    from the stored state before it and lambda carried backwards by G^dagger
    (the adjoint of psi -> G psi).  Returns (L, {gate: [dL/dp, ...]})."""
    B = len(bitstrings)
    psi = np.zeros((2,) * n_qubits, dtype=np.complex128)
    psi[(0,) * n_qubits] = 1.0
    before = {}
    for g, gate in enumerate(gates):
        if g in dgates:
            before[g] = psi
        psi = _apply(psi, np.asarray(gate.matrix, dtype=np.complex128), gate.qubits)
    lam = np.zeros_like(psi)
    L = 0.0
    for x in bitstrings:
        idx = tuple(int(b) for b in x)
        c = psi[idx]
        L += np.log(abs(c) ** 2) / B
        lam[idx] += np.conj(1.0 / c) / B
    grads = {}
    for g in range(len(gates) - 1, -1, -1):
        gate = gates[g]
        m = np.asarray(gate.matrix, dtype=np.complex128)
        if g in dgates:
            k = len(gate.qubits)
            lm = np.moveaxis(lam, list(gate.qubits), list(range(k))).reshape(2 ** k, -1)
            pm = np.moveaxis(before[g], list(gate.qubits), list(range(k))).reshape(2 ** k, -1)
            M = np.conj(lm) @ pm.T  # M[o, i] = d <lambda|psi_after> / d G[o, i]
            grads[g] = [2.0 * float(np.real(np.sum(M * d))) for d in dgates[g]]
        lam = _apply(lam, np.conj(m).T, gate.qubits)
    return float(L), grads
