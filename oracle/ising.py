"""Ising partition functions Z = sum_s exp(beta sum_e J_e s_u s_v).

Enumeration over all 2^N spin configurations (N <= ~22) and closed forms for
special graphs; independent of the tensor-network encoding.  The random
3-regular graph family is that of Sec. 4.1 of arXiv 2002.01935.

Test infrastructure only.
"""
from __future__ import annotations

import math
from typing import Sequence, Tuple

import numpy as np


def log_z_enumerate(n: int, edges: Sequence[Tuple[int, int]], J: Sequence[float],
                    beta: float) -> float:
    """ln Z by explicit enumeration, spins s = +1 for bit 0, -1 for bit 1."""
    if n > 24:
        raise ValueError("too many spins to enumerate")
    idx = np.arange(1 << n, dtype=np.int64)
    energy = np.zeros(1 << n, dtype=np.float64)
    for (u, v), j in zip(edges, J):
        su = 1.0 - 2.0 * ((idx >> u) & 1)
        sv = 1.0 - 2.0 * ((idx >> v) & 1)
        energy += j * su * sv
    x = beta * energy
    m = x.max()
    return float(m + math.log(np.exp(x - m).sum()))


def log_z_ring(J: Sequence[float], beta: float) -> float:
    """Closed ring: Z = prod 2cosh(beta J) + prod 2sinh(beta J) (transfer matrix)."""
    c = np.prod([2 * math.cosh(beta * j) for j in J])
    s = np.prod([2 * math.sinh(beta * j) for j in J])
    return math.log(c + s)


def log_z_tree(n: int, J: Sequence[float], beta: float) -> float:
    """Any tree graph on n vertices: Z = 2 prod_e 2cosh(beta J_e)."""
    return math.log(2.0) + sum(math.log(2 * math.cosh(beta * j)) for j in J)
