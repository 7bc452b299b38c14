"""Leaf derivatives of a network value, as environment contractions.

A network value c is multilinear in its leaves, so dc/dT_v[i] is the network
with T_v removed and T_v's labels left open at the values i: the
"environment" of v.  Contracting that network with the FP64 tree executor
gives the exact derivative (up to rounding), independent of any
reverse-mode bookkeeping.

Test infrastructure only.
"""
from __future__ import annotations

from typing import Callable, Dict, Sequence, Tuple

import numpy as np

from . import tree


def environment(tensors, labels, dims, v: int, tree_fn: Callable) -> np.ndarray:
    """dc/dT_v as an array shaped like T_v (closed networks only).

    ``tree_fn(labels, dims, open)`` returns an SSA tree for the reduced
    network (any tree gives the same value)."""
    rest_t = [t for i, t in enumerate(tensors) if i != v]
    rest_l = [l for i, l in enumerate(labels) if i != v]
    open_l = list(labels[v])
    # labels of T_v that occur nowhere else are not connected to the
    # environment: the derivative is constant (1) along them
    present = {l for ls in rest_l for l in ls}
    missing = [l for l in open_l if l not in present]
    for l in missing:
        rest_t.append(np.ones(dims[l]))
        rest_l.append([l])
    pairs = tree_fn(rest_l, dims, open_l)
    m, e = tree.contract(rest_t, rest_l, dims, open_l, pairs,
                         is_complex=any(np.iscomplexobj(t) for t in tensors))
    return m * (2.0 ** e)
