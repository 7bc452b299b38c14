"""The value of a tensor network as the literal nested sum of products.

Sec. 4.7.1 of arXiv 2002.01935: a network is the |E| nested summations of
the product of the entries of its |V| tensors; the open labels stay free.
Written out directly: broadcast every tensor onto the full label space,
multiply, and sum over the non-open labels.  Exponential in the number of
labels, so only for tiny networks (used to pin the tree executor).

Test infrastructure only.
"""
from __future__ import annotations

from typing import Dict, Sequence

import numpy as np


def nested_sum(tensors: Sequence[np.ndarray], labels: Sequence[Sequence[int]],
               dims: Dict[int, int], open_labels: Sequence[int] = (),
               max_entries: int = 1 << 24) -> np.ndarray:
    all_labels = sorted({l for ls in labels for l in ls} | set(open_labels))
    axis = {l: i for i, l in enumerate(all_labels)}
    shape = [dims[l] for l in all_labels]
    if int(np.prod(shape, dtype=np.float64)) > max_entries:
        raise ValueError("network too large for the nested sum")
    dt = np.complex128 if any(np.iscomplexobj(t) for t in tensors) else np.float64
    prod = np.ones(shape, dtype=dt)
    for t, ls in zip(tensors, labels):
        # place tensor axes on their label axes, size 1 elsewhere
        order = np.argsort([axis[l] for l in ls])
        tt = np.transpose(np.asarray(t, dtype=dt), order)
        bshape = [1] * len(all_labels)
        for l in ls:
            bshape[axis[l]] = dims[l]
        prod = prod * tt.reshape(bshape)
    summed = tuple(i for l, i in axis.items() if l not in set(open_labels))
    res = prod.sum(axis=summed) if summed else prod
    # remaining axes are the open labels in sorted order; reorder as requested
    kept = [l for l in all_labels if l in set(open_labels)]
    perm = [kept.index(l) for l in open_labels]
    return np.transpose(res, perm) if perm else np.asarray(res)
