"""ctypes driver of the FP64 tree executor in tn_oracle.c.

Test infrastructure only.  ``contract`` returns (mantissa, exp2) with
value = mantissa * 2**exp2; the mantissa is an ndarray over the open labels
(a 0-d array for a scalar network), complex128 or float64.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import build as _build

_lib = None


def load_library(path: str):
    """Load an oracle shared library built from tn_oracle.c."""
    lib = ctypes.CDLL(path)
    i64p = ctypes.POINTER(ctypes.c_longlong)
    lib.tno_contract.restype = ctypes.c_int
    lib.tno_contract.argtypes = [
        ctypes.c_int, ctypes.POINTER(ctypes.c_int), i64p, ctypes.c_int, i64p, i64p,
        ctypes.c_int, i64p, ctypes.c_int, ctypes.POINTER(ctypes.POINTER(ctypes.c_double)),
        ctypes.POINTER(ctypes.c_int), ctypes.c_int, i64p, ctypes.c_longlong,
        ctypes.c_longlong, ctypes.POINTER(ctypes.c_double), i64p]
    lib.tno_max_threads.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = load_library(_build.build())
    return _lib




def max_threads() -> int:
    return int(_load().tno_max_threads())


def _i64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def contract(tensors: Sequence[np.ndarray], labels: Sequence[Sequence[int]], dims: Dict[int, int],
             open_labels: Sequence[int], pairs: Sequence[Tuple[int, int]],
             sliced: Sequence[int] = (), slice_begin: int = 0, slice_count: int = -1,
             is_complex: Optional[bool] = None, lib=None) -> Tuple[np.ndarray, int]:
    """Contract with the given SSA tree; sum the selected slices."""
    lib = _load() if lib is None else lib
    n = len(tensors)
    if is_complex is None:
        is_complex = any(np.iscomplexobj(t) for t in tensors)
    dt = np.complex128 if is_complex else np.float64
    bufs = [np.ascontiguousarray(np.asarray(t, dtype=dt)) for t in tensors]
    ptrs = (ctypes.POINTER(ctypes.c_double) * n)(
        *[b.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for b in bufs])
    ranks = np.ascontiguousarray(np.array([len(l) for l in labels], dtype=np.int32))
    flat = _i64([l for ls in labels for l in ls] or [0])
    ids = sorted(dims)
    lid = _i64(ids or [0])
    ldim = _i64([dims[i] for i in ids] or [1])
    opn = _i64(list(open_labels) or [0])
    pr = np.ascontiguousarray(np.array([x for p in pairs for x in p] or [0], dtype=np.int32))
    sl = _i64(list(sliced) or [0])
    n_out = int(np.prod([dims[l] for l in open_labels])) if len(open_labels) else 1
    out = np.zeros(n_out, dtype=dt)
    e = np.zeros(1, dtype=np.int64)
    P = lambda a, t: a.ctypes.data_as(ctypes.POINTER(t))
    rc = lib.tno_contract(n, P(ranks, ctypes.c_int), P(flat, ctypes.c_longlong), len(ids),
                          P(lid, ctypes.c_longlong), P(ldim, ctypes.c_longlong), len(open_labels),
                          P(opn, ctypes.c_longlong), int(is_complex), ptrs,
                          P(pr, ctypes.c_int), len(sliced), P(sl, ctypes.c_longlong),
                          int(slice_begin), int(slice_count),
                          out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                          P(e, ctypes.c_longlong))
    if rc != 0:
        raise ValueError(f"oracle contraction failed (code {rc})")
    shape = tuple(dims[l] for l in open_labels)
    return out.reshape(shape), int(e[0])


def value(*args, **kw) -> np.ndarray:
    """mantissa * 2**exp2 as a plain ndarray (may over/underflow)."""
    m, e = contract(*args, **kw)
    return m * (2.0 ** e)


def contract_net(net, pairs, sliced=(), **kw):
    return contract(net.tensors, net.labels, net.dims, net.open, pairs, sliced, **kw)
