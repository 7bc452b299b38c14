"""ctypes binding of libtn.so, the C-ABI declared in include/tn.h.

Argument marshalling only: every step of a contraction runs in the
library's CUDA kernels.  Importing this module loads libtn.so and raises
ImportError if it has not been built (``paper_2002_01935_gb300.build``);
there is no fallback.

The functions mirror the C names (tn_create, tn_set_tensor, tn_contract,
tn_contract_ex, tn_contract_grad, tn_contract_grad_ex, tn_plan_info, tn_destroy,
tn_last_error); ``TensorNetwork`` wraps a handle for use with torch tensors.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtn.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libtn.so not built ({LIB_PATH}); run paper_2002_01935_gb300.build.build()")

_lib = ctypes.CDLL(LIB_PATH)

TN_OK, TN_EINVAL, TN_ENOMEM, TN_ECUDA, TN_ETIMEOUT, TN_EUNSUPPORTED = range(6)
TN_R32, TN_C64 = 0, 1
TN_MODE_FP32, TN_MODE_TF32_3M, TN_MODE_TF32_SPLIT, TN_MODE_BF16_SPLIT, TN_MODE_FP16_SPLIT = range(5)
TN_MEM_DEVICE, TN_MEM_HOST = 0, 1
MODES = {"fp32": TN_MODE_FP32, "tf32_3m": TN_MODE_TF32_3M, "tf32_split": TN_MODE_TF32_SPLIT,
         "bf16_split": TN_MODE_BF16_SPLIT, "fp16_split": TN_MODE_FP16_SPLIT}


class tn_options(ctypes.Structure):
    _fields_ = [("slice_begin", ctypes.c_int64), ("slice_count", ctypes.c_int64),
                ("no_graph", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("prof_events", ctypes.POINTER(ctypes.c_void_p)), ("prof_first", ctypes.c_int32),
                ("prof_count", ctypes.c_int32), ("slice_batch", ctypes.c_int32),
                ("persistent", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]


_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_vp = ctypes.c_void_p

_lib.tn_create.restype = ctypes.c_int
_lib.tn_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int32, _i32p, _i64p,
                           ctypes.c_int32, _i64p, _i64p, ctypes.c_int32, _i64p]
_lib.tn_set_tensor.restype = ctypes.c_int
_lib.tn_set_tensor.argtypes = [_vp, ctypes.c_int32, _vp, ctypes.c_int32]
_lib.tn_contract.restype = ctypes.c_int
_lib.tn_contract.argtypes = [_vp, _i32p, ctypes.c_int32, _i64p, ctypes.c_int, _vp, ctypes.c_int32,
                             _i64p, _vp]
_lib.tn_contract_ex.restype = ctypes.c_int
_lib.tn_contract_ex.argtypes = [_vp, _i32p, ctypes.c_int32, _i64p, ctypes.c_int,
                                ctypes.POINTER(tn_options), _vp, ctypes.c_int32, _i64p, _vp]
_lib.tn_contract_grad.restype = ctypes.c_int
_lib.tn_contract_grad.argtypes = [_vp, _i32p, ctypes.c_int32, _i64p, ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_double), ctypes.c_int64,
                                  ctypes.POINTER(_vp), _vp]
_lib.tn_contract_grad_ex.restype = ctypes.c_int
_lib.tn_contract_grad_ex.argtypes = [_vp, _i32p, ctypes.c_int32, _i64p, ctypes.c_int, _vp, ctypes.c_int32,
                                     ctypes.c_int64, _vp, ctypes.POINTER(_vp), ctypes.c_uint32,
                                     ctypes.c_int64, ctypes.c_int64, _vp]
_lib.tn_contract_grad_instances.restype = ctypes.c_int
_lib.tn_contract_grad_instances.argtypes = [_vp, _i32p, ctypes.c_int32, _i64p, ctypes.c_int, ctypes.c_int32,
                                            _i64p, _vp, ctypes.c_int32, ctypes.c_int64, _vp,
                                            ctypes.POINTER(_vp), ctypes.c_uint32, ctypes.c_int64,
                                            ctypes.c_int64, _vp]
_lib.tn_contract_instances_keep.restype = ctypes.c_int
_lib.tn_contract_instances_keep.argtypes = [_vp, _i32p, ctypes.c_int, ctypes.c_int32, _i64p, _vp, _vp,
                                            ctypes.c_int32, _vp]
_lib.tn_selftest_flow_timeout.restype = ctypes.c_int
_lib.tn_selftest_flow_timeout.argtypes = [_vp]
_lib.tn_contract_noalloc.restype = ctypes.c_int
_lib.tn_contract_noalloc.argtypes = [_vp, _i32p, ctypes.c_int32, _i64p, _vp, ctypes.c_int32, _i64p,
                                     _vp]
_lib.tn_contract_instances.restype = ctypes.c_int
_lib.tn_contract_instances.argtypes = [_vp, _i32p, ctypes.c_int, ctypes.c_int32, _i64p, _vp, _vp,
                                       ctypes.c_int32, _vp]
_lib.tn_plan_info.restype = ctypes.c_int
_lib.tn_plan_info.argtypes = [_vp, _i32p, ctypes.c_int32, _i64p, ctypes.c_int,
                              ctypes.POINTER(ctypes.c_double)]
_lib.tn_plan_steps.restype = ctypes.c_int
_lib.tn_plan_steps.argtypes = [_vp, _i32p, ctypes.c_int32, _i64p, ctypes.c_int, ctypes.c_int32,
                               _i32p, _i32p, _i32p]
_lib.tn_batch_create.restype = ctypes.c_int
_lib.tn_batch_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int32, ctypes.POINTER(_vp),
                                 ctypes.POINTER(_i32p), ctypes.c_int]
_lib.tn_batch_create_sliced.restype = ctypes.c_int
_lib.tn_batch_create_sliced.argtypes = [ctypes.POINTER(_vp), ctypes.c_int32, ctypes.POINTER(_vp),
                                        ctypes.POINTER(_i32p), _i32p, ctypes.POINTER(_i64p), ctypes.c_int]
_lib.tn_batch_contract.restype = ctypes.c_int
_lib.tn_batch_contract.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int32, _vp]
_lib.tn_batch_destroy.restype = None
_lib.tn_batch_destroy.argtypes = [_vp]
_lib.tn_destroy.restype = None
_lib.tn_destroy.argtypes = [_vp]
_lib.tn_last_error.restype = ctypes.c_char_p
_lib.tn_last_error.argtypes = []
_lib.tn_version.restype = ctypes.c_char_p
_lib.tn_version.argtypes = []

EXPORTS = ["tn_create", "tn_set_tensor", "tn_contract", "tn_contract_ex", "tn_contract_grad",
           "tn_contract_grad_ex", "tn_contract_grad_instances", "tn_contract_instances_keep",
           "tn_selftest_flow_timeout",
           "tn_contract_noalloc", "tn_contract_instances", "tn_autotune", "tn_plan_info", "tn_plan_steps",
           "tn_batch_create", "tn_batch_create_sliced",
           "tn_batch_contract", "tn_batch_destroy", "tn_destroy", "tn_last_error", "tn_version"]


class TNError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"tn status {status}: {msg}")
        self.status = status


def _check(rc: int) -> None:
    if rc != TN_OK:
        raise TNError(rc, tn_last_error())


def _arr(a, dt):
    return np.ascontiguousarray(np.asarray(a, dtype=dt))


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def tn_last_error() -> str:
    return _lib.tn_last_error().decode()


def tn_version() -> str:
    return _lib.tn_version().decode()


def tn_create(dtype: int, labels: Sequence[Sequence[int]], dims: Dict[int, int],
              open_labels: Sequence[int]) -> int:
    ranks = _arr([len(l) for l in labels], np.int32)
    flat = _arr([x for l in labels for x in l] or [0], np.int64)
    ids = sorted(dims)
    lid = _arr(ids or [0], np.int64)
    ldim = _arr([dims[i] for i in ids] or [1], np.int64)
    opn = _arr(list(open_labels) or [0], np.int64)
    h = _vp()
    _check(_lib.tn_create(ctypes.byref(h), dtype, len(labels), _p(ranks, ctypes.c_int32),
                          _p(flat, ctypes.c_int64), len(ids), _p(lid, ctypes.c_int64),
                          _p(ldim, ctypes.c_int64), len(open_labels), _p(opn, ctypes.c_int64)))
    _n_leaves[h.value] = len(labels)
    return h.value


def tn_set_tensor(h: int, v: int, ptr: int, mem: int = TN_MEM_DEVICE) -> None:
    _check(_lib.tn_set_tensor(h, v, ptr, mem))


def _hold(t, stream) -> None:
    """A temporary device tensor read by work queued on ``stream`` (a torch
    stream, or None for the current one): tell the caching allocator, so that
    its memory is not handed out again before that work has run."""
    if stream is not None and getattr(t, "is_cuda", False):
        t.record_stream(stream)


# Flattened trees of recent calls: most callers contract one tree many
# times, and flattening a few hundred pairs costs more than the device work
# of a small network.  An entry is reused only if the call's pair list
# equals the kept tuple copy (tuples are immutable, so any change is seen).
_tree_cache: Dict[int, Tuple[list, np.ndarray]] = {}


# leaves per handle made here: the library reads 2 * (n_tensors - 1) tree
# ids, so a pair list of another length is refused before the call (a short
# one would be read past its end)
_n_leaves: Dict[int, int] = {}


def _tree_of(h: int, pairs):
    n = _n_leaves.get(h)
    if n is not None and len(pairs) != n - 1:
        raise TNError(TN_EINVAL, f"the tree needs n_tensors - 1 = {n - 1} pairs, got {len(pairs)}")
    return _tree(pairs)


def _per_leaf(h: int, seq, name: str) -> None:
    """Arrays with one entry per leaf (gradient pointers, instance strides)
    are read n_tensors entries long by the library."""
    n = _n_leaves.get(h)
    if n is not None and seq is not None and len(seq) != n:
        raise TNError(TN_EINVAL, f"{name} needs n_tensors = {n} entries, got {len(seq)}")


def _tree(pairs):
    if not isinstance(pairs, list):
        return _arr([x for p in pairs for x in p] or [0], np.int32)
    hit = _tree_cache.get(id(pairs))
    if hit is not None and len(hit[0]) == len(pairs):
        # element by element, so that a list of lists (e.g. pairs read from
        # JSON) or of numpy rows is reused like a list of tuples
        try:
            same = all(len(p) == 2 and int(p[0]) == q[0] and int(p[1]) == q[1]
                       for p, q in zip(pairs, hit[0]))
        except (TypeError, ValueError):
            same = False
        if same:
            return hit[1]
    arr = _arr([x for p in pairs for x in p] or [0], np.int32)
    if len(_tree_cache) >= 64:
        _tree_cache.clear()
    _tree_cache[id(pairs)] = ([(int(p[0]), int(p[1])) for p in pairs], arr)
    return arr


def tn_contract_ex(h: int, pairs, sliced, mode: int, out_ptr: int, out_mem: int, exp_ptr: int,
                   stream: int = 0, slice_begin: int = 0, slice_count: int = 0,
                   no_graph: bool = False,
                   prof_events: Optional[Sequence[int]] = None, prof_first: int = 0,
                   slice_batch: int = 0, persistent: bool = False) -> None:
    tr = _tree_of(h, pairs)
    sl = _arr(list(sliced) or [0], np.int64)
    opt = tn_options(slice_begin, slice_count, int(no_graph), 0)
    opt.slice_batch = slice_batch
    opt.persistent = int(bool(persistent))
    if prof_events:
        evs = (ctypes.c_void_p * len(prof_events))(*prof_events)
        opt.prof_events = ctypes.cast(evs, ctypes.POINTER(ctypes.c_void_p))
        opt.prof_first = prof_first
        opt.prof_count = len(prof_events) - 1
    _check(_lib.tn_contract_ex(h, _p(tr, ctypes.c_int32), len(sliced), _p(sl, ctypes.c_int64), mode,
                               ctypes.byref(opt), out_ptr, out_mem,
                               ctypes.cast(exp_ptr, _i64p), stream))


def tn_contract(h: int, pairs, sliced, mode: int, out_ptr: int, out_mem: int, exp_ptr: int,
                stream: int = 0) -> None:
    tr = _tree_of(h, pairs)
    sl = _arr(list(sliced) or [0], np.int64)
    _check(_lib.tn_contract(h, _p(tr, ctypes.c_int32), len(sliced), _p(sl, ctypes.c_int64), mode,
                            out_ptr, out_mem, ctypes.cast(exp_ptr, _i64p), stream))


def tn_contract_grad(h: int, pairs, sliced, mode: int, adjoint: np.ndarray, adj_exp2: int,
                     grad_ptrs: Sequence[int], stream: int = 0) -> None:
    tr = _tree_of(h, pairs)
    _per_leaf(h, grad_ptrs, "grad_ptrs")
    sl = _arr(list(sliced) or [0], np.int64)
    adj = np.ascontiguousarray(adjoint)
    gp = (_vp * len(grad_ptrs))(*[g or None for g in grad_ptrs])
    _check(_lib.tn_contract_grad(h, _p(tr, ctypes.c_int32), len(sliced), _p(sl, ctypes.c_int64),
                                 mode, adj.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 int(adj_exp2), gp, stream))


TN_GRAD_ACCUMULATE = 1
TN_GRAD_KEPT_FORWARD = 2


def tn_contract_grad_ex(h: int, pairs, sliced, mode: int, adj_ptr: int, adj_mem: int, adj_exp2: int,
                        adj_exp2_dev: int, grad_ptrs: Sequence[int], flags: int = 0,
                        stream: int = 0, slice_begin: int = 0, slice_count: int = 0) -> None:
    """tn_contract_grad with a host or device adjoint (pointer to FP64) and
    optional accumulation (flags = TN_GRAD_ACCUMULATE)."""
    tr = _tree_of(h, pairs)
    _per_leaf(h, grad_ptrs, "grad_ptrs")
    sl = _arr(list(sliced) or [0], np.int64)
    gp = (_vp * len(grad_ptrs))(*[g or None for g in grad_ptrs])
    _check(_lib.tn_contract_grad_ex(h, _p(tr, ctypes.c_int32), len(sliced), _p(sl, ctypes.c_int64), mode,
                                    adj_ptr, adj_mem, int(adj_exp2), adj_exp2_dev or None, gp, flags,
                                    int(slice_begin), int(slice_count), stream))


def tn_contract_grad_instances(h: int, pairs, sliced, mode: int, n_inst: int, leaf_inst_stride,
                               adj_ptr: int, adj_mem: int, adj_exp2: int, adj_exp2_dev: int,
                               grad_ptrs: Sequence[int], flags: int = 0, stream: int = 0,
                               slice_begin: int = 0, slice_count: int = 0) -> None:
    """Reverse sweep of n_inst copies (leaf v of copy i at + i *
    leaf_inst_stride[v] elements; None: all shared) in one launch sequence."""
    tr = _tree_of(h, pairs)
    _per_leaf(h, grad_ptrs, "grad_ptrs")
    _per_leaf(h, leaf_inst_stride, "leaf_inst_stride")
    sl = _arr(list(sliced) or [0], np.int64)
    st = _arr(list(leaf_inst_stride), np.int64) if leaf_inst_stride is not None else None
    gp = (_vp * len(grad_ptrs))(*[g or None for g in grad_ptrs])
    _check(_lib.tn_contract_grad_instances(h, _p(tr, ctypes.c_int32), len(sliced), _p(sl, ctypes.c_int64),
                                           mode, n_inst, _p(st, ctypes.c_int64) if st is not None else None,
                                           adj_ptr, adj_mem, int(adj_exp2), adj_exp2_dev or None, gp, flags,
                                           int(slice_begin), int(slice_count), stream))


def tn_selftest_flow_timeout(stream: int = 0) -> int:
    """Failure-detection self-test: the status of a dataflow wait that is
    made to run out (TN_ETIMEOUT expected).  Does not raise for it."""
    return int(_lib.tn_selftest_flow_timeout(stream))


def tn_contract_noalloc(h: int, pairs, sliced, out_ptr: int, out_mem: int, exp_ptr: int,
                        stream: int = 0) -> None:
    """The contraction without any device allocation (fixed 8 MiB scratch)."""
    tr = _tree_of(h, pairs)
    sl = _arr(list(sliced) or [0], np.int64)
    _check(_lib.tn_contract_noalloc(h, _p(tr, ctypes.c_int32), len(sliced), _p(sl, ctypes.c_int64),
                                    out_ptr, out_mem, ctypes.cast(exp_ptr, _i64p), stream))


def tn_autotune(h: int, pairs, sliced, mode: int, reps: int = 3, stream: int = 0) -> List[int]:
    """Time every candidate kernel per node and keep the fastest in the
    cached plan; returns the per-node choice (0 untuned, 1..4 and 6 tile shape,
    8 tensor core, 9 tensor core with 128-column tiles)."""
    tr = _tree_of(h, pairs)
    sl = _arr(list(sliced) or [0], np.int64)
    ch = np.zeros(max(len(pairs), 1), dtype=np.int32)
    _check(_lib.tn_autotune(h, _p(tr, ctypes.c_int32), len(sliced), _p(sl, ctypes.c_int64), mode, reps,
                            _p(ch, ctypes.c_int32), stream))
    return ch[:len(pairs)].tolist()


def tn_plan_info(h: int, pairs, sliced, mode: int = TN_MODE_FP32) -> Dict[str, float]:
    tr = _tree_of(h, pairs)
    sl = _arr(list(sliced) or [0], np.int64)
    out = np.zeros(8, dtype=np.float64)
    _check(_lib.tn_plan_info(h, _p(tr, ctypes.c_int32), len(sliced), _p(sl, ctypes.c_int64), mode,
                             _p(out, ctypes.c_double)))
    keys = ["W", "C", "d_sliced", "flops", "ws_bytes", "n_tiled", "n_tensor_core", "n_generic"]
    return dict(zip(keys, out.tolist()))


def tn_plan_steps(h: int, pairs, sliced, mode: int = TN_MODE_FP32):
    """Launch steps of the per-slice sequence: list of dicts
    (wave, kind, cfg, launches, nodes)."""
    tr = _tree_of(h, pairs)
    sl = _arr(list(sliced) or [0], np.int64)
    ns = ctypes.c_int32(0)
    _check(_lib.tn_plan_steps(h, _p(tr, ctypes.c_int32), len(sliced), _p(sl, ctypes.c_int64), mode,
                              0, ctypes.byref(ns), None, None))
    n = ns.value
    info = np.zeros(5 * max(n, 1), dtype=np.int32)
    nodes = np.zeros(max(len(pairs), 1), dtype=np.int32)
    _check(_lib.tn_plan_steps(h, _p(tr, ctypes.c_int32), len(sliced), _p(sl, ctypes.c_int64), mode,
                              n, ctypes.byref(ns), _p(info, ctypes.c_int32), _p(nodes, ctypes.c_int32)))
    out, pos = [], 0
    for s in range(n):
        w, kind, cfg, cnt, nl = info[5 * s:5 * s + 5].tolist()
        out.append({"wave": bool(w), "kind": kind, "cfg": cfg, "launches": nl,
                    "nodes": nodes[pos:pos + cnt].tolist()})
        pos += cnt
    return out


def tn_destroy(h: int) -> None:
    _n_leaves.pop(h, None)
    _lib.tn_destroy(h)


class TensorNetwork:
    """A network handle bound to torch leaf tensors.

    ``tensors`` are torch tensors (complex64 or float32), on the GPU for
    device mode or in (pinned) host memory for host mode.  The handle
    borrows them: keep them alive while contractions that read them run.
    """

    def __init__(self, labels, dims, open_labels, tensors=None, complex_=True):
        import torch  # noqa: F401  (device memory, streams)
        self.dtype = TN_C64 if complex_ else TN_R32
        self.labels = [list(l) for l in labels]
        self.dims = dict(dims)
        self.open = list(open_labels)
        self.h = tn_create(self.dtype, self.labels, self.dims, self.open)
        self._keep: List = []
        if tensors is not None:
            self.set_tensors(tensors)

    def close(self):
        if self.h:
            tn_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tensors(self, tensors) -> None:
        import torch
        want = torch.complex64 if self.dtype == TN_C64 else torch.float32
        if len(tensors) > len(self.labels):
            raise TNError(TN_EINVAL, f"{len(tensors)} tensors for {len(self.labels)} leaves")
        for v, t in enumerate(tensors):
            # every call reads a whole leaf (stacked copies may hold more)
            if t.numel() < self._leaf_numel(v):
                raise TNError(TN_EINVAL, f"leaf {v}: {t.numel()} elements, the leaf has {self._leaf_numel(v)}")
        self._keep = []
        attached = getattr(self, "_attached", None) or [None] * len(tensors)
        for v, t in enumerate(tensors):
            if t.dtype != want:
                raise TypeError(f"leaf {v}: dtype {t.dtype}, expected {want}")
            if not t.is_contiguous():
                raise ValueError(f"leaf {v} must be contiguous")
            mem = TN_MEM_DEVICE if t.is_cuda else TN_MEM_HOST
            self._keep.append(t)
            key = (t.data_ptr(), mem)
            if attached[v] != key:  # unchanged pointers need no call
                tn_set_tensor(self.h, v, key[0], mem)
                attached[v] = key
        self._attached = attached

    @property
    def out_shape(self) -> Tuple[int, ...]:
        return tuple(self.dims[l] for l in self.open)

    # The library sees plain pointers: the extents it will read or write are
    # checked here, before any call, so that an undersized buffer raises
    # instead of being accessed out of bounds.

    def _leaf_numel(self, v: int) -> int:
        n = 1
        for l in self.labels[v]:
            n *= int(self.dims[l])
        return n

    def _extent(self, v: int, n_inst: int, strides) -> int:
        """Elements from leaf v's pointer that n_inst copies touch."""
        st = int(strides[v]) if strides is not None else 0
        return max(int(n_inst) - 1, 0) * st + self._leaf_numel(v)

    def _check_strides(self, n_inst: int, strides) -> None:
        if strides is not None and len(strides) != len(self.labels):
            raise TNError(TN_EINVAL, f"leaf_inst_stride needs {len(self.labels)} entries, got {len(strides)}")
        for v, t in enumerate(self._keep):
            if strides is not None and int(strides[v]) < 0:
                raise TNError(TN_EINVAL, f"leaf {v}: negative instance stride")
            need = self._extent(v, n_inst, strides)
            if t.numel() < need:
                raise TNError(TN_EINVAL, f"leaf {v}: {t.numel()} elements attached, "
                                         f"{n_inst} copies read {need}")

    def _check_grads(self, grads, n_inst: int = 1, strides=None) -> None:
        import torch
        if len(grads) != len(self.labels):
            raise TNError(TN_EINVAL, f"grads needs {len(self.labels)} entries (None to skip), got {len(grads)}")
        want = torch.complex64 if self.dtype == TN_C64 else torch.float32
        for v, g in enumerate(grads):
            if g is None:
                continue
            if g.dtype != want:
                raise TypeError(f"grads[{v}]: dtype {g.dtype}, expected {want}")
            if not g.is_cuda or not g.is_contiguous():
                raise TNError(TN_EINVAL, f"grads[{v}] must be a contiguous CUDA tensor")
            need = self._extent(v, n_inst, strides)
            if g.numel() < need:
                raise TNError(TN_EINVAL, f"grads[{v}]: {g.numel()} elements, {need} written")

    def contract(self, pairs, sliced=(), mode="fp32", out=None, out_exp=None, stream=None,
                 slice_begin=0, slice_count=0, no_graph=False,
                 prof_events=None, prof_first=0, slice_batch=0, persistent=False):
        """Return (mantissa, exp2) torch tensors; value = mantissa * 2**exp2.

        Device outputs by default (asynchronous on ``stream``); pass CPU
        ``out``/``out_exp`` tensors to receive host outputs (synchronous).
        ``persistent``: the whole call (every node of every slice) in one
        persistent dataflow launch (FP32 on the CUDA cores)."""
        import torch
        m = MODES[mode] if isinstance(mode, str) else int(mode)
        dev = torch.device("cuda")
        odt = torch.complex128 if self.dtype == TN_C64 else torch.float64
        if out is None:
            out = torch.empty(self.out_shape, dtype=odt, device=dev)
        if out_exp is None:
            out_exp = torch.empty((), dtype=torch.int64, device=out.device)
        if out.dtype != odt or out_exp.dtype != torch.int64:
            raise TypeError(f"out must be {odt} and out_exp torch.int64")
        n_out = math.prod(self.out_shape)
        if out.numel() != n_out or not out.is_contiguous() or out_exp.numel() != 1:
            raise TNError(TN_EINVAL, f"out must be a contiguous tensor of {n_out} elements, out_exp a scalar")
        if out_exp.is_cuda != out.is_cuda:
            raise TNError(TN_EINVAL, "out and out_exp must both be device or both host tensors")
        mem = TN_MEM_DEVICE if out.is_cuda else TN_MEM_HOST
        s = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
        evp = [e.cuda_event for e in prof_events] if prof_events else None
        tn_contract_ex(self.h, pairs, sliced, m, out.data_ptr(), mem, out_exp.data_ptr(), s,
                       slice_begin, slice_count, no_graph, evp, prof_first, slice_batch, persistent)
        return out, out_exp

    def grad(self, pairs, sliced, mode, adjoint, adj_exp2=0, grads=None, stream=None,
             accumulate=False, slice_begin=0, slice_count=0):
        """Leaf gradients conj(d value / d T_v) * adjoint, summed over slices
        and contracted over the open labels (torch's convention).

        ``adjoint``: shaped like the output, FP64 (complex128 for complex
        networks): a host array, or a CUDA torch tensor (read in stream
        order, no host synchronisation).  ``adj_exp2``: an int, or (with a
        CUDA adjoint) a CUDA int64 scalar tensor; the adjoint is
        adjoint * 2**adj_exp2.  ``grads``: torch tensors shaped like the
        leaves (device, leaf dtype; None entries are skipped), or None to
        allocate.  ``accumulate``: add into ``grads`` instead of overwriting.
        ``slice_begin``/``slice_count``: sweep only those slices (count 0:
        all).  Returns the list of gradient tensors (asynchronous)."""
        import torch
        m = MODES[mode] if isinstance(mode, str) else int(mode)
        cplx = self.dtype == TN_C64
        n_out = math.prod(self.out_shape)
        keep = None
        if isinstance(adjoint, torch.Tensor) and adjoint.is_cuda:
            want = torch.complex128 if cplx else torch.float64
            if adjoint.dtype != want:
                raise TypeError(f"adjoint dtype {adjoint.dtype}, expected {want}")
            if adjoint.numel() != n_out:
                raise ValueError("adjoint shape does not match the output")
            keep = adjoint.contiguous()
            adj_ptr, adj_mem = keep.data_ptr(), TN_MEM_DEVICE
        else:
            if isinstance(adjoint, torch.Tensor):
                adjoint = adjoint.detach().numpy()
            adj = np.ascontiguousarray(np.asarray(adjoint, dtype=np.complex128 if cplx else np.float64))
            if adj.size != n_out:
                raise ValueError("adjoint shape does not match the output")
            keep = adj
            adj_ptr, adj_mem = adj.ctypes.data, TN_MEM_HOST
        exp_host, exp_dev = 0, 0
        if isinstance(adj_exp2, torch.Tensor):
            if adj_mem != TN_MEM_DEVICE or not adj_exp2.is_cuda or adj_exp2.dtype != torch.int64:
                raise TypeError("a tensor adj_exp2 must be a CUDA int64 scalar, with a CUDA adjoint")
            if adj_exp2.numel() != 1:
                raise TNError(TN_EINVAL, "a tensor adj_exp2 must hold one exponent")
            exp_dev = adj_exp2.data_ptr()
        else:
            exp_host = int(adj_exp2)
        if grads is None:
            grads = [torch.empty_like(t, device="cuda") for t in self._keep]
        self._check_grads(grads)
        if keep is not adjoint:
            _hold(keep, stream)
        s = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
        tn_contract_grad_ex(self.h, pairs, sliced, m, adj_ptr, adj_mem, exp_host, exp_dev,
                            [g.data_ptr() if g is not None else 0 for g in grads],
                            TN_GRAD_ACCUMULATE if accumulate else 0, s, slice_begin, slice_count)
        self._grad_epoch = getattr(self, "_grad_epoch", 0) + 1
        del keep
        return grads

    def contract_instances_keep(self, pairs, mode, n_inst, leaf_inst_stride=None, stream=None):
        """contract_instances computed in the reverse sweep's state with the
        intermediates kept (tn_contract_instances_keep).  Returns (mantissa
        (n_inst, 2) float64, exp2 (n_inst,)) device tensors and a token for
        grad_instances(kept_forward=token)."""
        import torch
        m = MODES[mode] if isinstance(mode, str) else int(mode)
        self._check_strides(n_inst, leaf_inst_stride)
        out = torch.empty((n_inst, 2), dtype=torch.float64, device="cuda")
        ex = torch.empty(n_inst, dtype=torch.int64, device="cuda")
        st = _arr(list(leaf_inst_stride), np.int64) if leaf_inst_stride is not None else None
        s = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
        _check(_lib.tn_contract_instances_keep(self.h, _p(_tree_of(self.h, pairs), ctypes.c_int32), m, n_inst,
                                               _p(st, ctypes.c_int64) if st is not None else None,
                                               out.data_ptr(), ex.data_ptr(), TN_MEM_DEVICE, s))
        self._grad_epoch = getattr(self, "_grad_epoch", 0) + 1
        return out, ex, self._grad_epoch

    def grad_instances(self, pairs, sliced, mode, n_inst, leaf_inst_stride, adjoint, adj_exp2=0,
                       grads=None, stream=None, accumulate=False, kept_forward=None,
                       slice_begin=0, slice_count=0):
        """Reverse sweep of n_inst copies in one launch sequence (see
        tn_contract_grad_instances).  ``adjoint``: [n_inst, *output shape]
        FP64 (complex128 for complex networks), host array or CUDA tensor;
        ``adj_exp2``: int, or a CUDA int64 tensor of n_inst exponents (CUDA
        adjoint only).  ``grads``: per leaf a tensor shaped like the leaf
        (shared leaves: summed over the copies) or like the stacked copies
        (varying leaves), or None to skip.  ``kept_forward``: the token of a
        contract_instances_keep call; when no other gradient call ran on this
        handle since, the sweep reuses that forward (TN_GRAD_KEPT_FORWARD).
        Returns ``grads``."""
        import torch
        m = MODES[mode] if isinstance(mode, str) else int(mode)
        self._check_strides(n_inst, leaf_inst_stride)
        cplx = self.dtype == TN_C64
        n_out = math.prod(self.out_shape)
        if isinstance(adjoint, torch.Tensor) and adjoint.is_cuda:
            want = torch.complex128 if cplx else torch.float64
            if adjoint.dtype != want:
                raise TypeError(f"adjoint dtype {adjoint.dtype}, expected {want}")
            if adjoint.numel() != n_out * n_inst:
                raise ValueError("adjoint must hold n_inst outputs")
            keep = adjoint.contiguous()
            adj_ptr, adj_mem = keep.data_ptr(), TN_MEM_DEVICE
        else:
            if isinstance(adjoint, torch.Tensor):
                adjoint = adjoint.detach().numpy()
            keep = np.ascontiguousarray(np.asarray(adjoint, dtype=np.complex128 if cplx else np.float64))
            if keep.size != n_out * n_inst:
                raise ValueError("adjoint must hold n_inst outputs")
            adj_ptr, adj_mem = keep.ctypes.data, TN_MEM_HOST
        exp_host, exp_dev = 0, 0
        if isinstance(adj_exp2, torch.Tensor):
            if adj_mem != TN_MEM_DEVICE or not adj_exp2.is_cuda or adj_exp2.dtype != torch.int64 \
                    or adj_exp2.numel() != n_inst:
                raise TypeError("a tensor adj_exp2 must hold n_inst CUDA int64s, with a CUDA adjoint")
            exp_keep = adj_exp2.contiguous()
            if exp_keep is not adj_exp2:
                _hold(exp_keep, stream)
            exp_dev = exp_keep.data_ptr()
        else:
            exp_host = int(adj_exp2)
        if grads is None:  # attached tensors: stacked copies for varying leaves
            grads = [torch.empty_like(t, device="cuda") for t in self._keep]
        self._check_grads(grads, n_inst, leaf_inst_stride)
        if keep is not adjoint:
            _hold(keep, stream)
        s = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
        flags = TN_GRAD_ACCUMULATE if accumulate else 0
        if kept_forward is not None and kept_forward == getattr(self, "_grad_epoch", 0) and not sliced:
            flags |= TN_GRAD_KEPT_FORWARD
        tn_contract_grad_instances(self.h, pairs, sliced, m, n_inst, leaf_inst_stride, adj_ptr, adj_mem,
                                   exp_host, exp_dev, [g.data_ptr() if g is not None else 0 for g in grads],
                                   flags, s, slice_begin, slice_count)
        if not flags & TN_GRAD_KEPT_FORWARD:  # the sweep's workspace now holds another forward
            self._grad_epoch = getattr(self, "_grad_epoch", 0) + 1
        del keep
        return grads

    def autotune(self, pairs, sliced=(), mode="fp32", reps=3, stream=None):
        """Per-node kernel choice by measurement (see tn_autotune)."""
        import torch
        m = MODES[mode] if isinstance(mode, str) else int(mode)
        s = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
        return tn_autotune(self.h, pairs, sliced, m, reps, s)

    def plan_info(self, pairs, sliced=(), mode="fp32"):
        m = MODES[mode] if isinstance(mode, str) else int(mode)
        return tn_plan_info(self.h, pairs, sliced, m)

    def contract_instances(self, pairs, mode, n_inst, leaf_inst_stride=None, stream=None):
        """n_inst copies of this scalar network in one launch sequence; copy i
        reads leaf v at (attached pointer) + i * leaf_inst_stride[v] elements.
        Returns device tensors (mantissa (n_inst, 2) float64, exp2 (n_inst,))."""
        import torch
        m = MODES[mode] if isinstance(mode, str) else int(mode)
        self._check_strides(n_inst, leaf_inst_stride)
        out = torch.empty((n_inst, 2), dtype=torch.float64, device="cuda")
        ex = torch.empty(n_inst, dtype=torch.int64, device="cuda")
        strides = None
        if leaf_inst_stride is not None:
            self._strides = _arr(list(leaf_inst_stride), np.int64)
            strides = _p(self._strides, ctypes.c_int64)
        s = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
        tr = _tree_of(self.h, pairs)
        _check(_lib.tn_contract_instances(self.h, _p(tr, ctypes.c_int32), m, n_inst, strides,
                                          out.data_ptr(), ex.data_ptr(), TN_MEM_DEVICE, s))
        return out, ex

    def plan_steps(self, pairs, sliced=(), mode="fp32"):
        m = MODES[mode] if isinstance(mode, str) else int(mode)
        return tn_plan_steps(self.h, pairs, sliced, m)


class Batch:
    """Many scalar networks (TensorNetwork handles, each with its tree) run
    as one captured launch sequence.  ``sliced`` (optional) gives each
    network's sliced labels (empty: unsliced); sliced networks run their
    slice loops after the merged forest (tn_batch_create_sliced).
    ``contract`` returns (mantissa, exp2, latency_ns) device tensors:
    mantissa (n, 2) float64, exp2 (n,) int64, per-network completion time
    since the batch started."""

    def __init__(self, networks, trees, mode="fp32", sliced=None):
        import torch  # noqa: F401
        self.nets = list(networks)
        m = MODES[mode] if isinstance(mode, str) else int(mode)
        if len(trees) != len(self.nets):
            raise TNError(TN_EINVAL, "one tree per network")
        self._trees = [_tree_of(n.h, t) for n, t in zip(self.nets, trees)]
        hs = (_vp * len(self.nets))(*[n.h for n in self.nets])
        tp = (_i32p * len(self.nets))(*[t.ctypes.data_as(_i32p) for t in self._trees])
        h = _vp()
        if sliced is None or not any(len(s) for s in sliced):
            _check(_lib.tn_batch_create(ctypes.byref(h), len(self.nets), hs, tp, m))
        else:
            if len(sliced) != len(self.nets):
                raise TNError(TN_EINVAL, "one sliced-label list per network")
            self._sliced = [_arr(list(s) or [0], np.int64) for s in sliced]
            ns = _arr([len(s) for s in sliced], np.int32)
            sp = (_i64p * len(self.nets))(*[a.ctypes.data_as(_i64p) for a in self._sliced])
            _check(_lib.tn_batch_create_sliced(ctypes.byref(h), len(self.nets), hs, tp,
                                               ns.ctypes.data_as(_i32p), sp, m))
        self.h = h.value

    def contract(self, stream=None):
        import torch
        n = len(self.nets)
        out = torch.empty((n, 2), dtype=torch.float64, device="cuda")
        ex = torch.empty(n, dtype=torch.int64, device="cuda")
        lat = torch.empty(n, dtype=torch.int64, device="cuda")
        s = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
        _check(_lib.tn_batch_contract(self.h, out.data_ptr(), ex.data_ptr(), lat.data_ptr(),
                                      TN_MEM_DEVICE, s))
        return out, ex, lat

    def close(self):
        if self.h:
            _lib.tn_batch_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
