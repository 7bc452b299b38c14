"""Checkpoint and resume of a sliced contraction.

Slices are independent contractions whose values are summed (Sec. 4.7.1),
so a long sliced run can be cut into consecutive blocks of the slice range.
Each finished block leaves a partial result -- an FP64 mantissa (scalar or
open-output tensor) m and an int64 power-of-two exponent e, value m * 2^e --
which is written to a checkpoint directory before the next block starts.  A
resumed run reads the directory and contracts only the blocks still missing.
The partials are folded in block order with exponents aligned to the
largest one, so the result does not depend on where (or whether) the run
was interrupted.

The contraction of one block is a callable ``contract_block(begin, count)
-> (mantissa, exp2)``; ``library_block`` builds it from a network handle of
the binding (device contraction of that slice range, result copied to the
host).
"""
from __future__ import annotations

import os
from typing import Callable, List, Optional, Tuple

import numpy as np

# exponent of an exactly-zero partial: never the common exponent
ZERO_EXP = -(1 << 60)


def blocks(d_sliced: int, block: int) -> List[Tuple[int, int]]:
    """The (begin, count) blocks covering [0, d_sliced) in order."""
    if d_sliced < 1 or block < 1:
        raise ValueError("need d_sliced >= 1 and block >= 1")
    return [(b, min(block, d_sliced - b)) for b in range(0, d_sliced, block)]


def fold(partials) -> Tuple[np.ndarray, int]:
    """Sum of (mantissa, exp2) partials, in the given order, as one
    (mantissa, exp2): every mantissa is scaled exactly by a power of two to
    the largest exponent among the non-zero partials, then added in FP64."""
    parts = [(np.asarray(m), int(e)) for m, e in partials]
    if not parts:
        raise ValueError("nothing to fold")
    live = [e for m, e in parts if np.any(m != 0)]
    if not live:
        return np.zeros_like(parts[0][0]), 0
    e_max = max(live)
    acc = np.zeros_like(parts[0][0])
    for m, e in parts:
        if np.any(m != 0):
            # contributions more than 1100 binades down underflow, as in FP64
            shift = max(e - e_max, -1100)
            if np.iscomplexobj(m):
                acc = acc + (np.ldexp(m.real, shift) + 1j * np.ldexp(m.imag, shift))
            else:
                acc = acc + np.ldexp(m, shift)
    return acc, e_max


def _fsync_dir(path: str) -> None:
    try:
        fd = os.open(path, os.O_RDONLY)
    except OSError:
        return
    try:
        os.fsync(fd)
    except OSError:
        pass
    finally:
        os.close(fd)


class SliceCheckpoint:
    """The finished blocks of one sliced contraction, kept in the directory
    ``path``: ``meta.json`` names the problem (and, once a block is recorded,
    the partials' shape), and each finished block is one
    small ``block_<i>.npz`` written atomically (a rename), so recording costs
    the same for the first block and the ten-thousandth.  ``key`` names the
    problem (network, tree, sliced labels, mode): a directory written for
    another key, slice count or block size is refused, never mixed in."""

    def __init__(self, path: str, key: str, d_sliced: int, block: int):
        import json
        self.path, self.key, self.d_sliced, self.block = path, str(key), int(d_sliced), int(block)
        self.done: dict = {}  # block index -> (mantissa, exp2)
        self.shape = None     # mantissa shape, recorded with the first block
        meta = {"key": self.key, "d_sliced": self.d_sliced, "block": self.block}
        self._mpath = mpath = os.path.join(path, "meta.json")
        if os.path.exists(mpath):
            with open(mpath) as f:
                have = json.load(f)
            shape = have.pop("shape", None)
            if have != meta:
                raise ValueError(f"checkpoint {path} belongs to {have}, not {meta}")
            self.shape = tuple(shape) if shape is not None else None
            n_blocks = len(blocks(self.d_sliced, self.block))
            for name in sorted(os.listdir(path)):
                if not (name.startswith("block_") and name.endswith(".npz")):
                    continue
                # a damaged or foreign file counts as a missing block: that
                # block is contracted again instead of failing the run
                try:
                    with np.load(os.path.join(path, name), allow_pickle=False) as z:
                        idx, m, e = int(z["index"]), np.array(z["mantissa"]), int(z["exp2"])
                except Exception:
                    continue
                if not (0 <= idx < n_blocks) or name != f"block_{idx}.npz":
                    continue
                if self.shape is None or m.shape != self.shape:
                    continue
                self.done[idx] = (m, e)
        else:
            os.makedirs(path, exist_ok=True)
            self._write_meta(meta)
        self._meta = meta

    def _write_meta(self, meta: dict) -> None:
        import json
        tmp = self._mpath + ".tmp"
        with open(tmp, "w") as f:
            json.dump(meta, f)
            f.flush()
            os.fsync(f.fileno())
        os.replace(tmp, self._mpath)
        _fsync_dir(self.path)

    def record(self, index: int, mantissa, exp2: int) -> None:
        m = np.array(mantissa)
        if self.shape is None:
            # the first recorded block fixes the partials' shape; files of
            # another shape found later are not this problem's
            self.shape = m.shape
            self._write_meta(dict(self._meta, shape=list(m.shape)))
        elif m.shape != self.shape:
            raise ValueError(f"block {index}: mantissa shape {m.shape}, expected {self.shape}")
        self.done[int(index)] = (m, int(exp2))
        final = os.path.join(self.path, f"block_{int(index)}.npz")
        tmp = os.path.join(self.path, f"tmp_{int(index)}.npz")
        # written, flushed to the disk, then renamed (and the rename made
        # durable): a crash leaves either no file or a complete one
        with open(tmp, "wb") as f:
            np.savez(f, index=np.array(int(index)), mantissa=np.array(mantissa), exp2=np.array(int(exp2)))
            f.flush()
            os.fsync(f.fileno())
        os.replace(tmp, final)
        _fsync_dir(self.path)


def run(contract_block: Callable[[int, int], Tuple[np.ndarray, int]], d_sliced: int, block: int,
        path: str, key: str, on_block: Optional[Callable[[int], None]] = None) -> Tuple[np.ndarray, int]:
    """Contract every block of [0, d_sliced) not yet in the checkpoint
    directory ``path`` (recording each as it finishes) and return the folded
    (mantissa, exp2) of all of them.  ``on_block(i)`` is called after block
    i is recorded."""
    ck = SliceCheckpoint(path, key, d_sliced, block)
    bl = blocks(d_sliced, block)
    for i, (b, c) in enumerate(bl):
        if i in ck.done:
            continue
        m, e = contract_block(b, c)
        m = np.asarray(m)
        ck.record(i, m, ZERO_EXP if not np.any(m != 0) else int(e))
        if on_block is not None:
            on_block(i)
    return fold(ck.done[i] for i in range(len(bl)))


def library_block(tnw, pairs, sliced, mode: str = "fp32"):
    """``contract_block`` for a network handle of the binding: the slice
    range [begin, begin + count) contracted on the device, the
    (mantissa, exp2) copied to the host."""
    def contract_block(begin: int, count: int):
        m, e = tnw.contract(pairs, sliced, mode, slice_begin=begin, slice_count=count)
        return m.cpu().numpy(), int(e.cpu())
    return contract_block
