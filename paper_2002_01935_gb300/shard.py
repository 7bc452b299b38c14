"""Slice sharding across ranks.

Slices are independent contractions whose results are summed (Sec. 4.7.1):
rank r of a world of size P contracts one contiguous block of the slice
range on its own GPU, and the partial results -- each an FP64 mantissa
tensor m with an int64 power-of-two exponent e, value m * 2^e -- are
combined with one exchange: the largest exponent over the ranks, then the
sum of the mantissas rescaled to it.  The same two collectives serve any
torch.distributed backend (NCCL between GPUs, gloo on the host).
"""
from __future__ import annotations

from typing import Tuple

# exponent given to a partial result that is exactly zero, so that it never
# sets the common exponent (any real exponent is far above it)
ZERO_EXP = -(1 << 60)


def slice_range(rank: int, world: int, d_sliced: int) -> Tuple[int, int]:
    """Contiguous block [begin, begin + count) of the slice range owned by
    ``rank``; blocks differ in length by at most one, the first
    ``d_sliced % world`` ranks take the longer ones, and every slice is
    owned exactly once (a rank may own none when d_sliced < world)."""
    if world < 1 or not 0 <= rank < world or d_sliced < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, d_sliced >= 0")
    base, extra = divmod(d_sliced, world)
    begin = rank * base + min(rank, extra)
    return begin, base + (1 if rank < extra else 0)


def combine(mantissa, exp2: int, group=None):
    """Sum the partial results of all ranks: returns (mantissa, exp2) with
    the same meaning on every rank.  ``mantissa`` is a float64 tensor (any
    shape, the same on every rank), on the device the backend expects."""
    import torch
    import torch.distributed as dist

    if mantissa.dtype not in (torch.float64, torch.complex128):
        raise TypeError("mantissa must be float64 or complex128")
    m = torch.view_as_real(mantissa) if mantissa.is_complex() else mantissa
    e_local = ZERO_EXP if not bool(torch.any(m != 0)) else int(exp2)
    e = torch.tensor([e_local], dtype=torch.int64, device=m.device)
    dist.all_reduce(e, op=dist.ReduceOp.MAX, group=group)
    e_max = int(e.item())
    if e_max == ZERO_EXP:
        return mantissa.clone(), 0
    # exact rescaling by a power of two (ldexp); contributions more than
    # 1100 binades below the largest underflow to zero, as in FP64 itself
    shift = max(e_local - e_max, -1100) if e_local != ZERO_EXP else -1100
    part = torch.ldexp(m, torch.tensor(float(shift), dtype=torch.float64, device=m.device))
    dist.all_reduce(part, op=dist.ReduceOp.SUM, group=group)
    out = torch.view_as_complex(part) if mantissa.is_complex() else part
    return out, e_max


def combine_grads(grads, group=None):
    """Sum gradient buffers over the ranks, in place: each rank swept its own
    block of slices (tn_contract_grad_ex with a slice range) or its own
    networks (e.g. a block of bitstrings), and the gradient of the whole sum
    is the sum of the parts -- one all-reduce of all buffers together.  The
    sum is taken in float64 (rounded once back to the buffers' dtype), so
    that it does not depend on the backend's reduction order beyond FP64
    rounding.  ``grads``: tensors (None entries are skipped), on the device
    the backend expects."""
    import torch
    import torch.distributed as dist

    live = [g for g in grads if g is not None]
    if not live:
        return grads
    if not all(g.is_contiguous() for g in live):
        raise ValueError("gradient buffers must be contiguous")
    parts = [torch.view_as_real(g).reshape(-1) if g.is_complex() else g.reshape(-1) for g in live]
    flat = torch.cat([p.to(torch.float64) for p in parts])
    dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    off = 0
    for g, p in zip(live, parts):
        n = p.numel()
        src = flat[off:off + n].to(p.dtype)
        if g.is_complex():
            torch.view_as_real(g).reshape(-1).copy_(src)
        else:
            g.reshape(-1).copy_(src)
        off += n
    return grads
