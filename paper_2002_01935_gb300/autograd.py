"""torch.autograd.Function around the contraction and its reverse sweep.

``contract(tnw, pairs, sliced, mode, *leaves)`` returns the network value
as a complex128 / float64 torch tensor (mantissa * 2^exp2 folded in; use
``TensorNetwork.contract`` directly for values beyond the FP64 range).  Its
backward calls tn_contract_grad: every leaf's gradient is computed by the
hand-written reverse tree sweep on the GPU (per-slice recomputation of the
forward intermediates), with the holomorphic convention of torch:
grad_leaf = conj(d value / d leaf) * grad_output.
"""
from __future__ import annotations

import torch

from . import binding


class _Contract(torch.autograd.Function):
    @staticmethod
    def forward(ctx, tnw, pairs, sliced, mode, *leaves):
        leaves = [t.detach().contiguous() for t in leaves]
        tnw.set_tensors(leaves)
        m, e = tnw.contract(pairs, sliced, mode)
        value = m * torch.pow(torch.tensor(2.0, dtype=torch.float64, device=m.device), e.double())
        ctx.tnw, ctx.pairs, ctx.sliced, ctx.mode = tnw, pairs, sliced, mode
        ctx.save_for_backward(*leaves)
        return value

    @staticmethod
    def backward(ctx, grad_out):
        # one handle may serve several forward calls: re-attach this call's leaves
        ctx.tnw.set_tensors(list(ctx.saved_tensors))
        # the adjoint stays on the device: no host synchronisation
        adj = grad_out.detach().to(device=ctx.saved_tensors[0].device,
                                   dtype=torch.complex128 if ctx.tnw.dtype == binding.TN_C64
                                   else torch.float64).contiguous()
        # leaves that need no gradient get none (NULL: skipped by the sweep)
        need = ctx.needs_input_grad[4:]
        grads = [torch.empty_like(t) if nd else None for t, nd in zip(ctx.saved_tensors, need)]
        grads = ctx.tnw.grad(ctx.pairs, ctx.sliced, ctx.mode, adj, grads=grads)
        return (None, None, None, None, *grads)


def contract(tnw: "binding.TensorNetwork", pairs, sliced, mode, *leaves) -> torch.Tensor:
    return _Contract.apply(tnw, pairs, list(sliced), mode, *leaves)
