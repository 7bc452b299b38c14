"""torch.autograd.Function around the contraction and its reverse sweep.

``contract(tnw, pairs, sliced, mode, *leaves)`` returns the network value
as a complex128 / float64 torch tensor (mantissa * 2^exp2 folded in; use
``TensorNetwork.contract`` directly for values beyond the FP64 range).  Its
backward calls tn_contract_grad: every leaf's gradient is computed by the
hand-written reverse tree sweep on the GPU (per-slice recomputation of the
forward intermediates), with the holomorphic convention of torch:
grad_leaf = conj(d value / d leaf) * grad_output.

``contract_batch(tnw, pairs, mode, leaves, batch)`` is the same for B
scalar networks that share the tree and every leaf except those in
``batch`` (e.g. the output-state leaves of B bitstrings of one circuit,
Eq. trans-amp): the forward runs the B copies in one launch sequence
keeping the intermediates (tn_contract_instances_keep), the backward runs
the reverse sweeps of all B networks in one launch sequence
(tn_contract_grad_instances) on them, with the adjoints on the device; the
shared leaves' gradients are summed over the batch in the library.
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


class _ContractBatch(torch.autograd.Function):
    @staticmethod
    def forward(ctx, tnw, pairs, mode, batch_ids, n_batch, *tensors):
        n = len(tensors) - len(batch_ids)
        shared = [t.detach().contiguous() for t in tensors[:n]]
        stacks = [t.detach().contiguous() for t in tensors[n:]]
        leaves = list(shared)
        strides = [0] * n
        for v, st in zip(batch_ids, stacks):
            if st.shape[0] != n_batch:
                raise ValueError(f"batch leaf {v}: leading dimension {st.shape[0]}, expected {n_batch}")
            leaves[v] = st
            strides[v] = st[0].numel()
        tnw.set_tensors(leaves)
        # forward in the sweep's state with the intermediates kept: the
        # backward reuses them unless another gradient call intervened
        mant, ex, token = tnw.contract_instances_keep(pairs, mode, n_batch, strides)
        value = mant * torch.pow(torch.tensor(2.0, dtype=torch.float64, device=mant.device),
                                 ex.double()).unsqueeze(1)
        if tnw.dtype == binding.TN_C64:
            value = torch.complex(value[:, 0], value[:, 1])
        else:
            value = value[:, 0].contiguous()
        ctx.tnw, ctx.pairs, ctx.mode, ctx.batch_ids, ctx.token = tnw, pairs, mode, list(batch_ids), token
        ctx.save_for_backward(*shared, *stacks)
        return value

    @staticmethod
    def backward(ctx, grad_out):
        tnw = ctx.tnw
        saved = ctx.saved_tensors
        nb = len(ctx.batch_ids)
        n = len(saved) - nb
        shared, stacks = list(saved[:n]), list(saved[n:])
        need = ctx.needs_input_grad[5:]
        cplx = tnw.dtype == binding.TN_C64
        adj = grad_out.detach().to(device=shared[0].device,
                                   dtype=torch.complex128 if cplx else torch.float64).contiguous()
        # one reverse sweep over all networks: shared leaves' gradients
        # summed over the batch, batch leaves' per network
        g_shared = [torch.empty_like(t) if nd else None for t, nd in zip(shared, need[:n])]
        g_stack = [torch.empty_like(st) if nd else None for st, nd in zip(stacks, need[n:])]
        n_batch = adj.shape[0]
        leaves = list(shared)
        grads = list(g_shared)
        strides = [0] * n
        for j, v in enumerate(ctx.batch_ids):
            leaves[v] = stacks[j]
            grads[v] = g_stack[j]
            strides[v] = stacks[j][0].numel()
        tnw.set_tensors(leaves)
        tnw.grad_instances(ctx.pairs, [], ctx.mode, n_batch, strides, adj, grads=grads, kept_forward=ctx.token)
        return (None, None, None, None, None, *g_shared, *g_stack)


def contract_batch(tnw: "binding.TensorNetwork", pairs, mode, leaves, batch) -> torch.Tensor:
    """Values of B scalar networks sharing a tree: ``leaves`` gives every
    leaf (those replaced per network may be None), ``batch`` maps leaf
    index -> tensor [B, *leaf shape].  Returns a [B] complex128 / float64
    tensor, differentiable in every leaf tensor (unsliced trees)."""
    ids = sorted(batch)
    stacks = [batch[v] for v in ids]
    if not stacks:
        raise ValueError("contract_batch needs at least one batch leaf")
    n_batch = stacks[0].shape[0]
    # placeholders for the batch positions (never read: detached, no gradient)
    shared = [l if l is not None else batch[v][0].detach() for v, l in enumerate(leaves)]
    return _ContractBatch.apply(tnw, pairs, mode, ids, n_batch, *shared, *stacks)
