"""torch.autograd.Function around the cache-backed embedding bag.

Forward: sum-pooled lookups through the HBM cache (agile_embedding_bag).
Backward: the gradient rows G = scatter-add of grad_out over the bag indices, applied as
an SGD step T -= lr * G directly to the table's cached pages (fused optimiser): the
table lives on the backing store, not in a torch tensor, so there is no gradient tensor
to return for it.  Modified lines reach the store through the queues on eviction or at
agile_flush.  A scalar ``anchor`` tensor with requires_grad=True ties the op into the
autograd graph; its gradient is zero.
"""
from __future__ import annotations

import torch

from . import AGILE_ASYNC, agile_embedding_bag, agile_embedding_bag_backward


class CachedEmbeddingBag(torch.autograd.Function):
    @staticmethod
    def forward(ctx, anchor, handle, table_byte0, rows, dim, idx, offsets, lr, mode):
        nb = offsets.numel() - 1
        out = torch.empty((nb, dim), dtype=torch.float32, device=idx.device)
        stream = torch.cuda.current_stream(idx.device).cuda_stream
        agile_embedding_bag(handle, table_byte0, rows, dim, idx.data_ptr(), offsets.data_ptr(), nb,
                            out.data_ptr(), mode, stream)
        ctx.save_for_backward(idx, offsets)
        ctx.meta = (handle, table_byte0, rows, dim, float(lr), mode)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        idx, offsets = ctx.saved_tensors
        handle, table_byte0, rows, dim, lr, mode = ctx.meta
        g = grad_out.contiguous().to(torch.float32)
        stream = torch.cuda.current_stream(idx.device).cuda_stream
        agile_embedding_bag_backward(handle, table_byte0, rows, dim, idx.data_ptr(), offsets.data_ptr(),
                                     offsets.numel() - 1, idx.numel(), g.data_ptr(), lr, 0, mode, stream)
        return (torch.zeros((), device=g.device), None, None, None, None, None, None, None, None)


def cached_embedding_bag(handle, table_byte0, rows, dim, idx, offsets, lr, mode=AGILE_ASYNC, anchor=None):
    if anchor is None:
        anchor = torch.zeros((), device=idx.device, requires_grad=True)
    return CachedEmbeddingBag.apply(anchor, handle, table_byte0, rows, dim, idx, offsets, lr, mode)
