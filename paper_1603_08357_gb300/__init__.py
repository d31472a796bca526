"""GB300 (sm_103a) cluster labelling after Komura's generalized GPU CCL
(arXiv 1603.08357): the C-ABI library libccl.so and its Python binding.

``binding`` exposes the C functions under their C names; ``label`` and
``label_batched`` are conveniences over them that allocate the output and
raise on a non-OK status.
"""
from .binding import *  # noqa: F401,F403
from .binding import CclError, Context, check, ccl_context_create, ccl_label, ccl_label_batched, \
    ccl_sync, LIB_PATH  # noqa: F401

_default_ctx = {}


def default_context(device: int = 0):
    ctx = _default_ctx.get(device)
    if ctx is None:
        ctx = _default_ctx[device] = ccl_context_create(device)
    return ctx


def label(n_sites, nnz, row_ptr, col_idx, open_bits, ctx=None, stream=None, sync=True):
    """Labels one instance held in CUDA tensors; returns an int32 CUDA tensor."""
    import torch
    ctx = ctx or default_context(row_ptr.device.index or 0)
    out = torch.empty(n_sites, dtype=torch.int32, device=row_ptr.device)
    check(ccl_label(ctx, n_sites, nnz, row_ptr, col_idx, open_bits, out, stream), "ccl_label")
    if sync:
        check(ccl_sync(ctx, stream), "ccl_sync")
    return out


def label_batched(site_off, ent_off, row_ptr, col_idx, open_bits, ctx=None, stream=None, sync=True):
    """Labels K concatenated instances held in CUDA tensors (offsets on the host)."""
    import torch
    ctx = ctx or default_context(row_ptr.device.index or 0)
    K = len(site_off) - 1
    out = torch.empty(int(site_off[-1]), dtype=torch.int32, device=row_ptr.device)
    check(ccl_label_batched(ctx, K, site_off, ent_off, row_ptr, col_idx, open_bits, out, stream),
          "ccl_label_batched")
    if sync:
        check(ccl_sync(ctx, stream), "ccl_sync")
    return out
