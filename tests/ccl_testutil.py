"""Helpers shared by the GPU tests: moving generator output to the device and
calling the library through its C ABI."""
import numpy as np
import torch

import paper_1603_08357_gb300 as ccl

DEV = torch.device("cuda:0")


def to_dev(lat):
    rp = torch.from_numpy(np.ascontiguousarray(lat.row_ptr, np.int32)).to(DEV)
    ci = torch.from_numpy(np.ascontiguousarray(lat.col_idx, np.int32)).to(DEV)
    bits = torch.from_numpy(np.ascontiguousarray(lat.open_bits, np.uint32).view(np.int32)).to(DEV)
    return rp, ci, bits


def gpu_label(ctx, lat, stream=None, expect_status=ccl.CCL_OK):
    rp, ci, bits = to_dev(lat)
    out = torch.full((max(lat.n, 1),), -7, dtype=torch.int32, device=DEV)
    st = ccl.ccl_label(ctx, lat.n, lat.nnz, rp, ci if lat.nnz else None, bits if lat.nnz else None,
                       out, stream)
    assert st == ccl.CCL_OK, ccl.ccl_status_string(st)
    st = ccl.ccl_sync(ctx, stream)
    assert st == expect_status, ccl.ccl_status_string(st)
    return out[:lat.n].cpu().numpy()


def batch_to_dev(b):
    rp = torch.from_numpy(b.row_ptr).to(DEV)
    ci = torch.from_numpy(b.col_idx if b.col_idx.size else np.zeros(1, np.int32)).to(DEV)
    bits = torch.from_numpy(b.open_bits.view(np.int32)).to(DEV)
    return rp, ci, bits


def gpu_label_batched(ctx, b, stream=None):
    rp, ci, bits = batch_to_dev(b)
    out = torch.full((max(b.n_total, 1),), -7, dtype=torch.int32, device=DEV)
    st = ccl.ccl_label_batched(ctx, b.k, b.site_off, b.ent_off, rp, ci, bits, out, stream)
    assert st == ccl.CCL_OK, ccl.ccl_status_string(st)
    st = ccl.ccl_sync(ctx, stream)
    assert st == ccl.CCL_OK, ccl.ccl_status_string(st)
    return out[:b.n_total].cpu().numpy()
