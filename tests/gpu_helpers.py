"""Helpers for the GPU tests: device buffers from torch, decode through the C ABI."""
from __future__ import annotations

import numpy as np

import paper_2602_08190_gb300 as zf

SENTINEL = 0xA5


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def out_specs(x: np.ndarray, offsets: np.ndarray | None = None):
    """(numpy dtype, element count) of each output buffer of a column."""
    if offsets is not None:
        return [(np.uint8, int(offsets[-1])), (np.int32, len(offsets))]
    return [(x.dtype, len(x))]


def compress(x, scheme, chunk_rows=1 << 20, offsets=None, offsets_scheme=-1):
    col = zf.Column(x, offsets)
    p = zf.zf_plan(None, col, scheme=scheme, chunk_rows=chunk_rows, offsets_scheme=offsets_scheme)
    return zf.zf_compress_host(p, col)


class Gpu:
    def __init__(self, **kcfg):
        self.torch = torch_cuda()
        self.ctx = zf.zf_ctx_create(0)
        if kcfg:
            zf.zf_ctx_set_kcfg(self.ctx, **kcfg)

    def close(self):
        zf.zf_ctx_destroy(self.ctx)

    def alloc(self, specs):
        t = self.torch
        bufs = []
        for dt, n in specs:
            nb = max(16, np.dtype(dt).itemsize * n)
            b = t.full((nb,), SENTINEL, dtype=t.uint8, device="cuda")
            bufs.append(b)
        # the library runs on its own streams: the fills must be done first
        t.cuda.synchronize()
        return bufs

    def decode(self, handles, specs, resident=False, expect=zf.ZF_OK):
        """Decode compressed handles into fresh buffers; returns numpy arrays."""
        bufs = self.alloc(specs)
        outs = [b.data_ptr() for b in bufs]
        caps = [b.numel() for b in bufs]
        if resident:
            res = [zf.zf_upload(self.ctx, h) for h in handles]
            zf.zf_decompress_resident(self.ctx, res, outs, caps)
        else:
            res = []
            zf.zf_transfer_decompress(self.ctx, handles, outs, caps)
        st, stats = zf.zf_sync(self.ctx, raise_on_error=False)
        for r in res:
            zf.zf_resident_free(r)
        assert st == expect, (st, zf.zf_last_error(self.ctx))
        self.last_stats = stats
        host = []
        for b, (dt, n) in zip(bufs, specs):
            a = b.cpu().numpy()
            host.append(a[: np.dtype(dt).itemsize * n].view(dt))
        return host
