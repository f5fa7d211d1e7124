"""zf_decompress_device_noalloc: decoding with no allocation at all, for
callers that may not call cudaMalloc while running (engines that reserved
all device memory at start-up, code inside a fixed memory budget).  Its
output must equal the regular entry point's output on two calls in a row.
This file sorts last so a failure here comes after every other test."""
import numpy as np
import pytest

import zf_workloads as W
from gpu_helpers import Gpu, compress, out_specs

zf = pytest.importorskip("paper_2602_08190_gb300")
pytestmark = pytest.mark.gpu


def _device_bytes(torch, b: bytes):
    host = torch.frombuffer(bytearray(b), dtype=torch.uint8)
    return host.to("cuda")


def _prices_with_exceptions():
    x = W.decimal_prices(12, 5, 0, 70_001)
    x[::997] = np.nan
    x[5::1999] = np.inf
    x[7::2999] = -0.0
    x[11::3001] = 1.0 / 3.0
    return x


def test_noalloc_matches_transfer_decompress_twice():
    import torch
    # int32 first: the first call on a device must already allow the larger
    # shared-memory slices of the 8-byte columns after it
    cols = [
        (W.uniform_int(11, 0, 0, (1 << 20) + 777, 0, 4096).astype(np.int32), zf.ZF_FOR_BP, 65536),
        (W.sorted_keys(11, 3 << 20), zf.ZF_DELTA_BP, 1 << 18),
        (W.dates_rle(11, 3 << 20), zf.ZF_RLE, 1 << 18),
        (W.dict_codes(11, 3, 0, 500000), zf.ZF_DICT_BP, 65536),
        (W.decimal_prices(11, 5, 0, (1 << 20) + 333), zf.ZF_FLOAT2INT, 65536),
        (_prices_with_exceptions(), zf.ZF_FLOAT2INT, 16384),
        (_prices_with_exceptions(), zf.ZF_RAW, 16384),
    ]
    g = Gpu()
    try:
        for x, scheme, cr in cols:
            h = compress(x, scheme, cr)
            try:
                ref, = g.decode([h], out_specs(x))     # the regular entry point
                assert np.array_equal(ref.view(np.uint8), x.view(np.uint8))
                dcol = _device_bytes(torch, zf.zf_compressed_bytes(h))
                stream = torch.cuda.Stream()
                for call in range(2):                  # two calls in a row share the scratch array
                    out = torch.full((x.nbytes,), 0x5A, dtype=torch.uint8, device="cuda")
                    torch.cuda.synchronize()           # the fill runs on another stream
                    st = zf.zf_decompress_device_noalloc(dcol.data_ptr(), dcol.numel(), out.data_ptr(),
                                                         out.numel(), stream.cuda_stream)
                    assert st == zf.ZF_OK, (scheme, call, st)
                    got = out.cpu().numpy()               # bytes: NaN patterns compare too
                    assert np.array_equal(got, ref.view(np.uint8)), (scheme, call)
            finally:
                zf.zf_compressed_free(h)
    finally:
        g.close()


def test_noalloc_rejects_beyond_limits():
    import torch
    x = np.arange(4097 * 1024, dtype=np.int32)         # 4097 chunks: above the fixed scratch size
    h = compress(x, zf.ZF_FOR_BP, 1024)
    try:
        dcol = _device_bytes(torch, zf.zf_compressed_bytes(h))
        out = torch.empty(x.nbytes, dtype=torch.uint8, device="cuda")
        assert zf.zf_decompress_device_noalloc(dcol.data_ptr(), dcol.numel(), out.data_ptr(), out.numel()) \
            == zf.ZF_EINVAL
        assert zf.zf_decompress_device_noalloc(dcol.data_ptr(), dcol.numel(), out.data_ptr(), 16) == zf.ZF_EINVAL
    finally:
        zf.zf_compressed_free(h)


def test_noalloc_rejects_unordered_float2int_exceptions():
    """Chunk 0's first two exception rows swapped: the device check reports
    ZF_ECORRUPT, and the next call on the intact column decodes it."""
    import torch
    x = _prices_with_exceptions()
    h = compress(x, zf.ZF_FLOAT2INT, 16384)
    try:
        raw = bytearray(zf.zf_compressed_bytes(h))
        c0 = int.from_bytes(raw[64:72], "little")                   # directory entry 0: chunk offset
        n_aux = int.from_bytes(raw[c0 + 12:c0 + 16], "little")
        off1 = int.from_bytes(raw[c0 + 28:c0 + 32], "little")       # exception rows section
        assert n_aux >= 2
        bad = bytearray(raw)
        e = c0 + off1
        bad[e:e + 4], bad[e + 4:e + 8] = raw[e + 4:e + 8], raw[e:e + 4]
        out = torch.empty(x.nbytes, dtype=torch.uint8, device="cuda")
        dbad = _device_bytes(torch, bytes(bad))
        st = zf.zf_decompress_device_noalloc(dbad.data_ptr(), len(bad), out.data_ptr(), out.numel())
        assert st == zf.ZF_ECORRUPT
        good = _device_bytes(torch, bytes(raw))
        assert zf.zf_decompress_device_noalloc(good.data_ptr(), len(raw), out.data_ptr(), out.numel()) == zf.ZF_OK
        assert np.array_equal(out.cpu().numpy(), x.view(np.uint8))
    finally:
        zf.zf_compressed_free(h)
