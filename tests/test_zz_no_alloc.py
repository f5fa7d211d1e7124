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


def test_noalloc_matches_transfer_decompress_twice():
    import torch
    cols = [
        (W.sorted_keys(11, 3 << 20), zf.ZF_DELTA_BP, 1 << 18),
        (W.dates_rle(11, 3 << 20), zf.ZF_RLE, 1 << 18),
        (W.uniform_int(11, 0, 0, (1 << 20) + 777, 0, 4096).astype(np.int32), zf.ZF_FOR_BP, 65536),
        (W.dict_codes(11, 3, 0, 500000), zf.ZF_DICT_BP, 65536),
    ]
    g = Gpu()
    try:
        for x, scheme, cr in cols:
            h = compress(x, scheme, cr)
            try:
                ref, = g.decode([h], out_specs(x))     # the regular entry point
                assert np.array_equal(ref, x)
                dcol = _device_bytes(torch, zf.zf_compressed_bytes(h))
                stream = torch.cuda.Stream()
                for call in range(2):                  # two calls in a row share the scratch array
                    out = torch.full((x.nbytes,), 0x5A, dtype=torch.uint8, device="cuda")
                    torch.cuda.synchronize()           # the fill runs on another stream
                    st = zf.zf_decompress_device_noalloc(dcol.data_ptr(), dcol.numel(), out.data_ptr(),
                                                         out.numel(), stream.cuda_stream)
                    assert st == zf.ZF_OK, (scheme, call, st)
                    got = out.cpu().numpy().view(x.dtype)
                    assert np.array_equal(got, ref), (scheme, call)
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
