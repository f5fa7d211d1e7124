"""The selector's column statistics: the oracle's definitions pinned by
closed forms on special columns, and the library's extractor equal to the
oracle's on varied columns (float32 rounding)."""
import ctypes
import math

import numpy as np
import pytest

import zf_workloads as W
from oracle import features as OF

zf = pytest.importorskip("paper_2602_08190_gb300")


def lib_features(x, offsets=None):
    L = ctypes.CDLL(zf.LIB_PATH)
    L.zf_column_features.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    c = zf.Column(x, offsets)
    out = np.zeros(32, np.float32)
    assert L.zf_column_features(ctypes.byref(c.c), out.ctypes.data) == 0
    return out


def test_oracle_features_constant_column():
    f = OF.features(np.full(1000, 7, np.int32))
    assert f[0] == 1 and f[1] == 0 and f[2] == 0 and f[31] == 1
    assert f[5] == 0 and f[6] == pytest.approx(1 / 20) and f[7] == pytest.approx(1 / 1000)
    assert f[8] == pytest.approx(math.log2(1000) / 16) and f[9] == 0
    assert f[10] == 1 and f[11] == 0 and f[12] == 0 and f[13] == 0 and f[14] == 0
    assert f[15] == 0 and f[16] == 0 and f[17] == 1 and f[18] == 1 and f[19] == 0 and f[20] == 0
    assert f[21] == pytest.approx(3 / 64)            # log2(7 + 1) = 3
    assert f[22] == 0 and f[23] == pytest.approx(8 / 4000)


def test_oracle_features_arange():
    n = 5000
    f = OF.features(np.arange(n, dtype=np.int64))
    assert f[7] == 1 and f[8] == 0 and f[9] == 1 and f[10] == 1 and f[11] == 1
    assert f[12] == 0 and f[13] == 0 and f[16] == 0          # every difference is 1
    assert f[14] == pytest.approx((n - 1).bit_length() / 64)
    assert f[15] == pytest.approx(math.log2(n) / 20)          # uniform over n distinct values
    assert f[17] == pytest.approx(1 / n) and f[18] == pytest.approx(8 / n) and f[19] == pytest.approx(1 / n)
    assert f[25] == pytest.approx(min(1.0, (n * 8 + n * (n - 1).bit_length() / 8) / (n * 8)))


def test_oracle_features_alternating_and_windows():
    x = np.tile(np.array([0, 1], np.int32), 5000)
    f = OF.features(x)
    assert f[9] == 1 and f[19] == pytest.approx(0.5) and f[15] == pytest.approx(1 / 20)
    assert f[10] == pytest.approx(5000 / 9999) and f[11] == pytest.approx(5000 / 9999)
    big = np.zeros(1_000_000, np.int32)
    assert [ln for _, ln in OF.windows(len(big))] == [4096] * 64
    assert OF.windows(len(big))[-1][0] == len(big) - 4096 and OF.windows(262144) == [(0, 262144)]


def test_oracle_byte_features():
    t = np.frombuffer(b"a" * 1000, np.uint8).copy()
    f = OF.features(t, np.array([0, 1000], np.int32))
    assert f[2] == 1 and f[28] == 0 and f[30] == pytest.approx(1 / 256)
    assert f[29] == pytest.approx(996 / 997)                   # every 4-gram but the first repeats
    assert f[27] == pytest.approx(math.log2(1001) / 16)


def _columns():
    yield "keys", W.sorted_keys(1, 300000), None
    yield "dates", W.dates_rle(1, 100000), None
    yield "codes", W.dict_codes(1, 3, 0, 50000), None
    yield "cents", W.lognormal_cents(1, 5, 0, 20000), None
    yield "extremes", np.array([2**63 - 1, -2**63, 0, 5, -1], np.int64), None
    yield "uniform_big", W.uniform_int(2, 2, 0, 700_000, -5, 50).astype(np.int32), None
    yield "empty", np.zeros(0, np.int32), None
    t, o = W.text_column(1, 500000)
    yield "text", t, o


@pytest.mark.parametrize("case", list(_columns()), ids=lambda c: c[0])
def test_library_features_equal_oracle(case):
    name, x, o = case
    a = lib_features(x, o)
    b = OF.features(x, o)
    assert np.allclose(a, b, rtol=1e-6, atol=1e-6), (name, np.max(np.abs(a - b)))
