"""The integer-only Float2Int value (csrc/zf_f2i.h) against the definition.

The GPU decoder computes the double nearest d / 10^e with integer multiplies
by reciprocals of 5^e (Section 2.1 Float2Int; the Eisel-Lemire idea).  Here
the same header is compiled for the host and every result is compared with
the IEEE division d / 10^e, which is exactly the definition for |d| <= 2^53
and e <= 18 (both operands are doubles exactly, and IEEE division rounds the
exact quotient to nearest).  The reciprocal table is re-derived from exact
integer arithmetic and compared with the committed header.
"""
from __future__ import annotations

import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2602_08190_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <cstdint>
#include <vector>
#include "zf_f2i.h"
static const zf::F2IRecip kTab[19] = {ZF_F2I_RECIP_ROWS};
int main(int argc, char** argv) {
    FILE* fi = fopen(argv[1], "rb");
    FILE* fo = fopen(argv[2], "wb");
    int64_t rec[2];
    while (fread(rec, 8, 2, fi) == 2) {
        const zf::F2IRecip& r = kTab[rec[1]];
        uint64_t bits = argv[3][0] == '1'
            ? zf::f2i_bits_u32((uint32_t)rec[0], (uint32_t)rec[1], r, 1052 - (int32_t)r.s - (int32_t)rec[1])
            : zf::f2i_bits(rec[0], (uint32_t)rec[1], r);
        fwrite(&bits, 8, 1, fo);
    }
    fclose(fi);
    fclose(fo);
    return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    d = tmp_path_factory.mktemp("f2i")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    exe = d / "h"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, "-o", str(exe), str(src)], check=True)

    def run(dv: np.ndarray, ev: np.ndarray, u32: bool = False) -> np.ndarray:
        inp = d / "in.bin"
        out = d / "out.bin"
        np.stack([dv.astype(np.int64), ev.astype(np.int64)], 1).tofile(inp)
        subprocess.run([str(exe), str(inp), str(out), "1" if u32 else "0"], check=True)
        return np.fromfile(out, np.uint64)
    return run


def definition(dv: np.ndarray, ev: np.ndarray) -> np.ndarray:
    p = np.array([10.0 ** e for e in range(19)])   # exact: every 10^e, e <= 22, is a double
    return (dv.astype(np.float64) / p[ev]).view(np.uint64)


def check(run, dv, ev, u32=False):
    dv = np.asarray(dv, np.int64)
    ev = np.asarray(ev, np.int64)
    if u32:   # the 32-bit path: integers in [0, 2^32), e >= 1
        assert dv.min() >= 0 and dv.max() < 2**32 and ev.min() >= 1
    got, want = run(dv, ev, u32), definition(dv, ev)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, [(int(dv[i]), int(ev[i]), hex(int(got[i])), hex(int(want[i]))) for i in bad[:5]]


def test_table_matches_exact_integer_derivation(tmp_path):
    out = tmp_path / "t.h"
    subprocess.run([sys.executable, os.path.join(CSRC, "gen_f2i_table.py"), str(out)], check=True,
                   capture_output=True)
    assert out.read_text() == open(os.path.join(CSRC, "zf_f2i_table.h")).read()
    # and each row is the rounded-up reciprocal it claims to be
    rows = [l.strip().rstrip("\\").strip().rstrip(",") for l in out.read_text().splitlines() if l.strip().startswith("{0x")]
    for e, row in enumerate(rows):
        r64, hi, lo, s = [int(x.strip().rstrip("ul"), 0) for x in row.strip("{}").split(",")]
        if e == 0:
            continue
        p = 5 ** e
        assert 2 ** s <= p < 2 ** (s + 1)
        assert (r64 - 1) * p < 2 ** (64 + s) <= r64 * p
        r128 = (hi << 64) | lo
        assert (r128 - 1) * p < 2 ** (128 + s) <= r128 * p


def test_small_integers_every_exponent(harness):
    a = np.arange(0, 200_001, dtype=np.int64)
    for e in range(19):
        check(harness, np.concatenate([a, -a[1:]]), np.full(2 * a.size - 1, e))


def test_random_magnitudes_up_to_2_53(harness):
    rng = np.random.default_rng(11)
    n = 400_000
    bits = rng.integers(1, 54, n)
    a = (rng.integers(0, 2**62, n, dtype=np.int64) >> (62 - bits)) + 1
    a = np.minimum(a, 2**53)
    d = np.where(rng.integers(0, 2, n) == 1, -a, a)
    e = rng.integers(0, 19, n)
    check(harness, d, e)


def test_extremes_and_exact_quotients(harness):
    d, e = [], []
    for ee in range(19):
        for a in [1, 2, 3, 5, 9, 10, 2**52 - 1, 2**52, 2**52 + 1, 2**53 - 1, 2**53] + [2**k for k in range(54)] + \
                 [10**k for k in range(16)]:
            for sgn in (1, -1):
                d.append(sgn * a)
                e.append(ee)
        # multiples of 5^e: the quotient is an integer, the result exact
        p = 5 ** ee
        rng = np.random.default_rng(ee)
        for k in rng.integers(1, max(2, 2**53 // p), 2000):
            d.append(int(k) * p)
            e.append(ee)
    check(harness, d, e)


def test_quotients_next_to_halfway_points(harness):
    # a / 5^e as close as an integer a can get to a point halfway between two
    # doubles: the cases the 64-bit product cannot decide alone
    rng = np.random.default_rng(3)
    d, e = [], []
    for ee in range(1, 19):
        p = 5 ** ee
        for _ in range(3000):
            E = int(rng.integers(-20, 53))          # binade of the quotient
            if 2 ** E * p > 2 ** 53:
                continue
            n = int(rng.integers(2 ** 52, 2 ** 53))  # significand below the halfway point
            # halfway point h = (2n + 1) * 2^(E - 53); a ~ h * 5^e
            num = (2 * n + 1) * p
            sh = 53 - E
            base = num >> sh if sh > 0 else num << -sh
            for a in (base - 1, base, base + 1, base + 2):
                if 0 < a <= 2 ** 53:
                    d.append(a)
                    e.append(ee)
    assert len(d) > 50_000
    check(harness, d, e)


def test_u32_path_small_integers_every_exponent(harness):
    a = np.arange(0, 200_001, dtype=np.int64)
    for e in range(1, 19):
        check(harness, a, np.full(a.size, e), u32=True)


def test_u32_path_random_and_extreme_magnitudes(harness):
    rng = np.random.default_rng(12)
    n = 400_000
    bits = rng.integers(1, 33, n)
    a = rng.integers(0, 2**32, n, dtype=np.int64) >> (32 - bits)
    e = rng.integers(1, 19, n)
    ext = [2**32 - 1, 2**32 - 2, 2**31, 2**31 - 1, 2**31 + 1, 1, 2, 3] + [10**k for k in range(10)] + \
          [5**k for k in range(14)]
    d = np.concatenate([a, np.repeat(ext, 18)])
    e = np.concatenate([e, np.tile(np.arange(1, 19), len(ext))])
    check(harness, d, e, u32=True)


def test_u32_path_next_to_halfway_points(harness):
    # integers below 2^32 whose quotient lies closest to a halfway point: the
    # cases the 32-bit path hands to the general one
    rng = np.random.default_rng(4)
    d, e = [], []
    for ee in range(1, 19):
        p = 5 ** ee
        for _ in range(4000):
            E = int(rng.integers(-45, 32))
            if 2 ** E * p > 2 ** 32:
                continue
            n = int(rng.integers(2 ** 52, 2 ** 53))
            num = (2 * n + 1) * p
            sh = 53 - E
            base = num >> sh if sh > 0 else num << -sh
            for a in (base - 1, base, base + 1, base + 2):
                if 0 <= a < 2 ** 32:
                    d.append(a)
                    e.append(ee)
    assert len(d) > 20_000
    check(harness, d, e, u32=True)
