#!/usr/bin/env python
"""Write zf_f2i_table.h: the reciprocals of 5^e that the Float2Int decoder
multiplies by, computed with exact integer arithmetic (Python integers).

For e = 1..18, with s = floor(log2(5^e)):
  R64  = ceil(2^(64 + s)  / 5^e)   one 64-bit word in (2^63, 2^64)
  R128 = ceil(2^(128 + s) / 5^e)   two 64-bit words, in (2^127, 2^128)
Both are rounded up, so a product with them never falls below the exact
quotient.  Entry 0 is unused (e = 0 needs no division).

Run:  python gen_f2i_table.py [output path]   (default: zf_f2i_table.h beside this file)
"""
import os
import sys

EMAX = 18


def entries():
    out = [(0, 0, 0, 0)]
    for e in range(1, EMAX + 1):
        p = 5 ** e
        s = p.bit_length() - 1
        r64 = -(-(1 << (64 + s)) // p)
        r128 = -(-(1 << (128 + s)) // p)
        assert (1 << 63) < r64 < (1 << 64) and (1 << 127) < r128 < (1 << 128)
        out.append((r64, r128 >> 64, r128 & ((1 << 64) - 1), s))
    return out


def render() -> str:
    lines = [
        "// zf_f2i_table.h -- written by gen_f2i_table.py (exact integer arithmetic); do not edit.",
        "// Row e (1..18): { ceil(2^(64+s)/5^e), ceil(2^(128+s)/5^e) high word, low word, s = floor(log2 5^e) }.",
        "#pragma once",
        "#define ZF_F2I_RECIP_ROWS \\",
    ]
    rows = entries()
    for i, (r64, hi, lo, s) in enumerate(rows):
        sep = ", \\" if i + 1 < len(rows) else ""
        lines.append(f"    {{0x{r64:016x}ull, 0x{hi:016x}ull, 0x{lo:016x}ull, {s}u}}{sep}")
    return "\n".join(lines) + "\n"


if __name__ == "__main__":
    path = sys.argv[1] if len(sys.argv) > 1 else os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                                "zf_f2i_table.h")
    with open(path, "w") as f:
        f.write(render())
    print(path)
