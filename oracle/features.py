"""Column statistics of the learned selector, written out plainly in numpy
(float64) -- test infrastructure.  Same definitions as the library's
feature extractor, re-implemented from the written list (see the module's
tests): a sample of whole columns up to 262,144 rows (bytes), else 64
windows of 4,096 consecutive rows at floor(i (n - 4096) / 63); pairs, runs
and 1024-row blocks stay inside a window."""
from __future__ import annotations

import math

import numpy as np


def windows(n: int) -> list[tuple[int, int]]:
    if n <= 262144:
        return [(0, n)] if n else []
    return [(i * (n - 4096) // 63, 4096) for i in range(64)]


def bits(x: int) -> int:
    return int(x).bit_length()


def _entropy(counts) -> float:
    c = np.asarray(counts, dtype=np.float64)
    p = c / c.sum()
    return float(-(p * np.log2(p)).sum())


def int_features(x: np.ndarray) -> np.ndarray:
    f = np.zeros(32)
    n = len(x)
    size = x.dtype.itemsize
    f[0 if size == 4 else 1] = 1.0
    f[3] = math.log2(n + 1) / 32
    f[4] = math.log2(n * size + 1) / 40
    f[31] = 1.0
    ws = windows(n)
    if not ws:
        return f
    M = 1 << 64
    vals, pair_d, pair_ge, pair_gt = [], [], 0, 0
    runs, runs1, wbits, bbits = 0, 0, [], []
    for s0, ln in ws:
        w = [int(v) for v in x[s0:s0 + ln]]
        vals += w
        wbits.append(bits((max(w) - min(w)) % M))
        # runs
        k = 0
        while k < ln:
            e = k
            while e + 1 < ln and w[e + 1] == w[k]:
                e += 1
            runs += 1
            runs1 += e == k
            k = e + 1
        # pairs and per-block difference widths
        for b0 in range(0, ln, 1024):
            ds = []
            for j in range(b0 + 1, min(ln, b0 + 1024)):
                d = (w[j] - w[j - 1]) % M
                if d >= 1 << 63:
                    d -= M
                ds.append(d)
            bbits.append(bits((max(ds) - min(ds)) % M) if ds else 0)
        for j in range(1, ln):
            d = (w[j] - w[j - 1]) % M
            if d >= 1 << 63:
                d -= M
            pair_d.append(d)
            pair_ge += w[j] >= w[j - 1]
            pair_gt += w[j] > w[j - 1]
    S, P = len(vals), len(pair_d)
    uniq, cnt = np.unique(np.array(vals, dtype=np.int64), return_counts=True)
    D = len(uniq)
    f[5] = bits((max(vals) - min(vals)) % M) / 64
    f[6] = math.log2(D + 1) / 20
    f[7] = D / S
    f[8] = math.log2(S / runs) / 16
    f[9] = runs1 / runs
    f[10] = pair_ge / P if P else 0.0
    f[11] = pair_gt / P if P else 0.0
    f[12] = bits((max(pair_d) - min(pair_d)) % M) / 64 if P else 0.0
    f[13] = float(np.mean(bbits)) / 64
    f[14] = float(np.mean(wbits)) / 64
    f[15] = _entropy(cnt) / 20
    if P:
        _, dcnt = np.unique(np.array(pair_d, dtype=np.int64), return_counts=True)
        f[16] = _entropy(dcnt) / 20
    top = np.sort(cnt)[::-1]
    f[17] = top[0] / S
    f[18] = top[:8].sum() / S
    f[19] = sum(1 for v in vals if v == 0) / S
    f[20] = sum(1 for v in vals if v < 0) / S
    logs = np.array([math.log2(abs(v) + 1) for v in vals])
    f[21] = logs.mean() / 64
    f[22] = logs.std() / 64
    f[23] = min(1.0, runs * (size + 4) / (S * size))
    f[24] = f[14] * 64 / (8 * size)
    f[25] = min(1.0, (D * size + S * bits(D - 1) / 8) / (S * size))
    f[26] = f[13] * 64 / (8 * size)
    return f


def byte_features(data: np.ndarray, offsets: np.ndarray) -> np.ndarray:
    f = np.zeros(32)
    n = len(offsets) - 1
    nb = int(offsets[-1])
    f[2] = 1.0
    f[3] = math.log2(n + 1) / 32
    f[4] = math.log2(nb + 1) / 40
    f[31] = 1.0
    counts = np.zeros(256, np.int64)
    rep = grams = 0
    for s0, ln in windows(nb):
        w = bytes(data[s0:s0 + ln])
        counts += np.bincount(np.frombuffer(w, np.uint8), minlength=256)
        seen = set()
        for k in range(ln - 3):
            g = w[k:k + 4]
            grams += 1
            rep += g in seen
            seen.add(g)
    f[27] = math.log2(nb / max(n, 1) + 1) / 16
    nz = counts[counts > 0]
    f[28] = _entropy(nz) / 8 if counts.sum() else 0.0
    f[29] = rep / grams if grams else 0.0
    f[30] = len(nz) / 256
    return f


def features(x: np.ndarray, offsets: np.ndarray | None = None) -> np.ndarray:
    if offsets is not None:
        return byte_features(x, offsets)
    return int_features(x)
