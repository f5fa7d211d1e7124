"""Counter-based generators.  See the package docstring."""
from __future__ import annotations

import numpy as np

__all__ = [
    "splitmix64", "hash_u64", "uniform_int", "uniform_unit",
    "geometric_gaps", "sorted_keys", "run_lengths_geometric", "dates_rle",
    "zipf_cdf", "zipf_ranks", "vocabulary", "text_column", "lognormal_cents", "decimal_prices",
    "dict_codes", "rle_distribution", "DATE_LO", "DATE_HI", "parallel_rows", "FACT_COLUMNS", "fact_column",
    "fact_pieces", "SELECTOR_FAMILIES", "selector_column",
]

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
# TPC-H date span 1992-01-01 .. 1998-12-31 as days since 1970-01-01.
DATE_LO = 8035
DATE_HI = 10591  # inclusive; 2,557 distinct days


def splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser (Steele, Lea, Flood 2014) on a uint64 array."""
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def hash_u64(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """Random 64-bit word number ``idx`` of stream ``(seed, stream)``."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        key = splitmix64(np.uint64((seed * 0x100000001B3 + stream * 0x9E37) & 0xFFFFFFFFFFFFFFFF))
        return splitmix64(idx ^ key)


def uniform_int(seed: int, stream: int, start: int, n: int, lo: int, hi: int) -> np.ndarray:
    """Rows ``start .. start+n`` of integers uniform on ``[lo, hi)`` (int64 array).

    A power-of-two range takes the top bits of the hash word; other ranges use
    the 32x32 multiply-high reduction.
    """
    span = hi - lo
    assert 0 < span <= (1 << 32)
    h = hash_u64(seed, stream, np.arange(start, start + n, dtype=np.uint64))
    if span & (span - 1) == 0:
        k = span.bit_length() - 1
        v = (h >> np.uint64(64 - k)) if k else np.zeros(n, np.uint64)
    else:
        v = ((h >> np.uint64(32)) * np.uint64(span)) >> np.uint64(32)
    return v.astype(np.int64) + lo


def uniform_unit(seed: int, stream: int, start: int, n: int) -> np.ndarray:
    """Doubles uniform on (0, 1): top 53 bits of the hash word, offset by half a step."""
    h = hash_u64(seed, stream, np.arange(start, start + n, dtype=np.uint64))
    return ((h >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


_GROUP_LSB = {2: np.uint64(0x5555555555555555), 3: np.uint64(0x1249249249249249)}


def _first_success(h: np.ndarray, bits: int) -> np.ndarray:
    """1-based index of the first all-zero ``bits``-wide group of ``h`` (0 if none).

    For 2- and 3-bit groups the zero groups are found with word-wide bit
    operations and the lowest one located through its isolated bit."""
    if bits in _GROUP_LSB:
        x = h
        for k in range(1, bits):
            x = x | (h >> np.uint64(k))
        z = ~x & _GROUP_LSB[bits]
        if bits == 3:
            z &= np.uint64((1 << 63) - 1)   # 21 whole groups; bit 63 is not a group start
        low = z & (~z + np.uint64(1))       # isolate the lowest set bit
        pos = np.zeros(h.shape, np.int64)
        nz = low != 0
        pos[nz] = np.log2(low[nz].astype(np.float64)).astype(np.int64) // bits + 1
        return pos
    groups = 64 // bits
    out = np.zeros(h.shape, np.int64)
    mask = np.uint64((1 << bits) - 1)
    todo = np.ones(h.shape, bool)
    for g in range(groups):
        z = ((h >> np.uint64(g * bits)) & mask) == 0
        hit = todo & z
        out[hit] = g + 1
        todo &= ~z
        if not todo.any():
            break
    return out


def geometric_gaps(seed: int, stream: int, start: int, n: int, bits: int) -> np.ndarray:
    """Geometric variates on {1, 2, ...} with success probability 2**-bits.

    Each trial succeeds when ``bits`` fresh random bits are all zero, so the
    draw is integer-only (mean 4 for bits=2, mean 8 for bits=3).  Trials run
    over successive words of the stream until one succeeds.
    """
    idx = np.arange(start, start + n, dtype=np.uint64)
    out = np.zeros(n, np.int64)
    done = np.zeros(n, bool)
    base = np.zeros(n, np.int64)
    per_word = 64 // bits
    rnd = 0
    while not done.all():
        sel = ~done
        h = hash_u64(seed, stream + 7919 * rnd, idx[sel])
        f = _first_success(h, bits)
        got = f > 0
        o = base[sel]
        o[got] += f[got]
        o[~got] += per_word
        out_sel = out[sel]
        out_sel[got] = o[got]
        out[sel] = out_sel
        b = base[sel]
        b[~got] += per_word
        base[sel] = b
        d = done[sel]
        d[got] = True
        done[sel] = d
        rnd += 1
    return out


def sorted_keys(seed: int, n: int, start_key: int = 0, start_row: int = 0, mean_bits: int = 2) -> np.ndarray:
    """Strictly increasing int64 keys whose gaps are geometric (mean 4 by default).

    ``start_key`` is the key before row ``start_row`` so that a long column can
    be produced piecewise; key(row) = start_key + sum of the gaps up to row.
    """
    g = geometric_gaps(seed, 101, start_row, n, mean_bits)
    return start_key + np.cumsum(g, dtype=np.int64)


def run_lengths_geometric(seed: int, stream: int, start_run: int, nruns: int, bits: int = 3) -> np.ndarray:
    return geometric_gaps(seed, stream, start_run, nruns, bits)


def dates_rle(seed: int, n: int, mean_bits: int = 3) -> np.ndarray:
    """int32 date column: runs of geometric length (mean 8) of a day drawn
    uniformly from the 2,557 TPC-H days, each run independent of the last."""
    est = n // (1 << mean_bits) + 1024
    while True:
        lens = parallel_rows(lambda a, c: run_lengths_geometric(seed, 201, a, c, mean_bits), est, piece=1 << 22)
        if lens.sum() >= n:
            break
        est *= 2
    vals = parallel_rows(lambda a, c: uniform_int(seed, 202, a, c, DATE_LO, DATE_HI + 1), est, piece=1 << 22)
    out = np.repeat(vals.astype(np.int32), lens)
    return np.ascontiguousarray(out[:n])


def zipf_cdf(n: int, s: float) -> np.ndarray:
    """CDF of the finite Zipf law P(k) ~ k**-s on ranks 1..n."""
    w = np.arange(1, n + 1, dtype=np.float64) ** (-s)
    c = np.cumsum(w)
    return c / c[-1]


def zipf_ranks(seed: int, stream: int, start: int, n: int, cdf: np.ndarray) -> np.ndarray:
    """0-based Zipf ranks sampled by binary search of the CDF."""
    u = uniform_unit(seed, stream, start, n)
    r = np.searchsorted(cdf, u, side="left")
    return np.minimum(r, len(cdf) - 1).astype(np.int64)


def vocabulary(seed: int, nwords: int = 5000, lmin: int = 3, lmax: int = 12) -> list[bytes]:
    """``nwords`` distinct lowercase words of length lmin..lmax, in draw order
    (a repeated draw is skipped)."""
    words: list[bytes] = []
    seen: set[bytes] = set()
    start = 0
    while len(words) < nwords:
        batch = 2 * (nwords - len(words)) + 64
        lens = uniform_int(seed, 301, start, batch, lmin, lmax + 1)
        letters = uniform_int(seed, 302, start * lmax, batch * lmax, 0, 26).reshape(batch, lmax) + ord("a")
        rows = letters.astype(np.uint8)
        for i in range(batch):
            w = rows[i, : lens[i]].tobytes()
            if w in seen:
                continue
            seen.add(w)
            words.append(w)
            if len(words) == nwords:
                break
        start += batch
    return words


def text_column(seed: int, total_bytes: int, nwords: int = 5000, zipf_s: float = 1.1,
                wmin: int = 1, wmax: int = 8) -> tuple[np.ndarray, np.ndarray]:
    """A string column of exactly ``total_bytes`` bytes.

    Each row holds ``wmin..wmax`` words (uniform) drawn Zipf(s) from a seeded
    vocabulary and joined by single spaces; rows are concatenated with no
    separator.  Rows are drawn until the bytes reach the target and the last
    row is cut to fit exactly.  Returns (bytes uint8[total], offsets int32[rows+1]).
    """
    vocab = vocabulary(seed, nwords)
    vlen = np.array([len(w) for w in vocab], np.int64)
    vbytes = np.frombuffer(b"".join(vocab), np.uint8)
    vstart = np.concatenate([[0], np.cumsum(vlen)[:-1]])
    cdf = zipf_cdf(nwords, zipf_s)
    mean_row = (wmin + wmax) / 2 * (float((vlen * np.diff(np.concatenate([[0.0], cdf]))).sum()) + 1)
    rows_est = int(total_bytes / mean_row * 1.05) + 16
    while True:
        nw = uniform_int(seed, 401, 0, rows_est, wmin, wmax + 1)
        row_words_start = np.concatenate([[0], np.cumsum(nw)])
        ranks = zipf_ranks(seed, 402, 0, int(row_words_start[-1]), cdf)
        wl = vlen[ranks]
        # Bytes per row: word lengths plus (words-1) spaces.
        wl_cum = np.concatenate([[0], np.cumsum(wl)])
        row_bytes = wl_cum[row_words_start[1:]] - wl_cum[row_words_start[:-1]] + (nw - 1)
        if row_bytes.sum() >= total_bytes:
            break
        rows_est = int(rows_est * 1.3) + 16
    row_end = np.cumsum(row_bytes)
    nrows = int(np.searchsorted(row_end, total_bytes, side="left")) + 1
    nwords_used = int(row_words_start[nrows])
    ranks = ranks[:nwords_used]
    wl = wl[:nwords_used]
    # Each word is followed by a space except the last word of a row.
    last_in_row = np.zeros(nwords_used, bool)
    last_in_row[row_words_start[1:nrows + 1] - 1] = True
    tok_len = wl + (~last_in_row).astype(np.int64)
    tok_start = np.concatenate([[0], np.cumsum(tok_len)[:-1]])
    full = int(tok_len.sum())
    buf = np.full(full, ord(" "), np.uint8)
    # Scatter word bytes: position of byte j of word k is tok_start[k] + j.
    rep_word = np.repeat(np.arange(nwords_used), wl)
    within = np.arange(int(wl.sum())) - np.repeat(np.concatenate([[0], np.cumsum(wl)[:-1]]), wl)
    buf[tok_start[rep_word] + within] = vbytes[vstart[ranks[rep_word]] + within]
    offsets = np.concatenate([[0], row_end[:nrows]]).astype(np.int64)
    offsets[-1] = min(offsets[-1], total_bytes)
    assert offsets[-1] == total_bytes and full >= total_bytes
    return np.ascontiguousarray(buf[:total_bytes]), offsets.astype(np.int32)


def lognormal_cents(seed: int, stream: int, start: int, n: int, mu: float = 11.5, sigma: float = 1.0) -> np.ndarray:
    """Scaled decimals: round(exp(N(mu, sigma))) clipped to [1, 2**40) (Box-Muller)."""
    u1 = uniform_unit(seed, stream, start, n)
    u2 = uniform_unit(seed, stream + 1, start, n)
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    v = np.rint(np.exp(mu + sigma * z))
    return np.clip(v, 1, (1 << 40) - 1).astype(np.int64)


def decimal_prices(seed: int, stream: int, start: int, n: int, decimals: int = 2) -> np.ndarray:
    """float64 prices with ``decimals`` digits after the point: log-normal
    cents (lognormal_cents) divided by 10**decimals, i.e. the double nearest
    each decimal value, as parsing its text would give."""
    return lognormal_cents(seed, stream, start, n) / float(10 ** decimals)


def dict_codes(seed: int, stream: int, start: int, n: int, ndistinct: int = 25, zipf_s: float = 1.1) -> np.ndarray:
    """Low-cardinality int32 column: ``ndistinct`` values drawn uniformly from
    int32 once per seed, chosen per row with Zipf(s) frequencies."""
    vals = uniform_int(seed, stream + 17, 0, ndistinct, -(1 << 31), 1 << 31)
    r = zipf_ranks(seed, stream, start, n, zipf_cdf(ndistinct, zipf_s))
    return vals[r].astype(np.int32)


def rle_distribution(seed: int, kind: str, n: int, a: int = 1, b: int = 1) -> np.ndarray:
    """Group-size distributions of the RLE microbenchmark (Section 5.2.2).

    ``even``: every group has ``a`` elements; ``random``: sizes uniform on
    [a, b]; ``outlier``: mostly size 1 with one group of ``b`` elements in
    every ``a`` groups; ``mixed``: the first half even-``a``, the second half
    random [1, b].  Group values are uniform int32 and differ from their
    neighbour so that every group is one run.  Returns int32[n].
    """
    est = n + 1024
    if kind == "even":
        lens = np.full(est, a, np.int64)
    elif kind == "random":
        lens = uniform_int(seed, 501, 0, est, a, b + 1)
    elif kind == "outlier":
        lens = np.ones(est, np.int64)
        lens[a - 1::a] = b
    elif kind == "mixed":
        h = est // 2
        lens = np.concatenate([np.full(h, a, np.int64), uniform_int(seed, 502, 0, est - h, 1, b + 1)])
    else:
        raise ValueError(kind)
    vals = uniform_int(seed, 503, 0, est, -(1 << 31), 1 << 31)
    # Force neighbours to differ so that the declared groups are the runs.
    same = np.concatenate([[False], vals[1:] == vals[:-1]])
    vals[same] ^= 1
    out = np.repeat(vals.astype(np.int32), lens)
    return np.ascontiguousarray(out[:n])


def parallel_rows(fn, n: int, piece: int = 1 << 24, workers: int = 0) -> np.ndarray:
    """``fn(start, count)`` over [0, n) in pieces on a thread pool (numpy
    releases the GIL), concatenated.  ``fn`` must be a pure function of the
    row range (the counter-based generators are)."""
    import concurrent.futures as cf
    import os
    if n <= piece:
        return fn(0, n)
    starts = list(range(0, n, piece))
    workers = workers or min(16, os.cpu_count() or 1)
    with cf.ThreadPoolExecutor(workers) as ex:
        parts = list(ex.map(lambda s: fn(s, min(piece, n - s)), starts))
    return np.concatenate(parts)


# The 16 columns of the synthetic fact table, 100 bytes per row:
# (name, numpy dtype, kind)
FACT_COLUMNS = (
    [("qty_%d" % i, np.int32, "uniform_1_50") for i in range(2)]
    + [("price_%d" % i, np.int64, "lognormal_cents") for i in range(7)]
    + [("key_%d" % i, np.int64, "sorted_keys") for i in range(2)]
    + [("date_%d" % i, np.int32, "dates") for i in range(3)]
    + [("code_%d" % i, np.int32, "codes_25") for i in range(2)]
)


def fact_column(seed: int, idx: int, n: int) -> np.ndarray:
    """Column ``idx`` of the fact table (n rows), each column its own stream."""
    name, dt, kind = FACT_COLUMNS[idx]
    s = seed * 1000 + idx
    if kind == "uniform_1_50":
        return parallel_rows(lambda a, c: uniform_int(s, 11, a, c, 1, 51).astype(np.int32), n)
    if kind == "lognormal_cents":
        return parallel_rows(lambda a, c: lognormal_cents(s, 21, a, c), n)
    if kind == "sorted_keys":
        gaps = parallel_rows(lambda a, c: geometric_gaps(s, 101, a, c, 2), n)
        return np.cumsum(gaps, dtype=np.int64)
    if kind == "dates":
        return dates_rle(s, n)
    if kind == "codes_25":
        return parallel_rows(lambda a, c: dict_codes(s, 31, a, c), n)
    raise ValueError(kind)


def fact_pieces(seed: int, idx: int, n: int, lo_bytes: int = 4 << 20, hi_bytes: int = 64 << 20) -> list[int]:
    """Row counts of the uneven pieces a fact column is streamed in: sizes
    log-uniform over [lo_bytes, hi_bytes] of uncompressed bytes, rounded to a
    multiple of 1,024 rows (the last piece takes the remainder)."""
    itemsize = np.dtype(FACT_COLUMNS[idx][1]).itemsize
    out, total, k = [], 0, 0
    lo, hi = np.log(lo_bytes), np.log(hi_bytes)
    while total < n:
        u = float(uniform_unit(seed * 1000 + idx, 77, k, 1)[0])
        rows = int(np.exp(lo + (hi - lo) * u) / itemsize) // 1024 * 1024
        rows = max(1024, min(rows, n - total))
        out.append(rows)
        total += rows
        k += 1
    return out


SELECTOR_FAMILIES = ("uniform", "zipf", "sorted", "runs", "text")


def selector_column(seed: int, cap_rows: int | None = None):
    """One column of the selector's training / held-out sets (seeded).

    Family = seed mod 5: uniform (range 2^1..2^40), zipf (2..100,000
    distinct values, s in [0.8, 1.5]), sorted (geometric gaps, mean 2..16),
    runs (geometric run lengths, mean 2..256) or text (Zipf words from a
    100..20,000-word vocabulary).  Integer families pick int32 or int64 by
    seed.  Rows are log-uniform over [1M, 64M], cut to ``cap_rows`` when
    given.  Returns (values or bytes, offsets or None, meta)."""
    fam = SELECTOR_FAMILIES[seed % 5]
    u = uniform_unit(seed, 900, 0, 8)
    rows = int(round(np.exp(np.log(1 << 20) + u[0] * (np.log(64 << 20) - np.log(1 << 20)))))
    if cap_rows:
        rows = min(rows, cap_rows)
    meta = {"family": fam, "rows": rows}
    if fam == "text":
        vocab = int(np.exp(np.log(100) + u[1] * (np.log(20000) - np.log(100))))
        s = 0.8 + 0.7 * u[2]
        target = min(rows * 12, 8 << 20)          # about 12 bytes per row of 1-2 words, at most 8 MiB
        data, offs = text_column(seed, target, nwords=vocab, zipf_s=s, wmin=1, wmax=2)
        meta.update(vocab=vocab, zipf_s=s, bytes=len(data))
        return data, offs, meta
    i64 = u[3] < 0.5
    dt = np.int64 if i64 else np.int32
    meta["dtype"] = "int64" if i64 else "int32"
    if fam == "uniform":
        k = 1 + int(u[1] * (40 if i64 else 30))
        lo = int(uniform_int(seed, 901, 0, 1, -(1 << 30), 1 << 30)[0]) if not i64 else \
            int(uniform_int(seed, 901, 0, 1, -(1 << 31), 1 << 31)[0]) << 8
        span = 1 << k
        h = hash_u64(seed, 902, np.arange(rows, dtype=np.uint64))
        x = (lo + (h >> np.uint64(64 - k)).astype(np.int64)) if k < 64 else h.astype(np.int64)
        meta.update(bits=k)
        return x.astype(dt), None, meta
    if fam == "zipf":
        nd = int(np.exp(np.log(2) + u[1] * (np.log(100000) - np.log(2))))
        s = 0.8 + 0.7 * u[2]
        vals = uniform_int(seed, 903, 0, nd, -(1 << 31), 1 << 31)
        if i64:
            vals = vals * 4099
        r = parallel_rows(lambda a, c: zipf_ranks(seed, 904, a, c, zipf_cdf(nd, s)), rows)
        meta.update(ndistinct=nd, zipf_s=s)
        return vals[r].astype(dt), None, meta
    if fam == "sorted":
        bits = 1 + int(u[1] * 4)
        g = parallel_rows(lambda a, c: geometric_gaps(seed, 905, a, c, bits), rows)
        meta.update(gap_bits=bits)
        return np.cumsum(g).astype(dt), None, meta
    # runs
    mean_bits = 1 + int(u[1] * 8)
    vrange = 1 << (2 + int(u[2] * 28))
    est = rows // (1 << mean_bits) + 1024
    while True:
        lens = geometric_gaps(seed, 906, 0, est, mean_bits)
        if lens.sum() >= rows:
            break
        est *= 2
    vals = uniform_int(seed, 907, 0, est, 0, min(vrange, 1 << 32)) - (vrange // 2)
    meta.update(run_bits=mean_bits, value_range=vrange)
    return np.repeat(vals, lens)[:rows].astype(dt), None, meta
