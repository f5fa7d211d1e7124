#!/usr/bin/env python
"""Throughput of compressed-column transfer + decode on GB300.

Headline workload (one step): the batched fact table -- 16 columns x 400M
rows (2 int32 uniform 1-50 in FOR, 7 int64 log-normal cents in FOR, 2 int64
sorted keys in delta, 3 int32 RLE dates, 2 int32 25-value Zipf codes in
dictionary; 100 B/row, 40 GB), cut into 1,771 uneven pieces of 4-64 MB
uncompressed, each piece a pinned single-chunk compressed column, all decoded
by the persistent work-queue kernel (one launch per stage on the transfer
path, one launch for everything when resident).  Each configuration's stage
size, and whether the transfer is replayed from a captured CUDA graph or
launched plainly, are chosen by timing the transfer on the host clock.

  value   uncompressed GB/s of the decode with the compressed pieces already
          resident in HBM (zf_decompress_resident), CUDA events on the
          decode stream (inputs and outputs far larger than L2).
  e2e     the same metric end to end through zf_transfer_decompress +
          zf_sync: every piece copied host-to-device from pinned memory,
          decoded, and the step's status word read back; host wall clock.
          Beside it the raw link at the call's own pieces (zf_measure_copy:
          the same copies without decoding) and the fraction of
          link x compression ratio reached.
  roofline  the batched kernel's resident launch: algorithmic bytes
          (compressed read + plain written) over its CUDA-event duration,
          against the measured HBM copy peak.
  configs  every other configuration measured the same way in the same run:
          c1 (Fully-Parallel, one stream), c2 (Group-Parallel pair),
          c3_lz77 and c3_strdict (the 256 MB text column, two schemes),
          ans, float2int; each with resident and end-to-end GB/s, raw link at
          its pieces, fraction of link x CR, and its dominant launch's
          algorithmic bytes, duration and fraction of HBM.
  cpu_baseline  the CPU oracle decoding a bounded sample of the fact table's
          pieces on all host cores (threads over chunks), and on one thread.

Every configuration's decode is compared with the generator's column before
timing (whole columns on one GPU; sampled rows on replicas).

--impl reference times the CPU oracle alone on the fact table (a bounded
sample of its pieces, encoded and decoded by the oracle).
With torchrun (--gpus N) every rank decodes its own replica (no collective
on the data path); value sums the ranks' bytes over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "end-to-end uncompressed GB/s (H2D+decode) vs raw PCIe copy; decode % HBM peak"
N_ROWS = 1 << 26
CHUNK_ROWS = 1 << 20
FACT_ROWS = 400_000_000
# Schemes of the fact table's column kinds: FOR for small integers and
# scaled decimals, delta for sorted keys, RLE for dates, dictionary for the
# 25-value codes.
FACT_SCHEMES = {"uniform_1_50": "for_bp", "lognormal_cents": "for_bp", "sorted_keys": "delta_bp",
                "dates": "rle", "codes_25": "dict_bp"}
FACT_WORKLOAD = ("batched: 16-column fact table x {rows:,} rows (2 int32 uniform 1-50 FOR, 7 int64 log-normal "
                 "cents FOR, 2 int64 sorted keys delta, 3 int32 RLE dates, 2 int32 25-value Zipf codes dictionary; "
                 "100 B/row), {pieces} uneven pieces of 4-64 MB uncompressed in pinned memory, one persistent "
                 "work-queue kernel per stage")

# Committed ncu summaries that give each roofline kernel's DRAM traffic per
# launch; a figure is used only while the kernel sources hash as recorded.
KERNEL_SOURCES = ("paper_2602_08190_gb300/csrc/zf_device.cuh", "paper_2602_08190_gb300/csrc/zf_kernels.cu",
                  "paper_2602_08190_gb300/csrc/zf_f2i.h", "paper_2602_08190_gb300/csrc/zf_strdict.cuh")
TRAFFIC_PROFILES = {"c4": "profiles/batched_fact_table_decode.md", "c2": "profiles/delta_i64_decode_64M_rows.md"}


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profile_fields(rel: str) -> dict:
    path = os.path.join(ROOT, rel)
    fields = {}
    if os.path.exists(path):
        with open(path) as f:
            for line in f:
                if ":" in line and line.startswith("- "):
                    k, v = line[2:].split(":", 1)
                    fields[k.strip()] = v.strip().strip("`")
    return fields


def measured_traffic(name: str, units: float):
    """DRAM bytes (read + write) per launch from the committed ncu summary
    of config `name`, scaled from the captured launch's units (rows) to
    `units` when they differ, or None if the kernel sources changed since
    the counters were taken.  Returns (bytes or None, note)."""
    rel = TRAFFIC_PROFILES.get(name)
    if not rel:
        return None, "no capture"
    f = profile_fields(rel)
    if not f or f.get("kernel source hash") != kernel_source_hash():
        return None, "kernel changed since the capture" if f else "no capture"
    try:
        b = int(f["dram bytes read"]) + int(f["dram bytes write"])
        u = float(f["captured units"])
    except (KeyError, ValueError):
        return None, "capture incomplete"
    if u == units:
        return b, f"ncu capture of this launch ({rel})"
    return int(round(b * units / u)), f"ncu capture of {int(u):,} of {int(units):,} units, scaled ({rel})"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.first = 0
        self.windows: list[list[int]] = []   # [start, end) sample indices of the timed regions

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # nvidia-smi takes a moment to start: wait for its first sample so
            # that the samples kept (those after it) fall in the timed region
            t0 = time.perf_counter()
            while not self.lines and time.perf_counter() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        self.first = len(self.lines)
        return self

    def window_start(self):
        self.windows.append([len(self.lines), -1])

    def window_end(self):
        if self.windows and self.windows[-1][1] < 0:
            self.windows[-1][1] = len(self.lines) + 1   # the sample in flight at the end belongs to it

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        if self.windows:
            during = [l for a, b in self.windows for l in self.lines[a:(b if b >= 0 else None)]]
        else:
            during = self.lines[self.first:]
        during = during or self.lines[-1:]
        for line in during:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample(blobs, budget_s: float, threads: int = 1):
    """Decode chunk blobs [(bytes, numpy dtype)] with the CPU oracle until
    `budget_s` seconds pass, `threads` host threads taking them round-robin
    (the oracle's C decoder runs outside the GIL); returns (bytes, seconds,
    chunks decoded)."""
    import concurrent.futures
    import oracle
    t0 = time.perf_counter()

    def worker(w):
        nb = nc = 0
        i = w
        while True:
            blob, dt = blobs[i % len(blobs)]
            nb += oracle.decode_chunk(blob, dt).nbytes
            nc += 1
            i += threads
            if time.perf_counter() - t0 >= budget_s:
                return nb, nc

    with concurrent.futures.ThreadPoolExecutor(threads) as ex:
        res = list(ex.map(worker, range(threads)))
    return sum(r[0] for r in res), time.perf_counter() - t0, sum(r[1] for r in res)


def chunk_blobs(serialized: bytes, dtype, limit: int = 1 << 62):
    """(blob, dtype) of the chunks of a serialized single-part column."""
    import oracle
    out = []
    for c in range(min(limit, oracle.column_info(serialized)["n_chunks"])):
        off, ln, r0, rows = oracle.chunk_span(serialized, c)
        out.append((serialized[off:off + ln], dtype))
    return out


def max_over_ranks(values, dist, device: str):
    """Each value's largest over the ranks: the slowest rank sets the whole
    job's time.  Unchanged on a single process (dist None)."""
    if not dist:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def whole_job_gbs(total_bytes: float, ms: float) -> float:
    """GB/s of `total_bytes` (every rank's bytes) over the job's time."""
    return total_bytes / (ms * 1e-3) / 1e9


def host_threads() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


# ---------------------------------------------------------------- configurations
class Cfg:
    """One measured configuration: compressed handles, the device buffers
    their outputs land in, and what the decode must reproduce.

    parts[i] = [(buffer index, byte offset, bytes), ...] for the output
    parts of handle i (two for a string column: bytes, then int32 offsets).
    expects[b] = the numpy array buffer b must equal (or a strided sample:
    (stride, array of every stride-th element))."""

    def __init__(self, name, workload, handles, buf_bytes, parts, expects, kernel, kernel_idx=None,
                 batched=False, stage_mb=64, compare_batched=False):
        self.name, self.workload, self.handles = name, workload, handles
        self.buf_bytes, self.parts, self.expects = buf_bytes, parts, expects
        self.kernel = kernel
        self.kernel_idx = list(range(len(handles))) if kernel_idx is None else kernel_idx
        self.batched, self.stage_mb = batched, stage_mb
        self.compare_batched = compare_batched     # also time the resident decode in the batched kernel

    def free(self, zf):
        for h in self.handles:
            zf.zf_compressed_free(h)
        self.handles = []


def compress(zf, x, scheme, chunk_rows, offsets=None):
    col = zf.Column(x, offsets)
    return zf.zf_compress_host(zf.zf_plan(None, col, scheme=scheme, chunk_rows=chunk_rows), col)


def single(zf, name, workload, cols, kernel, kernel_idx=None):
    """A configuration of whole columns [(array, scheme, chunk_rows) or
    ((bytes, offsets), scheme, chunk_rows)], each into its own buffers."""
    handles, buf_bytes, parts, expects = [], [], [], []
    for x, scheme, cr in cols:
        arrays = list(x) if isinstance(x, tuple) else [x]
        handles.append(compress(zf, arrays[0], scheme, cr, arrays[1] if len(arrays) > 1 else None))
        p = []
        for a in arrays:
            p.append((len(buf_bytes), 0, a.nbytes))
            buf_bytes.append(a.nbytes)
            expects.append(a)
        parts.append(p)
    return Cfg(name, workload, handles, buf_bytes, parts, expects, kernel, kernel_idx)


def build_c1(zf, seed):
    import zf_workloads as W
    x = W.uniform_int(seed, 0, 0, 1 << 20, 0, 4096).astype(np.int32)
    return single(zf, "c1", "fully_parallel: 1,048,576 int32 uniform on [0, 4096), FOR + 12-bit packing, 65,536-row "
                  "chunks, one stream (a single stage: copy, then decode)", [(x, zf.ZF_FOR_BP, 65536)],
                  "tiles_kernel<FOR_BP, int32>")


def build_c2(zf, seed, rows):
    import zf_workloads as W
    keys, dates = W.sorted_keys(seed, rows), W.dates_rle(seed, rows)
    cfg = single(zf, "c2", f"group_parallel: {rows:,} int64 sorted keys (gaps geometric mean 4; delta + bit-packing, "
                 f"1024-row blocks) + {rows:,} int32 dates (2,557 days, runs geometric mean 8; RLE), 1M-row chunks, "
                 "double-buffered transfer", [(keys, zf.ZF_DELTA_BP, CHUNK_ROWS), (dates, zf.ZF_RLE, CHUNK_ROWS)],
                 "tiles_kernel<DELTA_BP, int64> (the keys)", kernel_idx=[0])
    cfg.compare_batched = True
    return cfg


def build_c3(zf, seed, text, scheme, chunk_mb):
    t, o = text
    if scheme == "lz77":
        return single(zf, "c3_lz77", f"non_parallel: {t.nbytes:,}-byte string column, Zipf(1.1) words from a 5,000-word "
                      "vocabulary (3-12 letters), 1-8 words per row; LZ77 in 64 KiB blocks, one warp per block; "
                      "int32 offsets delta-packed", [((t, o), zf.ZF_LZ77, 0)],
                      "lz_kernel (+ the offsets' delta launch)")
    cb = int(chunk_mb * (1 << 20))
    return single(zf, "c3_strdict", f"group_parallel string dictionary: the same {t.nbytes:,}-byte text column as "
                  f"bit-packed codes into a sorted dictionary of tokens, {cb:,}-byte chunks; int32 offsets "
                  "delta-packed", [((t, o), zf.ZF_STRDICT, cb)], "tiles_kernel<STRDICT, bytes> (+ the offsets' delta launch)")


def build_ans(zf, seed, rows):
    import zf_workloads as W
    u = W.uniform_int(seed, 11, 0, rows, 0, 4)
    x = np.array([65, 78, 78, 82], np.int32)[u]
    return single(zf, "ans", f"ans: {rows:,} int32 return-flag-like rows ('A','N','R' at 1/4, 1/2, 1/4), dictionary + "
                  "range ANS, 1M-row chunks", [(x, zf.ZF_ANS, CHUNK_ROWS)], "ans_kernel")


def build_f2i(zf, seed, rows):
    import zf_workloads as W
    x = W.decimal_prices(seed, 7, 0, rows)
    return single(zf, "float2int", f"float2int: {rows:,} float64 prices with two decimals (log-normal cents / 100), "
                  "Float2Int + bit-packing, 1M-row chunks", [(x, zf.ZF_FLOAT2INT, CHUNK_ROWS)],
                  "tiles_kernel<FLOAT2INT, float64>")


def build_c4(zf, seed, rows, keep: bool, stride: int = 1009):
    """The fact table, column by column: generate, cut into its uneven
    pieces, compress every piece (one single-chunk column per piece).  With
    `keep` the whole columns are kept for the exact check, else every
    `stride`-th row."""
    import zf_workloads as W
    scheme_of = {"for_bp": zf.ZF_FOR_BP, "dict_bp": zf.ZF_DICT_BP, "delta_bp": zf.ZF_DELTA_BP, "rle": zf.ZF_RLE}
    handles, buf_bytes, parts, expects = [], [], [], []
    for ci, (name, dt, kind) in enumerate(W.FACT_COLUMNS):
        x = W.fact_column(seed, ci, rows)
        isz = x.itemsize
        r0 = 0
        for n in W.fact_pieces(seed, ci, rows):
            handles.append(compress(zf, x[r0:r0 + n], scheme_of[FACT_SCHEMES[kind]], (n + 1023) // 1024 * 1024))
            parts.append([(ci, r0 * isz, n * isz)])
            r0 += n
        buf_bytes.append(x.nbytes)
        expects.append(x if keep else (stride, x[::stride].copy()))
        del x
    return Cfg("c4", FACT_WORKLOAD.format(rows=rows, pieces=len(handles)), handles, buf_bytes, parts, expects,
               "tiles_kernel<-1, -1> (batched work queue; one launch when resident)", batched=True)


def make_workload(seed: int, rows: int = N_ROWS):
    import zf_workloads as W
    return W.sorted_keys(seed, rows), W.dates_rle(seed, rows)


def verify(cfg: Cfg, bufs):
    """The decode of this run equals the generator's columns."""
    for b, (buf, want) in enumerate(zip(bufs, cfg.expects)):
        if isinstance(want, tuple):
            stride, sample = want
            got = buf.view(-1)[: cfg.buf_bytes[b]].cpu().numpy().view(sample.dtype)[::stride]
        else:
            got, sample = buf[: cfg.buf_bytes[b]].cpu().numpy().view(want.dtype), want
        if not np.array_equal(got.view(np.uint8), sample.view(np.uint8)):
            raise AssertionError(f"{cfg.name}: decoded buffer {b} differs from the generator's column")


def measure(zf, torch, cfg: Cfg, args, local: int, streams, flush, barrier=None, clk=None):
    """Time one configuration: resident decode (CUDA events on the decode
    stream, L2 flushed before each step), its dominant launch alone, the end
    to end transfer (host wall clock around zf_transfer_decompress +
    zf_sync, graph replay on or off as the sweep chose) and the raw link at the call's own
    pieces (zf_measure_copy).  `clk` (a Clocks) records the timed loops as
    its sampling windows.  Returns (record, step times in ms, sizes) for the
    caller's reduction over ranks."""
    copy_s, comp_s = streams
    ctx = zf.zf_ctx_create(local, copy_s.cuda_stream, comp_s.cuda_stream)
    flags = zf.ZF_KCFG_GRAPH | (zf.ZF_KCFG_BATCHED if cfg.batched else 0)
    zf.zf_ctx_set_kcfg(ctx, args.tile_rows, args.threads, args.ctas_per_sm, int(cfg.stage_mb * (1 << 20)), flags)
    if args.slots:
        zf.zf_ctx_set_ring(ctx, args.slots)
    bufs = [torch.empty(max(16, n), dtype=torch.uint8, device="cuda") for n in cfg.buf_bytes]
    outs, caps = [], []
    for p in cfg.parts:
        for b, off, n in p:
            outs.append(bufs[b].data_ptr() + off)
            caps.append(n)
    kouts, kcaps = [], []
    for i in cfg.kernel_idx:
        for b, off, n in cfg.parts[i]:
            kouts.append(bufs[b].data_ptr() + off)
            kcaps.append(n)
    raw = sum(zf.zf_compressed_info(h)[0] for h in cfg.handles)
    comp = sum(zf.zf_compressed_info(h)[1] for h in cfg.handles)
    kraw = sum(zf.zf_compressed_info(cfg.handles[i])[0] for i in cfg.kernel_idx)
    kcomp = sum(zf.zf_compressed_info(cfg.handles[i])[1] for i in cfg.kernel_idx)
    # parity of this run's outputs before timing
    torch.cuda.synchronize()
    zf.zf_transfer_decompress(ctx, cfg.handles, outs, caps)
    zf.zf_sync(ctx)
    verify(cfg, bufs)
    tuned = None
    if not args.no_tune:
        # the geometry: zf_tune's exhaustive search of the resident decode (tile rows x threads, 15
        # points), then the pipeline stage size by timing the transfer at each candidate
        t0 = time.perf_counter()
        # one search per output column (each a single class: the context keeps a geometry per class)
        by_col = {}
        for i, p in enumerate(cfg.parts):
            by_col.setdefault(p[0][0], []).append(i)
        npts, per_class = 0, []
        for b, idx in by_col.items():
            oo = [bufs[bb].data_ptr() + off for i in idx for bb, off, n in cfg.parts[i]]
            cc = [n for i in idx for bb, off, n in cfg.parts[i]]
            pts, best = zf.zf_tune(ctx, [cfg.handles[i] for i in idx], oo, cc, transfer=False, reps=args.tune_reps)
            npts += len(pts)
            per_class.append((best.tile_rows, best.threads))
        stage_ms = {}
        for st_mb in [m for m in (2, 4, 8, 16, 32, 64, 128) if comp <= 1500 * (m << 20) or m == 128]:
            # each stage size with and without graph replay: a replayed graph costs the host less,
            # plain launches let the copies start while the host still enqueues
            for graph in (True, False):
                fl = flags if graph else flags & ~zf.ZF_KCFG_GRAPH
                zf.zf_ctx_set_kcfg(ctx, 0, 0, args.ctas_per_sm, st_mb << 20, fl)
                tt = []
                for _ in range(1 + max(3, args.tune_reps)):
                    t1 = time.perf_counter()
                    zf.zf_transfer_decompress(ctx, cfg.handles, outs, caps)
                    st, stats = zf.zf_sync(ctx)
                    tt.append((time.perf_counter() - t1) * 1e3)   # host wall clock, as the e2e steps are timed
                stage_ms[(st_mb, graph)] = float(np.min(tt[1:]))   # the fastest repeat: host hiccups only add time
        st_best, graph_best = min(stage_ms, key=stage_ms.get)
        if not graph_best:
            flags &= ~zf.ZF_KCFG_GRAPH
        zf.zf_ctx_set_kcfg(ctx, 0, 0, args.ctas_per_sm, st_best << 20, flags)
        tuned = {"per_column_tile_rows_threads": sorted(set(per_class)), "stage_bytes": st_best << 20,
                 "graph_replay": graph_best, "resident_points": npts,
                 "stage_ms": {f"{k[0]}{'' if k[1] else ' no graph'}": round(v, 4) for k, v in stage_ms.items()},
                 "search_s": round(time.perf_counter() - t0, 2)}
        zf.zf_transfer_decompress(ctx, cfg.handles, outs, caps)
        zf.zf_sync(ctx)
        verify(cfg, bufs)
    res = [zf.zf_upload(ctx, h) for h in cfg.handles]
    kres = [res[i] for i in cfg.kernel_idx]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def resident(rs, o, c):
        with torch.cuda.stream(comp_s):
            flush.fill_(1)
            e0.record(comp_s)
            zf.zf_decompress_resident(ctx, rs, o, c)
            e1.record(comp_s)
        st, stats = zf.zf_sync(ctx)
        return e0.elapsed_time(e1), stats.n_launches

    def e2e():
        t0 = time.perf_counter()
        zf.zf_transfer_decompress(ctx, cfg.handles, outs, caps)
        st, stats = zf.zf_sync(ctx)
        return (time.perf_counter() - t0) * 1e3, stats.n_launches

    # the raw link at the call's own pieces, measured on a second context
    # (so the measured rate does not reorder the timed context's graph) and
    # interleaved with the end-to-end steps, so both see the same host
    lctx = zf.zf_ctx_create(local, copy_s.cuda_stream, comp_s.cuda_stream)
    stage = tuned["stage_bytes"] if tuned else int(cfg.stage_mb * (1 << 20))
    zf.zf_ctx_set_kcfg(lctx, args.tile_rows, args.threads, args.ctas_per_sm, stage, flags | zf.ZF_KCFG_KEEP_ORDER)
    link_acc = []

    def e2e_and_link():
        ms, nl = e2e()
        link_acc.append(zf.zf_measure_copy(lctx, cfg.handles, 1))
        return ms, nl

    for _ in range(args.warmup):
        resident(res, outs, caps)
        resident(kres, kouts, kcaps)
        e2e()
    launches = 0
    t_res, t_k, t_e = [], [], []
    import gc
    gc.collect()
    gc.disable()   # no collector pauses inside the timed loops
    for loop, fn, acc in ((0, lambda: resident(res, outs, caps), t_res), (1, lambda: resident(kres, kouts, kcaps), t_k),
                          (2, e2e_and_link, t_e)):
        if barrier:
            barrier()
        if clk:
            clk.window_start()
        for _ in range(args.steps):
            ms, nl = fn()
            acc.append(ms)
            launches += nl
        if barrier:
            barrier()
        if clk:
            clk.window_end()
    gc.enable()
    # the decode after timing is still exact (graph replays included, when used)
    verify(cfg, bufs)
    link_ms = float(np.mean(link_acc))
    link_med = float(np.median(link_acc))
    batched_ms = None
    if cfg.compare_batched:
        # the same resident decode through the batched work-queue kernel
        zf.zf_ctx_set_kcfg(ctx, args.tile_rows, args.threads, args.ctas_per_sm, stage, zf.ZF_KCFG_BATCHED)
        bt = []
        for i in range(args.warmup + args.steps):
            ms, nl = resident(res, outs, caps)
            if i >= args.warmup:
                bt.append(ms)
        batched_ms = float(np.mean(bt))
        verify(cfg, bufs)
    for r in res:
        zf.zf_resident_free(r)
    zf.zf_ctx_destroy(lctx)
    zf.zf_ctx_destroy(ctx)
    del bufs
    hbm, kind = peaks()
    tr, tk, te = float(np.mean(t_res)), float(np.mean(t_k)), float(np.mean(t_e))
    link = comp / (link_ms * 1e-3) / 1e9
    cr = raw / comp
    rec = {
        "workload": cfg.workload, "raw_bytes": raw, "comp_bytes": comp, "compression_ratio": round(cr, 3),
        "resident_gbs": round(raw / (tr * 1e-3) / 1e9, 2), "resident_ms": round(tr, 4),
        "e2e": {"gbs": round(raw / (te * 1e-3) / 1e9, 2), "ms": round(te, 4),
                "ms_min_median_max": [round(float(np.min(t_e)), 4), round(float(np.median(t_e)), 4),
                                      round(float(np.max(t_e)), 4)],
                "gbs_median_step": round(raw / (float(np.median(t_e)) * 1e-3) / 1e9, 2),
                "raw_h2d_link_gbs": round(link, 2), "link_ms": round(link_ms, 4),
                "link_ms_min_median_max": [round(float(np.min(link_acc)), 4), round(link_med, 4),
                                           round(float(np.max(link_acc)), 4)],
                "link_x_cr_gbs": round(link * cr, 2), "frac_of_link_x_cr": round(link_ms / te, 4),
                "frac_of_link_x_cr_medians": round(link_med / float(np.median(t_e)), 4),
                "link_sampling": "one copy-only pass of the same pieces after every timed end-to-end step"},
        "kernel": {"name": cfg.kernel, "algorithmic_bytes_per_launch": kraw + kcomp, "launch_ms": round(tk, 4),
                   "achieved_gbs": round((kraw + kcomp) / (tk * 1e-3) / 1e9, 1), "peak_gbs": hbm, "peak_kind": kind,
                   "frac": round((kraw + kcomp) / (tk * 1e-3) / 1e9 / hbm, 4)},
        "parity": "decode equals the generator's columns before and after timing",
        "launches": launches,
    }
    rec["geometry"] = tuned if tuned else "built-in (no search)"
    if batched_ms is not None:
        rec["resident_batched"] = {"gbs": round(raw / (batched_ms * 1e-3) / 1e9, 2), "ms": round(batched_ms, 4),
                                   "vs_single_scheme": round(tr / batched_ms, 4)}
    return rec, (tr, tk, te), (raw, comp, kraw + kcomp, link)


# ---------------------------------------------------------------- CPU oracle legs
def fact_sample_blobs(seed: int, rows: int):
    """A bounded sample of the fact table for the oracle: the first `rows`
    rows of every column, cut into that column's own first pieces, each
    piece encoded by the oracle (one chunk per piece, the scheme of its
    column kind).  Returns [(chunk blob, numpy dtype)], columns interleaved."""
    import oracle
    import zf_workloads as W
    per_col = []
    for ci, (name, dt, kind) in enumerate(W.FACT_COLUMNS):
        x = W.fact_column(seed, ci, rows)
        blobs, r0 = [], 0
        for n in W.fact_pieces(seed, ci, FACT_ROWS):
            n = min(n, rows - r0)
            if n <= 0:
                break
            buf = oracle.encode(x[r0:r0 + n], oracle.SCHEMES[FACT_SCHEMES[kind]], (n + 1023) // 1024 * 1024)
            blobs += chunk_blobs(buf, np.dtype(dt))
            r0 += n
        per_col.append(blobs)
    return [col[k] for k in range(max(len(c) for c in per_col)) for col in per_col if k < len(col)]


def cpu_baseline_of(blobs, budget_s: float):
    """The oracle on all host cores (2/3 of the budget) and on one thread."""
    import oracle
    oracle.build()
    nt = host_threads()
    b, s, n = oracle_sample(blobs, budget_s * 2 / 3, nt)
    b1, s1, n1 = oracle_sample(blobs, budget_s / 3, 1)
    return {"value": round(b / s / 1e9, 4), "unit": "GB/s", "cores": nt, "kind": "oracle",
            "sample": f"{n} chunk decodes taken round-robin over the fact table's 16 columns' pieces on {nt} host "
                      f"threads (uncompressed GB/s)", "single_thread_value": round(b1 / s1 / 1e9, 4)}


def run_reference(args, rank: int):
    """CPU oracle arm: each step decodes a bounded sample of the fact table,
    encoded by the oracle itself, on all host cores."""
    import oracle
    oracle.build()
    rows = min(args.fact_rows, args.ref_rows)
    blobs = fact_sample_blobs(1, rows)
    nt = host_threads()
    for _ in range(args.warmup):
        oracle_sample(blobs, 0.0, nt)
    tot_b, tot_s, tot_n = 0, 0.0, 0
    step_s = args.ref_step_s if args.ref_step_s is not None else min(2.0, max(0.3, 60.0 / args.steps))
    for _ in range(args.steps):
        b, s, n = oracle_sample(blobs, step_s, nt)
        tot_b += b
        tot_s += s
        tot_n += n
    v = tot_b / tot_s / 1e9
    desc = (f"{tot_n} chunk decodes over the first {rows:,} rows of each fact-table column (its own uneven pieces, "
            f"oracle-encoded), {nt} host threads, about {step_s:.2f} s per step")
    line = {"metric": METRIC, "value": round(v, 4), "unit": "GB/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(tot_s / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64/int32", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": FACT_WORKLOAD.format(rows=args.fact_rows, pieces="its"), "sample": desc},
            "cpu_baseline": {"value": round(v, 4), "unit": "GB/s", "cores": nt, "kind": "oracle", "sample": desc},
            "e2e": {"value": round(v, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


SELECTOR_METRIC = "learned selector: mean regret vs exhaustive class search on held-out columns"


def selector_dataset(zf, ctx, seeds, cap_rows: int, reps: int = 2):
    """Features and measured per-class transfer+decode times of the columns
    with the given seeds (columns are generated a few ahead on host threads
    while the GPU measures the current one)."""
    import concurrent.futures
    import zf_workloads as W
    F, T, fam, dts = [], [], [], []
    seeds = list(seeds)
    ex = concurrent.futures.ThreadPoolExecutor(4)
    ahead = [ex.submit(W.selector_column, s, cap_rows) for s in seeds[:8]]
    for i, s in enumerate(seeds):
        x, o, meta = ahead[i].result()
        ahead[i] = None
        if i + 8 < len(seeds):
            ahead.append(ex.submit(W.selector_column, seeds[i + 8], cap_rows))
        col = zf.Column(x, o)
        F.append(zf.zf_column_features(col))
        T.append(zf.zf_measure_classes(ctx, col, reps))
        fam.append(meta["family"])
        dts.append(meta.get("dtype", "bytes"))
    ex.shutdown()
    return np.array(F, np.float32), np.array(T, np.float32), fam, dts


def selector_eval(zf, ctx, F, T, n_train, epochs=400, batch=256, lr=1e-3, seed=1):
    """Train the MLP on the first n_train columns (on the GPU), evaluate the
    rest; returns a dict of regrets and the trained network."""
    mask = T >= 0
    y = np.where(mask, T, np.inf).argmin(1).astype(np.int32)
    Ftr, Fte = F[:n_train], F[n_train:]
    net = zf.zf_mlp_create(0, seed)
    t0 = time.perf_counter()
    # the library standardizes the features (statistics of the training rows, kept by the network)
    losses = zf.zf_mlp_train(net, Ftr, y[:n_train], mask[:n_train], epochs, batch, lr, seed=seed)
    train_s = time.perf_counter() - t0
    pred = zf.zf_mlp_predict(net, Fte, mask[n_train:])
    Tte, yte = T[n_train:], y[n_train:]
    best = Tte[np.arange(len(yte)), yte]

    def regret(choice):
        return float(np.mean((Tte[np.arange(len(yte)), choice] - best) / best))

    # the method without the network: one static class (per value type),
    # the best one on the training columns
    def static_choice(Ttr, Tev):
        mtr = Ttr >= 0
        btr = np.where(mtr, Ttr, np.inf).min(1)
        best_k, best_r = -1, np.inf
        for k in range(Ttr.shape[1]):
            if not mtr[:, k].all():
                continue
            r = np.mean((Ttr[:, k] - btr) / btr)
            if r < best_r:
                best_k, best_r = k, r
        return best_k
    is_bytes = F[:, 2] > 0.5
    static = np.zeros(len(yte), np.int32)
    for grp in (False, True):
        tr = is_bytes[:n_train] == grp
        te = is_bytes[n_train:] == grp
        if te.any():
            static[te] = static_choice(T[:n_train][tr], Tte[te])
    return {"regret": regret(pred), "accuracy": float((pred == yte).mean()), "static_regret": regret(static),
            "static_classes": sorted(set(static.tolist())), "loss_first": float(losses[0]),
            "loss_last": float(losses[-1]), "train_s": round(train_s, 3), "pred": pred, "labels": yte}, net


def run_selector(args, zf, torch):
    import zf_workloads as W
    n_train, n_test = args.sel_train, args.sel_test
    ctx = zf.zf_ctx_create(0)
    t0 = time.perf_counter()
    F, T, fam, dts = selector_dataset(zf, ctx, range(1, n_train + n_test + 1), args.sel_cap)
    collect_s = time.perf_counter() - t0
    res, net = selector_eval(zf, ctx, F, T, n_train)
    # the rule-based heuristic (zf_plan selector 0) on the held-out columns
    heur = []
    for i, s in enumerate(range(n_train + 1, n_train + n_test + 1)):
        x, o, meta = W.selector_column(s, args.sel_cap)
        col = zf.Column(x, o)
        p = zf.zf_plan(None, col, selector=0)
        k = p.scheme * 2 if o is None else (zf.ZF_LZ77 * 2)
        tt = T[n_train + i]
        b = tt[tt >= 0].min()
        heur.append((tt[k] - b) / b if tt[k] >= 0 else np.nan)
    # the trained network inside zf_plan, and its inference time
    zf.zf_ctx_set_selector(ctx, net)
    x, o, meta = W.selector_column(n_train + 1, args.sel_cap)
    col = zf.Column(x, o)
    zf.zf_plan(ctx, col, selector=1)
    t1 = time.perf_counter()
    for _ in range(20):
        zf.zf_plan(ctx, col, selector=1)
    plan_us = (time.perf_counter() - t1) / 20 * 1e6
    Fn = F[n_train:].astype(np.float32)
    m = (T[n_train:] >= 0).astype(np.uint8)
    zf.zf_mlp_predict(net, Fn, m)
    t1 = time.perf_counter()
    for _ in range(20):
        zf.zf_mlp_predict(net, Fn, m)
    infer_us = (time.perf_counter() - t1) / 20 * 1e6
    line = {"metric": SELECTOR_METRIC, "value": round(res["regret"], 4), "unit": "fraction", "n_gpus": 1,
            "steps": 1, "warmup": 1, "higher_is_better": False, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"selector: {n_train} train + {n_test} held-out seeded columns "
                                   f"(uniform/zipf/sorted/runs/text; int32/int64/bytes), rows log-uniform 1M-64M "
                                   f"capped at {args.sel_cap} for label collection, 12 classes = 6 schemes x "
                                   f"{{4, 32}} MiB chunks, labels = fastest measured transfer+decode",
                       "collect_s": round(collect_s, 1)},
            "selector": {"regret": round(res["regret"], 4), "accuracy": round(res["accuracy"], 4),
                         "static_class_regret": round(res["static_regret"], 4),
                         "static_classes": res["static_classes"],
                         "heuristic_regret": round(float(np.nanmean(heur)), 4),
                         "loss_first_epoch": round(res["loss_first"], 4), "loss_last_epoch": round(res["loss_last"], 4),
                         "gpu_train_s": res["train_s"], "plan_us_with_features": round(plan_us, 1),
                         "predict_us_batch": round(infer_us, 1), "predict_batch": n_test,
                         "label_counts": np.bincount(np.where(T >= 0, T, np.inf).argmin(1), minlength=12).tolist()}}
    print(json.dumps(line), flush=True)
    zf.zf_mlp_destroy(net)
    zf.zf_ctx_destroy(ctx)


def run_profile(args, zf, torch):
    """Resident decode of one workload column, nothing else (ncu target)."""
    import zf_workloads as W
    ctx = zf.zf_ctx_create(0)
    if any((args.tile_rows, args.threads, args.ctas_per_sm)):
        zf.zf_ctx_set_kcfg(ctx, args.tile_rows, args.threads, args.ctas_per_sm, 0, 0)
    hs, outs, caps, bufs = [], [], [], []
    if args.profile == "for":
        # the Fully-Parallel column at scale: int32 uniform on [0, 4096) (the top
        # 12 bits of the counter-based generator), FOR + 12-bit packing,
        # 65,536-row chunks
        cols = [(W.uniform_int(1, 0, 0, args.rows, 0, 4096).astype(np.int32), zf.ZF_FOR_BP, 65536)]
    elif args.profile == "ans":
        # a return-flag-like column: 'A', 'N', 'R' as int32 with shares 1/4, 1/2, 1/4
        # (uniform on [0, 4) from the counter-based generator, 1 and 2 both 'N'),
        # dictionary + ANS in 1M-row chunks
        u = W.uniform_int(1, 11, 0, args.rows, 0, 4)
        cols = [(np.array([65, 78, 78, 82], np.int32)[u], zf.ZF_ANS, CHUNK_ROWS)]
    elif args.profile == "float":
        # float64 prices with two decimals (log-normal cents / 100), Float2Int + packing, 1M-row chunks
        cols = [(W.decimal_prices(1, 7, 0, args.rows), zf.ZF_FLOAT2INT, CHUNK_ROWS)]
    elif args.profile == "fact":
        # the fact table (--fact-rows rows per column) as its uneven pieces, one batched launch per step
        zf.zf_ctx_set_kcfg(ctx, args.tile_rows, args.threads, args.ctas_per_sm, 0, zf.ZF_KCFG_BATCHED)
        cfg = build_c4(zf, 1, args.fact_rows, keep=False)
        bufs = [torch.empty(n, dtype=torch.uint8, device="cuda") for n in cfg.buf_bytes]
        hs = cfg.handles
        for p in cfg.parts:
            for b, off, n in p:
                outs.append(bufs[b].data_ptr() + off)
                caps.append(n)
        cols = []
    elif args.profile in ("strdict", "lz77"):
        # the text column (Zipf words), as a string dictionary in 4 MiB chunks or as LZ77 blocks
        t, o = W.text_column(1, int(args.text_mb * (1 << 20)))
        cols = [((t, o), zf.ZF_STRDICT if args.profile == "strdict" else zf.ZF_LZ77,
                 int(args.text_chunk_mb * (1 << 20)) if args.profile == "strdict" else 0)]
    else:
        keys, dates = make_workload(1, args.rows)
        cols = [(x, s, CHUNK_ROWS) for x, s, on in ((keys, zf.ZF_DELTA_BP, args.profile in ("keys", "both")),
                                                   (dates, zf.ZF_RLE, args.profile in ("dates", "both"))) if on]
    for x, s, cr in cols:
        parts = list(x) if isinstance(x, tuple) else [x]
        c = zf.Column(*parts)
        h = zf.zf_compress_host(zf.zf_plan(ctx, c, scheme=s, chunk_rows=cr), c)
        hs.append(h)
        for p in parts:
            b = torch.empty(p.nbytes, dtype=torch.uint8, device="cuda")
            bufs.append(b)
            outs.append(b.data_ptr())
            caps.append(p.nbytes)
    rs = [zf.zf_upload(ctx, h) for h in hs]
    ms = []
    for i in range(args.warmup + args.steps):
        zf.zf_decompress_resident(ctx, rs, outs, caps)
        st, stats = zf.zf_sync(ctx)
        if i >= args.warmup:
            ms.append(stats.total_ms)
    raw = sum(caps)
    comp = sum(zf.zf_compressed_info(h)[1] for h in hs)
    hbm, kind = peaks()
    alg = (raw + comp) / np.median(ms) / 1e6
    print(json.dumps({"profile": args.profile, "rows": args.rows, "raw_bytes": raw, "comp_bytes": comp,
                      "ms": round(float(np.median(ms)), 4), "gbs": round(raw / np.median(ms) / 1e6, 1),
                      "algorithmic_gbs": round(alg, 1), "frac_of_" + kind + "_hbm": round(alg / hbm, 4)}))
    for r in rs:
        zf.zf_resident_free(r)
    for h in hs:
        zf.zf_compressed_free(h)
    zf.zf_ctx_destroy(ctx)




def run_ans_sweep(args, zf, torch):
    """Section 5.2.3's trade of compression ratio against decode throughput as
    the ANS chunk size changes: the return-flag-like column at every chunk
    size (rows per chunk) and stream length (rows per independent rANS
    stream) of the grid, resident decode timed with CUDA events (median of
    --steps after --warmup), the decode checked against the column first."""
    import zf_workloads as W
    u = W.uniform_int(1, 11, 0, args.rows, 0, 4)
    x = np.array([65, 78, 78, 82], np.int32)[u]
    col = zf.Column(x)
    ctx = zf.zf_ctx_create(0)
    out = torch.empty(x.nbytes, dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    points = []
    for cr in (1 << 16, 1 << 18, 1 << 20, 1 << 22):
        for L in (32, 64, 128, 256, 512, 1024, 2048, 4096):
            h = zf.zf_compress_host(zf.zf_plan(ctx, col, scheme=zf.ZF_ANS, chunk_rows=cr, ans_stream_rows=L), col)
            raw, comp, nch = zf.zf_compressed_info(h)
            r = zf.zf_upload(ctx, h)
            zf.zf_decompress_resident(ctx, [r], [out.data_ptr()], [x.nbytes])
            zf.zf_sync(ctx)
            assert np.array_equal(out.cpu().numpy().view(np.int32), x), (cr, L)
            ms = []
            for i in range(args.warmup + args.steps):
                flush.fill_(1)
                torch.cuda.synchronize()
                zf.zf_decompress_resident(ctx, [r], [out.data_ptr()], [x.nbytes])
                st, stats = zf.zf_sync(ctx)
                if i >= args.warmup:
                    ms.append(stats.total_ms)
            t = float(np.median(ms))
            points.append({"chunk_rows": cr, "stream_rows": L, "compression_ratio": round(raw / comp, 3),
                           "comp_bytes": comp, "ms": round(t, 4), "gbs": round(raw / t / 1e6, 1),
                           "algorithmic_gbs": round((raw + comp) / t / 1e6, 1)})
            zf.zf_resident_free(r)
            zf.zf_compressed_free(h)
    print(json.dumps({"workload": f"ans sweep: {args.rows:,} int32 rows 'A','N','R' at 1/4, 1/2, 1/4",
                      "metric": "compression ratio and resident decode GB/s per (chunk rows, stream rows)",
                      "points": points}), flush=True)
    zf.zf_ctx_destroy(ctx)


def run_johnson(args, zf, torch):
    """Section 3.3's ordering of a call's columns for the two-stage flow
    (copy, then decode) by Johnson's rule, on a mixed call: a 64 MiB LZ77
    text column (decode-heavy), 64M RLE dates and 64M FOR integers (copy-
    heavy).  Each column's decode rate is measured by zf_tune (resident, its
    own class) and the link by zf_measure_copy, so the library orders by
    measured times; the same call is then timed end to end in Johnson's
    order, in the order given, and in the reverse of Johnson's order (both
    with ZF_KCFG_KEEP_ORDER)."""
    import zf_workloads as W
    t, o = W.text_column(1, 64 << 20)
    dates = W.dates_rle(1, args.rows)
    ints = W.uniform_int(1, 0, 0, args.rows, 0, 4096).astype(np.int32)
    cols = [((t, o), zf.ZF_LZ77, 0, "lz77 text"), ((ints,), zf.ZF_FOR_BP, 65536, "for int32"),
            ((dates,), zf.ZF_RLE, CHUNK_ROWS, "rle dates")]
    copy_s, comp_s = torch.cuda.Stream(), torch.cuda.Stream()
    ctx = zf.zf_ctx_create(0, copy_s.cuda_stream, comp_s.cuda_stream)
    hs, outs, caps, bufs, per = [], [], [], [], []
    for arrays, scheme, cr, name in cols:
        col = zf.Column(*arrays)
        h = zf.zf_compress_host(zf.zf_plan(ctx, col, scheme=scheme, chunk_rows=cr), col)
        hs.append(h)
        o_, c_ = [], []
        for a in arrays:
            b = torch.empty(a.nbytes, dtype=torch.uint8, device="cuda")
            bufs.append(b)
            o_.append(b.data_ptr())
            c_.append(a.nbytes)
        per.append((o_, c_))
    # measured decode time of each column (its class's best point) and the link
    dec_ms = []
    for h, (o_, c_) in zip(hs, per):
        pts, best = zf.zf_tune(ctx, [h], o_, c_, transfer=False, reps=3)
        dec_ms.append(min(p.ms for p in pts))
    link_ms = zf.zf_measure_copy(ctx, hs, 5)
    comp = [zf.zf_compressed_info(h)[1] for h in hs]
    copy_ms = [link_ms * c / sum(comp) for c in comp]
    jo = [int(i) for i in zf.zf_johnson_order(np.array(copy_ms, np.float32), np.array(dec_ms, np.float32))]
    raw = sum(zf.zf_compressed_info(h)[0] for h in hs)

    def timed(order, flags):
        zf.zf_ctx_set_kcfg(ctx, 0, 0, 0, 64 << 20, flags | zf.ZF_KCFG_GRAPH)
        oo = [x for i in order for x in per[i][0]]
        cc = [x for i in order for x in per[i][1]]
        hh = [hs[i] for i in order]
        ms = []
        for k in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            zf.zf_transfer_decompress(ctx, hh, oo, cc)
            zf.zf_sync(ctx)
            if k >= args.warmup:
                ms.append((time.perf_counter() - t0) * 1e3)
        return float(np.median(ms))
    given = list(range(len(cols)))
    res = {"library (Johnson, measured rates)": timed(given, 0),
           "johnson order, kept": timed(jo, zf.ZF_KCFG_KEEP_ORDER),
           "given order, kept": timed(given, zf.ZF_KCFG_KEEP_ORDER),
           "reverse of johnson, kept": timed(jo[::-1], zf.ZF_KCFG_KEEP_ORDER)}
    # the decode after all of them is still exact
    for (arrays, *_r), (o_, c_) in zip(cols, per):
        for a, ptr, n in zip(arrays, o_, c_):
            got = next(b for b in bufs if b.data_ptr() == ptr)[:n].cpu().numpy().view(a.dtype)
            assert np.array_equal(got, a)
    print(json.dumps({"workload": "johnson: 64 MiB LZ77 text + %d int32 FOR + %d int32 RLE dates in one call" % (
        args.rows, args.rows), "columns": [c[3] for c in cols], "copy_ms": [round(x, 4) for x in copy_ms],
        "decode_ms": [round(x, 4) for x in dec_ms], "johnson_order": [cols[i][3] for i in jo],
        "e2e_ms": {k: round(v, 4) for k, v in res.items()},
        "e2e_gbs": {k: round(raw / v / 1e6, 1) for k, v in res.items()}}), flush=True)
    for h in hs:
        zf.zf_compressed_free(h)
    zf.zf_ctx_destroy(ctx)


ALL_CONFIGS = ("c1", "c2", "c3_lz77", "c3_strdict", "ans", "float2int", "c4")


def build_config(zf, name, args, seed, world, text_cache):
    import zf_workloads as W
    if name in ("c3_lz77", "c3_strdict") and "text" not in text_cache:
        text_cache["text"] = W.text_column(seed, int(args.text_mb * (1 << 20)))
    if name == "c1":
        return build_c1(zf, seed)
    if name == "c2":
        return build_c2(zf, seed, args.rows)
    if name == "c3_lz77":
        return build_c3(zf, seed, text_cache["text"], "lz77", args.text_chunk_mb)
    if name == "c3_strdict":
        return build_c3(zf, seed, text_cache["text"], "strdict", args.text_chunk_mb)
    if name == "ans":
        return build_ans(zf, seed, args.rows)
    if name == "float2int":
        return build_f2i(zf, seed, args.rows)
    if name == "c4":
        return build_c4(zf, seed, args.fact_rows, keep=world == 1)
    raise ValueError(name)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="zipflow", choices=["zipflow", "reference"])
    ap.add_argument("--ref-step-s", type=float, default=None,
                    help="CPU seconds per reference step (default: 2 s, less for long runs so that "
                         "all steps take about a minute)")
    ap.add_argument("--ref-rows", type=int, default=4_000_000, help="fact-table rows per column in the reference sample")
    ap.add_argument("--cpu-budget-s", type=float, default=12.0, help="CPU seconds for the cpu_baseline sample")
    ap.add_argument("--tile-rows", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--stage-mb", type=float, default=0)
    ap.add_argument("--slots", type=int, default=0)
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    ap.add_argument("--no-tune", action="store_true", help="time the built-in geometry (no zf_tune search first)")
    ap.add_argument("--tune-reps", type=int, default=1, help="timed runs per point of the geometry search")
    ap.add_argument("--profile", choices=["keys", "dates", "both", "for", "float", "ans", "strdict", "lz77", "fact"],
                    default=None,
                    help="only decode the resident column(s) --steps times (for ncu captures)")
    ap.add_argument("--rows", type=int, default=N_ROWS, help="rows per column of c2, ans, float2int and profiles")
    ap.add_argument("--fact-rows", type=int, default=FACT_ROWS, help="rows per column of the fact table (c4)")
    ap.add_argument("--workload", default="all",
                    help="all (the headline fact table plus every other configuration), selector, ans_sweep, johnson, "
                         "or a "
                         "comma list "
                         f"of {', '.join(ALL_CONFIGS)}")
    ap.add_argument("--text-mb", type=float, default=256, help="string column size (c3), MiB")
    ap.add_argument("--text-chunk-mb", type=float, default=4, help="string-dictionary chunk size, MiB")
    ap.add_argument("--sel-train", type=int, default=2000)
    ap.add_argument("--sel-test", type=int, default=200)
    ap.add_argument("--sel-cap", type=int, default=2_000_000, help="row cap for label collection")
    args = ap.parse_args()
    assert args.warmup >= 3 or args.profile, "at least 3 warm-up steps"

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args, rank)
        return

    import torch
    import paper_2602_08190_gb300 as zf
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.profile:
        assert world == 1
        return run_profile(args, zf, torch)
    if args.workload == "selector":
        assert world == 1
        return run_selector(args, zf, torch)
    if args.workload == "ans_sweep":
        assert world == 1
        return run_ans_sweep(args, zf, torch)
    if args.workload == "johnson":
        assert world == 1
        return run_johnson(args, zf, torch)
    names = list(ALL_CONFIGS) if args.workload == "all" else args.workload.split(",")
    assert all(n in ALL_CONFIGS for n in names), names
    head = "c4" if "c4" in names else names[0]
    order = [n for n in names if n != head] + [head]
    streams = (torch.cuda.Stream(), torch.cuda.Stream())
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    seed = 1 + rank

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    records, text_cache = {}, {}
    launches = 0
    with Clocks(local) as clk:
        for name in order:
            cfg = build_config(zf, name, args, seed, world, text_cache)
            if name == head:
                rec, times, sizes = measure(zf, torch, cfg, args, local, streams, flush, barrier, clk)
                clk_summary = clk.summary()         # the headline's timed loops only
                head_cfg = cfg
                head_times, head_sizes = times, sizes
            else:
                rec, times, sizes = measure(zf, torch, cfg, args, local, streams, flush, None)
                cfg.free(zf)
            launches += rec.pop("launches")
            if name in TRAFFIC_PROFILES:
                units = args.fact_rows if name == "c4" else args.rows
                rec["kernel"]["traffic"], rec["kernel"]["traffic_note"] = measured_traffic(name, units)
            records[name] = rec
            if name in ("c3_strdict",):
                text_cache.clear()
    t_res, t_k, t_e = max_over_ranks(list(head_times), dist, "cuda")
    raw, comp, kbytes, link = head_sizes
    rec = records.pop(head)
    line = None
    if rank == 0:
        # the oracle on a bounded sample of the headline's own chunks
        import oracle
        blobs = []
        per = max(1, 48 // max(1, len(head_cfg.handles)))
        for h in head_cfg.handles[:: max(1, len(head_cfg.handles) // 48)][:48]:
            ser = zf.zf_compressed_bytes(h)
            dt = {0: np.int32, 1: np.int64, 2: np.uint8, 3: np.float64}[oracle.column_info(ser)["dtype"]]
            blobs += chunk_blobs(ser, np.dtype(dt), per)
        hbm, kind = peaks()
        achieved = kbytes / (t_k * 1e-3) / 1e9
        e2e = whole_job_gbs(world * raw, t_e)
        line = {
            "metric": METRIC, "value": round(whole_job_gbs(world * raw, t_res), 2), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_res, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64/int32", "data": "synthetic",
            "config": {"workload": rec["workload"], "raw_bytes_per_step": raw, "comp_bytes_per_step": comp,
                       "compression_ratio": rec["compression_ratio"],
                       "l2": "inputs and outputs far larger than L2 (and a 256 MiB write before every resident step)",
                       "parallelism": "replicas" if world > 1 else "single",
                       "geometry": rec.get("geometry")},
            "e2e": {"value": round(e2e, 2), "unit": "GB/s", "h2d_bytes_per_step": comp, "d2h_bytes_per_step": 8,
                    "ms_per_step": round(t_e, 4), "raw_h2d_link_gbs": rec["e2e"]["raw_h2d_link_gbs"],
                    "raw_link_at": "the call's own pieces (zf_measure_copy: the same copies, no decode)",
                    "link_x_cr_gbs": rec["e2e"]["link_x_cr_gbs"],
                    "target_0.9_link_x_cr_gbs": round(0.9 * rec["e2e"]["link_x_cr_gbs"], 2),
                    "frac_of_link_x_cr": round(e2e / world / rec["e2e"]["link_x_cr_gbs"], 4),
                    "ms_min_median_max": rec["e2e"]["ms_min_median_max"],
                    "gbs_median_step": rec["e2e"]["gbs_median_step"],
                    "frac_of_link_x_cr_medians": rec["e2e"]["frac_of_link_x_cr_medians"],
                    "link_ms_min_median_max": rec["e2e"]["link_ms_min_median_max"],
                    "link_sampling": rec["e2e"]["link_sampling"]},
            "roofline": {"bound": "hbm", "kernel": rec["kernel"]["name"], "achieved": round(achieved, 1), "peak": hbm,
                         "peak_kind": kind, "unit": "GB/s", "frac": round(achieved / hbm, 4),
                         "traffic": rec["kernel"].get("traffic"), "traffic_note": rec["kernel"].get("traffic_note"),
                         "algorithmic_bytes_per_launch": kbytes, "launch_ms": round(t_k, 4)},
            "cpu_baseline": cpu_baseline_of(blobs, args.cpu_budget_s),
            "clocks": clk_summary,
            "gpu_launches": launches,
            "configs": records,
        }
        print(json.dumps(line), flush=True)
    head_cfg.free(zf)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
