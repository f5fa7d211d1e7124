#!/usr/bin/env python
"""Throughput of compressed-column transfer + decode on GB300.

Workload (one step): a 64M-row int64 sorted key column (gaps geometric, mean
4) in delta + bit-packing with 1024-row blocks, and a 64M-row int32 date
column (2,557 distinct days, runs geometric, mean 8) in RLE, both in 1M-row
chunks (805,306,368 uncompressed bytes per step).

  value   uncompressed GB/s of the decode with the compressed columns already
          resident in HBM (zf_decompress_resident), CUDA events on the
          decode stream, L2 flushed before every step.
  e2e     the same metric end to end through zf_transfer_decompress +
          zf_sync: pinned-host chunks copied host-to-device, decoded,
          and the step's status word read back, host wall clock per step.
  roofline  the dominant kernel (delta decode of the keys) timed alone:
          algorithmic bytes (compressed read + plain written) per launch over
          its CUDA-event duration, against the measured HBM copy peak.
  cpu_baseline  the CPU oracle decoding a bounded sample of the same chunks on
          all host cores (threads over chunks), and on one thread.

--impl reference times the CPU oracle alone on the same metric.
With torchrun (--gpus N) every rank decodes its own replica (no collective on
the data path); value sums the ranks' bytes over the slowest rank's time.
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
WORKLOAD = ("group_parallel: 64M int64 sorted keys (gaps geometric mean 4; delta + bit-packing, 1024-row "
            "blocks) + 64M int32 dates (2,557 days, runs geometric mean 8; RLE), 1M-row chunks")


KERNEL_SOURCES = ("paper_2602_08190_gb300/csrc/zf_device.cuh", "paper_2602_08190_gb300/csrc/zf_kernels.cu")
TRAFFIC_PROFILE = "profiles/delta_i64_decode_32M_rows.md"


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic():
    """DRAM bytes per 64M-row delta launch from the committed ncu summary,
    or None if the kernel sources changed since those counters were taken."""
    path = os.path.join(ROOT, TRAFFIC_PROFILE)
    if not os.path.exists(path):
        return None
    fields = {}
    with open(path) as f:
        for line in f:
            if ":" in line and line.startswith("- "):
                k, v = line[2:].split(":", 1)
                fields[k.strip()] = v.strip().strip("`")
    if fields.get("kernel source hash") != kernel_source_hash():
        return None
    try:
        return int(fields["dram bytes per 64M-row launch (scaled)"])
    except (KeyError, ValueError):
        return None


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

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
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
        during = self.lines[self.first:] or self.lines[-1:]
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


def make_workload(seed: int, rows: int = N_ROWS):
    import zf_workloads as W
    keys = W.sorted_keys(seed, rows)
    dates = W.dates_rle(seed, rows)
    return keys, dates


def oracle_sample(handles, dtypes, budget_s: float, threads: int = 1):
    """Decode chunks of each column with the CPU oracle until `budget_s`
    seconds pass, `threads` host threads taking the chunks round-robin (the
    oracle's C decoder runs outside the GIL); returns (bytes, seconds,
    description)."""
    import concurrent.futures
    import oracle
    import paper_2602_08190_gb300 as zf
    per_col = []
    for h, dt in zip(handles, dtypes):
        b = zf.zf_compressed_bytes(h)
        nch = oracle.column_info(b)["n_chunks"]
        blobs = []
        for c in range(nch):
            off, ln, r0, rows = oracle.chunk_span(b, c)
            blobs.append((b[off:off + ln], dt))
        per_col.append(blobs)
    order = [col[k] for k in range(max(len(c) for c in per_col)) for col in per_col if k < len(col)]
    t0 = time.perf_counter()

    def worker(w):
        nb = nc = 0
        i = w
        while True:
            blob, dt = order[i % len(order)]
            nb += oracle.decode_chunk(blob, dt).nbytes
            nc += 1
            i += threads
            if time.perf_counter() - t0 >= budget_s:
                return nb, nc

    with concurrent.futures.ThreadPoolExecutor(threads) as ex:
        res = list(ex.map(worker, range(threads)))
    dt_s = time.perf_counter() - t0
    done_bytes = sum(r[0] for r in res)
    done_chunks = sum(r[1] for r in res)
    return done_bytes, dt_s, (f"{done_chunks} chunks of 1M rows taken round-robin over the columns, "
                              f"{threads} host thread{'s' if threads > 1 else ''}")


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


def run_reference(args, rank: int):
    """CPU oracle arm: each step decodes a bounded sample of the workload."""
    import oracle
    import paper_2602_08190_gb300 as zf
    oracle.build()
    keys, dates = make_workload(1)
    hk = zf.zf_compress_host(zf.zf_plan(None, zf.Column(keys), scheme=zf.ZF_DELTA_BP, chunk_rows=CHUNK_ROWS),
                             zf.Column(keys))
    hd = zf.zf_compress_host(zf.zf_plan(None, zf.Column(dates), scheme=zf.ZF_RLE, chunk_rows=CHUNK_ROWS),
                             zf.Column(dates))
    nt = host_threads()
    for _ in range(args.warmup):
        oracle_sample([hk, hd], [np.int64, np.int32], 0.0, nt)
    tot_b, tot_s = 0, 0.0
    desc = ""
    for _ in range(args.steps):
        step_s = args.ref_step_s if args.ref_step_s is not None else min(2.0, max(0.3, 60.0 / args.steps))
        b, s, desc = oracle_sample([hk, hd], [np.int64, np.int32], step_s, nt)
        tot_b += b
        tot_s += s
    v = tot_b / tot_s / 1e9
    line = {"metric": METRIC, "value": round(v, 4), "unit": "GB/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(tot_s / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64/int32", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "sample": desc},
            "cpu_baseline": {"value": round(v, 4), "unit": "GB/s", "cores": nt, "kind": "oracle", "sample": desc},
            "e2e": {"value": round(v, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    zf.zf_compressed_free(hk)
    zf.zf_compressed_free(hd)
    print(json.dumps(line), flush=True)


# Schemes of the fact table's column kinds: FOR for small integers and
# scaled decimals, delta for sorted keys, RLE for dates, dictionary for the
# 25-value codes.
FACT_SCHEMES = {"uniform_1_50": "for_bp", "lognormal_cents": "for_bp", "sorted_keys": "delta_bp",
                "dates": "rle", "codes_25": "dict_bp"}
FACT_ROWS = 400_000_000
BATCHED_WORKLOAD = ("batched: 16-column fact table x 400M rows (2 int32 uniform 1-50, 7 int64 log-normal cents, "
                    "2 int64 sorted keys, 3 int32 RLE dates, 2 int32 25-value Zipf codes; 100 B/row, 40 GB), "
                    "streamed in uneven 4-64 MB pieces, one work-queue launch per stage, CUDA graph")


def build_fact_table(zf, rows: int = FACT_ROWS, seed: int = 1, keep: bool = True):
    """Generate the fact table column by column, cut each column into its
    uneven pieces and compress every piece (one single-chunk compressed
    column per piece).  Returns (columns or None, [(handle, col, row0, rows)])."""
    import zf_workloads as W
    scheme_of = {"raw": zf.ZF_RAW, "for_bp": zf.ZF_FOR_BP, "dict_bp": zf.ZF_DICT_BP, "delta_bp": zf.ZF_DELTA_BP,
                 "rle": zf.ZF_RLE}
    cols, pieces = [], []
    for ci, (name, dt, kind) in enumerate(W.FACT_COLUMNS):
        x = W.fact_column(seed, ci, rows)
        scheme = scheme_of[FACT_SCHEMES[kind]]
        r0 = 0
        for n in W.fact_pieces(seed, ci, rows):
            part = zf.Column(x[r0:r0 + n])
            h = zf.zf_compress_host(zf.zf_plan(None, part, scheme=scheme, chunk_rows=(n + 1023) // 1024 * 1024),
                                    part)
            pieces.append((h, ci, r0, n))
            r0 += n
        cols.append(x if keep else None)
    return cols, pieces


def run_batched(args, zf, torch):
    """The batched workload: every piece of the 16 columns in one call."""
    import zf_workloads as W
    rows = args.rows if args.rows != N_ROWS else FACT_ROWS
    cols, pieces = build_fact_table(zf, rows)
    copy_s, comp_s = torch.cuda.Stream(), torch.cuda.Stream()
    ctx = zf.zf_ctx_create(0, copy_s.cuda_stream, comp_s.cuda_stream)
    stage = int((args.stage_mb or 64) * (1 << 20))
    zf.zf_ctx_set_kcfg(ctx, args.tile_rows, args.threads, args.ctas_per_sm, stage,
                       zf.ZF_KCFG_BATCHED | zf.ZF_KCFG_GRAPH)
    if args.slots:
        zf.zf_ctx_set_ring(ctx, args.slots)
    dev = [torch.empty(rows * np.dtype(dt).itemsize, dtype=torch.uint8, device="cuda")
           for _, dt, _ in W.FACT_COLUMNS]
    handles = [h for h, _, _, _ in pieces]
    outs, caps = [], []
    for h, ci, r0, n in pieces:
        isz = np.dtype(W.FACT_COLUMNS[ci][1]).itemsize
        outs.append(dev[ci].data_ptr() + r0 * isz)
        caps.append(n * isz)
    raw = sum(caps)
    comp = sum(zf.zf_compressed_info(h)[1] for h in handles)
    # correctness of this run's outputs before timing
    zf.zf_transfer_decompress(ctx, handles, outs, caps)
    zf.zf_sync(ctx)
    for ci, x in enumerate(cols):
        assert np.array_equal(dev[ci].cpu().numpy().view(x.dtype), x), W.FACT_COLUMNS[ci][0]
    res = [zf.zf_upload(ctx, h) for h in handles]
    e2e_ms, dev_ms, launches = [], [], 0
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        zf.zf_transfer_decompress(ctx, handles, outs, caps)
        st, stats = zf.zf_sync(ctx)
        if i >= args.warmup:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
            launches += stats.n_launches
    for i in range(args.warmup + args.steps):
        zf.zf_decompress_resident(ctx, res, outs, caps)
        st, stats = zf.zf_sync(ctx)
        if i >= args.warmup:
            dev_ms.append(stats.total_ms)
            launches += stats.n_launches
    t_e2e, t_dev = float(np.mean(e2e_ms)), float(np.mean(dev_ms))
    line = {"metric": METRIC, "value": round(raw / (t_dev * 1e-3) / 1e9, 2), "unit": "GB/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_dev, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64/int32", "data": "synthetic",
            "config": {"workload": BATCHED_WORKLOAD, "raw_bytes_per_step": raw, "comp_bytes_per_step": comp,
                       "compression_ratio": round(raw / comp, 3), "pieces": len(pieces), "stage_bytes": stage,
                       "l2": "inputs and outputs far larger than L2"},
            "e2e": {"value": round(raw / (t_e2e * 1e-3) / 1e9, 2), "unit": "GB/s", "h2d_bytes_per_step": comp,
                    "d2h_bytes_per_step": 8, "ms_per_step": round(t_e2e, 3)},
            "gpu_launches": launches}
    print(json.dumps(line), flush=True)
    for r in res:
        zf.zf_resident_free(r)
    for h in handles:
        zf.zf_compressed_free(h)
    zf.zf_ctx_destroy(ctx)


TEXT_WORKLOAD = ("non_parallel: {:,}-byte string column, Zipf(1.1) words from a 5,000-word vocabulary "
                 "(3-12 letters), 1-8 words per row; LZ77 in 64 KiB blocks (one warp per block), int32 offsets "
                 "delta-packed in 65,536-row chunks")
TEXT_STRDICT_WORKLOAD = ("group_parallel string dictionary: {:,}-byte string column, Zipf(1.1) words from a "
                         "5,000-word vocabulary (3-12 letters), 1-8 words per row; tokens (words with their space) "
                         "as bit-packed dictionary codes in {:,}-byte chunks, int32 offsets delta-packed in "
                         "65,536-row chunks")


def run_text(args, zf, torch):
    """The Non-Parallel workload: decode of a 256 MB LZ77 string column (or,
    with --text-scheme strdict, the same column as a string dictionary)."""
    import zf_workloads as W
    t, o = W.text_column(1, int(args.text_mb * (1 << 20)))
    col = zf.Column(t, o)
    strdict = args.text_scheme == "strdict"
    chunk = int(args.text_chunk_mb * (1 << 20))
    plan = zf.zf_plan(None, col, scheme=zf.ZF_STRDICT if strdict else zf.ZF_LZ77, chunk_rows=chunk if strdict else 0)
    h = zf.zf_compress_host(plan, col)
    raw, comp, nch = zf.zf_compressed_info(h)
    copy_s, comp_s = torch.cuda.Stream(), torch.cuda.Stream()
    ctx = zf.zf_ctx_create(0, copy_s.cuda_stream, comp_s.cuda_stream)
    zf.zf_ctx_set_kcfg(ctx, args.tile_rows, args.threads, args.ctas_per_sm, int(args.stage_mb * (1 << 20)), 0)
    if args.slots:
        zf.zf_ctx_set_ring(ctx, args.slots)
    ob = torch.empty(t.nbytes, dtype=torch.uint8, device="cuda")
    oo = torch.empty(o.nbytes, dtype=torch.uint8, device="cuda")
    outs, caps = [ob.data_ptr(), oo.data_ptr()], [t.nbytes, o.nbytes]
    zf.zf_transfer_decompress(ctx, [h], outs, caps)
    zf.zf_sync(ctx)
    assert np.array_equal(ob.cpu().numpy(), t) and np.array_equal(oo.cpu().numpy().view(np.int32), o)
    r = zf.zf_upload(ctx, h)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    dev_ms, e2e_ms, launches = [], [], 0
    for i in range(args.warmup + args.steps):
        with torch.cuda.stream(comp_s):
            flush.fill_(1)
        zf.zf_decompress_resident(ctx, [r], outs, caps)
        st, stats = zf.zf_sync(ctx)
        if i >= args.warmup:
            dev_ms.append(stats.total_ms)
            launches += stats.n_launches
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        zf.zf_transfer_decompress(ctx, [h], outs, caps)
        st, stats = zf.zf_sync(ctx)
        if i >= args.warmup:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
            launches += stats.n_launches
    td, te = float(np.mean(dev_ms)), float(np.mean(e2e_ms))
    line = {"metric": METRIC, "value": round(raw / (td * 1e-3) / 1e9, 2), "unit": "GB/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(td, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8/int32", "data": "synthetic",
            "config": {"workload": (TEXT_STRDICT_WORKLOAD.format(t.nbytes, plan.chunk_rows) if strdict
                                    else TEXT_WORKLOAD.format(t.nbytes)),
                       "raw_bytes_per_step": raw, "comp_bytes_per_step": comp,
                       "compression_ratio": round(raw / comp, 3), "chunks": nch,
                       "l2": "flushed (256 MiB write) before every resident step"},
            "e2e": {"value": round(raw / (te * 1e-3) / 1e9, 2), "unit": "GB/s", "h2d_bytes_per_step": comp,
                    "d2h_bytes_per_step": 8, "ms_per_step": round(te, 4)},
            "gpu_launches": launches}
    print(json.dumps(line), flush=True)
    zf.zf_resident_free(r)
    zf.zf_compressed_free(h)
    zf.zf_ctx_destroy(ctx)


SELECTOR_METRIC = "learned selector: mean regret vs exhaustive class search on held-out columns"


def selector_dataset(zf, ctx, seeds, cap_rows: int, reps: int = 2):
    """Features and measured per-class transfer+decode times of the columns
    with the given seeds."""
    import zf_workloads as W
    F, T, fam, dts = [], [], [], []
    for s in seeds:
        x, o, meta = W.selector_column(s, cap_rows)
        col = zf.Column(x, o)
        F.append(zf.zf_column_features(col))
        T.append(zf.zf_measure_classes(ctx, col, reps))
        fam.append(meta["family"])
        dts.append(meta.get("dtype", "bytes"))
    return np.array(F, np.float32), np.array(T, np.float32), fam, dts


def selector_eval(zf, ctx, F, T, n_train, epochs=400, batch=256, lr=1e-3, seed=1):
    """Train the MLP on the first n_train columns (on the GPU), evaluate the
    rest; returns a dict of regrets and the trained network."""
    mask = T >= 0
    y = np.where(mask, T, np.inf).argmin(1).astype(np.int32)
    Ftr, Fte = F[:n_train], F[n_train:]
    mean = Ftr.mean(0)
    std = Ftr.std(0)
    std[std == 0] = 1.0
    net = zf.zf_mlp_create(0, seed)
    t0 = time.perf_counter()
    losses = zf.zf_mlp_train(net, (Ftr - mean) / std, y[:n_train], mask[:n_train], epochs, batch, lr, seed=seed)
    train_s = time.perf_counter() - t0
    pred = zf.zf_mlp_predict(net, (Fte - mean) / std, mask[n_train:])
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
            "loss_last": float(losses[-1]), "train_s": round(train_s, 3), "mean": mean, "std": std,
            "pred": pred, "labels": yte}, net


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
    zf.zf_ctx_set_selector(ctx, net, res["mean"], res["std"])
    x, o, meta = W.selector_column(n_train + 1, args.sel_cap)
    col = zf.Column(x, o)
    zf.zf_plan(ctx, col, selector=1)
    t1 = time.perf_counter()
    for _ in range(20):
        zf.zf_plan(ctx, col, selector=1)
    plan_us = (time.perf_counter() - t1) / 20 * 1e6
    Fn = ((F[n_train:] - res["mean"]) / res["std"]).astype(np.float32)
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="zipflow", choices=["zipflow", "reference"])
    ap.add_argument("--ref-step-s", type=float, default=None,
                    help="CPU seconds per reference step (default: 2 s, less for long runs so that "
                         "all steps take about a minute)")
    ap.add_argument("--cpu-budget-s", type=float, default=12.0, help="CPU seconds for the cpu_baseline sample")
    ap.add_argument("--tile-rows", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--stage-mb", type=float, default=0)
    ap.add_argument("--slots", type=int, default=0)
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    ap.add_argument("--no-graph", action="store_true", help="enqueue transfers call by call (no CUDA graph)")
    ap.add_argument("--profile", choices=["keys", "dates", "both", "for", "float", "ans", "strdict", "lz77"], default=None,
                    help="only decode the resident column(s) --steps times (for ncu captures)")
    ap.add_argument("--rows", type=int, default=N_ROWS, help="rows per column (profile / batched runs)")
    ap.add_argument("--workload", choices=["group_parallel", "batched", "selector", "text"], default="group_parallel",
                    help="group_parallel: the benchmark line; batched: the 40 GB fact table; "
                         "selector: train and evaluate the learned selector")
    ap.add_argument("--text-mb", type=float, default=256, help="string column size (text workload), MiB")
    ap.add_argument("--text-scheme", choices=["lz77", "strdict"], default="lz77",
                    help="byte scheme of the text workload")
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
    if args.workload == "batched":
        assert world == 1
        return run_batched(args, zf, torch)
    if args.workload == "selector":
        assert world == 1
        return run_selector(args, zf, torch)
    if args.workload == "text":
        assert world == 1
        return run_text(args, zf, torch)
    keys, dates = make_workload(1 + rank)
    ck, cd = zf.Column(keys), zf.Column(dates)
    copy_s, comp_s = torch.cuda.Stream(), torch.cuda.Stream()
    ctx = zf.zf_ctx_create(local, copy_s.cuda_stream, comp_s.cuda_stream)
    # transfers replay a captured CUDA graph (the same host buffers every step)
    zf.zf_ctx_set_kcfg(ctx, args.tile_rows, args.threads, args.ctas_per_sm, int(args.stage_mb * (1 << 20)),
                       0 if args.no_graph else zf.ZF_KCFG_GRAPH)
    if args.slots:
        zf.zf_ctx_set_ring(ctx, args.slots)
    hk = zf.zf_compress_host(zf.zf_plan(ctx, ck, scheme=zf.ZF_DELTA_BP, chunk_rows=CHUNK_ROWS), ck)
    hd = zf.zf_compress_host(zf.zf_plan(ctx, cd, scheme=zf.ZF_RLE, chunk_rows=CHUNK_ROWS), cd)
    raw_k, comp_k, _ = zf.zf_compressed_info(hk)
    raw_d, comp_d, _ = zf.zf_compressed_info(hd)
    raw, comp = raw_k + raw_d, comp_k + comp_d
    out_k = torch.empty(raw_k, dtype=torch.uint8, device="cuda")
    out_d = torch.empty(raw_d, dtype=torch.uint8, device="cuda")
    outs, caps = [out_k.data_ptr(), out_d.data_ptr()], [raw_k, raw_d]
    rk, rd = zf.zf_upload(ctx, hk), zf.zf_upload(ctx, hd)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    def resident_step(cols, o, c):
        with torch.cuda.stream(comp_s):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(comp_s)
            zf.zf_decompress_resident(ctx, cols, o, c)
            e1.record(comp_s)
        st, stats = zf.zf_sync(ctx)
        return e0.elapsed_time(e1), stats.n_launches

    def e2e_step():
        t0 = time.perf_counter()
        zf.zf_transfer_decompress(ctx, [hk, hd], outs, caps)
        st, stats = zf.zf_sync(ctx)
        return (time.perf_counter() - t0) * 1e3, stats

    # correctness of this run's outputs (cheap full compare) before timing
    zf.zf_transfer_decompress(ctx, [hk, hd], outs, caps)
    zf.zf_sync(ctx)
    assert np.array_equal(out_k.cpu().numpy().view(np.int64), keys)
    assert np.array_equal(out_d.cpu().numpy().view(np.int32), dates)

    for _ in range(args.warmup):
        resident_step([rk, rd], outs, caps)
        e2e_step()
        resident_step([rk], outs[:1], caps[:1])

    launches = 0
    with Clocks(local) as clk:
        barrier()
        dev_ms = []
        for _ in range(args.steps):
            ms, nl = resident_step([rk, rd], outs, caps)
            dev_ms.append(ms)
            launches += nl
        barrier()
        e2e_ms, e2e_ev = [], []
        for _ in range(args.steps):
            ms, stats = e2e_step()
            e2e_ms.append(ms)
            e2e_ev.append(stats.total_ms)
            launches += stats.n_launches
        barrier()
        kern_ms = []
        for _ in range(args.steps):
            ms, nl = resident_step([rk], outs[:1], caps[:1])
            kern_ms.append(ms)
            launches += nl
        barrier()

    # raw link: best-of-10 pinned H2D copy of the same compressed bytes
    src = torch.empty(comp, dtype=torch.uint8, pin_memory=True)
    dst = torch.empty(comp, dtype=torch.uint8, device="cuda")
    best = 1e9
    for _ in range(10):
        with torch.cuda.stream(copy_s):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(copy_s)
            dst.copy_(src, non_blocking=True)
            e1.record(copy_s)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    link_gbs = comp / best / 1e6

    t_dev = float(np.mean(dev_ms))
    t_e2e = float(np.mean(e2e_ms))
    t_kern = float(np.mean(kern_ms))
    t_dev, t_e2e, t_kern = max_over_ranks([t_dev, t_e2e, t_kern], dist, "cuda")
    value = whole_job_gbs(world * raw, t_dev)
    e2e = whole_job_gbs(world * raw, t_e2e)
    hbm, peak_kind = peaks()
    kern_bytes = comp_k + raw_k
    achieved = kern_bytes / (t_kern * 1e-3) / 1e9
    cr = raw / comp
    line = None
    if rank == 0:
        import oracle
        oracle.build()
        nt = host_threads()
        cpu_b, cpu_s, cpu_desc = oracle_sample([hk, hd], [np.int64, np.int32], args.cpu_budget_s * 2 / 3, nt)
        one_b, one_s, _ = oracle_sample([hk, hd], [np.int64, np.int32], args.cpu_budget_s / 3, 1)
        traffic = measured_traffic()
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(t_dev, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64/int32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "raw_bytes_per_step": raw, "comp_bytes_per_step": comp,
                       "compression_ratio": round(cr, 3), "l2": "flushed (256 MiB write) before every resident step",
                       "parallelism": "replicas" if world > 1 else "single"},
            "e2e": {"value": round(e2e, 2), "unit": "GB/s", "h2d_bytes_per_step": comp, "d2h_bytes_per_step": 8,
                    "ms_per_step": round(t_e2e, 4), "event_ms_per_step": round(float(np.mean(e2e_ev)), 4),
                    "raw_h2d_link_gbs": round(link_gbs, 2), "target_0.9_link_x_cr_gbs": round(0.9 * link_gbs * cr, 2),
                    "frac_of_link_x_cr": round(e2e / world / (link_gbs * cr), 4)},
            "roofline": {"bound": "hbm", "kernel": "tiles_kernel<delta_bp, int64>", "achieved": round(achieved, 1),
                         "peak": hbm, "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / hbm, 4),
                         "traffic": traffic, "algorithmic_bytes_per_launch": kern_bytes,
                         "launch_ms": round(t_kern, 4)},
            "cpu_baseline": {"value": round(cpu_b / cpu_s / 1e9, 4), "unit": "GB/s", "cores": nt, "kind": "oracle",
                             "sample": cpu_desc, "single_thread_value": round(one_b / one_s / 1e9, 4)},
            "clocks": clk.summary(),
            "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)
    zf.zf_resident_free(rk)
    zf.zf_resident_free(rd)
    zf.zf_compressed_free(hk)
    zf.zf_compressed_free(hd)
    zf.zf_ctx_destroy(ctx)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
