"""ctypes declarations of the C ABI in include/zf.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libzf.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libzf.so is not built ({LIB_PATH}); run __graft_entry__.build() or "
                      "python paper_2602_08190_gb300/build.py")
_L = ctypes.CDLL(LIB_PATH)

__all__ = [
    "ZF_OK", "ZF_EINVAL", "ZF_ENOMEM", "ZF_ECUDA", "ZF_ECORRUPT", "ZF_ETIMEOUT", "ZF_EUNSUPPORTED", "ZF_EBUSY",
    "ZF_I32", "ZF_I64", "ZF_BYTES", "ZF_F64", "ZF_RAW", "ZF_FOR_BP", "ZF_DICT_BP", "ZF_DELTA_BP", "ZF_RLE", "ZF_LZ77",
    "ZF_FLOAT2INT", "ZF_STRDICT", "ZF_ANS",
    "ZF_KCFG_BATCHED", "ZF_KCFG_GRAPH", "SCHEME_NAMES", "ZfError", "zf_column", "zf_kcfg", "zf_plan_opts",
    "zf_plan_t", "zf_stats", "Column", "zf_ctx_create", "zf_ctx_destroy", "zf_last_error", "zf_ctx_set_kcfg",
    "zf_ctx_set_ring", "zf_plan", "zf_compress_host", "zf_compressed_info", "zf_compressed_free",
    "zf_compressed_bytes", "zf_compressed_from_bytes", "zf_transfer_decompress", "zf_sync", "zf_upload",
    "zf_resident_free", "zf_decompress_resident", "zf_decompress_device_noalloc", "zf_tune", "zf_tune_point",
    "zf_ctx_tuned_geometry", "zf_measure_copy", "zf_johnson_order", "ZF_KCFG_KEEP_ORDER", "zf_ctx_rates", "zf_mlp_get_scaling", "zf_tune_chunk_rows",
    "zf_column_features", "zf_measure_classes", "zf_ctx_set_selector", "zf_mlp_create", "zf_mlp_destroy",
    "zf_mlp_get_params", "zf_mlp_set_params", "zf_mlp_forward", "zf_mlp_grad", "zf_mlp_adam", "zf_mlp_train",
    "zf_mlp_predict", "ZF_MLP_PARAMS", "ZF_MLP_CLASSES", "EXPORTED", "LIB_PATH",
]
ZF_MLP_PARAMS, ZF_MLP_CLASSES = 7052, 12

(ZF_OK, ZF_EINVAL, ZF_ENOMEM, ZF_ECUDA, ZF_ECORRUPT, ZF_ETIMEOUT, ZF_EUNSUPPORTED, ZF_EBUSY) = range(8)
ZF_I32, ZF_I64, ZF_BYTES, ZF_F64 = range(4)
ZF_RAW, ZF_FOR_BP, ZF_DICT_BP, ZF_DELTA_BP, ZF_RLE, ZF_LZ77, ZF_FLOAT2INT, ZF_STRDICT, ZF_ANS = range(9)
ZF_KCFG_BATCHED, ZF_KCFG_GRAPH, ZF_KCFG_KEEP_ORDER = 1, 2, 4
SCHEME_NAMES = ["raw", "for_bp", "dict_bp", "delta_bp", "rle", "lz77", "float2int", "strdict", "ans"]
_STATUS = ["ok", "einval", "enomem", "ecuda", "ecorrupt", "etimeout", "eunsupported", "ebusy"]


class ZfError(RuntimeError):
    def __init__(self, status: int, call: str, detail: str = ""):
        name = _STATUS[status] if 0 <= status < len(_STATUS) else str(status)
        super().__init__(f"{call} -> {name}" + (f": {detail}" if detail else ""))
        self.status = status


class zf_column(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("data", ctypes.c_void_p), ("n", ctypes.c_uint64),
                ("offsets", ctypes.c_void_p)]


class zf_kcfg(ctypes.Structure):
    _fields_ = [("tile_rows", ctypes.c_uint32), ("threads", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32),
                ("stage_bytes", ctypes.c_uint32), ("flags", ctypes.c_uint32)]


class zf_plan_opts(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int32), ("chunk_rows", ctypes.c_uint32), ("selector", ctypes.c_int32),
                ("offsets_scheme", ctypes.c_int32), ("ans_stream_rows", ctypes.c_uint32)]


class zf_plan_t(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int32), ("chunk_rows", ctypes.c_uint32), ("offsets_scheme", ctypes.c_int32),
                ("kcfg", zf_kcfg), ("predicted_ms", ctypes.c_float), ("label", ctypes.c_int32),
                ("ans_stream_rows", ctypes.c_uint32)]


class zf_tune_point(ctypes.Structure):
    _fields_ = [("kcfg", zf_kcfg), ("ms", ctypes.c_float)]


class zf_stats(ctypes.Structure):
    _fields_ = [("raw_bytes", ctypes.c_uint64), ("comp_bytes", ctypes.c_uint64), ("n_chunks", ctypes.c_uint32),
                ("n_stages", ctypes.c_uint32), ("n_launches", ctypes.c_uint32), ("device_error", ctypes.c_uint32),
                ("total_ms", ctypes.c_float), ("copy_ms", ctypes.c_float), ("decode_ms", ctypes.c_float)]


_vp, _u32, _u64, _i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32
_SIGS = {
    "zf_ctx_create": [ctypes.c_int, _vp, _vp, ctypes.POINTER(_vp)],
    "zf_ctx_destroy": [_vp],
    "zf_ctx_set_kcfg": [_vp, ctypes.POINTER(zf_kcfg)],
    "zf_ctx_set_ring": [_vp, _u32, _u64],
    "zf_plan": [_vp, ctypes.POINTER(zf_column), ctypes.POINTER(zf_plan_opts), ctypes.POINTER(zf_plan_t)],
    "zf_compress_host": [ctypes.POINTER(zf_plan_t), ctypes.POINTER(zf_column), ctypes.POINTER(_vp)],
    "zf_compressed_info": [_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u64), ctypes.POINTER(_u32)],
    "zf_compressed_free": [_vp],
    "zf_compressed_bytes": [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_u64)],
    "zf_compressed_from_bytes": [_vp, _u64, ctypes.POINTER(_vp)],
    "zf_transfer_decompress": [_vp, ctypes.POINTER(_vp), _u32, ctypes.POINTER(_vp), ctypes.POINTER(_u64)],
    "zf_sync": [_vp, ctypes.POINTER(zf_stats)],
    "zf_upload": [_vp, _vp, ctypes.POINTER(_vp)],
    "zf_resident_free": [_vp],
    "zf_decompress_resident": [_vp, ctypes.POINTER(_vp), _u32, ctypes.POINTER(_vp), ctypes.POINTER(_u64)],
    "zf_decompress_device_noalloc": [_vp, _u64, _vp, _u64, _vp],
    "zf_column_features": [ctypes.POINTER(zf_column), _vp],
    "zf_measure_classes": [_vp, ctypes.POINTER(zf_column), _u32, _vp],
    "zf_ctx_set_selector": [_vp, _vp, _vp, _vp],
    "zf_mlp_create": [ctypes.c_int, _u64, ctypes.POINTER(_vp)],
    "zf_mlp_destroy": [_vp],
    "zf_mlp_get_params": [_vp, _vp],
    "zf_mlp_set_params": [_vp, _vp],
    "zf_mlp_forward": [_vp, _vp, _u32, _vp, _vp],
    "zf_mlp_grad": [_vp, _vp, _vp, _vp, _u32, _vp, _vp, _vp],
    "zf_mlp_adam": [_vp, _vp, ctypes.c_float, _vp],
    "zf_mlp_train": [_vp, _vp, _vp, _vp, _u32, _u32, _u32, ctypes.c_float, _u64, _vp],
    "zf_mlp_predict": [_vp, _vp, _vp, _u32, _vp],
    "zf_ctx_tuned_geometry": [_vp, ctypes.c_int32, ctypes.c_int32, _u32, ctypes.POINTER(zf_kcfg)],
    "zf_measure_copy": [_vp, ctypes.POINTER(_vp), _u32, _u32, ctypes.POINTER(ctypes.c_float)],
    "zf_ctx_rates": [_vp, ctypes.c_int32, ctypes.c_int32, _u32, ctypes.POINTER(ctypes.c_float),
                     ctypes.POINTER(ctypes.c_float)],
    "zf_mlp_get_scaling": [_vp, _vp, _vp],
    "zf_tune_chunk_rows": [_vp, ctypes.POINTER(zf_column), ctypes.c_int32, _vp, _u32, _u32, _vp,
                           ctypes.POINTER(_u32)],
    "zf_johnson_order": [_vp, _vp, _u32, _vp],
    "zf_tune": [_vp, ctypes.POINTER(_vp), _u32, ctypes.POINTER(_vp), ctypes.POINTER(_u64), ctypes.c_int32, _u32,
                ctypes.POINTER(zf_tune_point), _u32, ctypes.POINTER(_u32), ctypes.POINTER(zf_kcfg)],
}
for _name, _args in _SIGS.items():
    _f = getattr(_L, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int
_L.zf_last_error.argtypes = [_vp]
_L.zf_last_error.restype = ctypes.c_char_p
EXPORTED = sorted(list(_SIGS) + ["zf_last_error"])


def _check(st: int, call: str, ctx=None):
    if st != ZF_OK:
        detail = _L.zf_last_error(ctx).decode() if ctx else ""
        raise ZfError(st, call, detail)


class Column:
    """A host column kept alive for the duration of a call (numpy arrays)."""

    def __init__(self, data: np.ndarray, offsets: np.ndarray | None = None):
        self.data = np.ascontiguousarray(data)
        if offsets is None:
            kinds = {np.dtype(np.int32): ZF_I32, np.dtype(np.int64): ZF_I64, np.dtype(np.float64): ZF_F64}
            if self.data.dtype not in kinds:
                raise TypeError(f"columns are int32, int64 or float64 (or uint8 bytes with offsets), "
                                f"not {self.data.dtype}")
            dt = kinds[self.data.dtype]
            self.offsets = None
            n = len(self.data)
        else:
            if self.data.dtype != np.uint8:
                raise TypeError(f"a string column's bytes are uint8, not {self.data.dtype}")
            self.offsets = np.ascontiguousarray(offsets, dtype=np.int32)
            dt = ZF_BYTES
            n = len(self.offsets) - 1
        self.c = zf_column(dt, self.data.ctypes.data if self.data.size else None, n,
                           self.offsets.ctypes.data if self.offsets is not None else None)


def zf_ctx_create(device: int = 0, copy_stream: int | None = None, compute_stream: int | None = None) -> int:
    out = _vp()
    _check(_L.zf_ctx_create(device, copy_stream or None, compute_stream or None, ctypes.byref(out)), "zf_ctx_create")
    return out.value


def zf_ctx_destroy(ctx: int) -> None:
    _check(_L.zf_ctx_destroy(ctx), "zf_ctx_destroy")


def zf_last_error(ctx: int) -> str:
    return _L.zf_last_error(ctx).decode()


def zf_ctx_set_kcfg(ctx: int, tile_rows=0, threads=0, ctas_per_sm=0, stage_bytes=0, flags=0) -> None:
    k = zf_kcfg(tile_rows, threads, ctas_per_sm, stage_bytes, flags)
    _check(_L.zf_ctx_set_kcfg(ctx, ctypes.byref(k)), "zf_ctx_set_kcfg", ctx)


def zf_ctx_set_ring(ctx: int, slots: int, slot_bytes: int = 0) -> None:
    _check(_L.zf_ctx_set_ring(ctx, slots, slot_bytes), "zf_ctx_set_ring", ctx)


def zf_plan(ctx: int | None, col: Column, scheme: int = -1, chunk_rows: int = 0, selector: int = 0,
            offsets_scheme: int = -1, ans_stream_rows: int = 0) -> zf_plan_t:
    o = zf_plan_opts(scheme, chunk_rows, selector, offsets_scheme, ans_stream_rows)
    p = zf_plan_t()
    _check(_L.zf_plan(ctx, ctypes.byref(col.c), ctypes.byref(o), ctypes.byref(p)), "zf_plan", ctx)
    return p


def zf_compress_host(plan: zf_plan_t, col: Column) -> int:
    out = _vp()
    _check(_L.zf_compress_host(ctypes.byref(plan), ctypes.byref(col.c), ctypes.byref(out)), "zf_compress_host")
    return out.value


def zf_compressed_info(c: int) -> tuple[int, int, int]:
    raw, comp, n = _u64(), _u64(), _u32()
    _check(_L.zf_compressed_info(c, ctypes.byref(raw), ctypes.byref(comp), ctypes.byref(n)), "zf_compressed_info")
    return raw.value, comp.value, n.value


def zf_compressed_free(c: int) -> None:
    _check(_L.zf_compressed_free(c), "zf_compressed_free")


def zf_compressed_bytes(c: int) -> bytes:
    p, n = _vp(), _u64()
    _check(_L.zf_compressed_bytes(c, ctypes.byref(p), ctypes.byref(n)), "zf_compressed_bytes")
    return ctypes.string_at(p.value, n.value) if n.value else b""


def zf_compressed_from_bytes(data: bytes) -> int:
    out = _vp()
    buf = ctypes.create_string_buffer(bytes(data), len(data))
    _check(_L.zf_compressed_from_bytes(buf, len(data), ctypes.byref(out)), "zf_compressed_from_bytes")
    return out.value


def _arrays(cols, outs, caps):
    n = len(outs)
    return ((_vp * max(1, len(cols)))(*cols), (_vp * max(1, n))(*outs), (_u64 * max(1, n))(*caps))


def zf_transfer_decompress(ctx: int, cols: list[int], outs: list[int], caps: list[int]) -> None:
    c, o, k = _arrays(cols, outs, caps)
    _check(_L.zf_transfer_decompress(ctx, c, len(cols), o, k), "zf_transfer_decompress", ctx)


def zf_sync(ctx: int, raise_on_error: bool = True) -> tuple[int, zf_stats]:
    s = zf_stats()
    st = _L.zf_sync(ctx, ctypes.byref(s))
    if raise_on_error:
        _check(st, "zf_sync", ctx)
    return st, s


def zf_upload(ctx: int, c: int) -> int:
    out = _vp()
    _check(_L.zf_upload(ctx, c, ctypes.byref(out)), "zf_upload", ctx)
    return out.value


def zf_resident_free(r: int) -> None:
    _check(_L.zf_resident_free(r), "zf_resident_free")


def zf_decompress_resident(ctx: int, cols: list[int], outs: list[int], caps: list[int]) -> None:
    c, o, k = _arrays(cols, outs, caps)
    _check(_L.zf_decompress_resident(ctx, c, len(cols), o, k), "zf_decompress_resident", ctx)


def zf_decompress_device_noalloc(d_column: int, column_bytes: int, d_out: int, out_bytes: int,
                                 stream: int | None = None) -> int:
    """Decode a serialized integer or float64 column already in device memory
    without allocating; returns the zf_status (0 = ok) instead of raising."""
    return int(_L.zf_decompress_device_noalloc(d_column, column_bytes, d_out, out_bytes, stream or None))


def zf_tune(ctx: int, cols: list[int], outs: list[int], caps: list[int], transfer: bool = False,
            reps: int = 3) -> tuple[list[zf_tune_point], zf_kcfg]:
    c, o, k = _arrays(cols, outs, caps)
    pts = (zf_tune_point * 256)()
    n = _u32()
    best = zf_kcfg()
    _check(_L.zf_tune(ctx, c, len(cols), o, k, 1 if transfer else 0, reps, pts, 256, ctypes.byref(n),
                      ctypes.byref(best)), "zf_tune", ctx)
    return [pts[i] for i in range(min(n.value, 256))], best


def zf_ctx_tuned_geometry(ctx: int, scheme: int, dtype: int, bmax: int) -> zf_kcfg:
    out = zf_kcfg()
    _check(_L.zf_ctx_tuned_geometry(ctx, scheme, dtype, bmax, ctypes.byref(out)), "zf_ctx_tuned_geometry", ctx)
    return out


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def zf_column_features(col: Column) -> np.ndarray:
    out = np.zeros(32, np.float32)
    _check(_L.zf_column_features(ctypes.byref(col.c), out.ctypes.data), "zf_column_features")
    return out


def zf_measure_classes(ctx: int, col: Column, reps: int = 3) -> np.ndarray:
    out = np.zeros(ZF_MLP_CLASSES, np.float32)
    _check(_L.zf_measure_classes(ctx, ctypes.byref(col.c), reps, out.ctypes.data), "zf_measure_classes", ctx)
    return out


def zf_ctx_set_selector(ctx: int, net: int | None, mean=None, std=None) -> None:
    m = _f32(mean) if mean is not None else None
    sd = _f32(std) if std is not None else None
    _check(_L.zf_ctx_set_selector(ctx, net, m.ctypes.data if m is not None else None,
                                  sd.ctypes.data if sd is not None else None), "zf_ctx_set_selector", ctx)


def zf_mlp_create(device: int = 0, seed: int = 0) -> int:
    out = _vp()
    _check(_L.zf_mlp_create(device, seed, ctypes.byref(out)), "zf_mlp_create")
    return out.value


def zf_mlp_destroy(net: int) -> None:
    _check(_L.zf_mlp_destroy(net), "zf_mlp_destroy")


def zf_mlp_get_params(net: int) -> np.ndarray:
    out = np.zeros(ZF_MLP_PARAMS, np.float32)
    _check(_L.zf_mlp_get_params(net, out.ctypes.data), "zf_mlp_get_params")
    return out


def zf_mlp_set_params(net: int, params) -> None:
    p = _f32(params)
    assert p.size == ZF_MLP_PARAMS
    _check(_L.zf_mlp_set_params(net, p.ctypes.data), "zf_mlp_set_params")


def zf_mlp_forward(net: int, d_x: int, batch: int, d_logits: int, stream: int | None = None) -> None:
    _check(_L.zf_mlp_forward(net, d_x, batch, d_logits, stream or None), "zf_mlp_forward")


def zf_mlp_grad(net: int, d_x: int, d_y: int, d_mask: int, batch: int, d_grad: int, d_loss: int | None = None,
                stream: int | None = None) -> None:
    _check(_L.zf_mlp_grad(net, d_x, d_y, d_mask, batch, d_grad, d_loss or None, stream or None), "zf_mlp_grad")


def zf_mlp_adam(net: int, d_grad: int, lr: float, stream: int | None = None) -> None:
    _check(_L.zf_mlp_adam(net, d_grad, lr, stream or None), "zf_mlp_adam")


def zf_mlp_train(net: int, x, y, mask, epochs: int, batch: int, lr: float, seed: int = 0) -> np.ndarray:
    x = _f32(x)
    y = np.ascontiguousarray(y, dtype=np.int32)
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    losses = np.zeros(epochs, np.float32)
    _check(_L.zf_mlp_train(net, x.ctypes.data, y.ctypes.data, m.ctypes.data, len(y), epochs, batch, lr, seed,
                           losses.ctypes.data), "zf_mlp_train")
    return losses


def zf_mlp_predict(net: int, x, mask) -> np.ndarray:
    x = _f32(x)
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    out = np.zeros(len(x), np.int32)
    _check(_L.zf_mlp_predict(net, x.ctypes.data, m.ctypes.data, len(x), out.ctypes.data), "zf_mlp_predict")
    return out


def zf_measure_copy(ctx: int, cols: list[int], reps: int = 5) -> float:
    """Milliseconds of the fastest host-to-device copy of the columns in the
    transfer's own pieces (no decode)."""
    arr = (_vp * len(cols))(*cols)
    ms = ctypes.c_float()
    _check(_L.zf_measure_copy(ctx, arr, len(cols), reps, ctypes.byref(ms)), "zf_measure_copy", ctx)
    return ms.value


def zf_johnson_order(copy_ms, decode_ms) -> np.ndarray:
    """Johnson's-rule order (indices) of jobs with the given stage times."""
    c = np.ascontiguousarray(copy_ms, np.float32)
    d = np.ascontiguousarray(decode_ms, np.float32)
    assert c.shape == d.shape
    out = np.zeros(max(1, len(c)), np.uint32)
    _check(_L.zf_johnson_order(c.ctypes.data, d.ctypes.data, len(c), out.ctypes.data), "zf_johnson_order")
    return out[:len(c)].astype(np.int64)


def zf_ctx_rates(ctx: int, scheme: int, dtype: int, bmax: int) -> tuple[float, float]:
    """(decode GB/s measured for the class, link GB/s measured), 0 if none."""
    d, l = ctypes.c_float(), ctypes.c_float()
    _check(_L.zf_ctx_rates(ctx, scheme, dtype, bmax, ctypes.byref(d), ctypes.byref(l)), "zf_ctx_rates", ctx)
    return d.value, l.value


def zf_mlp_get_scaling(net: int) -> tuple[np.ndarray, np.ndarray]:
    """(mean, std) of the input standardization the network fitted."""
    m, sd = np.zeros(32, np.float32), np.zeros(32, np.float32)
    _check(_L.zf_mlp_get_scaling(net, m.ctypes.data, sd.ctypes.data), "zf_mlp_get_scaling")
    return m, sd


def zf_tune_chunk_rows(ctx: int, col: Column, scheme: int, chunk_rows, reps: int = 3) -> tuple[np.ndarray, int]:
    """(ms per candidate chunk size, -1 where it does not fit; index of the fastest)."""
    cr = np.ascontiguousarray(chunk_rows, np.uint32)
    ms = np.zeros(len(cr), np.float32)
    best = _u32()
    _check(_L.zf_tune_chunk_rows(ctx, ctypes.byref(col.c), scheme, cr.ctypes.data, len(cr), reps, ms.ctypes.data,
                                 ctypes.byref(best)), "zf_tune_chunk_rows", ctx)
    return ms, best.value
