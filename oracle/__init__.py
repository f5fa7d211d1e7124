"""CPU oracle for the compressed-column codecs -- test infrastructure.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``zf_oracle.c`` (plain C,
compiled on first use with gcc) and ``mlp.py`` (the selector network in
float64 numpy).  Nothing here is shared with the GPU library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "zf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

RAW, FOR_BP, DICT_BP, DELTA_BP, RLE, LZ77, FLOAT2INT, STRDICT, ANS = range(9)
I32, I64, BYTES, F64 = range(4)
OK, EINVAL, ENOMEM, ECUDA, ECORRUPT = 0, 1, 2, 3, 4
SCHEMES = {"raw": RAW, "for_bp": FOR_BP, "dict_bp": DICT_BP, "delta_bp": DELTA_BP, "rle": RLE, "lz77": LZ77,
           "float2int": FLOAT2INT, "strdict": STRDICT, "ans": ANS}
_DT = {np.dtype(np.int32): I32, np.dtype(np.int64): I64, np.dtype(np.uint8): BYTES, np.dtype(np.float64): F64}
_NP = {I32: np.int32, I64: np.int64, BYTES: np.uint8, F64: np.float64}


def build(force: bool = False, src: str = _SRC, out: str = _LIB) -> str:
    """Compile the oracle's C file into a shared library (default: next to it)."""
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O1", "-std=c11", "-Wall", "-ffp-contract=off", "-shared", "-fPIC", "-o", tmp, src, "-lm"],
                       check=True)
        os.replace(tmp, out)
    return out


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what}: status {code}")
        self.code = code


class Oracle:
    """One loaded copy of the C oracle (the tests also load deliberately broken copies)."""

    def __init__(self, so_path: str):
        L = ctypes.CDLL(so_path)
        u8p, u64p, u32p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint32)
        L.orc_bits.restype = ctypes.c_uint32
        L.orc_bits.argtypes = [ctypes.c_uint64]
        L.orc_packed_bytes.restype = ctypes.c_uint64
        L.orc_packed_bytes.argtypes = [ctypes.c_uint64, ctypes.c_uint32]
        L.orc_pack.restype = ctypes.c_uint64
        L.orc_pack.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint32, u8p]
        L.orc_unpack_one.restype = ctypes.c_uint64
        L.orc_unpack_one.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint32]
        L.orc_encode_bound.restype = ctypes.c_uint64
        L.orc_encode_bound.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32]
        L.orc_encode.restype = ctypes.c_int
        L.orc_encode.argtypes = [ctypes.c_int, ctypes.c_int, u8p, ctypes.c_uint64, ctypes.c_uint32, u8p,
                                 ctypes.c_uint64, u64p]
        L.orc_encode_ans.restype = ctypes.c_int
        L.orc_encode_ans.argtypes = [ctypes.c_int, u8p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, u8p,
                                     ctypes.c_uint64, u64p]
        L.orc_encode_strdict.restype = ctypes.c_int
        L.orc_encode_strdict.argtypes = [u8p, ctypes.c_uint64, u8p, ctypes.c_uint64, ctypes.c_uint32, u8p,
                                         ctypes.c_uint64, u64p]
        L.orc_decode.restype = ctypes.c_int
        L.orc_decode.argtypes = [u8p, ctypes.c_uint64, u8p, ctypes.c_uint64]
        L.orc_decode_chunk.restype = ctypes.c_int
        L.orc_decode_chunk.argtypes = [u8p, ctypes.c_uint64, u8p, ctypes.c_uint64]
        L.orc_column_info.restype = ctypes.c_int
        L.orc_column_info.argtypes = [u8p, ctypes.c_uint64, u32p, u32p, u64p, u32p, u64p]
        L.orc_chunk_span.restype = ctypes.c_int
        L.orc_chunk_span.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint32, u64p, u64p, u64p, u32p]
        self.L = L

    def bits(self, x: int) -> int:
        return int(self.L.orc_bits(int(x) & 0xFFFFFFFFFFFFFFFF))

    def pack(self, u, b: int) -> bytes:
        u = np.ascontiguousarray(np.asarray(u, dtype=np.uint64))
        if len(u) == 0:
            u = np.zeros(1, np.uint64)[:0]
        out = np.zeros(max(1, int(self.L.orc_packed_bytes(len(u), b))), np.uint8)
        uu = u if len(u) else np.zeros(1, np.uint64)
        n = self.L.orc_pack(_ptr(uu), len(u), b, _ptr(out))
        return bytes(out[:n])

    def unpack(self, buf: bytes, n: int, b: int) -> np.ndarray:
        a = np.frombuffer(bytes(buf) + b"\0" * 16, np.uint8)
        return np.array([self.L.orc_unpack_one(_ptr(a), i, b) for i in range(n)], dtype=np.uint64)

    def encode(self, x: np.ndarray, scheme: int, chunk_rows: int, ans_stream_rows: int | None = None) -> bytes:
        """Serialize column ``x`` (int32, int64 or uint8 bytes) with one scheme
        (ANS: ``ans_stream_rows`` rows per stream, 512 if None)."""
        x = np.ascontiguousarray(x)
        dt = _DT[x.dtype]
        cap = int(self.L.orc_encode_bound(scheme, dt, len(x), chunk_rows))
        if cap == 0:
            raise OracleError(EINVAL, "encode bound")
        out = np.empty(cap, np.uint8)
        n = ctypes.c_uint64(0)
        xx = x if len(x) else np.zeros(1, x.dtype)
        if ans_stream_rows is not None:
            assert scheme == ANS
            st = self.L.orc_encode_ans(dt, _ptr(xx), len(x), chunk_rows, ans_stream_rows, _ptr(out), cap,
                                       ctypes.byref(n))
        else:
            st = self.L.orc_encode(scheme, dt, _ptr(xx), len(x), chunk_rows, _ptr(out), cap, ctypes.byref(n))
        if st:
            raise OracleError(st, "encode")
        return bytes(out[: n.value])

    def column_info(self, buf: bytes) -> dict:
        a = np.frombuffer(buf, np.uint8)
        s, d, nch = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
        n, tot = ctypes.c_uint64(), ctypes.c_uint64()
        st = self.L.orc_column_info(_ptr(a), len(a), ctypes.byref(s), ctypes.byref(d), ctypes.byref(n),
                                    ctypes.byref(nch), ctypes.byref(tot))
        if st:
            raise OracleError(st, "column_info")
        return {"scheme": s.value, "dtype": d.value, "n_rows": n.value, "n_chunks": nch.value,
                "total_bytes": tot.value, "flags": int.from_bytes(buf[40:44], "little")}

    def decode(self, buf: bytes) -> np.ndarray:
        info = self.column_info(buf)
        out = np.empty(max(1, info["n_rows"]), _NP[info["dtype"]])
        a = np.frombuffer(buf, np.uint8)
        st = self.L.orc_decode(_ptr(a), len(a), _ptr(out), out.nbytes)
        if st:
            raise OracleError(st, "decode")
        return out[: info["n_rows"]]

    def chunk_span(self, buf: bytes, c: int) -> tuple[int, int, int, int]:
        a = np.frombuffer(buf, np.uint8)
        off, ln, r0 = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        rows = ctypes.c_uint32()
        st = self.L.orc_chunk_span(_ptr(a), len(a), c, ctypes.byref(off), ctypes.byref(ln), ctypes.byref(r0),
                                   ctypes.byref(rows))
        if st:
            raise OracleError(st, "chunk_span")
        return off.value, ln.value, r0.value, rows.value

    def decode_chunk(self, blob: bytes, dtype) -> np.ndarray:
        """Decode one chunk blob on its own (for sampled checks of large columns)."""
        a = np.frombuffer(blob, np.uint8)
        rows = int.from_bytes(blob[8:12], "little")
        out = np.empty(max(1, rows), dtype)
        st = self.L.orc_decode_chunk(_ptr(a), len(a), _ptr(out), out.nbytes)
        if st:
            raise OracleError(st, "decode_chunk")
        return out[:rows]

    def encode_strdict(self, data: np.ndarray, offsets: np.ndarray, chunk_bytes: int) -> bytes:
        """Serialize a byte column (rows at ``offsets``) in string-dictionary chunks."""
        data = np.ascontiguousarray(data, dtype=np.uint8)
        offsets = np.ascontiguousarray(offsets, dtype=np.int32)
        cap = int(self.L.orc_encode_bound(STRDICT, BYTES, len(data), chunk_bytes))
        if cap == 0:
            raise OracleError(EINVAL, "encode bound")
        out = np.empty(cap, np.uint8)
        n = ctypes.c_uint64(0)
        dd = data if len(data) else np.zeros(1, np.uint8)
        st = self.L.orc_encode_strdict(_ptr(dd), len(data), _ptr(offsets), len(offsets) - 1, chunk_bytes,
                                       _ptr(out), cap, ctypes.byref(n))
        if st:
            raise OracleError(st, "encode_strdict")
        return bytes(out[: n.value])

    # ---- string columns: a byte part (LZ77 or string dictionary) followed by an int32 offsets part ----
    def encode_strings(self, data: np.ndarray, offsets: np.ndarray, block: int = 65536,
                       offsets_scheme: int = DELTA_BP, offsets_chunk_rows: int = 65536,
                       scheme: int = LZ77) -> bytes:
        if scheme == STRDICT:
            a = bytearray(self.encode_strdict(data, offsets, block))
        else:
            a = bytearray(self.encode(np.ascontiguousarray(data, dtype=np.uint8), scheme, block))
        a[40] |= 1  # flag: an offsets part follows
        b = self.encode(np.ascontiguousarray(offsets, dtype=np.int32), offsets_scheme, offsets_chunk_rows)
        return bytes(a) + b

    def decode_strings(self, buf: bytes) -> tuple[np.ndarray, np.ndarray]:
        info = self.column_info(buf)
        return self.decode(buf[: info["total_bytes"]]), self.decode(buf[info["total_bytes"]:])


def default() -> Oracle:
    global _lib
    with _lock:
        if _lib is None:
            _lib = Oracle(build())
    return _lib


def _delegate(name):
    def f(*a, **k):
        return getattr(default(), name)(*a, **k)
    f.__name__ = name
    f.__doc__ = getattr(Oracle, name).__doc__
    return f


for _n in ("bits", "pack", "unpack", "encode", "column_info", "decode", "chunk_span", "decode_chunk",
           "encode_strdict", "encode_strings", "decode_strings"):
    globals()[_n] = _delegate(_n)
