"""CPU oracle for SipTreeHash (arXiv:1612.06257, Section 3): ctypes loader.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only ``tests/``,
``__graft_entry__`` and ``bench.py``'s CPU legs may import it.  The C source
``sipo.c`` is compiled with gcc into ``liboracle_sipo.so`` beside it.  Its
readings of the points Section 3 leaves open, and what pins each function,
are listed in ``sipo.h``.

SipTreeHash uses SipHash-2-4 lanes (``ROUNDS["siptree"]``), SipTreeHash13
SipHash-1-3 (``ROUNDS["siptree13"]``), Section 5.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(_HERE, "sipo.c")
HDR = os.path.join(_HERE, "sipo.h")
LIB_PATH = os.path.join(_HERE, "liboracle_sipo.so")

ROUNDS = {"siptree": (2, 4), "siptree13": (1, 3)}

_lock = threading.Lock()
_lib = None
_u64p = ctypes.POINTER(ctypes.c_uint64)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False, src: str = SRC, out: str = LIB_PATH) -> str:
    """Compile sipo.c (or a copy of it) with gcc (plain -O2)."""
    newest = max(os.path.getmtime(p) for p in (src, HDR))
    if not force and os.path.exists(out) and os.path.getmtime(out) >= newest:
        return out
    tmp = out + ".tmp.%d" % os.getpid()
    subprocess.run(["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-Wall", "-Wextra",
                    "-I", _HERE, "-o", tmp, src], check=True)
    os.replace(tmp, out)
    return out


def _buf(data: bytes):
    return (ctypes.c_uint8 * max(1, len(data))).from_buffer_copy(data if data else b"\0")


def _key(key):
    return (ctypes.c_uint64 * 4)(*[int(k) & 0xFFFFFFFFFFFFFFFF for k in key])


class SipOracle:
    """The C functions of one build of sipo.c."""

    def __init__(self, path: str):
        L = ctypes.CDLL(path)
        L.sipo_siphash.argtypes = [ctypes.c_uint64, ctypes.c_uint64, _u8p, ctypes.c_size_t,
                                   ctypes.c_int, ctypes.c_int]
        L.sipo_siphash.restype = ctypes.c_uint64
        L.sipo_tree_lanes.argtypes = [_u64p, _u8p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int,
                                      _u64p]
        L.sipo_tree_hash.argtypes = [_u64p, _u8p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int]
        L.sipo_tree_hash.restype = ctypes.c_uint64
        L.sipo_tree_batch.argtypes = [_u64p, ctypes.c_int, _u8p, _i64p, ctypes.c_int64,
                                      ctypes.c_int64, ctypes.c_int, ctypes.c_int, _u64p]
        L.sipo_tree_batch.restype = ctypes.c_int
        self.L = L

    def siphash(self, k0: int, k1: int, msg: bytes, c: int = 2, d: int = 4) -> int:
        return int(self.L.sipo_siphash(k0 & 0xFFFFFFFFFFFFFFFF, k1 & 0xFFFFFFFFFFFFFFFF,
                                       _buf(msg), len(msg), c, d))

    def tree_lanes(self, key, msg: bytes, c: int = 2, d: int = 4):
        out = (ctypes.c_uint64 * 4)()
        self.L.sipo_tree_lanes(_key(key), _buf(msg), len(msg), c, d, out)
        return [int(x) for x in out]

    def tree_hash(self, key, msg: bytes, c: int = 2, d: int = 4) -> int:
        return int(self.L.sipo_tree_hash(_key(key), _buf(msg), len(msg), c, d))

    def tree_batch(self, keys: np.ndarray, per_message_keys: bool, data: np.ndarray,
                   offsets: np.ndarray, c: int = 2, d: int = 4, first: int = 0,
                   last: int | None = None, out: np.ndarray | None = None) -> np.ndarray:
        """SipTreeHash of messages [first, last) of a batch (host numpy
        arrays, laid out as for the HighwayHash oracle); uint64 [last-first].
        The C call releases the GIL."""
        n = offsets.shape[0] - 1
        last = n if last is None else last
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        data = np.ascontiguousarray(data, dtype=np.uint8)
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        if out is None:
            out = np.zeros(last - first, dtype=np.uint64)
        keep = _buf(b"")
        dptr = data.ctypes.data_as(_u8p) if data.size else keep
        rc = self.L.sipo_tree_batch(keys.ctypes.data_as(_u64p), int(per_message_keys), dptr,
                                    offsets.ctypes.data_as(_i64p), first, last, c, d,
                                    out.ctypes.data_as(_u64p))
        if rc != 0:
            raise ValueError("oracle rejected the batch (offsets or rounds)")
        return out


def lib() -> SipOracle:
    global _lib
    with _lock:
        if _lib is None:
            _lib = SipOracle(build())
    return _lib


def siphash(k0, k1, msg, c=2, d=4):
    return lib().siphash(k0, k1, msg, c, d)


def tree_lanes(key, msg, c=2, d=4):
    return lib().tree_lanes(key, msg, c, d)


def tree_hash(key, msg, c=2, d=4):
    return lib().tree_hash(key, msg, c, d)


def tree_batch(keys, per_message_keys, data, offsets, c=2, d=4, first=0, last=None, out=None):
    return lib().tree_batch(keys, per_message_keys, data, offsets, c, d, first, last, out)
