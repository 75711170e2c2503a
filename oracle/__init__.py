"""CPU oracle for HighwayHash (arXiv:1612.06257, Section 4): ctypes loader.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product library (``paper_1612_06257_gb300``) never imports it and
shares no code with it: the C source ``hho.c`` is compiled here with gcc into
``liboracle_hho.so`` beside it.

Pin status of each C function is listed in ``hho.h``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hho.c")
_HDR = os.path.join(_HERE, "hho.h")
LIB_PATH = os.path.join(_HERE, "liboracle_hho.so")

_lock = threading.Lock()
_lib = None

_u64p = ctypes.POINTER(ctypes.c_uint64)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_i64p = ctypes.POINTER(ctypes.c_int64)


class State(ctypes.Structure):
    """The 1024-bit state of Section 4.2 (four vectors of four u64 lanes)."""

    _fields_ = [
        ("v0", ctypes.c_uint64 * 4),
        ("v1", ctypes.c_uint64 * 4),
        ("mul0", ctypes.c_uint64 * 4),
        ("mul1", ctypes.c_uint64 * 4),
    ]

    def as_lists(self):
        return ([int(x) for x in self.v0], [int(x) for x in self.v1],
                [int(x) for x in self.mul0], [int(x) for x in self.mul1])

    @classmethod
    def from_lists(cls, v0, v1, mul0, mul1):
        s = cls()
        for i in range(4):
            s.v0[i], s.v1[i], s.mul0[i], s.mul1[i] = v0[i], v1[i], mul0[i], mul1[i]
        return s


def build(force: bool = False, src: str = _SRC, out: str = LIB_PATH) -> str:
    """Compile hho.c (or another source file) into a shared library with gcc
    (plain -O2, no architecture flags)."""
    deps = [src, _HDR]
    newest_src = max(os.path.getmtime(p) for p in deps)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= newest_src:
        return out
    tmp = out + ".tmp.%d" % os.getpid()
    subprocess.run(["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-Wall", "-Wextra",
                    "-I", _HERE, "-o", tmp, src], check=True)
    os.replace(tmp, out)
    return out


def _u64arr(vals):
    return (ctypes.c_uint64 * len(vals))(*[int(v) & 0xFFFFFFFFFFFFFFFF for v in vals])


def _bytes_ptr(data: bytes):
    return (ctypes.c_uint8 * max(1, len(data))).from_buffer_copy(data if data else b"\0")


class OracleLib:
    """The oracle's C functions, bound from one build of the library."""

    State = State

    def __init__(self, path: str):
        L = ctypes.CDLL(path)
        sp = ctypes.POINTER(State)
        L.hho_constants.argtypes = [_u64p, _u64p]
        L.hho_init.argtypes = [sp, _u64p]
        L.hho_zipper_merge.argtypes = [_u64p, _u64p]
        L.hho_update.argtypes = [sp, _u64p]
        L.hho_permute.argtypes = [_u64p, _u64p]
        L.hho_remainder.argtypes = [sp, _u8p, ctypes.c_size_t]
        L.hho_finalize.argtypes = [sp, ctypes.c_int]
        L.hho_output.argtypes = [sp, _u64p]
        L.hho_hash_rounds.argtypes = [_u64p, _u8p, ctypes.c_size_t, ctypes.c_int,
                                      ctypes.c_int, _u64p]
        L.hho_hash_rounds.restype = ctypes.c_int
        for name in ("hho_hash64", "hho_hash128", "hho_hash256"):
            getattr(L, name).argtypes = [_u64p, _u8p, ctypes.c_size_t, _u64p]
        L.hho_hash_batch.argtypes = [_u64p, ctypes.c_int, _u8p, _i64p, ctypes.c_int64,
                                     ctypes.c_int64, ctypes.c_int, _u64p]
        L.hho_hash_batch.restype = ctypes.c_int
        self.L = L
        self.path = path

    def constants(self):
        """Section 4.4: (C0, C1) as lists of four u64 lanes, lane 0 first."""
        c0, c1 = _u64arr([0] * 4), _u64arr([0] * 4)
        self.L.hho_constants(c0, c1)
        return list(c0), list(c1)

    def zipper_merge(self, v):
        out = _u64arr([0] * 4)
        self.L.hho_zipper_merge(_u64arr(v), out)
        return list(out)

    def permute(self, v0):
        out = _u64arr([0] * 4)
        self.L.hho_permute(_u64arr(v0), out)
        return list(out)

    def init_state(self, key) -> State:
        s = State()
        self.L.hho_init(ctypes.byref(s), _u64arr(key))
        return s

    def update(self, s: State, packet) -> State:
        self.L.hho_update(ctypes.byref(s), _u64arr(packet))
        return s

    def remainder(self, s: State, tail: bytes) -> State:
        self.L.hho_remainder(ctypes.byref(s), _bytes_ptr(tail), len(tail))
        return s

    def finalize(self, s: State, rounds: int = 4) -> State:
        self.L.hho_finalize(ctypes.byref(s), rounds)
        return s

    def output(self, s: State):
        h = _u64arr([0] * 4)
        self.L.hho_output(ctypes.byref(s), h)
        return list(h)

    def hash_rounds(self, key, msg: bytes, bits: int = 64, rounds: int = 4):
        out = _u64arr([0] * 4)
        rc = self.L.hho_hash_rounds(_u64arr(key), _bytes_ptr(msg), len(msg), bits, rounds, out)
        if rc != 0:
            raise ValueError("bad bits")
        return list(out)[: bits // 64]

    def hash64(self, key, msg: bytes) -> int:
        out = _u64arr([0])
        self.L.hho_hash64(_u64arr(key), _bytes_ptr(msg), len(msg), out)
        return int(out[0])

    def hash128(self, key, msg: bytes):
        out = _u64arr([0] * 2)
        self.L.hho_hash128(_u64arr(key), _bytes_ptr(msg), len(msg), out)
        return list(out)

    def hash256(self, key, msg: bytes):
        out = _u64arr([0] * 4)
        self.L.hho_hash256(_u64arr(key), _bytes_ptr(msg), len(msg), out)
        return list(out)

    def hash_batch(self, keys: np.ndarray, per_message_keys: bool, data: np.ndarray,
                   offsets: np.ndarray, bits: int = 64, first: int = 0,
                   last: int | None = None, out: np.ndarray | None = None) -> np.ndarray:
        """Hash messages [first, last) of a batch (numpy arrays, host memory).

        keys: uint64 [4] (shared) or [n, 4] (per message); data: uint8 [total];
        offsets: int64 [n + 1].  Returns uint64 [last - first, bits // 64].
        The C call releases the GIL, so threads may hash disjoint ranges at once.
        """
        n = offsets.shape[0] - 1
        last = n if last is None else last
        words = bits // 64
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        data = np.ascontiguousarray(data, dtype=np.uint8)
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        if out is None:
            out = np.zeros((last - first, words), dtype=np.uint64)
        keep = _bytes_ptr(b"")
        dptr = data.ctypes.data_as(_u8p) if data.size else keep
        rc = self.L.hho_hash_batch(keys.ctypes.data_as(_u64p), int(per_message_keys), dptr,
                                   offsets.ctypes.data_as(_i64p), first, last, bits,
                                   out.ctypes.data_as(_u64p))
        if rc != 0:
            raise ValueError("oracle rejected the batch (bits or offsets)")
        return out


def lib() -> OracleLib:
    """The default oracle build (compiled on first use)."""
    global _lib
    with _lock:
        if _lib is None:
            _lib = OracleLib(build())
    return _lib


def constants():
    return lib().constants()


def zipper_merge(v):
    return lib().zipper_merge(v)


def permute(v0):
    return lib().permute(v0)


def init_state(key) -> State:
    return lib().init_state(key)


def update(s: State, packet) -> State:
    return lib().update(s, packet)


def remainder(s: State, tail: bytes) -> State:
    return lib().remainder(s, tail)


def finalize(s: State, rounds: int = 4) -> State:
    return lib().finalize(s, rounds)


def output(s: State):
    return lib().output(s)


def hash_rounds(key, msg: bytes, bits: int = 64, rounds: int = 4):
    return lib().hash_rounds(key, msg, bits, rounds)


def hash64(key, msg: bytes) -> int:
    return lib().hash64(key, msg)


def hash128(key, msg: bytes):
    return lib().hash128(key, msg)


def hash256(key, msg: bytes):
    return lib().hash256(key, msg)


def hash_batch(keys, per_message_keys, data, offsets, bits=64, first=0, last=None, out=None):
    return lib().hash_batch(keys, per_message_keys, data, offsets, bits, first, last, out)
