"""Thin ctypes binding of libhh (include/hh.h): argument marshalling only.

Every function here has the name of the C entry point it calls.  Tensors are
PyTorch tensors on the context's CUDA device (PyTorch supplies device memory
and streams); every step of the hash runs in libhh's CUDA kernels.  There is
no CPU fallback: if libhh.so has not been built, loading raises.

HighwayHash here is the keyed hash of arXiv:1612.06257, Section 4, with the
readings stated in include/hh.h; agreement with any released HighwayHash
library is not claimed.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

try:
    import torch
except ImportError:  # the host-buffer entry point needs only numpy
    torch = None

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhh.so")

HH_OK = 0
HH_ERR_INVALID_ARG = 1
HH_ERR_CUDA = 2
HH_ERR_NO_MEMORY = 3
HH_ERR_TIMEOUT = 4
HH_ERR_TOO_LARGE = 5
HH_ERR_BAD_OFFSETS = 6
HH_ERR_NO_DEVICE = 7
HH_ERR_BAD_KEY_INDEX = 8
HH_ERR_BAD_CHUNK = 9

HH_KEY_SHARED = 0
HH_KEY_PER_MESSAGE = 1

HH_KERNEL_AUTO = 0
HH_KERNEL_NAIVE = 1
HH_KERNEL_STAGED = 2
HH_KERNEL_STAGED_UNSORTED = 3
HH_KERNEL_STAGED_BULK = 4

# Every symbol include/hh.h declares.
EXPORTS = (
    "hh_init", "hh_destroy", "hh_reserve", "hh_hash64_batch", "hh_hash128_batch",
    "hh_hash256_batch", "hh_hash_fixed", "hh_hash_host", "hh_get_device_error",
    "hh_set_kernel", "hh_last_launch_count", "hh_status_string", "hh_set_staged_shape",
    "hh_update_microbench", "hh_hash_batch_noalloc", "hh_hash_segments", "hh_autotune",
    "hh_tune_save", "hh_tune_describe", "hh_set_tune_param", "hh_prng_fill",
    "hh_stats_round_table", "hh_stats_toggle_counts", "hh_stats_avalanche", "hh_stream_init",
    "hh_stream_update", "hh_stream_finish", "hh_siptree_batch",
)

HH_SIPTREE = 24
HH_SIPTREE13 = 13

HH_REGIME_FIXED = 0
HH_REGIME_RAGGED = 1
HH_REGIME_BULK = 2

_lock = threading.Lock()
_lib = None

_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int


class HHError(RuntimeError):
    """A libhh call returned a status other than HH_OK."""

    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s: %s (status %d)" % (where, hh_status_string(status), status))


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libhh.so and declare its signatures.  Raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(
                "libhh.so is not built (%s); run paper_1612_06257_gb300.build.build() "
                "or __graft_entry__.build().  There is no CPU fallback." % path)
        L = ctypes.CDLL(path)
        L.hh_init.argtypes = [ctypes.POINTER(_vp), _int, ctypes.c_char_p]
        L.hh_destroy.argtypes = [_vp]
        L.hh_reserve.argtypes = [_vp, _i64]
        batch = [_vp, _vp, _int, _vp, _vp, _i64, _vp, _vp]
        L.hh_hash64_batch.argtypes = batch
        L.hh_hash128_batch.argtypes = batch
        L.hh_hash256_batch.argtypes = batch
        L.hh_hash_fixed.argtypes = [_vp, _int, _vp, _int, _vp, _i64, _i64, _vp, _vp]
        L.hh_hash_host.argtypes = [_vp, _int, _vp, _int, _vp, _vp, _i64, _vp]
        L.hh_get_device_error.argtypes = [_vp, _vp]
        L.hh_set_kernel.argtypes = [_vp, _int]
        L.hh_last_launch_count.argtypes = [_vp]
        L.hh_set_staged_shape.argtypes = [_vp, _int, _int, _int, _int]
        L.hh_update_microbench.argtypes = [_vp, _int, _i64, _i64, _vp, _vp]
        L.hh_hash_batch_noalloc.argtypes = [_int, _vp, _int, _vp, _vp, _i64, _vp, _vp, _vp]
        L.hh_autotune.argtypes = [_vp, _i64]
        L.hh_tune_save.argtypes = [_vp, ctypes.c_char_p]
        L.hh_set_tune_param.argtypes = [_vp, ctypes.c_char_p, _int]
        L.hh_stream_init.argtypes = [_vp, _vp, _int, _i64, _vp, _vp]
        L.hh_stream_update.argtypes = [_vp, _vp, _vp, _vp, _i64, _vp]
        L.hh_stream_finish.argtypes = [_vp, _int, _vp, _vp, _vp, _i64, _vp, _vp]
        L.hh_prng_fill.argtypes = [_vp, _int, _vp, ctypes.c_uint64, _i64, _vp, _vp]
        L.hh_stats_round_table.argtypes = [_vp, ctypes.POINTER(ctypes.c_uint64), _int, _int,
                                           _vp, _vp]
        L.hh_stats_toggle_counts.argtypes = [_vp, _vp, _int, _vp, _vp]
        L.hh_stats_avalanche.argtypes = [_vp, _int, ctypes.c_uint64, _i64, _vp, _vp]
        L.hh_tune_describe.argtypes = [_vp, ctypes.c_char_p, _i64]
        L.hh_hash_segments.argtypes = [_vp, _int, _vp, ctypes.c_int32, _vp, _vp, _i64, _vp, _vp,
                                       _i64, _vp, _vp, _vp]
        L.hh_siptree_batch.argtypes = [_vp, _int, _vp, _int, _vp, _vp, _i64, _vp, _vp]
        L.hh_status_string.argtypes = [_int]
        L.hh_status_string.restype = ctypes.c_char_p
        _lib = L
        return L


def hh_status_string(status: int) -> str:
    return load_library().hh_status_string(int(status)).decode()


def _check(status: int, where: str) -> None:
    if status != HH_OK:
        raise HHError(status, where)


class Context:
    """An hh_ctx* and the CUDA device it lives on."""

    def __init__(self, ptr: int, device: int):
        self.ptr = ptr
        self.device = device

    def __del__(self):
        try:
            if self.ptr:
                hh_destroy(self)
        except Exception:
            pass


def hh_init(device: int = 0, tune_cache_path: str | None = None) -> Context:
    p = _vp()
    path = tune_cache_path.encode() if tune_cache_path else None
    _check(load_library().hh_init(ctypes.byref(p), int(device), path), "hh_init")
    return Context(p.value, int(device))


def hh_destroy(ctx: Context) -> None:
    if ctx.ptr:
        ptr, ctx.ptr = ctx.ptr, None
        _check(load_library().hh_destroy(ptr), "hh_destroy")


def hh_reserve(ctx: Context, max_messages: int) -> None:
    """Size the context's sort scratch for batches of up to max_messages (the
    hash calls never allocate; beyond it they raise HH_ERR_TOO_LARGE)."""
    _check(load_library().hh_reserve(ctx.ptr, int(max_messages)), "hh_reserve")


def _stream_ptr(stream, device):
    if stream is None:
        return torch.cuda.current_stream(device).cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


_I64 = (torch.int64,) + ((torch.uint64,) if hasattr(torch, "uint64") else ())


def _dev_ptr(t, name, dtypes, device):
    if t is None:
        return None
    if t.get_device() != device:  # -1 for CPU tensors
        raise ValueError("%s must be a CUDA tensor on device %d" % (name, device))
    if t.dtype not in dtypes:
        raise ValueError("%s has dtype %s, expected one of %s" % (name, t.dtype, dtypes))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return t.data_ptr()


def _batch(fn_name, words, ctx, keys, key_mode, data, offsets, n=None, out=None, stream=None):
    n = offsets.numel() - 1 if n is None else int(n)
    if out is None:
        out = torch.empty(n * words, dtype=torch.int64, device=data.device)
    if out.numel() < n * words:
        raise ValueError("out holds %d words, need %d" % (out.numel(), n * words))
    dev = ctx.device
    i64 = _I64
    args = (ctx.ptr, _dev_ptr(keys, "keys", i64, dev), int(key_mode),
            _dev_ptr(data, "bytes", (torch.uint8,), dev),
            _dev_ptr(offsets, "offsets", (torch.int64,), dev), n,
            _dev_ptr(out, "out", i64, dev), _stream_ptr(stream, dev))
    _check(getattr(load_library(), fn_name)(*args), fn_name)
    return out


def hh_hash64_batch(ctx, keys, key_mode, data, offsets, n=None, out=None, stream=None):
    """64-bit hashes of a ragged batch; returns out (int64 [n], uint64 bit patterns)."""
    return _batch("hh_hash64_batch", 1, ctx, keys, key_mode, data, offsets, n, out, stream)


def hh_hash128_batch(ctx, keys, key_mode, data, offsets, n=None, out=None, stream=None):
    return _batch("hh_hash128_batch", 2, ctx, keys, key_mode, data, offsets, n, out, stream)


def hh_hash256_batch(ctx, keys, key_mode, data, offsets, n=None, out=None, stream=None):
    return _batch("hh_hash256_batch", 4, ctx, keys, key_mode, data, offsets, n, out, stream)


def hh_siptree_batch(ctx, variant, keys, key_mode, data, offsets, n=None, out=None,
                     stream=None):
    """SipTreeHash (HH_SIPTREE) or SipTreeHash13 (HH_SIPTREE13) of a ragged
    batch; returns out (int64 [n], uint64 bit patterns)."""
    n = offsets.numel() - 1 if n is None else int(n)
    if out is None:
        out = torch.empty(n, dtype=torch.int64, device=data.device)
    if out.numel() < n:
        raise ValueError("out holds %d words, need %d" % (out.numel(), n))
    dev = ctx.device
    st = load_library().hh_siptree_batch(
        ctx.ptr, int(variant), _dev_ptr(keys, "keys", _I64, dev), int(key_mode),
        _dev_ptr(data, "bytes", (torch.uint8,), dev),
        _dev_ptr(offsets, "offsets", (torch.int64,), dev), n, _dev_ptr(out, "out", _I64, dev),
        _stream_ptr(stream, dev))
    _check(st, "hh_siptree_batch")
    return out


def hh_hash_fixed(ctx, bits, keys, key_mode, data, msg_len, n, out=None, stream=None):
    words = {64: 1, 128: 2, 256: 4}.get(int(bits))
    if words is None:
        raise ValueError("bits must be 64, 128 or 256")
    if out is None:
        out = torch.empty(int(n) * words, dtype=torch.int64, device=data.device)
    dev = ctx.device
    i64 = _I64
    st = load_library().hh_hash_fixed(
        ctx.ptr, int(bits), _dev_ptr(keys, "keys", i64, dev), int(key_mode),
        _dev_ptr(data, "bytes", (torch.uint8,), dev), int(msg_len), int(n),
        _dev_ptr(out, "out", i64, dev), _stream_ptr(stream, dev))
    _check(st, "hh_hash_fixed")
    return out


def hh_hash_segments(ctx, bits, key_table, key_index, data, starts, lengths, out=None,
                     stream=None, n_device=None):
    """Hash segments data[starts[i] : starts[i] + lengths[i]] with key
    key_table[key_index[i]] (key_index None: row 0 for all).  key_table: int64
    [k, 4]; key_index: int32 [n]; starts, lengths: int64 [n]; all on the
    context's device.  n_device: optional int64 [1] device tensor holding the
    live message count (the arrays are then a capacity).  Returns out (int64
    [n * bits // 64])."""
    words = {64: 1, 128: 2, 256: 4}.get(int(bits))
    if words is None:
        raise ValueError("bits must be 64, 128 or 256")
    n = starts.numel()
    if lengths.numel() != n or (key_index is not None and key_index.numel() != n):
        raise ValueError("starts, lengths and key_index must have n entries")
    if out is None:
        out = torch.empty(n * words, dtype=torch.int64, device=data.device)
    dev = ctx.device
    i64 = _I64
    st = load_library().hh_hash_segments(
        ctx.ptr, int(bits), _dev_ptr(key_table, "key_table", i64, dev),
        int(key_table.numel() // 4), _dev_ptr(key_index, "key_index", (torch.int32,), dev),
        _dev_ptr(data, "bytes", (torch.uint8,), dev), int(data.numel()),
        _dev_ptr(starts, "starts", (torch.int64,), dev),
        _dev_ptr(lengths, "lengths", (torch.int64,), dev), n,
        _dev_ptr(n_device, "n_device", (torch.int64,), dev),
        _dev_ptr(out, "out", i64, dev), _stream_ptr(stream, dev))
    _check(st, "hh_hash_segments")
    return out


def hh_hash_host(ctx, bits, keys: np.ndarray, key_mode, data: np.ndarray, offsets: np.ndarray,
                 out: np.ndarray | None = None) -> np.ndarray:
    """Host-buffer call: numpy arrays in host memory (pinned for full speed)."""
    words = {64: 1, 128: 2, 256: 4}.get(int(bits))
    if words is None:
        raise ValueError("bits must be 64, 128 or 256")
    n = offsets.shape[0] - 1
    for name, a, dt in (("keys", keys, np.uint64), ("bytes", data, np.uint8),
                        ("offsets", offsets, np.int64)):
        if a.dtype != dt or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("%s must be a contiguous %s array" % (name, np.dtype(dt).name))
    if out is None:
        out = np.empty(n * words, dtype=np.uint64)
    st = load_library().hh_hash_host(ctx.ptr, int(bits), keys.ctypes.data, int(key_mode),
                                     data.ctypes.data if data.size else None,
                                     offsets.ctypes.data, n, out.ctypes.data)
    _check(st, "hh_hash_host")
    return out


def hh_get_device_error(ctx, stream=None) -> int:
    """Synchronise the stream; return (and clear) the device error word."""
    st = load_library().hh_get_device_error(ctx.ptr, _stream_ptr(stream, ctx.device))
    if st == HH_ERR_CUDA or st == HH_ERR_INVALID_ARG:
        raise HHError(st, "hh_get_device_error")
    return st


def hh_set_kernel(ctx, kernel: int) -> None:
    _check(load_library().hh_set_kernel(ctx.ptr, int(kernel)), "hh_set_kernel")


def hh_set_staged_shape(ctx, regime: int, window: int, stages: int,
                        messages_per_thread: int = 1) -> None:
    _check(load_library().hh_set_staged_shape(ctx.ptr, int(regime), int(window), int(stages),
                                              int(messages_per_thread)), "hh_set_staged_shape")


def hh_update_microbench(ctx, variant: int, updates: int, threads: int, out=None, stream=None):
    """Run the Update-rate microbenchmark; returns out (int64 [threads])."""
    if out is None:
        out = torch.empty(int(threads), dtype=torch.int64, device="cuda:%d" % ctx.device)
    st = load_library().hh_update_microbench(ctx.ptr, int(variant), int(updates), int(threads),
                                             _dev_ptr(out, "out", (torch.int64,), ctx.device),
                                             _stream_ptr(stream, ctx.device))
    _check(st, "hh_update_microbench")
    return out


def hh_autotune(ctx, max_device_bytes: int = 1 << 30) -> None:
    _check(load_library().hh_autotune(ctx.ptr, int(max_device_bytes)), "hh_autotune")


def hh_stream_init(ctx, keys, key_mode: int, n: int, states=None, stream=None):
    """New stream states (int64 [n, 16]) from the keys."""
    if states is None:
        states = torch.empty(int(n), 16, dtype=torch.int64, device="cuda:%d" % ctx.device)
    st = load_library().hh_stream_init(ctx.ptr, _dev_ptr(keys, "keys", _I64, ctx.device),
                                       int(key_mode), int(n),
                                       _dev_ptr(states, "states", _I64, ctx.device),
                                       _stream_ptr(stream, ctx.device))
    _check(st, "hh_stream_init")
    return states


def hh_stream_update(ctx, states, data, offsets, stream=None):
    """Append piece m = data[offsets[m]:offsets[m+1]] (whole 32-byte packets) to stream m."""
    n = offsets.numel() - 1
    st = load_library().hh_stream_update(ctx.ptr, _dev_ptr(states, "states", _I64, ctx.device),
                                         _dev_ptr(data, "bytes", (torch.uint8,), ctx.device),
                                         _dev_ptr(offsets, "offsets", (torch.int64,), ctx.device),
                                         n, _stream_ptr(stream, ctx.device))
    _check(st, "hh_stream_update")
    return states


def hh_stream_finish(ctx, bits, states, data, offsets, out=None, stream=None):
    """Append the last pieces and return the hashes (int64 [n * bits // 64])."""
    words = {64: 1, 128: 2, 256: 4}.get(int(bits))
    if words is None:
        raise ValueError("bits must be 64, 128 or 256")
    n = offsets.numel() - 1
    if out is None:
        out = torch.empty(n * words, dtype=torch.int64, device=data.device)
    st = load_library().hh_stream_finish(ctx.ptr, int(bits),
                                         _dev_ptr(states, "states", _I64, ctx.device),
                                         _dev_ptr(data, "bytes", (torch.uint8,), ctx.device),
                                         _dev_ptr(offsets, "offsets", (torch.int64,), ctx.device),
                                         n, _dev_ptr(out, "out", _I64, ctx.device),
                                         _stream_ptr(stream, ctx.device))
    _check(st, "hh_stream_finish")
    return out


def hh_prng_fill(ctx, bits, key, counter0: int, n: int, out=None, stream=None):
    """out[i] = HighwayHash(key, 8-byte LE counter0 + i); returns int64 [n * bits // 64]."""
    words = {64: 1, 128: 2, 256: 4}.get(int(bits))
    if words is None:
        raise ValueError("bits must be 64, 128 or 256")
    if out is None:
        out = torch.empty(int(n) * words, dtype=torch.int64, device="cuda:%d" % ctx.device)
    st = load_library().hh_prng_fill(ctx.ptr, int(bits), _dev_ptr(key, "key", _I64, ctx.device),
                                     int(counter0) & ((1 << 64) - 1), int(n),
                                     _dev_ptr(out, "out", _I64, ctx.device),
                                     _stream_ptr(stream, ctx.device))
    _check(st, "hh_prng_fill")
    return out


def hh_stats_round_table(ctx, key, nbytes: int, rounds: int, table=None, stream=None):
    """Hashes of all nbytes-byte inputs with `rounds` finalisation rounds;
    key: 4 ints (host).  Returns int64 [2 ** (8 * nbytes)]."""
    if table is None:
        table = torch.empty(1 << (8 * int(nbytes)), dtype=torch.int64,
                            device="cuda:%d" % ctx.device)
    k = (ctypes.c_uint64 * 4)(*[int(x) & ((1 << 64) - 1) for x in key])
    st = load_library().hh_stats_round_table(ctx.ptr, k, int(nbytes), int(rounds),
                                             _dev_ptr(table, "table", _I64, ctx.device),
                                             _stream_ptr(stream, ctx.device))
    _check(st, "hh_stats_round_table")
    return table


def hh_stats_toggle_counts(ctx, table, m: int, counts=None, stream=None):
    """Adds toggle counts into counts (int64 [m * 64], zeroed when created here)."""
    if counts is None:
        counts = torch.zeros(int(m) * 64, dtype=torch.int64, device="cuda:%d" % ctx.device)
    st = load_library().hh_stats_toggle_counts(ctx.ptr, _dev_ptr(table, "table", _I64, ctx.device),
                                               int(m), _dev_ptr(counts, "counts", _I64, ctx.device),
                                               _stream_ptr(stream, ctx.device))
    _check(st, "hh_stats_toggle_counts")
    return counts


def hh_stats_avalanche(ctx, size: int, seed: int, iterations: int, counts=None, stream=None):
    """Adds avalanche flip counts into counts (int64 [8 * size * 64])."""
    if counts is None:
        counts = torch.zeros(8 * int(size) * 64, dtype=torch.int64, device="cuda:%d" % ctx.device)
    st = load_library().hh_stats_avalanche(ctx.ptr, int(size), int(seed) & ((1 << 64) - 1),
                                           int(iterations),
                                           _dev_ptr(counts, "counts", _I64, ctx.device),
                                           _stream_ptr(stream, ctx.device))
    _check(st, "hh_stats_avalanche")
    return counts


def hh_set_tune_param(ctx, name: str, value: int) -> None:
    _check(load_library().hh_set_tune_param(ctx.ptr, name.encode(), int(value)),
           "hh_set_tune_param")


def hh_tune_save(ctx, path: str) -> None:
    _check(load_library().hh_tune_save(ctx.ptr, path.encode()), "hh_tune_save")


def hh_tune_describe(ctx) -> str:
    buf = ctypes.create_string_buffer(8192)
    _check(load_library().hh_tune_describe(ctx.ptr, buf, len(buf)), "hh_tune_describe")
    return buf.value.decode()


def hh_last_launch_count(ctx) -> int:
    return int(load_library().hh_last_launch_count(ctx.ptr))
