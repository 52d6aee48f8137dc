"""Thin ctypes binding of libfalcon (C ABI in include/falcon.h).

Argument marshalling only: every step of compression and decompression runs in
the CUDA kernels of ``_build/libfalcon.so``.  PyTorch supplies device memory and
streams.  There is no CPU fallback: if the library is missing or a call fails,
an exception is raised.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

F64, F32 = 0, 1
OK, ERR_INVALID, ERR_CAPACITY, ERR_CORRUPT, ERR_CUDA, ERR_TIMEOUT, ERR_UNSUPPORTED = range(7)
HEADER_BYTES = 32
MAX_BLOCK = 1025

_lock = threading.Lock()
_lib = None


class FalconError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        name = _load().falcon_status_string(status).decode() if _lib is not None else str(status)
        super().__init__(f"libfalcon {what}: {name} (status {status})")


def _load():
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"libfalcon is not built ({path}); run paper_2511_04140_gb300/build.py")
            L = ctypes.CDLL(path)
            c = ctypes
            vp, sz, u64, u32, ci = c.c_void_p, c.c_size_t, c.c_uint64, c.c_uint32, c.c_int
            L.falcon_abi_version.restype = ci
            L.falcon_status_string.restype = c.c_char_p
            L.falcon_status_string.argtypes = [ci]
            L.falcon_bound.restype = sz
            L.falcon_bound.argtypes = [u64, ci, u32]
            L.falcon_stream_info.restype = ci
            L.falcon_stream_info.argtypes = [vp, sz, c.POINTER(u64), c.POINTER(ci), c.POINTER(u32), c.POINTER(u64)]
            L.falcon_compress.restype = ci
            L.falcon_compress.argtypes = [vp, u64, ci, u32, vp, sz, c.POINTER(sz), vp]
            L.falcon_decompress.restype = ci
            L.falcon_decompress.argtypes = [vp, sz, vp, sz, c.POINTER(u64), vp]
            L.falcon_workspace_bytes.restype = sz
            L.falcon_workspace_bytes.argtypes = [u64]
            L.falcon_compress_async.restype = ci
            L.falcon_compress_async.argtypes = [vp, u64, ci, u32, vp, sz, vp, sz, vp, vp]
            L.falcon_decompress_async.restype = ci
            L.falcon_decompress_async.argtypes = [vp, sz, vp, vp, sz, vp, sz, vp, vp]
            L.falcon_release.restype = ci
            _lib = L
    return _lib


def lib():
    return _load()


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    raise TypeError(f"unsupported dtype {t.dtype}")


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _check(st: int, what: str):
    if st != OK:
        raise FalconError(st, what)


def bound(n: int, dtype_code: int, block: int = 1024) -> int:
    return _load().falcon_bound(n, dtype_code, block)


def workspace_bytes(nchunks: int) -> int:
    return _load().falcon_workspace_bytes(nchunks)


def stream_info(header) -> tuple:
    """(n, dtype_code, block, num_chunks) from a host copy of the first 32 bytes."""
    buf = bytes(header)[:HEADER_BYTES]
    n, nc = ctypes.c_uint64(), ctypes.c_uint64()
    dt, blk = ctypes.c_int(), ctypes.c_uint32()
    _check(_load().falcon_stream_info(buf, len(buf), ctypes.byref(n), ctypes.byref(dt), ctypes.byref(blk),
                                      ctypes.byref(nc)), "stream_info")
    return n.value, dt.value, blk.value, nc.value


def compress(x: torch.Tensor, block: int = 1024, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Compresses a contiguous CUDA FP64/FP32 tensor; returns a uint8 CUDA tensor view of the stream."""
    if not x.is_cuda or not x.is_contiguous():
        raise ValueError("x must be a contiguous CUDA tensor")
    code = _dtype_code(x)
    n = x.numel()
    cap = bound(n, code, block)
    if out is None:
        out = torch.empty(max(cap, 32), dtype=torch.uint8, device=x.device)
    nbytes = ctypes.c_size_t()
    _check(_load().falcon_compress(x.data_ptr(), n, code, block, out.data_ptr(), out.numel(),
                                   ctypes.byref(nbytes), _stream_ptr(stream)), "compress")
    return out[:nbytes.value]


def decompress(s: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Decompresses a uint8 CUDA tensor holding one stream; returns the values."""
    if not s.is_cuda or s.dtype != torch.uint8:
        raise ValueError("s must be a uint8 CUDA tensor")
    hdr = s[:HEADER_BYTES].cpu().numpy().tobytes() if s.numel() >= HEADER_BYTES else b""
    if len(hdr) < HEADER_BYTES:
        raise FalconError(ERR_CORRUPT, "decompress")
    n, code, _, _ = stream_info(hdr)
    dtype = torch.float64 if code == F64 else torch.float32
    if out is None:
        out = torch.empty(max(n, 1), dtype=dtype, device=s.device)
    n_out = ctypes.c_uint64()
    _check(_load().falcon_decompress(s.data_ptr(), s.numel(), out.data_ptr(), out.numel() * out.element_size(),
                                     ctypes.byref(n_out), _stream_ptr(stream)), "decompress")
    return out[:n_out.value]


def compress_async(x: torch.Tensor, block: int, out: torch.Tensor, workspace: torch.Tensor,
                   result: torch.Tensor, stream=None) -> None:
    """Enqueues compression without synchronising; result (uint64[2] on device) receives
    [stream bytes, status]."""
    _check(_load().falcon_compress_async(x.data_ptr(), x.numel(), _dtype_code(x), block, out.data_ptr(),
                                         out.numel(), workspace.data_ptr(), workspace.numel(),
                                         result.data_ptr(), _stream_ptr(stream)), "compress_async")


def decompress_async(s: torch.Tensor, nbytes: int, header: bytes, out: torch.Tensor, workspace: torch.Tensor,
                     result: torch.Tensor, stream=None) -> None:
    """Enqueues decompression of s[:nbytes] (header: host copy of its first 32 bytes)."""
    hdr = bytes(header)[:HEADER_BYTES]
    _check(_load().falcon_decompress_async(s.data_ptr(), nbytes, hdr, out.data_ptr(),
                                           out.numel() * out.element_size(), workspace.data_ptr(),
                                           workspace.numel(), result.data_ptr(), _stream_ptr(stream)),
           "decompress_async")


def release() -> None:
    _load().falcon_release()
