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

F64, F32, F16 = 0, 1, 2
OK, ERR_INVALID, ERR_CAPACITY, ERR_CORRUPT, ERR_CUDA, ERR_TIMEOUT, ERR_UNSUPPORTED = range(7)
HEADER_BYTES = 32
MAX_BLOCK = 1025

_lock = threading.Lock()
_lib = None
COMPRESS, DECOMPRESS = 0, 1
# compression schedulers of the host pipeline (falcon_scheduler, Sec. 3.1)
SCHED_EVENT_DRIVEN, SCHED_SYNC_BASED, SCHED_PRE_ALLOCATION = 0, 1, 2
# codec variants (falcon_variant): Falcon and the ablations of Sec. 5.4.2
VARIANT_FALCON, VARIANT_SPARSE, VARIANT_DENSE, VARIANT_ELF = 0, 1, 2, 3


class Series(ctypes.Structure):
    """falcon_series (include/falcon.h)."""
    _fields_ = [("d_in", ctypes.c_void_p), ("d_out", ctypes.c_void_p), ("n", ctypes.c_uint64),
                ("in_bytes", ctypes.c_uint64), ("out_capacity", ctypes.c_uint64), ("dtype", ctypes.c_int32),
                ("block_size", ctypes.c_uint32), ("h_header", ctypes.c_void_p)]


class Completion(ctypes.Structure):
    """falcon_completion (include/falcon.h)."""
    _fields_ = [("tag", ctypes.c_uint64), ("status", ctypes.c_int32), ("op", ctypes.c_int32),
                ("h_out", ctypes.c_void_p), ("out_bytes", ctypes.c_uint64), ("values", ctypes.c_uint64),
                ("latency_s", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    """falcon_server_stats (include/falcon.h)."""
    _fields_ = [(k, ctypes.c_uint64) for k in (
        "submitted", "completed", "failed", "batches", "multi_request_batches", "max_batch", "max_in_flight",
        "device_capacity", "device_in_use", "device_peak", "host_capacity", "host_in_use", "host_peak")]


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
            L.falcon_compress_variant_async.restype = ci
            L.falcon_compress_variant_async.argtypes = [vp, u64, ci, u32, ci, vp, sz, vp, sz, vp, vp]
            L.falcon_variant_bound.restype = sz
            L.falcon_variant_bound.argtypes = [u64, ci, u32, ci]
            L.falcon_decompress_async.restype = ci
            L.falcon_decompress_async.argtypes = [vp, sz, vp, vp, sz, vp, sz, vp, vp]
            L.falcon_aggregate_async.restype = ci
            L.falcon_aggregate_async.argtypes = [vp, sz, vp, vp, sz, vp, vp]
            L.falcon_aggregate.restype = ci
            L.falcon_aggregate.argtypes = [vp, sz, c.POINTER(Stats), vp]
            L.falcon_release.restype = ci
            L.falcon_batch_workspace_bytes.restype = sz
            L.falcon_batch_workspace_bytes.argtypes = [ci, c.POINTER(Series), ci]
            L.falcon_batch_plan.restype = ci
            L.falcon_batch_plan.argtypes = [ci, c.POINTER(Series), ci, vp, sz, vp, vp]
            L.falcon_batch_launch.restype = ci
            L.falcon_batch_launch.argtypes = [vp, vp]
            L.falcon_batch_forget.restype = ci
            L.falcon_batch_forget.argtypes = [vp]
            L.falcon_set_launch_config.restype = ci
            L.falcon_set_launch_config.argtypes = [ci, ci]
            L.falcon_set_cta_warps.restype = ci
            L.falcon_set_cta_warps.argtypes = [ci, ci]
            L.falcon_pipeline_compress.restype = ci
            L.falcon_pipeline_compress.argtypes = [vp, u64, ci, u32, u64, ci, vp, sz, vp, c.POINTER(sz)]
            L.falcon_pipeline_compress_with.restype = ci
            L.falcon_pipeline_compress_with.argtypes = [vp, u64, ci, u32, u64, ci, ci, vp, sz, vp, c.POINTER(sz)]
            L.falcon_pipeline_decompress.restype = ci
            L.falcon_pipeline_decompress.argtypes = [vp, vp, u64, ci, vp, sz, c.POINTER(u64)]
            L.falcon_compress_noalloc.restype = ci
            L.falcon_compress_noalloc.argtypes = [vp, u64, ci, u32, vp, sz, vp, vp]
            L.falcon_server_create.restype = ci
            L.falcon_server_create.argtypes = [ci, sz, sz, ci, ci, sz, c.POINTER(vp)]
            L.falcon_server_submit.restype = ci
            L.falcon_server_submit.argtypes = [vp, ci, vp, u64, ci, u32, u64]
            L.falcon_server_poll.restype = ci
            L.falcon_server_poll.argtypes = [vp, c.POINTER(Completion), ci, ci, c.POINTER(ci)]
            L.falcon_server_free_output.restype = ci
            L.falcon_server_free_output.argtypes = [vp, vp]
            L.falcon_server_get_stats.restype = ci
            L.falcon_server_get_stats.argtypes = [vp, c.POINTER(ServerStats)]
            L.falcon_server_destroy.restype = ci
            L.falcon_server_destroy.argtypes = [vp]
            _lib = L
    return _lib


def lib():
    return _load()


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.float16:
        return F16
    raise TypeError(f"unsupported dtype {t.dtype}")


def torch_dtype(code: int) -> torch.dtype:
    """The torch dtype of a stream's dtype code (FALCON_F64 / F32 / F16)."""
    return {F64: torch.float64, F32: torch.float32, F16: torch.float16}[code]


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _check(st: int, what: str):
    if st != OK:
        raise FalconError(st, what)


def bound(n: int, dtype_code: int, block: int = 1024) -> int:
    return _load().falcon_bound(n, dtype_code, block)


def variant_bound(n: int, dtype_code: int, block: int, variant: int) -> int:
    return _load().falcon_variant_bound(n, dtype_code, block, variant)


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
    dtype = torch_dtype(code)
    if out is None:
        out = torch.empty(max(n, 1), dtype=dtype, device=s.device)
    n_out = ctypes.c_uint64()
    _check(_load().falcon_decompress(s.data_ptr(), s.numel(), out.data_ptr(), out.numel() * out.element_size(),
                                     ctypes.byref(n_out), _stream_ptr(stream)), "decompress")
    return out[:n_out.value]


class Stats(ctypes.Structure):
    """falcon_stats: the aggregate of a stream (analytics on compressed data)."""
    _fields_ = [("count", ctypes.c_uint64), ("nan_count", ctypes.c_uint64), ("min", ctypes.c_double),
                ("max", ctypes.c_double), ("sum", ctypes.c_double), ("status", ctypes.c_uint64)]


STATS_BYTES = 48


def aggregate(s: torch.Tensor, stream=None) -> dict:
    """Aggregate of the stream in a uint8 CUDA tensor, computed from its records without
    writing the values: count, nan_count, min / max (totalOrder, non-NaN), sum."""
    if not s.is_cuda or s.dtype != torch.uint8:
        raise ValueError("s must be a uint8 CUDA tensor")
    st = Stats()
    _check(_load().falcon_aggregate(s.data_ptr(), s.numel(), ctypes.byref(st), _stream_ptr(stream)), "aggregate")
    return {"count": st.count, "nan_count": st.nan_count, "min": st.min, "max": st.max, "sum": st.sum}


def aggregate_async(s: torch.Tensor, nbytes: int, header: bytes, workspace: torch.Tensor, stats: torch.Tensor,
                    stream=None) -> None:
    """Enqueues the aggregate of s[:nbytes] into stats (uint8 CUDA tensor of STATS_BYTES,
    8-byte aligned; read it with stats_of)."""
    hdr = bytes(header)[:HEADER_BYTES]
    _check(_load().falcon_aggregate_async(s.data_ptr(), nbytes, hdr, workspace.data_ptr(), workspace.numel(),
                                          stats.data_ptr(), _stream_ptr(stream)), "aggregate_async")


def stats_of(stats: torch.Tensor) -> dict:
    st = Stats.from_buffer_copy(stats.cpu().numpy().tobytes())
    return {"count": st.count, "nan_count": st.nan_count, "min": st.min, "max": st.max, "sum": st.sum,
            "status": st.status}


def compress_async(x: torch.Tensor, block: int, out: torch.Tensor, workspace: torch.Tensor,
                   result: torch.Tensor, stream=None) -> None:
    """Enqueues compression without synchronising; result (uint64[2] on device) receives
    [stream bytes, status]."""
    _check(_load().falcon_compress_async(x.data_ptr(), x.numel(), _dtype_code(x), block, out.data_ptr(),
                                         out.numel(), workspace.data_ptr(), workspace.numel(),
                                         result.data_ptr(), _stream_ptr(stream)), "compress_async")


def compress_variant_async(x: torch.Tensor, block: int, variant: int, out: torch.Tensor, workspace: torch.Tensor,
                           result: torch.Tensor, stream=None) -> None:
    """compress_async for a codec variant (VARIANT_*); size `out` with variant_bound."""
    _check(_load().falcon_compress_variant_async(x.data_ptr(), x.numel(), _dtype_code(x), block, variant,
                                                 out.data_ptr(), out.numel(), workspace.data_ptr(),
                                                 workspace.numel(), result.data_ptr(), _stream_ptr(stream)),
           "compress_variant_async")


def compress_variant(x: torch.Tensor, block: int, variant: int, stream=None) -> torch.Tensor:
    """Compresses x with a codec variant (allocates the output and a workspace, synchronises);
    returns the stream as a uint8 CUDA tensor."""
    code = _dtype_code(x)
    out = torch.empty(max(variant_bound(x.numel(), code, block, variant), 32), dtype=torch.uint8, device=x.device)
    ws = torch.empty(workspace_bytes((x.numel() + block - 1) // block), dtype=torch.uint8, device=x.device)
    res = torch.zeros(2, dtype=torch.int64, device=x.device)
    compress_variant_async(x, block, variant, out, ws, res, stream)
    (stream or torch.cuda.current_stream()).synchronize()
    nbytes, status = (int(v) for v in res.cpu())
    if status != OK:
        raise FalconError(status, "compress_variant")
    return out[:nbytes]


def decompress_async(s: torch.Tensor, nbytes: int, header: bytes, out: torch.Tensor, workspace: torch.Tensor,
                     result: torch.Tensor, stream=None) -> None:
    """Enqueues decompression of s[:nbytes] (header: host copy of its first 32 bytes)."""
    hdr = bytes(header)[:HEADER_BYTES]
    _check(_load().falcon_decompress_async(s.data_ptr(), nbytes, hdr, out.data_ptr(),
                                           out.numel() * out.element_size(), workspace.data_ptr(),
                                           workspace.numel(), result.data_ptr(), _stream_ptr(stream)),
           "decompress_async")


def compress_noalloc(x: torch.Tensor, block: int, out: torch.Tensor, result: torch.Tensor, stream=None) -> None:
    """falcon_compress_noalloc: as compress_async, with the library's static scratch."""
    _check(_load().falcon_compress_noalloc(x.data_ptr(), x.numel(), _dtype_code(x), block, out.data_ptr(),
                                           out.numel(), result.data_ptr(), _stream_ptr(stream)), "compress_noalloc")


def release() -> None:
    _load().falcon_release()


def set_launch_config(compress_ctas_per_sm: int = 0, decompress_ctas_per_sm: int = 0) -> None:
    """Caps the persistent grids at the given CTAs per SM (0 = occupancy limit)."""
    _check(_load().falcon_set_launch_config(compress_ctas_per_sm, decompress_ctas_per_sm), "set_launch_config")


def set_cta_warps(compress_warps: int = 4, decompress_warps: int = 4) -> None:
    """Warps per CTA of the persistent kernels (launch shape only, no output byte changes)."""
    _check(_load().falcon_set_cta_warps(compress_warps, decompress_warps), "set_cta_warps")


class Batch:
    """A planned batched launch over many series (the launches of one direction, each covering
    every (series, chunk) work item).

    compress:   Batch(COMPRESS, inputs=[tensor...], block=1024)       -> outputs: uint8 streams
    decompress: Batch(DECOMPRESS, inputs=[(stream_tensor, nbytes, header_bytes), ...])

    launch(stream) only enqueues work (capturable in a CUDA graph); results() reads
    [bytes-or-values, status] per series back to the host.
    """

    def __init__(self, direction: int, inputs, block: int = 1024, outputs=None, device=None):
        self.direction = direction
        self.inputs = list(inputs)
        n = len(self.inputs)
        arr = (Series * max(n, 1))()
        self._headers = []
        self.outputs = []
        for i, item in enumerate(self.inputs):
            sr = arr[i]
            if direction == COMPRESS:
                x = item
                code = _dtype_code(x)
                cap = bound(x.numel(), code, block)
                out = outputs[i] if outputs is not None else torch.empty(max(cap, 32), dtype=torch.uint8, device=x.device)
                sr.d_in, sr.d_out, sr.n = x.data_ptr(), out.data_ptr(), x.numel()
                sr.out_capacity, sr.dtype, sr.block_size = out.numel(), code, block
                sr.h_header = None
            else:
                s_t, nbytes, hdr = item
                hb = ctypes.create_string_buffer(bytes(hdr)[:HEADER_BYTES], HEADER_BYTES)
                self._headers.append(hb)
                nval, code, _, _ = stream_info(bytes(hdr))
                dtype = torch_dtype(code)
                out = outputs[i] if outputs is not None else torch.empty(max(nval, 1), dtype=dtype, device=s_t.device)
                sr.d_in, sr.d_out, sr.in_bytes = s_t.data_ptr(), out.data_ptr(), nbytes
                sr.out_capacity = out.numel() * out.element_size()
                sr.h_header = ctypes.cast(hb, ctypes.c_void_p)
            self.outputs.append(out)
        self._series = arr
        L = _load()
        ws_bytes = L.falcon_batch_workspace_bytes(direction, arr, n)
        if ws_bytes == 0:
            raise FalconError(ERR_INVALID, "batch_workspace_bytes")
        dev = device or (self.inputs[0].device if direction == COMPRESS and n else
                         (self.inputs[0][0].device if n else torch.device("cuda")))
        self.workspace = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
        self.results_dev = torch.zeros(2 * max(n, 1), dtype=torch.int64, device=dev)
        _check(L.falcon_batch_plan(direction, arr, n, self.workspace.data_ptr(), ws_bytes,
                                   self.results_dev.data_ptr(), _stream_ptr(None)), "batch_plan")

    def launch(self, stream=None) -> None:
        _check(_load().falcon_batch_launch(self.workspace.data_ptr(), _stream_ptr(stream)), "batch_launch")

    def results(self):
        r = self.results_dev.view(-1, 2)[:len(self.inputs)].cpu().tolist()
        return [(int(a), int(b)) for a, b in r]

    def streams(self):
        """Compressed streams (views of the output buffers) after a compress launch."""
        return [out[:nb] for out, (nb, st) in zip(self.outputs, self.results())]

    def close(self) -> None:
        if self.workspace is not None:
            _load().falcon_batch_forget(self.workspace.data_ptr())
            self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pipeline_compress(x: torch.Tensor, block: int = 1024, frame_values: int = 1 << 23, nstreams: int = 16,
                      out: torch.Tensor | None = None, scheduler: int = 0):
    """Streams a HOST tensor (pin it for overlap) through the GPU in frames; returns
    (uint8 host tensor of the concatenated frame streams, list of frame lengths).
    scheduler: SCHED_EVENT_DRIVEN (the paper's), SCHED_SYNC_BASED or SCHED_PRE_ALLOCATION."""
    if x.is_cuda or not x.is_contiguous():
        raise ValueError("x must be a contiguous host tensor")
    code = _dtype_code(x)
    n = x.numel()
    nframes = (n + frame_values - 1) // frame_values
    if out is None:
        cap = nframes * bound(frame_values, code, block) if nframes else 32
        out = torch.empty(cap, dtype=torch.uint8, pin_memory=torch.cuda.is_available())
    fb = (ctypes.c_uint64 * max(nframes, 1))()
    total = ctypes.c_size_t()
    _check(_load().falcon_pipeline_compress_with(x.data_ptr(), n, code, block, frame_values, nstreams, scheduler,
                                                 out.data_ptr(), out.numel(), fb, ctypes.byref(total)),
           "pipeline_compress")
    return out[:total.value], [int(fb[i]) for i in range(nframes)]


def pipeline_decompress(s: torch.Tensor, frame_bytes, nstreams: int = 16, out: torch.Tensor | None = None,
                        dtype=None, n: int | None = None) -> torch.Tensor:
    """Inverse of pipeline_compress: host frames -> host values."""
    nframes = len(frame_bytes)
    fb = (ctypes.c_uint64 * max(nframes, 1))(*frame_bytes)
    if out is None:
        if n is None or dtype is None:
            tot, code = 0, F64
            off = 0
            for b in frame_bytes:
                nv, code, _, _ = stream_info(s[off:off + HEADER_BYTES].numpy().tobytes())
                tot += nv
                off += b
            n, dtype = tot, torch_dtype(code)
        out = torch.empty(max(n, 1), dtype=dtype, pin_memory=torch.cuda.is_available())
    n_out = ctypes.c_uint64()
    _check(_load().falcon_pipeline_decompress(s.data_ptr(), fb, nframes, nstreams, out.data_ptr(),
                                              out.numel() * out.element_size(), ctypes.byref(n_out)),
           "pipeline_decompress")
    return out[:n_out.value]
