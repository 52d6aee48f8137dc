"""Continuous-batching compression server on one GPU (Python face of falcon_server_*).

The scheduler is native (the library's worker thread, see include/falcon.h):
  - admission in arrival order against a device-memory budget: every request in flight
    holds one block of a device arena of that size (input, output, workspace words), and
    its output one block of a page-locked host arena;
  - each pass of the worker turns everything admitted into ONE batched persistent launch per
    direction, with the uploads, the launch, the per-request result read-back (the paper's
    M-D2H) and, for decompression, the output copy (P-D2H) chained by device-side events;
    compression outputs are copied once their lengths are back.  Requests that arrive while
    a batch runs join the next one.
This module adds futures: a poller thread drains completions (the ctypes call releases the
GIL while it waits) and resolves each request's Future with a zero-copy tensor over the
host arena, whose space returns to the arena when the tensor is garbage collected.

Latency = time from submit() to completion, measured by the library.  Every result is
byte-identical to the same request processed alone (the codec is deterministic and
per-series).
"""
from __future__ import annotations

import concurrent.futures as cf
import ctypes
import threading
import time
import weakref

import numpy as np
import torch

from . import falcon

COMPRESS, DECOMPRESS = "compress", "decompress"
_OPS = {COMPRESS: falcon.COMPRESS, DECOMPRESS: falcon.DECOMPRESS}


class Server:
    """Server(budget_bytes=64 << 30).submit("compress", host_values)    -> Future[uint8 tensor]
    Server.submit("decompress", host_uint8_stream)                       -> Future[value tensor]

    Results are views of the server's page-locked output arena, valid until close(); clone()
    what must outlive the server.  Inputs must stay unchanged until their future resolves
    (the server keeps a reference).  Futures carry `.latency` (seconds)."""

    def __init__(self, budget_bytes: int = 64 << 30, host_budget_bytes: int = 16 << 30, device="cuda",
                 block: int = 1024, compute_streams: int = 16, max_batch: int = 1024,
                 max_batch_bytes: int = 64 << 20):
        self.device = torch.device(device)
        index = self.device.index if self.device.index is not None else torch.cuda.current_device()
        self.block = block
        self._L = falcon.lib()
        h = ctypes.c_void_p()
        falcon._check(self._L.falcon_server_create(index, budget_bytes, host_budget_bytes, compute_streams,
                                                   max_batch, max_batch_bytes, ctypes.byref(h)), "server_create")
        self._h = h.value
        self._lock = threading.Lock()
        self._futs: dict = {}
        self._tag = 0
        self._open = True
        self._closing = False
        self._poller = threading.Thread(target=self._poll_loop, name="falcon-server-poll", daemon=True)
        self._poller.start()

    # ------------------------------------------------------------------ public API
    def submit(self, op: str, payload: torch.Tensor, block: int | None = None) -> cf.Future:
        if op not in _OPS:
            raise ValueError(op)
        if payload.is_cuda:
            raise ValueError("payload must be a host tensor")
        payload = payload.contiguous()
        if op == COMPRESS:
            code, count = falcon._dtype_code(payload), payload.numel()
        else:
            if payload.dtype != torch.uint8:
                raise TypeError("a stream is a uint8 tensor")
            code, count = 0, payload.numel()
        f = cf.Future()
        with self._lock:
            if self._closing:
                raise RuntimeError("server is closed")
            tag = self._tag
            self._tag += 1
            self._futs[tag] = (f, payload)
        st = self._L.falcon_server_submit(self._h, _OPS[op], payload.data_ptr(), count, code, block or self.block, tag)
        if st != falcon.OK:
            with self._lock:
                self._futs.pop(tag, None)
            f.set_exception(falcon.FalconError(st, f"server {op}"))
        return f

    @property
    def stats(self) -> dict:
        s = falcon.ServerStats()
        falcon._check(self._L.falcon_server_get_stats(self._h, ctypes.byref(s)), "server_get_stats")
        d = {k: getattr(s, k) for k, _ in falcon.ServerStats._fields_}
        d["requests"] = d["submitted"]
        return d

    @property
    def in_use(self) -> int:
        return self.stats["device_in_use"]

    def close(self) -> None:
        with self._lock:
            if self._closing:
                return
            self._closing = True
        self._poller.join()
        with self._lock:
            self._open = False
        falcon._check(self._L.falcon_server_destroy(self._h), "server_destroy")

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------------ completions
    def _free(self, ptr: int) -> None:
        with self._lock:
            if self._open:
                self._L.falcon_server_free_output(self._h, ptr)

    def _wrap(self, c, payload) -> torch.Tensor:
        nbytes = int(c.out_bytes)
        if c.op == falcon.COMPRESS:
            dtype = torch.uint8
        else:
            dtype = falcon.torch_dtype(int(payload[5]))
        raw = (ctypes.c_uint8 * nbytes).from_address(c.h_out) if nbytes else bytearray(0)
        arr = np.frombuffer(raw, dtype=np.uint8)
        weakref.finalize(arr, self._free, c.h_out)        # arena space back when unreferenced
        t = torch.from_numpy(arr)
        return t if dtype == torch.uint8 else t.view(dtype)

    def _poll_loop(self) -> None:
        buf = (falcon.Completion * 256)()
        cnt = ctypes.c_int()
        while True:
            falcon._check(self._L.falcon_server_poll(self._h, buf, 256, 20000, ctypes.byref(cnt)), "server_poll")
            for i in range(cnt.value):
                c = buf[i]
                with self._lock:
                    f, payload = self._futs.pop(c.tag)
                f.latency = c.latency_s
                if c.status != falcon.OK:
                    f.set_exception(falcon.FalconError(c.status, "server request"))
                else:
                    f.set_result(self._wrap(c, payload))
                del f, payload                 # hold no output here: its space must return
            with self._lock:
                if self._closing and not self._futs:
                    return


def _bytes_of(op, payload, out):
    return payload.numel() * payload.element_size() if op == COMPRESS else out.numel() * out.element_size()


def run_load(server: Server, pool, rate: float, duration: float, seed: int = 0) -> dict:
    """Poisson arrivals at `rate` requests/s for `duration` seconds; each request is drawn
    uniformly from `pool` (list of (op, host tensor)).  Throughput counts original
    (uncompressed) bytes; latency runs from the scheduled arrival to the moment the client
    sees the result (as in run_one_at_a_time)."""
    arr = _arrivals(rate, duration, len(pool), seed)
    lock = threading.Lock()
    acc = {"bytes": 0, "done": 0, "failed": 0}
    lat: list = []
    all_done = threading.Event()

    def record(f, op, payload, t_arrival):
        # the client keeps only latency and byte counts; the output returns to the arena
        t_seen = time.perf_counter() - t0
        with lock:
            if f.exception() is None:
                lat.append(t_seen - t_arrival)
                acc["bytes"] += _bytes_of(op, payload, f.result())
            else:
                acc["failed"] += 1
            acc["done"] += 1
            if acc["done"] == len(arr):
                all_done.set()

    before = server.stats
    t0 = time.perf_counter()
    for t, i in arr:
        now = time.perf_counter() - t0
        if t > now:
            time.sleep(t - now)
        op, payload = pool[i]
        server.submit(op, payload).add_done_callback(lambda f, op=op, p=payload, t=t: record(f, op, p, t))
    if arr:
        all_done.wait()
    wall = time.perf_counter() - t0
    after = server.stats
    res = _summary(lat, acc["bytes"], wall, len(arr))
    res["failed"] = acc["failed"]
    res["batches"] = after["batches"] - before["batches"]
    res["multi_request_batches"] = after["multi_request_batches"] - before["multi_request_batches"]
    res["mean_batch"] = len(arr) / max(1, res["batches"])
    res.update({k: after[k] for k in ("max_batch", "max_in_flight", "device_peak")})
    return res


def _arrivals(rate: float, duration: float, npool: int, seed: int):
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            return out
        out.append((t, int(rng.integers(npool))))


def _summary(lat, nbytes, wall, n):
    lat = sorted(lat)
    q = lambda f: lat[min(len(lat) - 1, int(f * len(lat)))] * 1e3 if lat else None
    return {"requests": n, "p50_ms": q(0.5), "p99_ms": q(0.99), "gbs": nbytes / wall / 1e9, "wall_s": wall}


def run_one_at_a_time(pool, rate: float, duration: float, seed: int = 0, device="cuda", block: int = 1024) -> dict:
    """The same arrivals served strictly one request at a time (upload, one compress or
    decompress call, download, next): the queue-only baseline.  Its device and page-locked
    host buffers are allocated once, for the largest request, and reused, as the server's
    arenas are."""
    dev = torch.device(device)
    arr = _arrivals(rate, duration, len(pool), seed)
    stream = torch.cuda.Stream(dev)
    in_max = max(p.numel() * p.element_size() for _, p in pool)
    out_max = 0
    for op, p in pool:
        if op == COMPRESS:
            out_max = max(out_max, falcon.bound(p.numel(), falcon._dtype_code(p), block))
        else:
            n, code, _, _ = falcon.stream_info(p[:falcon.HEADER_BYTES].numpy().tobytes())
            out_max = max(out_max, n * torch.empty(0, dtype=falcon.torch_dtype(code)).element_size())
    d_in = torch.empty((in_max + 15) // 16 * 16, dtype=torch.uint8, device=dev)
    d_out = torch.empty(max(out_max, 32) // 8 * 8 + 8, dtype=torch.uint8, device=dev)
    h_out = torch.empty(max(out_max, 32), dtype=torch.uint8, pin_memory=True)
    t0 = time.perf_counter()
    lat, nbytes = [], 0
    with torch.cuda.stream(stream):
        for t, i in arr:
            now = time.perf_counter() - t0
            if t > now:
                time.sleep(t - now)
            op, payload = pool[i]
            nb = payload.numel() * payload.element_size()
            d_in[:nb].copy_(payload.view(torch.uint8), non_blocking=True)
            if op == COMPRESS:
                x = d_in[:nb].view(payload.dtype)
                s = falcon.compress(x, block, out=d_out, stream=stream)
                out = h_out[:s.numel()]
                out.copy_(s)
            else:
                y = falcon.decompress(d_in[:nb], out=d_out.view(falcon.torch_dtype(int(payload[5]))), stream=stream)
                out = h_out[:y.numel() * y.element_size()]
                out.copy_(y.view(torch.uint8))
            lat.append(time.perf_counter() - t0 - t)
            nbytes += nb if op == COMPRESS else out.numel()
    wall = time.perf_counter() - t0
    return _summary(lat, nbytes, wall, len(arr))


def make_pool(count: int = 256, seed: int = 5, min_bytes: int = 4 << 10, max_bytes: int = 256 << 20,
              device="cuda", block: int = 1024):
    """Request pool: sizes log-uniform in [min_bytes, max_bytes], FP64/FP32 50/50, random-walk
    data (2 places, generated on the GPU); half compress requests (values) and half
    decompress requests (streams produced by the library).  Payloads live in pinned host
    memory."""
    from . import synth
    rng = np.random.default_rng(seed)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    pool = []
    for i in range(count):
        nbytes = int(np.exp(rng.uniform(np.log(min_bytes), np.log(max_bytes))))
        dtype = np.float64 if rng.random() < 0.5 else np.float32
        n = max(1, nbytes // np.dtype(dtype).itemsize)
        vals = synth.random_walk_cuda(n, g, places=2, dtype=dtype, device=device)
        if i % 2 == 0:
            pool.append((COMPRESS, vals.cpu().pin_memory()))
        else:
            pool.append((DECOMPRESS, falcon.compress(vals, block).cpu().pin_memory()))
        del vals
    return pool
