"""Continuous-batching compression server on one GPU.

Requests (compress a host array, or decompress a host stream) are admitted in arrival order
while the device-memory budget allows, so new requests join while earlier ones are still on
the GPU.  The scheduler thread loops over four stages without blocking on any of them:

  1. admit   - reserve device memory for input, output and workspace, copy the input
               host -> device on the upload stream (pinned payloads overlap fully);
  2. launch  - every admitted request whose upload finished joins ONE batched launch per
               direction (falcon_batch_plan + falcon_batch_launch) on one of several compute
               streams, so batches overlap each other and the copies;
  3. size    - for compression, the per-series results (stream length, status) come back
               with a 16-byte-per-request copy (the paper's M-D2H);
  4. return  - the payload goes device -> host (P-D2H) into a pinned buffer; when that copy
               completes the request's future resolves and its memory budget is released.

Latency = time from submit() to the resolved future.  Every result is byte-identical to
the same request processed alone (the codec is deterministic and per-series).
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import threading
import time

import numpy as np
import torch

from . import falcon

COMPRESS, DECOMPRESS = "compress", "decompress"


class _Req:
    __slots__ = ("op", "payload", "block", "future", "t_submit", "t_done", "need", "d_in", "d_out", "nbytes",
                 "header", "ev", "host_out", "n", "dtype_code", "stage", "batch", "index")

    def __init__(self, op, payload, block):
        self.op = op
        self.payload = payload
        self.block = block
        self.future = cf.Future()
        self.t_submit = time.perf_counter()
        self.t_done = None
        self.stage = "queued"


class Server:
    """Continuous-batching server.

    Server(budget_bytes=64 << 30).submit("compress", host_tensor) -> Future[uint8 host tensor]
    Server.submit("decompress", host_uint8_tensor)                  -> Future[value host tensor]
    """

    def __init__(self, budget_bytes: int = 64 << 30, device="cuda", block: int = 1024,
                 compute_streams: int = 4, max_batch: int = 1024, idle_sleep: float = 20e-6):
        self.device = torch.device(device)
        self.budget = budget_bytes
        self.block = block
        self.max_batch = max_batch
        self.idle_sleep = idle_sleep
        self.in_use = 0
        self._pending = collections.deque()
        self._lock = threading.Lock()
        self._cv = threading.Condition(self._lock)
        self._running = True
        self.stats = {"batches": 0, "requests": 0, "max_batch": 0, "multi_request_batches": 0,
                      "max_in_flight": 0}
        with torch.cuda.device(self.device):
            self.up = torch.cuda.Stream(self.device)
            self.down = torch.cuda.Stream(self.device)
            self.plan_stream = torch.cuda.Stream(self.device)
            self.compute = [torch.cuda.Stream(self.device) for _ in range(compute_streams)]
        self._next_compute = 0
        self._thread = threading.Thread(target=self._loop, name="falcon-server", daemon=True)
        self._thread.start()

    # ------------------------------------------------------------------ public API
    def submit(self, op: str, payload: torch.Tensor, block: int | None = None) -> cf.Future:
        if op not in (COMPRESS, DECOMPRESS):
            raise ValueError(op)
        if payload.is_cuda:
            raise ValueError("payload must be a host tensor")
        r = _Req(op, payload.contiguous(), block or self.block)
        with self._cv:
            self._pending.append(r)
            self._cv.notify()
        return r.future

    def close(self) -> None:
        with self._cv:
            self._running = False
            self._cv.notify()
        self._thread.join()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------------ scheduler
    def _need(self, r: _Req) -> int:
        if r.op == COMPRESS:
            x = r.payload
            code = falcon._dtype_code(x)
            nc = (x.numel() + r.block - 1) // r.block
            return x.numel() * x.element_size() + falcon.bound(x.numel(), code, r.block) + falcon.workspace_bytes(nc) + 4096
        hdr = r.payload[:falcon.HEADER_BYTES].numpy().tobytes()
        n, code, blk, nc = falcon.stream_info(hdr)
        return r.payload.numel() + n * (8 if code == falcon.F64 else 4) + falcon.workspace_bytes(nc) + 4096

    def _fail(self, r: _Req, exc: Exception) -> None:
        self.in_use -= getattr(r, "need", 0) or 0
        r.t_done = time.perf_counter()
        if not r.future.done():
            r.future.set_exception(exc)

    def _admit(self, admitted: list) -> None:
        while True:
            with self._lock:
                if not self._pending:
                    return
                r = self._pending[0]
                try:
                    need = self._need(r)
                except Exception as exc:                     # malformed request: reject it
                    self._pending.popleft()
                    self._fail(r, exc)
                    continue
                if self.in_use + need > self.budget and self.in_use > 0:
                    return                                   # wait for memory to free up
                self._pending.popleft()
            r.need = need
            self.in_use += need
            with torch.cuda.stream(self.up):
                if r.op == COMPRESS:
                    r.d_in = r.payload.to(self.device, non_blocking=True)
                else:
                    r.header = r.payload[:falcon.HEADER_BYTES].numpy().tobytes()
                    r.n, r.dtype_code, _, _ = falcon.stream_info(r.header)
                    r.d_in = torch.empty(((r.payload.numel() + 15) // 16) * 16, dtype=torch.uint8, device=self.device)
                    r.d_in[:r.payload.numel()].copy_(r.payload, non_blocking=True)
                r.ev = torch.cuda.Event()
                r.ev.record(self.up)
            r.stage = "uploading"
            admitted.append(r)
            self.stats["max_in_flight"] = max(self.stats["max_in_flight"], len(admitted))

    def _launch_ready(self, admitted: list) -> None:
        ready = [r for r in admitted if r.stage == "uploading" and r.ev.query()]
        for op in (COMPRESS, DECOMPRESS):
            group = [r for r in ready if r.op == op][:self.max_batch]
            if not group:
                continue
            st = self.compute[self._next_compute % len(self.compute)]
            self._next_compute += 1
            try:
                with torch.cuda.stream(self.plan_stream):
                    if op == COMPRESS:
                        b = falcon.Batch(falcon.COMPRESS, [r.d_in for r in group], block=group[0].block
                                         if len({r.block for r in group}) == 1 else self.block, device=self.device)
                    else:
                        b = falcon.Batch(falcon.DECOMPRESS, [(r.d_in, r.payload.numel(), r.header) for r in group],
                                         device=self.device)
                st.wait_stream(self.up)
                b.launch(st)
            except Exception as exc:
                for r in group:
                    admitted.remove(r)
                    self._fail(r, exc)
                continue
            ev = torch.cuda.Event()
            ev.record(st)
            for i, r in enumerate(group):
                r.batch, r.index, r.stage, r.ev = b, i, "computing", ev
            self.stats["batches"] += 1
            self.stats["requests"] += len(group)
            self.stats["max_batch"] = max(self.stats["max_batch"], len(group))
            self.stats["multi_request_batches"] += len(group) > 1

    def _collect(self, admitted: list) -> None:
        for r in list(admitted):
            if r.stage == "computing" and r.ev.query():
                b = r.batch
                if not hasattr(b, "_res"):
                    with torch.cuda.stream(self.plan_stream):
                        b._res = b.results()                 # 16 bytes per request (M-D2H)
                nb, status = b._res[r.index]
                if status != 0:
                    admitted.remove(r)
                    self._fail(r, falcon.FalconError(status, r.op))
                    continue
                out = b.outputs[r.index]
                with torch.cuda.stream(self.down):
                    self.down.wait_event(r.ev)
                    if r.op == COMPRESS:
                        r.host_out = torch.empty(nb, dtype=torch.uint8, pin_memory=True)
                        r.host_out.copy_(out[:nb], non_blocking=True)
                    else:
                        r.host_out = torch.empty(nb, dtype=out.dtype, pin_memory=True)
                        r.host_out.copy_(out[:nb], non_blocking=True)
                    r.ev = torch.cuda.Event()
                    r.ev.record(self.down)
                r.stage = "returning"
            elif r.stage == "returning" and r.ev.query():
                admitted.remove(r)
                self.in_use -= r.need
                r.t_done = time.perf_counter()
                r.d_in = None
                r.batch = None
                r.future.latency = r.t_done - r.t_submit
                r.future.set_result(r.host_out)

    def _loop(self) -> None:
        admitted: list = []
        with torch.cuda.device(self.device):
            while True:
                with self._cv:
                    if not self._running and not self._pending and not admitted:
                        break
                    if not self._pending and not admitted:
                        self._cv.wait(timeout=0.05)
                        continue
                try:
                    self._admit(admitted)
                    self._launch_ready(admitted)
                    self._collect(admitted)
                except Exception as exc:                     # keep serving; fail what is in flight
                    for r in list(admitted):
                        admitted.remove(r)
                        self._fail(r, exc)
                if admitted:
                    time.sleep(self.idle_sleep)


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


def _bytes_of(op, payload, out):
    return payload.numel() * payload.element_size() if op == COMPRESS else out.numel() * out.element_size()


def run_load(server: Server, pool, rate: float, duration: float, seed: int = 0) -> dict:
    """Poisson arrivals at `rate` requests/s for `duration` seconds; each request is drawn
    uniformly from `pool` (list of (op, host tensor)).  Throughput counts original
    (uncompressed) bytes; latency runs from arrival to the resolved future."""
    arr = _arrivals(rate, duration, len(pool), seed)
    futs = []
    t0 = time.perf_counter()
    for t, i in arr:
        now = time.perf_counter() - t0
        if t > now:
            time.sleep(t - now)
        op, payload = pool[i]
        futs.append((server.submit(op, payload), op, payload))
    nbytes, lat = 0, []
    for f, op, payload in futs:
        out = f.result()
        lat.append(f.latency)
        nbytes += _bytes_of(op, payload, out)
    wall = time.perf_counter() - t0
    res = _summary(lat, nbytes, wall, len(futs))
    res.update({k: server.stats[k] for k in ("batches", "max_batch", "multi_request_batches", "max_in_flight")})
    return res


def run_one_at_a_time(pool, rate: float, duration: float, seed: int = 0, device="cuda", block: int = 1024) -> dict:
    """The same arrivals served strictly one request at a time (upload, one kernel launch,
    download, next): the queue-only baseline."""
    dev = torch.device(device)
    arr = _arrivals(rate, duration, len(pool), seed)
    stream = torch.cuda.Stream(dev)
    t0 = time.perf_counter()
    lat, nbytes = [], 0
    with torch.cuda.stream(stream):
        for t, i in arr:
            now = time.perf_counter() - t0
            if t > now:
                time.sleep(t - now)
            op, payload = pool[i]
            if op == COMPRESS:
                d = payload.to(dev, non_blocking=True)
                s = falcon.compress(d, block, stream=stream)
                out = torch.empty(s.numel(), dtype=torch.uint8, pin_memory=True)
                out.copy_(s)
            else:
                d = torch.empty(((payload.numel() + 15) // 16) * 16, dtype=torch.uint8, device=dev)
                d[:payload.numel()].copy_(payload, non_blocking=True)
                y = falcon.decompress(d[:payload.numel()], stream=stream)
                out = torch.empty(y.numel(), dtype=y.dtype, pin_memory=True)
                out.copy_(y)
            lat.append(time.perf_counter() - t0 - t)
            nbytes += _bytes_of(op, payload, out)
    wall = time.perf_counter() - t0
    return _summary(lat, nbytes, wall, len(arr))


def make_pool(count: int = 64, seed: int = 5, min_bytes: int = 4 << 10, max_bytes: int = 256 << 20,
              device="cuda", block: int = 1024):
    """Request pool: sizes log-uniform in [min_bytes, max_bytes], FP64/FP32 50/50, random-walk
    data (2 places); half compress requests (values) and half decompress requests (streams
    produced by the library).  Payloads live in pinned host memory."""
    from . import synth
    rng = np.random.default_rng(seed)
    pool = []
    for i in range(count):
        nbytes = int(np.exp(rng.uniform(np.log(min_bytes), np.log(max_bytes))))
        dtype = np.float64 if rng.random() < 0.5 else np.float32
        n = max(1, nbytes // np.dtype(dtype).itemsize)
        vals = synth.random_walk(n, seed=int(rng.integers(1 << 30)), places=2, dtype=dtype)
        host = torch.from_numpy(vals).pin_memory()
        if i % 2 == 0:
            pool.append((COMPRESS, host))
        else:
            s = falcon.compress(host.to(device), block)
            pool.append((DECOMPRESS, s.cpu().pin_memory()))
    return pool
