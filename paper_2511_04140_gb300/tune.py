"""Autotuner for the batched launch.

Tunes what the caller may change without changing the method:
  * block size B (a format parameter recorded in every stream header; it changes the bytes
    and the ratio, never losslessness),
  * the persistent grids' resident CTAs per SM for compression and decompression (launch
    shape only; output bytes are unchanged).
The plane-packing width is fixed by the kernel design (one 32-bit word per lane and bit
plane, i.e. four row bytes), so it is not a search dimension.

Each candidate is timed on a sample of the batch with CUDA events (compress + decompress,
inputs resident); the fastest candidate whose compression ratio is within `ratio_slack` of
the best ratio wins.
"""
from __future__ import annotations

import itertools

import torch

from . import falcon


def _time_ms(fn, reps: int) -> float:
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def measure(sample, block: int, c_ctas: int, d_ctas: int, reps: int = 3) -> dict:
    """Throughput and ratio of one candidate on `sample` (list of CUDA tensors)."""
    falcon.set_launch_config(c_ctas, d_ctas)
    try:
        comp = falcon.Batch(falcon.COMPRESS, sample, block=block)
        tc = _time_ms(comp.launch, reps)
        res = comp.results()
        if any(st != 0 for _, st in res):
            raise falcon.FalconError(max(st for _, st in res), "tune compress")
        streams = comp.streams()
        dec_in = [(s, s.numel(), s[:32].cpu().numpy().tobytes()) for s in streams]
        dec = falcon.Batch(falcon.DECOMPRESS, dec_in)
        td = _time_ms(dec.launch, reps)
        orig = sum(x.numel() * x.element_size() for x in sample)
        comp_bytes = sum(nb for nb, _ in res)
        comp.close()
        dec.close()
    finally:
        falcon.set_launch_config(0, 0)
    return {"block": block, "compress_ctas_per_sm": c_ctas, "decompress_ctas_per_sm": d_ctas,
            "compress_ms": tc, "decompress_ms": td, "gbs": 2 * orig / ((tc + td) * 1e6),
            "ratio": comp_bytes / orig}


def autotune(sample, blocks=(512, 1024, 1025), compress_ctas=(0, 3), decompress_ctas=(0, 2),
             reps: int = 3, ratio_slack: float = 0.02) -> dict:
    """Returns the chosen configuration and the table of all candidates."""
    table = [measure(sample, b, c, d, reps) for b, c, d in itertools.product(blocks, compress_ctas, decompress_ctas)]
    best_ratio = min(r["ratio"] for r in table)
    ok = [r for r in table if r["ratio"] <= best_ratio * (1 + ratio_slack)]
    best = max(ok, key=lambda r: r["gbs"])
    return {"choice": best, "table": table}


def apply(choice: dict) -> int:
    """Sets the chosen launch shape and returns the chosen block size."""
    falcon.set_launch_config(choice["compress_ctas_per_sm"], choice["decompress_ctas_per_sm"])
    return choice["block"]
