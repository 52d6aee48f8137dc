"""Autotuner for the batched launch.

Tunes what the caller may change without changing the method:
  * block size B (a format parameter recorded in every stream header; it changes the bytes
    and the ratio, never losslessness),
  * the persistent grids' threads per CTA (warps per CTA) and resident CTAs per SM, for
    compression and decompression (launch shape only; output bytes are unchanged).
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


def measure(sample, block: int, c_ctas: int, d_ctas: int, reps: int = 3, c_warps: int = 4,
            d_warps: int = 4) -> dict:
    """Throughput and ratio of one candidate on `sample` (list of CUDA tensors)."""
    falcon.set_launch_config(c_ctas, d_ctas)
    falcon.set_cta_warps(c_warps, d_warps)
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
        falcon.set_cta_warps(4, 4)
    return {"block": block, "compress_ctas_per_sm": c_ctas, "decompress_ctas_per_sm": d_ctas,
            "compress_warps_per_cta": c_warps, "decompress_warps_per_cta": d_warps,
            "compress_ms": tc, "decompress_ms": td, "gbs": 2 * orig / ((tc + td) * 1e6),
            "ratio": comp_bytes / orig}


def autotune(sample, blocks=(512, 1024, 1025), compress_ctas=(0, 3), decompress_ctas=(0, 2),
             compress_warps=(2, 4, 8), decompress_warps=(2, 4, 8), reps: int = 3,
             ratio_slack: float = 0.02) -> dict:
    """Returns the chosen configuration and the table of all candidates: every block size and
    CTA shape (warps per CTA) at the occupancy limit, then the resident-CTA caps at the best
    block size and shape."""
    table = [measure(sample, b, 0, 0, reps, cw, dw)
             for b, cw, dw in itertools.product(blocks, compress_warps, decompress_warps)]
    best_ratio = min(r["ratio"] for r in table)
    ok = [r for r in table if r["ratio"] <= best_ratio * (1 + ratio_slack)]
    first = max(ok, key=lambda r: r["gbs"])
    table += [measure(sample, first["block"], c, d, reps, first["compress_warps_per_cta"],
                      first["decompress_warps_per_cta"])
              for c, d in itertools.product(compress_ctas, decompress_ctas) if (c, d) != (0, 0)]
    ok = [r for r in table if r["ratio"] <= best_ratio * (1 + ratio_slack)]
    best = max(ok, key=lambda r: r["gbs"])
    return {"choice": best, "table": table}


def apply(choice: dict) -> int:
    """Sets the chosen launch shape and returns the chosen block size."""
    falcon.set_launch_config(choice["compress_ctas_per_sm"], choice["decompress_ctas_per_sm"])
    falcon.set_cta_warps(choice.get("compress_warps_per_cta", 4), choice.get("decompress_warps_per_cta", 4))
    return choice["block"]
