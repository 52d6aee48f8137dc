"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no codec arithmetic: it only produces decimal numbers and
converts them to binary floating point, correctly rounded, so that the CUDA
path and the CPU oracle can be fed the same bytes.  The paper's datasets
(Table 1, Sec. 5.1) are not available; these generators stand in for them and
cover the decimal-significand range the paper reports (3 to 17 digits).

Workloads (sizes as quoted for the method's throughput targets):
  * ``random_walk``      x_{i+1} = x_i + N(0, 0.5) from 20.0, rounded to
                         ``places`` decimals and stored as the nearest binary
                         value (1,048,576 FP64 values, 2 places, seed 0).
  * ``segments``         4096-value segments, each with its own decimal place
                         count drawn from 0..6, a sinusoid of amplitude 10^U(0,4)
                         plus AR(1) noise (phi = 0.95, innovation sd = 1% of the
                         amplitude), rounded to the segment's places; 1% of the
                         values replaced by outliers x * 10^U(3,8) kept at full
                         precision, 0.01% by special values (NaN with payloads,
                         +-inf, subnormals, -0.0).  67,108,864 values, FP64 or FP32.
  * ``series_batch``     independent series of log-uniform lengths, mixed dtype,
                         per-series places and outlier rate.
  * ``adversarial``      hand-picked edge values (specials, powers of ten and
                         their neighbours, 2^53 +- 1, 17-digit values ...).
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

__all__ = ["decimal_to_f64", "decimal_to_f32", "random_walk", "random_walk_cuda", "segments", "series_batch",
           "adversarial_f64", "adversarial_f32", "specials_f64", "specials_f32"]

_P10 = np.array([10.0 ** k for k in range(23)], dtype=np.float64)   # exact for k <= 22


def decimal_to_f64(k: np.ndarray, places: np.ndarray | int) -> np.ndarray:
    """Nearest FP64 to the decimal k * 10^-places (|k| < 2^53, places <= 22).

    Both operands of the division are exact binary values, so the IEEE
    division rounds the exact quotient once.
    """
    k = np.asarray(k, dtype=np.int64)
    places = np.broadcast_to(np.asarray(places, dtype=np.int64), k.shape)
    return k.astype(np.float64) / _P10[places]


def decimal_to_f32(k: np.ndarray, places: np.ndarray | int) -> np.ndarray:
    """Nearest FP32 to k * 10^-places, avoiding double rounding.

    The quotient is first rounded to FP64; that can only mislead the second
    rounding when it lands exactly on an FP32 midpoint, and those rare values
    are resolved against the exact rational.
    """
    k = np.asarray(k, dtype=np.int64)
    places = np.broadcast_to(np.asarray(places, dtype=np.int64), k.shape)
    d = decimal_to_f64(k, places)
    f = d.astype(np.float32)
    bits = d.view(np.uint64)
    exp = (bits >> np.uint64(52)) & np.uint64(0x7FF)
    low = bits & np.uint64((1 << 29) - 1)
    normal32 = (exp >= np.uint64(1023 - 126)) & (exp <= np.uint64(1023 + 127))
    tie = normal32 & (low == np.uint64(1 << 28))
    for i in np.flatnonzero(tie):
        exact = Fraction(int(k[i]), 10 ** int(places[i]))
        mid = Fraction(float(d[i]))
        lo = np.float32(d[i])
        if exact == mid:
            continue                              # exact tie: the cast already rounds to even
        # the two FP32 neighbours of the midpoint
        below = np.nextafter(np.float32(d[i]), np.float32(-np.inf)) if Fraction(float(lo)) > mid else lo
        above = np.nextafter(below, np.float32(np.inf))
        f[i] = above if exact > mid else below
    return f


def _specials(rng: np.random.Generator, count: int, dtype) -> np.ndarray:
    """Uniform over {qNaN payload, sNaN payload, +inf, -inf, subnormal, -0.0}."""
    kind = rng.integers(0, 6, size=count)
    if dtype == np.float64:
        ut = np.uint64
        payload = rng.integers(1, 1 << 51, size=count, dtype=np.uint64)
        sign = rng.integers(0, 2, size=count, dtype=np.uint64) << ut(63)
        qnan = ut(0x7FF8000000000000) | payload | sign
        snan = ut(0x7FF0000000000000) | payload | sign
        pinf = np.full(count, 0x7FF0000000000000, dtype=np.uint64)
        ninf = np.full(count, 0xFFF0000000000000, dtype=np.uint64)
        sub = rng.integers(1, 1 << 52, size=count, dtype=np.uint64) | sign
        nzero = np.full(count, 0x8000000000000000, dtype=np.uint64)
        out = np.choose(kind, [qnan, snan, pinf, ninf, sub, nzero])
        return out.astype(np.uint64).view(np.float64)
    ut = np.uint32
    payload = rng.integers(1, 1 << 22, size=count, dtype=np.uint32)
    sign = rng.integers(0, 2, size=count, dtype=np.uint32) << ut(31)
    qnan = ut(0x7FC00000) | payload | sign
    snan = ut(0x7F800000) | payload | sign
    pinf = np.full(count, 0x7F800000, dtype=np.uint32)
    ninf = np.full(count, 0xFF800000, dtype=np.uint32)
    sub = rng.integers(1, 1 << 23, size=count, dtype=np.uint32) | sign
    nzero = np.full(count, 0x80000000, dtype=np.uint32)
    out = np.choose(kind, [qnan, snan, pinf, ninf, sub, nzero])
    return out.astype(np.uint32).view(np.float32)


def specials_f64(count: int, seed: int = 0) -> np.ndarray:
    return _specials(np.random.default_rng(seed), count, np.float64)


def specials_f32(count: int, seed: int = 0) -> np.ndarray:
    return _specials(np.random.default_rng(seed), count, np.float32)


def random_walk(n: int, seed: int = 0, places: int = 2, start: float = 20.0, sigma: float = 0.5,
                dtype=np.float64, outlier_rate: float = 0.0) -> np.ndarray:
    """Random walk rounded to ``places`` decimals (the 1,048,576-value FP64 workload).

    With ``outlier_rate`` > 0 a fraction of the values is replaced by
    full-precision outliers x * 10^U(3,8), as in the segment workload.
    """
    rng = np.random.default_rng(seed)
    x = start + np.concatenate([[0.0], np.cumsum(rng.normal(0.0, sigma, size=max(n - 1, 0)))])
    x = x[:n]
    k = np.rint(x * 10.0 ** places).astype(np.int64)
    vals = decimal_to_f64(k, places) if dtype == np.float64 else decimal_to_f32(k, places)
    if outlier_rate > 0 and n > 0:
        cnt = rng.binomial(n, outlier_rate)
        pos = rng.choice(n, size=cnt, replace=False)
        mag = x[pos] * 10.0 ** rng.uniform(3, 8, size=cnt)
        vals[pos] = mag.astype(dtype)
    return vals


def segments(n: int = 1 << 26, seed: int = 1, dtype=np.float64, seg_len: int = 4096,
             outlier_rate: float = 0.01, special_rate: float = 1e-4) -> np.ndarray:
    """The 4096-value-segment sinusoid + AR(1) workload (see module doc)."""
    from scipy.signal import lfilter

    rng = np.random.default_rng(seed)
    nseg = (n + seg_len - 1) // seg_len
    places = rng.integers(0, 7, size=nseg)
    amp = 10.0 ** rng.uniform(0, 4, size=nseg)
    period = rng.uniform(64, 4096, size=nseg)
    phase = rng.uniform(0, 2 * np.pi, size=nseg)
    seg = np.arange(n) // seg_len
    t = (np.arange(n) % seg_len).astype(np.float64)
    innov = rng.standard_normal(n)
    ar = lfilter([1.0], [1.0, -0.95], innov)
    x = amp[seg] * np.sin(2 * np.pi * t / period[seg] + phase[seg]) + 0.01 * amp[seg] * ar
    pl = places[seg]
    k = np.rint(x * (10.0 ** pl)).astype(np.int64)
    vals = decimal_to_f64(k, pl) if dtype == np.float64 else decimal_to_f32(k, pl)
    n_out = rng.binomial(n, outlier_rate)
    pos = rng.choice(n, size=n_out, replace=False)
    vals[pos] = (x[pos] * 10.0 ** rng.uniform(3, 8, size=n_out)).astype(dtype)
    n_sp = rng.binomial(n, special_rate)
    pos = rng.choice(n, size=n_sp, replace=False)
    vals[pos] = _specials(rng, n_sp, dtype)
    return vals


def segments_f16(n: int = 1 << 26, seed: int = 1, seg_len: int = 4096, outlier_rate: float = 1e-4,
                 special_rate: float = 1e-5) -> np.ndarray:
    """Binary16 segments: the sinusoid + AR(1) construction with amplitude 10^U(-1, 1) and
    U{0..2} places, rounded to binary16 (1 to 4 significant digits, so chunks of both Cases);
    a few full-precision outliers and special values."""
    from scipy.signal import lfilter

    rng = np.random.default_rng(seed)
    nseg = (n + seg_len - 1) // seg_len
    places = rng.integers(0, 3, size=nseg)
    amp = 10.0 ** rng.uniform(-1, 1, size=nseg)
    period = rng.uniform(64, 4096, size=nseg)
    phase = rng.uniform(0, 2 * np.pi, size=nseg)
    seg = np.arange(n) // seg_len
    t = (np.arange(n) % seg_len).astype(np.float64)
    ar = lfilter([1.0], [1.0, -0.95], rng.standard_normal(n))
    x = amp[seg] * np.sin(2 * np.pi * t / period[seg] + phase[seg]) + 0.01 * amp[seg] * ar
    pl = places[seg]
    vals = (np.rint(x * 10.0 ** pl) / 10.0 ** pl).astype(np.float16)
    n_out = rng.binomial(n, outlier_rate)
    pos = rng.choice(n, size=n_out, replace=False)
    vals[pos] = (x[pos] * np.pi).astype(np.float16)
    n_sp = rng.binomial(n, special_rate)
    pos = rng.choice(n, size=n_sp, replace=False)
    vals[pos] = np.array([np.nan, np.inf, -np.inf, -0.0, 6e-8], dtype=np.float16)[rng.integers(0, 5, n_sp)]
    return vals


def series_batch(count: int = 4096, seed: int = 2, min_len: int = 1024, max_len: int = 1 << 22,
                 p_f64: float = 0.7, max_outlier_rate: float = 0.05):
    """Independent series: length floor(2^U(log2 min, log2 max)), FP64 with probability
    ``p_f64`` else FP32, places U{0..6}, outlier rate U(0, max_outlier_rate).
    Returns a list of numpy arrays."""
    rng = np.random.default_rng(seed)
    lengths = np.floor(2.0 ** rng.uniform(np.log2(min_len), np.log2(max_len), size=count))
    lengths = lengths.astype(np.int64)
    is64 = rng.random(count) < p_f64
    places = rng.integers(0, 7, size=count)
    rates = rng.uniform(0, max_outlier_rate, size=count)
    seeds = rng.integers(0, 2 ** 31, size=count)
    out = []
    for i in range(count):
        out.append(random_walk(int(lengths[i]), seed=int(seeds[i]), places=int(places[i]),
                               dtype=np.float64 if is64[i] else np.float32,
                               outlier_rate=float(rates[i])))
    return out


def adversarial_f64() -> np.ndarray:
    """Edge values for the FP64 path (specials, boundaries of the decimal ranges)."""
    v = [0.0, -0.0, 1.0, -1.0, 0.1, 0.5, 2.5, 1.11, 8.04, -0.0314, 111.0, 111.00000000000001,
         9.110900773177071, 1.23456789876543e-9, 7.15, 7150.0, 123456789012345.0,
         1234567890123456.0, 0.000001, 1e-22, 1e-23, 1e15, 1e15 - 1, 1e16,
         2.0 ** 53, 2.0 ** 53 + 2, 2.0 ** 53 - 1, 2.0 ** -1022, 2.0 ** -1074, 5e-324,
         np.finfo(np.float64).max, -np.finfo(np.float64).max, np.inf, -np.inf, np.nan,
         0.1 + 0.2, 1 / 3, 3.141592653589793, 2.718281828459045]
    for k in range(-25, 17):
        p = float(Fraction(10) ** k)
        v += [p, np.nextafter(p, np.inf), np.nextafter(p, -np.inf), -p]
    arr = np.array(v, dtype=np.float64)
    bits = np.array([0x7FF8000000000001, 0xFFF8000000000123, 0x7FF0000000000001,
                     0xFFF4000000000000, 0x0000000000000001, 0x800FFFFFFFFFFFFF],
                    dtype=np.uint64).view(np.float64)
    return np.concatenate([arr, bits])


def adversarial_f32() -> np.ndarray:
    v = [0.0, -0.0, 1.0, -1.0, 0.1, 0.5, 2.5, 1.11, 8.04, -0.0314, 111.0, 7.15, 9999999.0,
         1234567.0, 12345678.0, 0.000001, 1e-10, 1e-11, 1e7, 2.0 ** 24, 2.0 ** 24 + 2,
         2.0 ** -126, 2.0 ** -149, np.finfo(np.float32).max, np.inf, -np.inf, np.nan,
         3.1415927, 2.7182817]
    for k in range(-13, 9):
        p = np.float32(float(Fraction(10) ** k))
        v += [p, np.nextafter(p, np.float32(np.inf)), np.nextafter(p, np.float32(-np.inf)), -p]
    arr = np.array(v, dtype=np.float32)
    bits = np.array([0x7FC00001, 0xFFC00123, 0x7F800001, 0xFFA00000, 0x00000001, 0x807FFFFF],
                    dtype=np.uint32).view(np.float32)
    return np.concatenate([arr, bits])


def series_batch_cuda(count: int = 4096, seed: int = 2, min_len: int = 1024, max_len: int = 1 << 22,
                      p_f64: float = 0.7, max_outlier_rate: float = 0.05, device="cuda"):
    """The independent-series workload generated on the GPU (same distributions as
    ``series_batch``; different random stream).  Returns a list of CUDA tensors.

    Each series: random walk x_{i+1} = x_i + N(0, 0.5) from 20.0, rounded to a per-series
    number of places U{0..6} (the nearest binary value of the decimal, FP32 ties resolved
    exactly), a per-series fraction U(0, max_outlier_rate) replaced by full-precision
    outliers x * 10^U(3,8); FP64 with probability p_f64, else FP32."""
    import torch
    rng = np.random.default_rng(seed)
    lengths = np.floor(2.0 ** rng.uniform(np.log2(min_len), np.log2(max_len), size=count)).astype(np.int64)
    is64 = rng.random(count) < p_f64
    places = rng.integers(0, 7, size=count)
    rates = rng.uniform(0, max_outlier_rate, size=count)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return [random_walk_cuda(int(lengths[i]), g, places=int(places[i]),
                             dtype=np.float64 if is64[i] else np.float32, outlier_rate=float(rates[i]),
                             device=device) for i in range(count)]


def random_walk_cuda(n: int, generator, places: int = 2, dtype=np.float64, outlier_rate: float = 0.0,
                     device="cuda"):
    """``random_walk`` generated on the GPU from a torch Generator: x_{i+1} = x_i + N(0, 0.5)
    from 20.0, rounded to ``places`` decimals (the nearest binary value of the decimal, FP32
    ties resolved exactly), a fraction ``outlier_rate`` replaced by full-precision outliers
    x * 10^U(3,8).  Returns a CUDA tensor."""
    import torch
    g = generator
    steps = torch.randn(n, generator=g, device=device, dtype=torch.float64) * 0.5
    steps[0] = 0.0
    x = 20.0 + torch.cumsum(steps, 0)
    k = torch.round(x * (10.0 ** places))
    d = k / (10.0 ** places)                                 # exact operands: one rounding
    if dtype == np.float64:
        vals = d
    else:
        vals = d.to(torch.float32)
        bits = d.view(torch.int64)
        exp = (bits >> 52) & 0x7FF
        tie = ((bits & ((1 << 29) - 1)) == (1 << 28)) & (exp >= 1023 - 126) & (exp <= 1023 + 127)
        idx = torch.nonzero(tie).flatten()
        if idx.numel():
            fixed = decimal_to_f32(k[idx].to(torch.int64).cpu().numpy(), places)
            vals[idx] = torch.from_numpy(fixed).to(device)
    if outlier_rate > 0:
        mask = torch.rand(n, generator=g, device=device) < float(outlier_rate)
        if bool(mask.any()):
            u = torch.rand(n, generator=g, device=device, dtype=torch.float64) * 5 + 3
            big = (x * torch.pow(10.0, u)).to(vals.dtype)
            vals = torch.where(mask, big, vals)
    return vals.contiguous()
