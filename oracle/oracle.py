"""ctypes front end of the plain C oracle (``falcon_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it; the product
path (the CUDA library and its binding) never imports it.

The oracle follows the paper's definitions step by step (Alg. 2, Eq. 4-5,
Sec. 3.3, Sec. 4); see the header comment of ``falcon_oracle.c`` for the
readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "falcon_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

F64, F32, F16 = 0, 1, 2
OK, ERR_INVALID, ERR_CAPACITY, ERR_CORRUPT = 0, 1, 2, 3
# codec variants: Falcon and the ablations of Sec. 5.4.2 (Fal._Sparse, Fal._Dense, Fal._Elf)
FALCON, SPARSE, DENSE, ELF = 0, 1, 2, 3

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles the oracle with plain IEEE semantics (no contraction, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-pthread",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            c = ctypes
            L.oracle_pow10_f64.restype = c.c_double
            L.oracle_pow10_f64.argtypes = [c.c_int]
            L.oracle_pow10_f32.restype = c.c_float
            L.oracle_pow10_f32.argtypes = [c.c_int]
            L.oracle_is_special_f64.argtypes = [c.c_double]
            L.oracle_is_special_f32.argtypes = [c.c_float]
            L.oracle_floor_log10_f64.argtypes = [c.c_double]
            L.oracle_floor_log10_f32.argtypes = [c.c_float]
            L.oracle_dp_ds_f64.argtypes = [c.c_double, c.POINTER(c.c_int), c.POINTER(c.c_int)]
            L.oracle_dp_ds_f32.argtypes = [c.c_float, c.POINTER(c.c_int), c.POINTER(c.c_int)]
            L.oracle_dp_elf_f64.argtypes = [c.c_double, c.POINTER(c.c_int), c.POINTER(c.c_int)]
            L.oracle_dp_elf_f32.argtypes = [c.c_float, c.POINTER(c.c_int), c.POINTER(c.c_int)]
            L.oracle_chunk_transform_elf.argtypes = [c.c_void_p, c.c_uint32, c.c_int,
                                                     c.POINTER(c.c_int), c.POINTER(c.c_int),
                                                     c.POINTER(c.c_int), c.c_void_p]
            L.oracle_encode_z_storage.restype = c.c_size_t
            L.oracle_encode_z_storage.argtypes = [c.c_void_p, c.c_uint32, c.c_int, c.c_int, c.c_int,
                                                  c.c_int, c.c_void_p, c.c_size_t]
            L.oracle_compress_variant.argtypes = [c.c_void_p, c.c_uint64, c.c_int, c.c_uint32, c.c_int,
                                                  c.c_void_p, c.c_size_t, c.POINTER(c.c_size_t)]
            L.oracle_compress_mt.argtypes = [c.c_void_p, c.c_uint64, c.c_int, c.c_uint32, c.c_int, c.c_int,
                                             c.c_void_p, c.c_size_t, c.POINTER(c.c_size_t)]
            L.oracle_decompress_mt.argtypes = [c.c_void_p, c.c_size_t, c.c_void_p, c.c_size_t,
                                               c.POINTER(c.c_uint64), c.c_int]
            for name in ("oracle_zigzag64", "oracle_unzigzag64"):
                getattr(L, name).restype = c.c_uint64
                getattr(L, name).argtypes = [c.c_uint64]
            for name in ("oracle_zigzag32", "oracle_unzigzag32"):
                getattr(L, name).restype = c.c_uint32
                getattr(L, name).argtypes = [c.c_uint32]
            # binary16 (R18): values cross the boundary as their 16-bit patterns
            for name in ("oracle_zigzag16", "oracle_unzigzag16"):
                getattr(L, name).restype = c.c_uint16
                getattr(L, name).argtypes = [c.c_uint16]
            L.oracle_pow10_f16.restype = c.c_uint16
            L.oracle_pow10_f16.argtypes = [c.c_int]
            L.oracle_f16_div_pow10.restype = c.c_uint16
            L.oracle_f16_div_pow10.argtypes = [c.c_int32, c.c_int]
            L.oracle_half_to_double.restype = c.c_double
            L.oracle_half_to_double.argtypes = [c.c_uint16]
            L.oracle_is_special_f16.argtypes = [c.c_uint16]
            L.oracle_floor_log10_f16.argtypes = [c.c_uint16]
            L.oracle_dp_ds_f16.argtypes = [c.c_uint16, c.POINTER(c.c_int), c.POINTER(c.c_int)]
            L.oracle_dp_elf_f16.argtypes = [c.c_uint16, c.POINTER(c.c_int), c.POINTER(c.c_int)]
            L.oracle_aggregate.argtypes = [c.c_void_p, c.c_size_t, c.POINTER(c.c_uint64), c.POINTER(c.c_uint64),
                                           c.POINTER(c.c_double), c.POINTER(c.c_double), c.POINTER(c.c_double)]
            L.oracle_chunk_transform.argtypes = [c.c_void_p, c.c_uint32, c.c_int,
                                                 c.POINTER(c.c_int), c.POINTER(c.c_int),
                                                 c.POINTER(c.c_int), c.c_void_p]
            L.oracle_delta_zigzag.argtypes = [c.c_void_p, c.c_uint32, c.c_int, c.c_void_p]
            L.oracle_encode_z.restype = c.c_size_t
            L.oracle_encode_z.argtypes = [c.c_void_p, c.c_uint32, c.c_int, c.c_int, c.c_int,
                                          c.c_void_p, c.c_size_t]
            L.oracle_encode_chunk.restype = c.c_size_t
            L.oracle_encode_chunk.argtypes = [c.c_void_p, c.c_uint32, c.c_int, c.c_void_p,
                                              c.c_size_t]
            L.oracle_decode_chunk.argtypes = [c.c_void_p, c.c_size_t, c.c_uint32, c.c_int,
                                              c.c_void_p]
            L.oracle_bound_variant.restype = c.c_size_t
            L.oracle_bound_variant.argtypes = [c.c_uint64, c.c_int, c.c_uint32, c.c_int]
            L.oracle_bound.restype = c.c_size_t
            L.oracle_bound.argtypes = [c.c_uint64, c.c_int, c.c_uint32]
            L.oracle_compress.argtypes = [c.c_void_p, c.c_uint64, c.c_int, c.c_uint32,
                                          c.c_void_p, c.c_size_t, c.POINTER(c.c_size_t)]
            L.oracle_decompress.argtypes = [c.c_void_p, c.c_size_t, c.c_void_p, c.c_size_t,
                                            c.POINTER(c.c_uint64)]
            L.oracle_stream_info.argtypes = [c.c_void_p, c.c_size_t, c.POINTER(c.c_uint64),
                                             c.POINTER(c.c_int), c.POINTER(c.c_uint32),
                                             c.POINTER(c.c_uint64)]
            _lib = L
    return _lib


def _dtype_code(arr: np.ndarray) -> int:
    if arr.dtype == np.float64:
        return F64
    if arr.dtype == np.float32:
        return F32
    if arr.dtype == np.float16:
        return F16
    raise TypeError(f"unsupported dtype {arr.dtype}")


def _np_dtype(code: int):
    return {F64: np.float64, F32: np.float32, F16: np.float16}[code]


def _h(v) -> int:
    """The binary16 pattern of v (a float16 or its uint16 pattern)."""
    if isinstance(v, (int, np.integer)) and not isinstance(v, bool):
        return int(v) & 0xFFFF
    return int(np.array(v, dtype=np.float16).view(np.uint16))


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


# ----------------------------------------------------------------------------- scalar steps
def pow10(k: int, dtype=np.float64):
    L = lib()
    if dtype == np.float16:
        return np.array(L.oracle_pow10_f16(k), dtype=np.uint16).view(np.float16)[()]
    return L.oracle_pow10_f64(k) if dtype == np.float64 else np.float32(L.oracle_pow10_f32(k))


def f16_div_pow10(g: int, a: int) -> int:
    """fl16(g / 10^a) as a binary16 pattern (R18's Case-1 round trip and decode)."""
    return lib().oracle_f16_div_pow10(g, a)


def half_to_double(u: int) -> float:
    return lib().oracle_half_to_double(u & 0xFFFF)


def dp_ds(v, dtype=np.float64):
    """Alg. 2 DPAndDSCalculation -> (alpha, beta)."""
    L = lib()
    a, b = ctypes.c_int(), ctypes.c_int()
    if dtype == np.float64:
        L.oracle_dp_ds_f64(float(v), ctypes.byref(a), ctypes.byref(b))
    elif dtype == np.float16:
        L.oracle_dp_ds_f16(_h(v), ctypes.byref(a), ctypes.byref(b))
    else:
        L.oracle_dp_ds_f32(float(np.float32(v)), ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def dp_elf(v, dtype=np.float64):
    """Fal._Elf's trial-and-error decimal place (Sec. 1, Sec. 5.4.2) -> (alpha, beta)."""
    L = lib()
    a, b = ctypes.c_int(), ctypes.c_int()
    if dtype == np.float64:
        L.oracle_dp_elf_f64(float(v), ctypes.byref(a), ctypes.byref(b))
    elif dtype == np.float16:
        L.oracle_dp_elf_f16(_h(v), ctypes.byref(a), ctypes.byref(b))
    else:
        L.oracle_dp_elf_f32(float(np.float32(v)), ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def floor_log10(v, dtype=np.float64) -> int:
    L = lib()
    if dtype == np.float64:
        return L.oracle_floor_log10_f64(float(v))
    if dtype == np.float16:
        return L.oracle_floor_log10_f16(_h(v))
    return L.oracle_floor_log10_f32(float(np.float32(v)))


def is_special(v, dtype=np.float64) -> bool:
    L = lib()
    if dtype == np.float64:
        return bool(L.oracle_is_special_f64(float(v)))
    if dtype == np.float16:
        return bool(L.oracle_is_special_f16(_h(v)))
    return bool(L.oracle_is_special_f32(float(np.float32(v))))


def zigzag64(x: int) -> int:
    return lib().oracle_zigzag64(x & 0xFFFFFFFFFFFFFFFF)


def unzigzag64(z: int) -> int:
    return lib().oracle_unzigzag64(z & 0xFFFFFFFFFFFFFFFF)


def zigzag32(x: int) -> int:
    return lib().oracle_zigzag32(x & 0xFFFFFFFF)


def unzigzag32(z: int) -> int:
    return lib().oracle_unzigzag32(z & 0xFFFFFFFF)


def zigzag16(x: int) -> int:
    return lib().oracle_zigzag16(x & 0xFFFF)


def unzigzag16(z: int) -> int:
    return lib().oracle_unzigzag16(z & 0xFFFF)


# ----------------------------------------------------------------------------- chunk steps
def chunk_transform(vals: np.ndarray, elf: bool = False):
    """Eq. 4 on one chunk -> (alpha_max, beta_hat_max, case1, G as uint64 words); elf=True
    takes Fal._Elf's decimal places."""
    vals = np.ascontiguousarray(vals)
    g = np.zeros(max(len(vals), 1), dtype=np.uint64)
    a, b, c1 = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    fn = lib().oracle_chunk_transform_elf if elf else lib().oracle_chunk_transform
    fn(_ptr(vals), len(vals), _dtype_code(vals), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c1), _ptr(g))
    return a.value, b.value, bool(c1.value), g[:len(vals)]


def delta_zigzag(g: np.ndarray, dtype_code: int) -> np.ndarray:
    g = np.ascontiguousarray(g, dtype=np.uint64)
    z = np.zeros(max(len(g), 1), dtype=np.uint64)
    lib().oracle_delta_zigzag(_ptr(g), len(g), dtype_code, _ptr(z))
    return z[:len(g)]


def encode_z(z: np.ndarray, dtype_code: int, alpha_max: int, beta_hat: int, storage: int = 0) -> bytes:
    """Sec. 3.3 record of Z; storage 0 = adaptive, 1 = every row sparse, 2 = every row dense."""
    z = np.ascontiguousarray(z, dtype=np.uint64)
    cap = 16 + 8 * 64 * (len(z) + 64)
    out = np.zeros(cap, dtype=np.uint8)
    n = lib().oracle_encode_z_storage(_ptr(z), len(z), dtype_code, alpha_max, beta_hat, storage, _ptr(out), cap)
    if n == 0:
        raise RuntimeError("oracle_encode_z overflow")
    return out[:n].tobytes()


def encode_chunk(vals: np.ndarray) -> bytes:
    vals = np.ascontiguousarray(vals)
    cap = 16 + 8 * 64 * (len(vals) + 64)
    out = np.zeros(cap, dtype=np.uint8)
    n = lib().oracle_encode_chunk(_ptr(vals), len(vals), _dtype_code(vals), _ptr(out), cap)
    if n == 0:
        raise RuntimeError("oracle_encode_chunk overflow")
    return out[:n].tobytes()


def decode_chunk(rec: bytes, m: int, dtype=np.float64) -> np.ndarray:
    buf = np.frombuffer(rec, dtype=np.uint8).copy()
    out = np.zeros(max(m, 1), dtype=dtype)
    code = {np.dtype(np.float64): F64, np.dtype(np.float32): F32, np.dtype(np.float16): F16}[np.dtype(dtype)]
    st = lib().oracle_decode_chunk(_ptr(buf), len(buf), m, code, _ptr(out))
    if st != OK:
        raise ValueError(f"oracle_decode_chunk status {st}")
    return out[:m]


# ----------------------------------------------------------------------------- stream level
def bound(n: int, dtype_code: int, block: int, variant: int = FALCON) -> int:
    if variant != FALCON:
        return lib().oracle_bound_variant(n, dtype_code, block, variant)
    return lib().oracle_bound(n, dtype_code, block)


def compress(vals: np.ndarray, block: int = 1024, variant: int = FALCON, threads: int = 1) -> bytes:
    """The stream of `vals`; variant selects Falcon or one of its ablations; threads > 1 runs
    the multi-threaded driver (same bytes)."""
    vals = np.ascontiguousarray(vals)
    code = _dtype_code(vals)
    cap = bound(len(vals), code, block, variant)
    if cap == 0:
        raise ValueError("invalid arguments")
    out = np.empty(cap, dtype=np.uint8)
    nbytes = ctypes.c_size_t()
    if threads > 1:
        st = lib().oracle_compress_mt(_ptr(vals), len(vals), code, block, variant, threads, _ptr(out), cap,
                                      ctypes.byref(nbytes))
    elif variant != FALCON:
        st = lib().oracle_compress_variant(_ptr(vals), len(vals), code, block, variant, _ptr(out), cap,
                                           ctypes.byref(nbytes))
    else:
        st = lib().oracle_compress(_ptr(vals), len(vals), code, block, _ptr(out), cap, ctypes.byref(nbytes))
    if st != OK:
        raise ValueError(f"oracle_compress status {st}")
    return out[:nbytes.value].tobytes()


def stream_info(stream: bytes):
    buf = np.frombuffer(stream, dtype=np.uint8)
    n, nc = ctypes.c_uint64(), ctypes.c_uint64()
    dt, blk = ctypes.c_int(), ctypes.c_uint32()
    st = lib().oracle_stream_info(_ptr(buf), len(buf), ctypes.byref(n), ctypes.byref(dt),
                                  ctypes.byref(blk), ctypes.byref(nc))
    if st != OK:
        raise ValueError(f"oracle_stream_info status {st}")
    return n.value, dt.value, blk.value, nc.value


def decompress_status(stream: bytes, threads: int = 1):
    """Returns (status, values or None) without raising."""
    buf = np.frombuffer(stream, dtype=np.uint8)
    if len(buf) < 32:
        return ERR_CORRUPT, None
    try:
        n, dt, _, _ = stream_info(stream)
    except ValueError:
        return ERR_CORRUPT, None
    dtype = _np_dtype(dt)
    s = np.dtype(dtype).itemsize
    if n > (1 << 34):
        return ERR_CORRUPT, None
    out = np.zeros(max(n, 1), dtype=dtype)
    nout = ctypes.c_uint64()
    if threads > 1:
        st = lib().oracle_decompress_mt(_ptr(buf), len(buf), _ptr(out), n * s, ctypes.byref(nout), threads)
    else:
        st = lib().oracle_decompress(_ptr(buf), len(buf), _ptr(out), n * s, ctypes.byref(nout))
    if st != OK:
        return st, None
    return OK, out[:n]


def decompress(stream: bytes, threads: int = 1) -> np.ndarray:
    st, out = decompress_status(stream, threads)
    if st != OK:
        raise ValueError(f"oracle_decompress status {st}")
    return out


def chunk_records(stream: bytes):
    """Splits a stream into its chunk records (list of bytes), using the size array."""
    n, dt, blk, nc = stream_info(stream)
    sizes = np.frombuffer(stream, dtype="<u4", count=nc, offset=32)
    pos = 32 + 4 * nc
    recs = []
    for s in sizes:
        recs.append(stream[pos:pos + int(s)])
        pos += int(s)
    return recs


def aggregate(stream: bytes) -> dict:
    """R19's aggregate of a stream: count, nan_count, min / max in totalOrder (NaN if none),
    and the correctly rounded exact sum of the non-NaN values."""
    buf = np.frombuffer(stream, dtype=np.uint8)
    cnt, nan = ctypes.c_uint64(), ctypes.c_uint64()
    lo, hi, sm = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    st = lib().oracle_aggregate(_ptr(buf), len(buf), ctypes.byref(cnt), ctypes.byref(nan), ctypes.byref(lo),
                                ctypes.byref(hi), ctypes.byref(sm))
    if st != OK:
        raise ValueError(f"oracle_aggregate status {st}")
    return {"count": cnt.value, "nan_count": nan.value, "min": lo.value, "max": hi.value, "sum": sm.value}
