"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module only produces operand values and storage layouts. It holds none of the
fault-tolerant GEMM's arithmetic (no products, checksums, thresholds or corrections),
so both the CUDA path and the CPU oracle can be fed from it without sharing code.

Generator: SplitMix64 (Steele, Lea and Flood, OOPSLA 2014), used counter-style. The
value of logical element ``idx`` of matrix ``matrix_id`` under ``seed`` is
``mix(key + (idx + 1) * GOLDEN)`` with ``key = seed ^ (matrix_id << 56)``, where ``mix``
is the SplitMix64 finaliser. Uniform[-1, 1) draws are ``(x >> 11) * 2**-52 - 1``, a
multiple of 2**-52, so every value is exact in binary64.

The logical index of element (r, c) of an ``rows x cols`` matrix is ``r + c * rows``
(column-major), whatever storage layout is asked for, so the same seed gives the same
matrix in column-major and row-major storage.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

COL_MAJOR = 102
ROW_MAJOR = 101


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, matrix_id: int, idx: np.ndarray) -> np.ndarray:
    """Counter-based SplitMix64 outputs for the logical indexes ``idx`` (uint64)."""
    key = np.uint64((seed ^ (matrix_id << 56)) & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        z = key + (idx.astype(np.uint64) + np.uint64(1)) * GOLDEN
        return _mix(z)


def uniform(seed: int, matrix_id: int, count: int, chunk: int = 1 << 24) -> np.ndarray:
    """``count`` values exactly representable in binary64, uniform on [-1, 1)."""
    out = np.empty(count, dtype=np.float64)
    for s in range(0, count, chunk):
        e = min(count, s + chunk)
        x = splitmix64(seed, matrix_id, np.arange(s, e, dtype=np.uint64))
        out[s:e] = (x >> np.uint64(11)).astype(np.float64) * (2.0 ** -52) - 1.0
    return out


def _chunks(count: int, threads: int, fn, chunk: int = 1 << 22) -> None:
    """Run fn(s, e) over [0, count) in chunks, on `threads` threads (numpy releases the GIL
    in its array loops); fn writes disjoint slices, so the result is order-independent."""
    spans = [(s, min(count, s + chunk)) for s in range(0, count, chunk)]
    if threads <= 1 or len(spans) <= 1:
        for s, e in spans:
            fn(s, e)
        return
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(lambda se: fn(*se), spans))


def normal(seed: int, matrix_id: int, count: int, threads: int = 1) -> np.ndarray:
    """Standard normal values by the Box-Muller transform of two uniform streams (host libm):
    pair q gives values q (cosine) and n2 + q (sine), n2 = ceil(count / 2)."""
    n2 = (count + 1) // 2
    z = np.empty(2 * n2, dtype=np.float64)

    def work(s, e):
        idx = np.arange(s, e, dtype=np.uint64)
        x1 = splitmix64(seed, matrix_id, idx)
        x2 = splitmix64(seed, matrix_id ^ 0x55, idx)
        u1 = ((x1 >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)  # (0, 1]
        u2 = (x2 >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)          # [0, 1)
        r = np.sqrt(-2.0 * np.log(u1))
        z[s:e] = r * np.cos(2.0 * np.pi * u2)
        z[n2 + s:n2 + e] = r * np.sin(2.0 * np.pi * u2)

    _chunks(n2, threads, work)
    return z[:count]


def map_elementwise(fn, x: np.ndarray, out_dtype, threads: int = 1) -> np.ndarray:
    """fn applied to the elements of x (flattened in C order, reshaped back), in chunks on
    `threads` threads; fn must be elementwise (e.g. to_bf16_bits, to_e4m3_bits)."""
    flat = np.ascontiguousarray(x).reshape(-1)
    out = np.empty(flat.size, dtype=out_dtype)

    def work(s, e):
        out[s:e] = fn(flat[s:e])

    _chunks(flat.size, threads, work)
    return out.reshape(np.shape(x))


def randint(seed: int, matrix_id: int, count: int, lo: int, hi: int) -> np.ndarray:
    """Integers uniform on [lo, hi] (inclusive)."""
    x = splitmix64(seed, matrix_id, np.arange(0, count, dtype=np.uint64))
    return (x % np.uint64(hi - lo + 1)).astype(np.int64) + lo


def store(logical: np.ndarray, layout: int, ld: int | None = None, pad_value: float = np.nan) -> tuple[np.ndarray, int]:
    """Lay a logical ``rows x cols`` matrix out in BLAS storage.

    Returns ``(flat_buffer, ld)``. Column-major: element (r, c) at ``r + c*ld`` with
    ``ld >= rows``; row-major: at ``r*ld + c`` with ``ld >= cols``. Padding slots
    (``ld`` beyond the logical extent) hold ``pad_value`` (NaN by default) so that a
    kernel reading them would be caught.
    """
    rows, cols = logical.shape
    if layout == COL_MAJOR:
        ld = max(1, rows) if ld is None else ld
        buf = np.full(ld * cols if cols else 0, pad_value, dtype=logical.dtype)
        if rows and cols:
            buf.reshape(cols, ld)[:, :rows] = logical.T
    elif layout == ROW_MAJOR:
        ld = max(1, cols) if ld is None else ld
        buf = np.full(ld * rows if rows else 0, pad_value, dtype=logical.dtype)
        if rows and cols:
            buf.reshape(rows, ld)[:, :cols] = logical
    else:
        raise ValueError("layout must be COL_MAJOR (102) or ROW_MAJOR (101)")
    return buf, ld


def load(buf: np.ndarray, layout: int, rows: int, cols: int, ld: int) -> np.ndarray:
    """Inverse of :func:`store`: the logical ``rows x cols`` matrix held in ``buf``."""
    if rows == 0 or cols == 0:
        return np.zeros((rows, cols), dtype=buf.dtype)
    if layout == COL_MAJOR:
        return buf[: ld * cols].reshape(cols, ld)[:, :rows].T.copy()
    return buf[: ld * rows].reshape(rows, ld)[:, :cols].copy()


def uniform_matrix(seed: int, matrix_id: int, rows: int, cols: int) -> np.ndarray:
    """Logical ``rows x cols`` matrix of exact uniform[-1, 1) values."""
    return uniform(seed, matrix_id, rows * cols).reshape(cols, rows).T


def normal_matrix(seed: int, matrix_id: int, rows: int, cols: int, std: float = 1.0, threads: int = 1) -> np.ndarray:
    z = normal(seed, matrix_id, rows * cols, threads)
    if std != 1.0:
        z *= std
    return z.reshape(cols, rows).T


def pow2_row_scales(seed: int, matrix_id: int, count: int, lo: int = -8, hi: int = 8) -> np.ndarray:
    """Exact powers of two 2**u with u uniform on the integers [lo, hi]."""
    return np.ldexp(1.0, randint(seed, matrix_id, count, lo, hi).astype(np.int32))


# ---------------------------------------------------------------------------------------
# Reduced-precision storage formats. Encoding rounds to nearest, ties to even, on the
# host; it is input preparation only (both sides receive the same encoded bits).
# ---------------------------------------------------------------------------------------

def to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round binary64 values to bfloat16 (nearest, ties to even); returns uint16 bits."""
    f = np.asarray(x, dtype=np.float64)
    # binary64 -> binary32 rounding first could double-round; round directly instead:
    # bfloat16 keeps 8 significant bits, so round the binary64 significand at bit 45.
    b = f.view(np.uint64)
    sign = (b >> np.uint64(63)).astype(np.uint16)
    mag = np.abs(f)
    out = np.zeros(f.shape, dtype=np.uint16)
    finite = np.isfinite(mag)
    # Work in binary32 space by exact scaling: value = m * 2**e with m in [1, 2).
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        m, e = np.frexp(np.where(finite, mag, 0.0))  # mag = m * 2**e, m in [0.5, 1)
    # normal bf16 range: exponent (unbiased, value in [2**(e-1), 2**e)) from -125 to 128
    q = np.rint(m * 256.0)  # 8 significant bits, ties to even via rint
    carry = q >= 256.0
    q = np.where(carry, 128.0, q)
    e = np.where(carry, e + 1, e)
    ebias = e - 1 + 127  # biased exponent of value q/128 * 2**(e-1)
    normal_ = finite & (mag > 0) & (ebias >= 1) & (ebias <= 254)
    bits_n = (ebias.astype(np.int64) << 7) | (q.astype(np.int64) - 128)
    # subnormals: value = q_s * 2**-133 with q_s in [0, 127]
    sub = finite & (mag > 0) & (ebias < 1)
    qs = np.rint(np.ldexp(np.where(sub, mag, 0.0), 133))
    bits_s = qs.astype(np.int64)  # qs == 128 rolls into the smallest normal, still correct bits
    over = (finite & (ebias > 254)) | (~finite & ~np.isnan(f))
    bits = np.where(normal_, bits_n, 0)
    bits = np.where(sub, bits_s, bits)
    bits = np.where(over, 0x7F80, bits)
    bits = np.where(np.isnan(f), 0x7FC0, bits)
    out[:] = bits.astype(np.uint16)
    return out | (sign << np.uint16(15))


def bf16_bits_to_f64(bits: np.ndarray) -> np.ndarray:
    """Exact binary64 value of bfloat16 bit patterns."""
    return (np.asarray(bits, dtype=np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)


E4M3_MAX = 448.0


def to_e4m3_bits(x: np.ndarray) -> np.ndarray:
    """Round to OCP FP8 E4M3 (nearest, ties to even, saturating at +-448); uint8 bits."""
    f = np.asarray(x, dtype=np.float64)
    sign = (f < 0) | ((f == 0) & (np.signbit(f)))
    mag = np.minimum(np.abs(np.nan_to_num(f, nan=0.0)), E4M3_MAX)
    out = np.zeros(f.shape, dtype=np.int64)
    with np.errstate(divide="ignore"):
        m, e = np.frexp(mag)  # mag = m * 2**e, m in [0.5, 1)
    eb = e - 1 + 7  # biased exponent of a normal value in [2**(e-1), 2**e)
    normal_ = (mag > 0) & (eb >= 1)
    q = np.rint(m * 16.0)  # 4 significant bits (1 implicit + 3 stored)
    carry = q >= 16.0
    q = np.where(carry, 8.0, q)
    eb = np.where(carry, eb + 1, eb)
    bits_n = (eb.astype(np.int64) << 3) | (q.astype(np.int64) - 8)
    # subnormal range by the exponent before rounding (a carry may lift it to the smallest
    # normal, and qs == 8 is then the smallest normal's bit pattern)
    sub = (mag > 0) & ~normal_
    qs = np.rint(np.ldexp(np.where(sub, mag, 0.0), 9))  # subnormal step 2**-9
    out = np.where(normal_, bits_n, 0)
    out = np.where(sub, qs.astype(np.int64), out)
    out = np.minimum(out, 0x7E)  # 0x7E = 448; saturate (0x7F is NaN in E4M3)
    out = np.where(np.isnan(f), 0x7F, out)
    return (out | (sign.astype(np.int64) << 7)).astype(np.uint8)


def e4m3_bits_to_f64(bits: np.ndarray) -> np.ndarray:
    """Exact binary64 value of E4M3 bit patterns (0x7F/0xFF decode to NaN)."""
    b = np.asarray(bits, dtype=np.int64)
    s = np.where(b & 0x80, -1.0, 1.0)
    e = (b >> 3) & 0xF
    m = b & 0x7
    val = np.where(e == 0, np.ldexp(m.astype(np.float64), -9), np.ldexp((8 + m).astype(np.float64), (e - 10).astype(np.int32)))
    val = np.where((b & 0x7F) == 0x7F, np.nan, val)
    return s * val
