"""Block floating-point storage format of the populations (the library's BFP16 storage), written
out plainly in numpy.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): the tests use it as the reference for what the
CUDA library stores; it shares no code with the library.

The paper fixes no storage precision; this is the project's 16-bit format for the populations g,
which are deviations from the rest state (F = M (1 + eps g), Sec. 3).  Each velocity array is cut
into blocks of 8 consecutive cells (flat cell order).  A block of FP32 values v_k is stored as

    M   = max_k |v_k| = (1 + m / 2^23) * 2^(b - 127)   (b: biased exponent, m: mantissa bits),
    e   = b - 14 + [m >= 8387840],  e := 0 if e < 1,  e := 255 if any v_k is NaN or +-Inf;
    u_k = round-half-even(v_k * 2^(127 - e)) + 32768   (uint16; all 32768 when e is 0 or 255);
    value_k = (u_k - 32768) * 2^(e - 127)   (NaN for every value of a block with e = 255).

The mantissa test bumps the exponent exactly when M * 2^(127 - e) would reach 32766.5, so every
|u_k - 32768| <= 32766, the largest value keeps at least 15 bits, and decoded values encode back
to themselves.
"""
from __future__ import annotations

import numpy as np

BLOCK = 8
BUMP_MANTISSA = 8387840  # (32766.5 / 2^14 - 1) * 2^23: mantissa bits from which M 2^(14 - p) >= 32766.5


def block_exponents(v32: np.ndarray) -> np.ndarray:
    """Exponent byte of each block of 8 values of the FP32 array v32 (last axis, length a
    multiple of 8).  Returns an int64 array with the last axis divided by 8."""
    v = np.asarray(v32, dtype=np.float32)
    blocks = v.reshape(v.shape[:-1] + (v.shape[-1] // BLOCK, BLOCK))
    finite = np.isfinite(blocks).all(axis=-1)
    m = np.abs(np.where(finite[..., None], blocks, np.float32(0))).max(axis=-1).astype(np.float32)
    bits = m.view(np.uint32).astype(np.int64)
    b = (bits >> 23) + ((bits & 0x7FFFFF) >= BUMP_MANTISSA)
    e = np.where(b > 14, b - 14, 0)
    return np.where(finite, e, 255)


def encode(v32: np.ndarray):
    """(u, e): uint16 mantissas (offset binary) with the shape of v32 and the exponent bytes of
    its blocks, for FP32 values v32 (last axis a multiple of 8)."""
    v = np.asarray(v32, dtype=np.float32)
    e = block_exponents(v)
    ebig = np.repeat(e, BLOCK, axis=-1)
    live = (ebig > 0) & (ebig < 255)
    scale = np.where(live, np.ldexp(1.0, (127 - ebig).astype(np.int64)), 0.0)
    with np.errstate(invalid="ignore"):
        prod = np.where(live, v.astype(np.float64) * scale, 0.0)  # exact: a power-of-two scale
    q = np.rint(prod)  # round half to even
    assert np.all(np.abs(q) <= 32766), "block scale leaves two units of headroom"
    return (q + 32768).astype(np.uint16), e.astype(np.uint8)


def decode(u: np.ndarray, e: np.ndarray) -> np.ndarray:
    """FP64 values of stored mantissas u and block exponents e."""
    ebig = np.repeat(np.asarray(e, dtype=np.int64), BLOCK, axis=-1)
    val = (np.asarray(u, dtype=np.float64) - 32768.0) * np.ldexp(1.0, ebig - 127)
    return np.where(ebig == 255, np.nan, val)


def round_trip(v32: np.ndarray) -> np.ndarray:
    """What storing the FP32 values v32 keeps: decode(encode(v32))."""
    return decode(*encode(v32))
