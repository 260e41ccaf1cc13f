"""The arithmetic of the BF16 path's compact master of X, on the CPU.

On the FP32 bit pattern b of x the encoder forms t = b + 0x8080 and keeps
hi = t >> 16 (the BF16 operand the tensor cores read) and the byte
u = (t >> 8) & 0xFF; the decoder rebuilds (hi << 16) + (u << 8) - 0x8000.
This restates that integer map with numpy (the device code is checked on the
GPU by the identity-step test) and checks the properties the kernels rely on:
|x' - x| <= 2^-16 |x| over many magnitudes and both signs, zero maps to zero,
the sign never flips, hi is within one BF16 unit of round-to-nearest, and the
residual code u - 128 stays a signed byte.
"""
import numpy as np


def encode(x):
    b = np.asarray(x, dtype=np.float32).view(np.uint32)
    t = b.astype(np.uint64) + 0x8080
    hi = (t >> 16).astype(np.uint32) & 0xFFFF
    u = ((t >> 8) & 0xFF).astype(np.uint32)
    return hi, u


def decode(hi, u):
    bits = ((hi.astype(np.uint64) << 16) + (u.astype(np.uint64) << 8) - 0x8000).astype(np.uint32)
    return bits.view(np.float32)


def _values(n=400000, seed=0):
    rng = np.random.default_rng(seed)
    mag = 10.0 ** rng.uniform(-30, 30, n)
    sign = rng.choice([-1.0, 1.0], n)
    x = (sign * mag).astype(np.float32)
    # bit patterns around the rounding thresholds of the low half (0x7F7F..0x8081)
    # and around powers of two
    base = rng.integers(0x00800000, 0x7F000000, 2000, dtype=np.uint64) & ~np.uint64(0xFFFF)
    lows = np.array([0x0000, 0x007F, 0x0080, 0x00FF, 0x7F7F, 0x7F80, 0x7FFF, 0x8000, 0x8080, 0xFF7F, 0xFF80, 0xFFFF],
                    dtype=np.uint64)
    edge = (base[:, None] + lows[None, :]).astype(np.uint32).reshape(-1).view(np.float32)
    return np.concatenate([x, edge, -edge])


def test_relative_error_bound():
    x = _values()
    hi, u = encode(x)
    y = decode(hi, u)
    xd, yd = x.astype(np.float64), y.astype(np.float64)
    assert np.all(np.abs(yd - xd) <= 2.0 ** -16 * np.abs(xd))


def test_zero_sign_and_residual_range():
    hi, u = encode(np.array([0.0, -0.0], dtype=np.float32))
    assert np.all(decode(hi, u) == 0.0)
    x = _values(seed=1)
    hi, u = encode(x)
    y = decode(hi, u)
    assert np.all(np.signbit(y) == np.signbit(x))
    # the signed residual code u - 128 is (b - (hi << 16) + 0x80) >> 8, and that
    # difference stays within a signed 16-bit range (so the code is a signed byte)
    b = x.view(np.uint32).astype(np.int64)
    r = b - (hi.astype(np.int64) << 16) + 0x80
    assert np.all((r >= -0x8000) & (r <= 0x7FFF))
    assert np.all((u.astype(np.int64) - 128) == (r >> 8))
    # decoding is b rounded to a multiple of 2^8 (ties up): x' keeps 16 mantissa bits
    xb = decode(hi, u).view(np.uint32).astype(np.int64)
    assert np.all(xb == ((b + 0x80) >> 8) << 8)


def test_hi_is_a_bf16_rounding():
    """hi differs from round-to-nearest-even BF16 by at most one unit (it
    rounds up from 0x7F80 of the low half instead of 0x8000)."""
    x = _values(seed=2)
    hi, _ = encode(x)
    b = x.view(np.uint32).astype(np.int64)
    rne = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    assert np.all(np.abs(hi.astype(np.int64) - (rne & 0xFFFF)) <= 1)
    # and as the BF16 operand it is within (2^-8 + 2^-16) |x| of x (rounding up
    # from 0x7F80 moves at most 0x8080 units of the low half)
    h = (hi.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    assert np.all(np.abs(h - x.astype(np.float64)) <= (2.0 ** -8 + 2.0 ** -16) * np.abs(x.astype(np.float64)))
