"""Seeded, platform-independent random numbers for the synthetic workloads.

Counter-based: the value at position ``i`` of stream ``(seed, stream)`` is a
pure function of those three integers, so every machine (x86 or Arm, any numpy
version) produces the same integer and uniform bits; normals go through the C
library's log/cos/sin and may differ in the last bit between platforms.  Generator: SplitMix64 (Steele, Lea, Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014) applied to a
Weyl sequence keyed by (seed, stream); uniforms take the top 53 bits; normals
use the Box--Muller transform (Box & Muller, 1958).

This module holds no arithmetic of the refinement method itself.
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z):
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed, stream):
    with np.errstate(over="ignore"):
        k = _mix(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * _GOLDEN + np.uint64(stream & 0xFFFFFFFF))
    return k


def uint64(seed, stream, count, offset=0):
    """``count`` 64-bit words of stream ``(seed, stream)`` starting at ``offset``."""
    idx = np.arange(offset, offset + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _key(seed, stream) + (idx + np.uint64(1)) * _GOLDEN
        return _mix(z)


def uniform(seed, stream, count, offset=0):
    """Doubles uniform on (0, 1): (top 53 bits + 0.5) * 2^-53."""
    u = uint64(seed, stream, count, offset) >> np.uint64(11)
    return (u.astype(np.float64) + 0.5) * (2.0 ** -53)


def normal(seed, stream, count, offset=0):
    """Standard normal doubles by Box--Muller on pairs of uniforms."""
    m = (count + 1) // 2
    u = uniform(seed, stream, 2 * m, 2 * offset)
    u1, u2 = u[0::2], u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = rad * np.cos(2.0 * np.pi * u2)
    z[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return z[:count]
