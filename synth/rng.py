"""Counter-based random numbers for the synthetic inputs.

The generator is the SplitMix64 output function of Steele, Lea and Flood,
"Fast splittable pseudorandom number generators" (OOPSLA 2014): a 64-bit
state is advanced by the golden-ratio increment and passed through a
two-multiply xor-shift finaliser.  Here it is used counter-style: the value
for (seed, stream, index) is the finaliser applied to
``key(seed, stream) + (index + 1) * GOLDEN`` (mod 2^64), so every draw is a
pure function of its coordinates and does not depend on chunking, thread
count or device.

All arithmetic is on torch int64 tensors, whose multiplication wraps modulo
2^64 exactly like unsigned arithmetic; logical right shifts are emulated by
an arithmetic shift followed by a mask.  The same code therefore yields
bit-identical streams on the CPU and on a CUDA device.
"""
from __future__ import annotations

import torch

_MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB


def _signed(x: int) -> int:
    """Reinterpret an unsigned 64-bit integer as a signed int64."""
    x &= _MASK64
    return x - (1 << 64) if x >= (1 << 63) else x


def _mix_int(z: int) -> int:
    """SplitMix64 finaliser on a Python integer (exact, unsigned)."""
    z &= _MASK64
    z = ((z ^ (z >> 30)) * _M1) & _MASK64
    z = ((z ^ (z >> 27)) * _M2) & _MASK64
    return z ^ (z >> 31)


def _srl(x: torch.Tensor, s: int) -> torch.Tensor:
    """Logical right shift of int64 bit patterns."""
    return (x >> s) & ((1 << (64 - s)) - 1)


def mix64(z: torch.Tensor) -> torch.Tensor:
    """SplitMix64 finaliser on an int64 tensor (bit pattern = uint64)."""
    z = (z ^ _srl(z, 30)) * _signed(_M1)
    z = (z ^ _srl(z, 27)) * _signed(_M2)
    return z ^ _srl(z, 31)


def stream_key(seed: int, stream: int) -> int:
    """Per-(seed, stream) key as a signed int64 Python integer."""
    return _signed(_mix_int(_mix_int((seed & _MASK64) + GOLDEN) ^ (stream & _MASK64)))


def hash_u64(seed: int, stream: int, idx: torch.Tensor) -> torch.Tensor:
    """64 random bits (as int64 bit patterns) for each counter in ``idx``."""
    idx = idx.to(torch.int64)
    z = (idx + 1) * _signed(GOLDEN) + stream_key(seed, stream)
    return mix64(z)


def bits_below(h: torch.Tensor, nbits: int) -> torch.Tensor:
    """Top ``nbits`` bits of each draw as a non-negative int64 (nbits <= 62)."""
    return _srl(h, 64 - nbits)


def uniform01(seed: int, stream: int, idx: torch.Tensor) -> torch.Tensor:
    """Float64 uniforms in (0, 1]: ((top 53 bits) + 1) * 2^-53 (exact)."""
    h = hash_u64(seed, stream, idx)
    return (bits_below(h, 53) + 1).to(torch.float64) * (2.0 ** -53)


def below(seed: int, stream: int, idx: torch.Tensor, bound: torch.Tensor | int) -> torch.Tensor:
    """Integers in [0, bound) from the top 62 bits modulo ``bound``."""
    h = hash_u64(seed, stream, idx)
    return torch.remainder(bits_below(h, 62), bound)
