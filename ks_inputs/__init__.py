"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no arithmetic of the multiplication method: it only draws
coefficients.  Both the CUDA path (through the tests and ``bench.py``) and the
CPU oracle receive the same arrays from here.

Random numbers come from the splitmix64 generator (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014), used in its
counter form: draw ``i`` of stream ``seed`` is ``mix(seed + (i + 1) * gamma)``
with ``gamma = 0x9E3779B97F4A7C15``.

Coefficient encoding (the library's layout): a polynomial of length ``L`` with
coefficient bound ``b`` bits is a ``(L, in_limbs)`` uint64 array,
``in_limbs = ceil(b / 64)``, limbs little-endian.  Unsigned coefficients lie in
``[0, 2^b)``; signed ones in ``[-2^(b-1), 2^(b-1))``, stored two's complement
and sign-extended over all ``in_limbs`` limbs.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
MASK64 = (1 << 64) - 1


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Draws ``offset .. offset+n-1`` of the splitmix64 stream ``seed``."""
    with np.errstate(over="ignore"):
        idx = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & MASK64) + idx * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def in_limbs(coeff_bits: int) -> int:
    return (coeff_bits + 63) // 64


def random_poly(length: int, coeff_bits: int, is_signed: bool, seed: int) -> np.ndarray:
    """Uniform coefficients of ``coeff_bits`` bits, as a ``(length, in_limbs)`` uint64 array."""
    if length < 0 or coeff_bits < 1:
        raise ValueError("length >= 0 and coeff_bits >= 1 required")
    nl = in_limbs(coeff_bits)
    raw = splitmix64(seed, length * nl).reshape(length, nl)
    top_bits = coeff_bits - 64 * (nl - 1)  # bits used in the top limb, 1..64
    if top_bits < 64:
        raw[:, nl - 1] &= np.uint64((1 << top_bits) - 1)
    if is_signed:
        raw = sign_extend(raw, coeff_bits)
    return raw


def sign_extend(limbs: np.ndarray, coeff_bits: int) -> np.ndarray:
    """Reads each row as a ``coeff_bits``-bit two's complement value and sign-extends it."""
    limbs = limbs.copy()
    nl = limbs.shape[1]
    top_bits = coeff_bits - 64 * (nl - 1)
    if top_bits < 64:
        top = limbs[:, nl - 1]
        neg = (top >> np.uint64(top_bits - 1)) & np.uint64(1)
        ext = np.uint64(MASK64 ^ ((1 << top_bits) - 1))
        limbs[:, nl - 1] = np.where(neg == 1, top | ext, top)
    return limbs


def const_poly(length: int, coeff_bits: int, value: int) -> np.ndarray:
    """All coefficients equal to ``value`` (a Python int, two's complement if negative)."""
    nl = in_limbs(coeff_bits)
    v = value & ((1 << (64 * nl)) - 1)
    row = np.array([(v >> (64 * i)) & MASK64 for i in range(nl)], dtype=np.uint64)
    return np.tile(row, (length, 1))


def from_ints(values, coeff_bits: int) -> np.ndarray:
    """Encodes Python ints (any sign) as a limb array of ``in_limbs(coeff_bits)`` limbs."""
    nl = in_limbs(coeff_bits)
    out = np.zeros((len(values), nl), dtype=np.uint64)
    full = (1 << (64 * nl)) - 1
    for i, v in enumerate(values):
        v &= full
        for l in range(nl):
            out[i, l] = (v >> (64 * l)) & MASK64
    return out


def to_ints(limbs: np.ndarray, is_signed: bool) -> list[int]:
    """Decodes a ``(L, nl)`` limb array into Python ints."""
    limbs = np.asarray(limbs, dtype=np.uint64)
    nl = limbs.shape[1]
    width = 64 * nl
    out = []
    for row in limbs.tolist():
        v = 0
        for l in reversed(range(nl)):
            v = (v << 64) | int(row[l])
        if is_signed and v >> (width - 1):
            v -= 1 << width
        out.append(v)
    return out


def log_uniform_int(u: np.ndarray, lo: int, hi: int) -> np.ndarray:
    """Maps uniform 64-bit draws to integers log-uniform in ``[lo, hi]``."""
    x = (u >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    v = np.exp(math.log(lo) + x * (math.log(hi + 1) - math.log(lo)))
    return np.clip(np.floor(v).astype(np.int64), lo, hi)


def uneven_batch(n: int, seed: int, len_lo: int = 8, len_hi: int = 8192,
                 bits_lo: int = 4, bits_hi: int = 512):
    """Shapes of a batch of uneven products: ``(len_f, len_g, coeff_bits, is_signed)`` arrays.

    ``len_f`` and ``len_g`` are drawn independently log-uniform in ``[len_lo, len_hi]``,
    ``coeff_bits`` log-uniform in ``[bits_lo, bits_hi]`` (rounded down), and each
    product is signed with probability one half.
    """
    u = splitmix64(seed, 4 * n).reshape(n, 4)
    lf = log_uniform_int(u[:, 0], len_lo, len_hi)
    lg = log_uniform_int(u[:, 1], len_lo, len_hi)
    cb = log_uniform_int(u[:, 2], bits_lo, bits_hi)
    sg = (u[:, 3] >> np.uint64(63)).astype(np.int64)
    return lf, lg, cb, sg


def random_residues(length: int, p: int, seed: int) -> np.ndarray:
    """Residues uniform in ``[0, p)`` for a modulus ``p < 2^64`` (rejection sampling), ``(L, 1)``."""
    if not (2 <= p < (1 << 64)):
        raise ValueError("modulus must lie in [2, 2^64)")
    bits = (p - 1).bit_length()
    mask = np.uint64((1 << bits) - 1) if bits < 64 else np.uint64(MASK64)
    out = np.empty(0, dtype=np.uint64)
    offset = 0
    while out.size < length:
        need = length - out.size
        draw = splitmix64(seed, 2 * need + 16, offset) & mask
        offset += 2 * need + 16
        out = np.concatenate([out, draw[draw < np.uint64(p)][:need]])
    return out.reshape(length, 1)
