"""Whole-array forms of the definitions in ``oracle.montgomery``, so that
every element of a full-size output (2^26 products per vector, or 2^22
multi-limb products) can be compared with the definition in seconds.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): the library never
imports this module.

What each reduction returns is its plain definition (Section 1 for REDC,
the Ensure lines of Algorithms 1-4), exactly as ``mul_value`` states it:

* REDC                   ``T R^{-1} mod N``              in ``[0, N)``
* Algorithm 1 (SigRedc)  ``(T - m N) / R`` with ``m = T N^{-1} mods R``
                         (the one representative the algorithm picks, Eq. (5))
* Algorithm 2 (PRedc)    ``-T R^{-1} mod N``             in ``[0, N)``
* Algorithms 3 and 4     ``-T R^{-1} mods N``

with ``T = a b``.  Two evaluations are given:

``mul_value_u32``  numpy ``uint64``/``int64`` arithmetic for ``N < 2^32``:
    residues below N are multiplied in ``uint64`` (``N^2 < 2^64``), so every
    product and remainder is exact.  Algorithm 1 needs T itself: with
    ``|a|, |b| < 2^31`` the product fits ``int64``, ``T N^{-1} mod 2^32`` is
    the low word of a wrapping ``uint64`` product, and ``T - m N`` stays
    below ``2^63`` in absolute value.
``mul_value_obj``  numpy ``object`` arrays of Python integers: any width,
    nothing can overflow.

``ints_from_limbs`` / ``limbs_from_ints`` convert between little-endian
32-bit limb arrays (k limbs per element, element-major) and Python integers,
optionally read as k-limb two's complement.

Parity status: pinned by ``tests/test_oracle_bulk_pins.py`` against the scalar
``mul_value`` (itself pinned against the paper) on random and edge operands
of every variant at 32-bit, 64-bit and multi-limb widths.
"""

from __future__ import annotations

import numpy as np

from .montgomery import PLANTARD, REDC, SIGNED, SIGNED_PLANTARD, SIGNED_PLANTARD2

_U64 = np.uint64


def _mods_array(x, n):
    """``x mods n`` elementwise for ``0 <= x < n``: ``[-n/2, n/2)`` (Section 2)."""
    return np.where(2 * x >= n, x - n, x)


def mul_value_u32(variant: int, a, b, N: int, log2R: int, alpha: int = 0) -> np.ndarray:
    """The reduction of ``T = a b`` for every element, as ``int64``.

    ``a`` and ``b`` are integer arrays (any signed or unsigned dtype) with
    values below ``2^32`` in absolute value; ``N < 2^32`` is odd.  For
    Algorithm 1 the operands must satisfy ``|a|, |b| < 2^31`` and
    ``log2R <= 32`` (true for every admissible input of a 32-bit ctx, since
    ``2N < R``)."""
    if not (3 <= N < (1 << 32)) or N % 2 == 0:
        raise ValueError("mul_value_u32 needs an odd N < 2^32")
    a = np.asarray(a)
    b = np.asarray(b)
    R = 1 << log2R
    if variant == SIGNED:
        if log2R > 32:
            raise ValueError("Algorithm 1 path needs log2R <= 32")
        ai = a.astype(np.int64)
        bi = b.astype(np.int64)
        if np.abs(ai).max(initial=0) >= (1 << 31) or np.abs(bi).max(initial=0) >= (1 << 31):
            raise ValueError("Algorithm 1 path needs |a|, |b| < 2^31")
        T = ai * bi                                              # |T| < 2^62: exact
        Ninv = pow(N, -1, R)
        low = (T.view(_U64) * _U64(Ninv)) & _U64(R - 1)          # T N^{-1} mod R
        m = _mods_array(low.astype(np.int64), R)                 # ... mods R
        num = T - m * np.int64(N)                                # |num| < 2^63
        if np.any(num % R):
            raise AssertionError("T - mN not divisible by R")
        return num // R
    # residues of a and b in [0, N), multiplied exactly in uint64
    A = np.remainder(a.astype(np.int64), N).astype(_U64)
    B = np.remainder(b.astype(np.int64), N).astype(_U64)
    t = (A * B) % _U64(N)                                        # T mod N
    y = (t * _U64(pow(R, -1, N))) % _U64(N)                      # T R^{-1} mod N
    y = y.astype(np.int64)
    if variant == REDC:
        return y
    neg = np.where(y == 0, 0, N - y)                             # -T R^{-1} mod N
    if variant == PLANTARD:
        return neg
    if variant in (SIGNED_PLANTARD, SIGNED_PLANTARD2):
        return _mods_array(neg, N)
    raise ValueError(f"unknown variant {variant}")


def as_ints(x) -> np.ndarray:
    """An integer array as an ``object`` array of Python integers."""
    return np.asarray(x).astype(object)


def mul_value_obj(variant: int, a, b, N: int, log2R: int, alpha: int = 0) -> np.ndarray:
    """The reduction of ``T = a b`` for every element, in Python integers.

    ``a`` and ``b`` are ``object`` arrays of Python ints (or integer arrays,
    converted); the result is an ``object`` array."""
    A = a if getattr(a, "dtype", None) == object else as_ints(a)
    B = b if getattr(b, "dtype", None) == object else as_ints(b)
    R = 1 << log2R
    T = A * B
    if variant == SIGNED:
        m = _mods_array((T * pow(N, -1, R)) % R, R)              # T N^{-1} mods R
        num = T - m * N
        if np.any(num % R != 0):
            raise AssertionError("T - mN not divisible by R")
        return num // R
    y = ((T % N) * pow(R, -1, N)) % N                            # T R^{-1} mod N
    if variant == REDC:
        return y
    neg = (-y) % N                                               # -T R^{-1} mod N
    if variant == PLANTARD:
        return neg
    if variant in (SIGNED_PLANTARD, SIGNED_PLANTARD2):
        return _mods_array(neg, N)
    raise ValueError(f"unknown variant {variant}")


def ints_from_limbs(limbs, k: int, signed: bool = False) -> np.ndarray:
    """Elements of ``k`` little-endian 32-bit limbs as Python integers.

    ``limbs`` is a flat (or (n, k)) ``uint32``-compatible array; with
    ``signed`` each element is read as a k-limb two's complement integer."""
    arr = np.ascontiguousarray(np.asarray(limbs).reshape(-1, k).astype(np.uint32))
    raw = arr.astype("<u4").tobytes()
    w = 4 * k
    out = np.empty(arr.shape[0], dtype=object)
    out[:] = [int.from_bytes(raw[i * w:(i + 1) * w], "little", signed=signed)
              for i in range(arr.shape[0])]
    return out


def limbs_from_ints(x, k: int) -> np.ndarray:
    """Python integers (``object`` array or list) as ``k`` little-endian
    32-bit limbs each (two's complement for negative values), shape (n, k)."""
    w = 4 * k
    mod = 1 << (32 * k)
    raw = b"".join((int(v) % mod).to_bytes(w, "little") for v in x)
    return np.frombuffer(raw, dtype="<u4").reshape(-1, k).astype(np.uint32)
