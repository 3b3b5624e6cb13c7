"""Host model of the multi-limb kernels' blocked product (k >= 32 limbs).

The kernel forms out = a b mod 2^{32M} as a schoolbook over 16 x 16-limb
blocks: row I of blocks multiplies a's block I by every block of b, adds each
block product's low half into the output block it lands on (written by row
I-1, or zero in row 0), carries its high half to the next block in registers
and writes the block above the row first.  This model follows the same
steps with Python integers and checks the bounds the kernel relies on: every
column sum fits a 96-bit accumulator, every carry between columns fits 64
bits, and nothing carries past the block a row writes first (so that block
needs no read of earlier contents).  It is a check of the scheme, not of the
CUDA code, which the GPU parity tests compare with the oracle."""

import random

import pytest

B = 16
W = 1 << 32


def limbs(x, n):
    return [(x >> (32 * i)) & (W - 1) for i in range(n)]


def value(ls):
    return sum(v << (32 * i) for i, v in enumerate(ls))


def block_mac(ra, rb, o, has_old, hi, tc, low_only):
    """One block product accumulated: returns the carry past column 31."""
    carry = 0
    for col in range(B if low_only else 2 * B):
        s = carry
        if col < B:
            s += (o[col] if has_old else 0) + hi[col]
        elif col == B:
            s += tc
        for i in range(B):
            j = col - i
            if 0 <= j < B:
                s += ra[i] * rb[j]
        assert s < 1 << 96
        if col < B:
            o[col] = s & (W - 1)
        else:
            hi[col - B] = s & (W - 1)
        carry = s >> 32
        assert carry < 1 << 64
    return 0 if low_only else carry


def mul_blocked(a, b, KA, KB, M):
    NA, NB, NM = KA // B, KB // B, M // B
    out = [None] * M   # never read before written
    for I in range(min(NA, NM)):
        ra, hi, tc = a[B * I:B * I + B], [0] * B, 0
        for J in range(NB):
            if I + J >= NM:
                break
            o = out[B * (I + J):B * (I + J) + B]
            tc = block_mac(ra, b[B * J:B * J + B], o, I > 0, hi, tc, I + J == NM - 1)
            out[B * (I + J):B * (I + J) + B] = o
        if I + NB < NM:
            assert tc == 0
            out[B * (I + NB):B * (I + NB) + B] = hi
    return out


# (KA, KB, M) as the kernels call it at k = 32 and 64: a b, Algorithm 1's m,
# the Plantard family's m, and the truncated and rectangular cases
SHAPES = [(32, 32, 64), (32, 32, 32), (64, 64, 64), (64, 64, 128), (128, 128, 128),
          (16, 16, 32), (32, 16, 48), (16, 32, 32)]


@pytest.mark.parametrize("KA,KB,M", SHAPES)
def test_blocked_product_equals_integer_product(KA, KB, M):
    rnd = random.Random(KA * 1000 + KB * 10 + M)
    ones_a, ones_b = (1 << (32 * KA)) - 1, (1 << (32 * KB)) - 1
    cases = [(ones_a, ones_b), (ones_a - rnd.getrandbits(40), ones_b), (0, ones_b), (1, 1)]
    cases += [(rnd.getrandbits(32 * KA), rnd.getrandbits(32 * KB)) for _ in range(20)]
    for x, y in cases:
        got = mul_blocked(limbs(x, KA), limbs(y, KB), KA, KB, M)
        assert value(got) == (x * y) % (1 << (32 * M))
