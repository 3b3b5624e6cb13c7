"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these checks retypes the oracle's formula: each reaches the expected
value by another route -- the paper's printed numbers (Example 3.1), Qin's
identity (Theorem 2.1), brute-force search over all candidates on tiny inputs,
the range theorems of Sections 1 and 3, and the inequality criterion the
analysis of Section 3.3 derives.  The last tests plant mistakes in copies of
the oracle's functions and check that the pins catch them.
"""

import decimal
import itertools
import random

import pytest

import oracle as o
from oracle import exhaustive as sw
from conftest import read_golden


def odd_moduli(lo, hi):
    return [N for N in range(max(lo, 3), hi + 1) if N % 2]


# --------------------------------------------------------------------------
# mods notation (Section 2)
# --------------------------------------------------------------------------

def test_mods_is_the_unique_least_absolute_remainder():
    for n in range(1, 24):
        for x in range(-60, 61):
            # all y with y = x (mod n) and -n/2 <= y < n/2, found by search
            cands = [y for y in range(-n, n + 1) if (x - y) % n == 0 and -n <= 2 * y < n]
            assert len(cands) == 1
            assert o.mods(x, n) == cands[0]


def test_mods_even_modulus_keeps_minus_half():
    assert o.mods(8, 16) == -8 and o.mods(-8, 16) == -8 and o.mods(7, 16) == 7


# --------------------------------------------------------------------------
# Qin's identity (Theorem 2.1) pins the two inverses the oracle computes
# --------------------------------------------------------------------------

def test_qin_identity_for_oracle_constants():
    rnd = random.Random(7)
    cases = [(N, l) for l in range(2, 13) for N in odd_moduli(3, (1 << l) + 40)]
    cases += [(rnd.randrange(3, 1 << 64) | 1, l) for l in (32, 64, 128) for _ in range(200)]
    cases += [(rnd.randrange(1 << 255, 1 << 256) | 1, 256) for _ in range(50)]
    for N, l in cases:
        c = o.constants(N, l)
        assert 1 <= c.Ninv < c.R and 1 <= c.Rinv < N
        # R^{-1} R + N^{-1} N = 1 + N R
        assert c.Rinv * c.R + c.Ninv * N == 1 + N * c.R


def test_qin_identity_determines_the_inverses():
    # Theorem 2.1's proof: N^{-1} N = 1 + l R with l < N and R^{-1} = N - l.
    for l in range(3, 11):
        R = 1 << l
        for N in odd_moduli(3, 3 * R):
            c = o.constants(N, l)
            ell, rem = divmod(c.Ninv * N - 1, R)
            assert rem == 0 and 0 <= ell < N
            assert c.Rinv == N - ell


def test_nprime_sign_convention():
    # Section 1: N' = R - (N^{-1} mod R), so N N' = -1 (mod R).
    for l in (4, 8, 16, 32, 64):
        for N in (3, 5, 3329, 8380417, (1 << l) - 1 if l > 2 else 3):
            if N >= (1 << l):
                continue
            c = o.constants(N, l)
            assert (N * c.Nprime + 1) % c.R == 0
            assert 0 < c.Nprime < c.R


def test_constants_of_known_moduli():
    # values fixed by N N^{-1} = 1 (mod R), checked by multiplication
    for N, l in ((3329, 32), (8380417, 32), (3329, 64), (8380417, 64)):
        c = o.constants(N, l)
        assert (N * c.Ninv) % c.R == 1
        assert (c.R2_mod_N - c.R * c.R) % N == 0 and 0 <= c.R2_mod_N < N


# --------------------------------------------------------------------------
# Example 3.1 (Section 3.3): every printed value
# --------------------------------------------------------------------------

def test_example_3_1_printed_values():
    g = read_golden("example_3_1.txt")
    n, N, alpha, T = g["n"], g["N"], g["alpha"], g["T"]
    log2R = 2 * n
    c = o.constants(N, log2R)
    assert c.R == g["R"]
    assert N < (1 << (n - alpha - 1))
    assert o.precondition_ok(o.SIGNED_PLANTARD2, N, log2R, alpha)
    assert c.Ninv_s == g["Ninv_mods_R"]
    m = o.mods(T * c.Ninv_s, c.R)
    assert m == g["m"]
    assert (m * N - T) // (1 << n) == g["mN_minus_T_over_2n"]
    assert ((m >> n) + 1) * N == g["floor_m_over_2n_plus_1_times_N"]
    assert o.sigpredc2_alg(T, N, log2R, alpha) == g["algorithm_output"]
    assert o.sigpredc_value(T, N, c.R) == g["correct"]
    assert o.claimed_range(o.SIGNED_PLANTARD2, N) == (g["range_lo"], g["range_hi"])


def test_example_3_1_found_by_the_sweep():
    g = read_golden("example_3_1.txt")
    res = o.sweep(o.SIGNED_PLANTARD2, 2 * g["n"], g["alpha"], g["N"], g["N"])
    assert (g["N"], g["T"], g["algorithm_output"], g["correct"]) in res.examples


# --------------------------------------------------------------------------
# Definitions against brute force on tiny inputs
# --------------------------------------------------------------------------

def brute_r_times_R(T, N, R, sign, lo, hi):
    """All r in [lo, hi] with r R = sign T (mod N), by search."""
    return [r for r in range(lo, hi + 1) if (r * R - sign * T) % N == 0]


@pytest.mark.parametrize("l", [2, 3, 4, 5, 6])
def test_value_definitions_by_search(l):
    R = 1 << l
    for N in odd_moduli(3, 4 * R + 3):
        for T in range(-3 * N, 3 * N + 5):
            assert [o.redc_value(T, N, R)] == brute_r_times_R(T, N, R, +1, 0, N - 1)
            assert [o.predc_value(T, N, R)] == brute_r_times_R(T, N, R, -1, 0, N - 1)
            lo, hi = -(N // 2), (N - 1) // 2
            assert [o.sigpredc_value(T, N, R)] == brute_r_times_R(T, N, R, -1, lo, hi)


@pytest.mark.parametrize("l", [3, 4, 5, 6])
def test_sigredc_value_by_search_of_m(l):
    # Eq. (5) with m the unique m = T N^{-1} (mods R): search m in [-R/2, R/2)
    R = 1 << l
    for N in odd_moduli(3, R // 2 - 1):
        for T in range(-(N * R) // 2 + 1, (N * R) // 2, max(1, N // 3)):
            ms = [m for m in range(-R // 2, R // 2) if (T - m * N) % R == 0]
            assert len(ms) == 1
            assert o.sigredc_value(T, N, R) == (T - ms[0] * N) // R


# --------------------------------------------------------------------------
# Algorithms equal the definitions on their whole domains (theorems of
# Sections 1 and 3); outputs lie in the claimed ranges.
# --------------------------------------------------------------------------

@pytest.mark.parametrize("l", [3, 4, 5, 6, 7])
def test_redc_algorithm_exhaustive(l):
    R = 1 << l
    for N in odd_moduli(3, R - 1):
        for T in range(0, R * N):
            r = o.redc_alg(T, N, l)
            assert 0 <= r < N
            assert r == o.redc_value(T, N, R)


@pytest.mark.parametrize("l", [3, 4, 5, 6, 7])
def test_sigredc_algorithm_exhaustive(l):
    R = 1 << l
    for N in odd_moduli(3, R // 2 - 1):
        lo, hi = o.input_domain(o.SIGNED, N, l)
        for T in range(lo, hi + 1):
            r = o.sigredc_alg(T, N, l)
            assert -N < r < N                     # Algorithm 1's Ensure line
            assert (r * R - T) % N == 0
            assert r == o.sigredc_value(T, N, R)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_plantard_algorithms_exhaustive(n):
    l = 2 * n
    R = 1 << l
    for N in odd_moduli(3, 1 << n):
        if o.plantard_bound_ok(N, n):
            for T in range(0, N * N + 1):
                r = o.predc_alg(T, N, l)
                assert 0 <= r < N and r == o.predc_value(T, N, R)
                # the Remark after Algorithm 2: the raw formula is already < N
                m = (T * o.constants(N, l).Ninv) % R
                assert ((m >> n) + 1) * N >> n < N
        if N < (1 << (n - 1)):
            b = 1 << (2 * n - 2)
            for T in range(-b, b + 1):
                r = o.sigpredc1_alg(T, N, l)
                assert r == o.sigpredc_value(T, N, R)
        for alpha in (1, 2):
            if n - alpha - 1 >= 0 and N < (1 << (n - alpha - 1)):
                b = (1 << (2 * alpha)) * N * N
                for T in range(-b, b + 1):
                    assert o.sigpredc2_alg(T, N, l, alpha) == o.sigpredc_value(T, N, R)


@pytest.mark.parametrize("n", [4, 6, 8])
def test_plantard_exact_on_the_wider_domain(n):
    """Algorithm 2 returns -T R^{-1} mod N exactly for every 0 <= T <= N 2^n once
    N <= 2^{n-1} (a wider domain than the paper's T <= N^2, used by the lazy NTT).
    With m = T N^{-1} mod 2^{2n} = m1 2^n + m0 and k = (mN - T)/2^{2n}, the output is
    floor(k + d), d = (N 2^n + m0 N - T)/2^{2n}, and 0 <= d < 1 on that domain.
    Both conditions are needed: outside either, some (N, T) fail."""
    l = 2 * n
    R = 1 << l
    beyond_fails = 0
    for N in odd_moduli(3, 1 << (n - 1)):
        want = lambda T: (-T * pow(R, -1, N)) % N
        for T in range(0, (N << n) + 1):
            assert o.predc_alg(T, N, l) == want(T), (n, N, T)
        beyond_fails += sum(o.predc_alg(T, N, l) != want(T)
                            for T in range((N << n) + 1, (N << n) + (4 << n)))
    assert beyond_fails > 0                  # the bound on T is not vacuous
    N = (1 << (n - 1)) + 1                   # just above 2^{n-1}, inside 2^n / phi
    assert o.plantard_bound_ok(N, n)
    assert any(o.predc_alg(T, N, l) != (-T * pow(R, -1, N)) % N for T in range(0, (N << n) + 1))


def test_plantard_bound_exact_against_decimal():
    decimal.getcontext().prec = 80
    phi = (1 + decimal.Decimal(5).sqrt()) / 2
    for n in range(2, 40):
        bound = (decimal.Decimal(2) ** n) / phi
        base = int(bound)
        for N in range(max(1, base - 6), base + 7):
            assert o.plantard_bound_ok(N, n) == (decimal.Decimal(N) < bound)


# --------------------------------------------------------------------------
# Section 3.3's analysis: Algorithm 4 is right iff two inequalities hold.
# Count their violations independently and compare with the sweep.
# --------------------------------------------------------------------------

def inequality_failures(n, alpha):
    """(N, T) pairs where (mN-T)/2^n <= (floor(m/2^n)+2^a)N < (mN+R-T)/2^n fails.

    N^{-1} is found by search and m by searching the mods-R residue class,
    not through the oracle."""
    R = 1 << (2 * n)
    out = set()
    for N in odd_moduli(3, (1 << (n - alpha - 1)) - 1):
        ninv = next(x for x in range(1, R) if (N * x) % R == 1)
        b = (1 << (2 * alpha)) * N * N
        for T in range(-b, b + 1):
            m = (T * ninv) % R
            if 2 * m >= R:
                m -= R
            q = m // (1 << n)
            lhs = (m * N - T)                    # times 1/2^n
            mid = (q + (1 << alpha)) * N * (1 << n)
            rhs = (m * N + R - T)
            if not (lhs <= mid < rhs):
                out.add((N, T))
    return out


@pytest.mark.parametrize("n,alpha", [(4, 0), (5, 0), (6, 0), (5, 1), (6, 1), (7, 1)])
def test_alpha_counterexamples_match_the_inequality_criterion(n, alpha):
    res = o.sweep(o.SIGNED_PLANTARD2, 2 * n, alpha, 3, 1 << n)
    found = {(N, T) for (N, T, r, e) in res.examples}
    assert found == inequality_failures(n, alpha)
    if alpha >= 1:
        assert res.total == 0                    # Section 3.3: correct for alpha >= 1


def test_alpha0_fails_at_n8_and_alpha1_does_not():
    r0 = o.sweep(o.SIGNED_PLANTARD2, 16, 0, 3, 127, vectorised=True)
    r1 = o.sweep(o.SIGNED_PLANTARD2, 16, 1, 3, 63, vectorised=True)
    assert r0.total > 0 and r1.total == 0


# --------------------------------------------------------------------------
# Sweep: in-spec algorithms have no counterexample (theorems), both
# implementations agree, and out-of-domain inputs do produce failures.
# --------------------------------------------------------------------------

@pytest.mark.parametrize("variant,alpha", [(0, 0), (1, 0), (2, 0), (3, 0), (4, 1)])
def test_sweep_zero_in_spec(variant, alpha):
    for l in (6, 8):
        res = o.sweep(variant, l, alpha, 3, 63, vectorised=True)
        assert res.total == 0, (variant, l, res.examples[:3])


@pytest.mark.parametrize("variant,alpha", [(0, 0), (1, 0), (2, 0), (3, 0), (4, 0), (4, 1)])
def test_sweep_numpy_equals_python(variant, alpha):
    for dom in (sw.DOMAIN_DEFAULT, sw.DOMAIN_REDC):
        a = o.sweep(variant, 8 if variant < 2 else 6, alpha, 3, 33, domain=dom,
                    include_out_of_spec=True)
        b = o.sweep(variant, 8 if variant < 2 else 6, alpha, 3, 33, domain=dom,
                    include_out_of_spec=True, vectorised=True)
        assert a.counts == b.counts and a.examples == b.examples


def test_sweep_outside_domain_fails():
    # Algorithm 1 evaluated on REDC's domain [0, RN) leaves its range
    res = o.sweep(o.SIGNED, 8, 0, 3, 63, domain=sw.DOMAIN_REDC)
    assert res.total > 0
    # Plantard above N < 2^n / phi: the first odd N past the bound fails at n = 8
    res = o.sweep(o.PLANTARD, 16, 0, 151, 161, include_out_of_spec=True, vectorised=True)
    bad = sorted(N for N, c in res.counts.items() if c)
    assert bad and bad[0] == 159 and not o.plantard_bound_ok(159, 8)
    assert o.plantard_bound_ok(157, 8)


def test_sweep_expected_values_are_canonical():
    res = o.sweep(o.SIGNED_PLANTARD2, 12, 0, 3, 31)
    for N, T, r, e in res.examples:
        assert -(N // 2) <= e <= (N - 1) // 2
        assert ((e * (1 << 12)) + T) % N == 0        # e R = -T (mod N)


# --------------------------------------------------------------------------
# Multi-limb REDC and the domain maps
# --------------------------------------------------------------------------

def test_multilimb_redc_by_multiplication():
    rnd = random.Random(11)
    for k in (8, 12, 32, 64):
        l = 32 * k
        R = 1 << l
        for _ in range(20):
            N = rnd.randrange(1 << (l - 1), R) | 1
            a, b = rnd.randrange(N), rnd.randrange(N)
            r = o.mul_value(o.REDC, a, b, N, l)
            assert 0 <= r < N and (r * R - a * b) % N == 0
            assert o.from_limbs(o.to_limbs(r, k)) == r


def test_limbs_little_endian():
    assert o.to_limbs(0x0000000100000002, 2) == [2, 1]
    assert o.from_limbs([0xFFFFFFFF, 0, 1]) == 0xFFFFFFFF + (1 << 64)


@pytest.mark.parametrize("variant,l", [(0, 16), (1, 16), (2, 16), (3, 16), (4, 16),
                                       (0, 32), (1, 32), (2, 64), (3, 64), (4, 64)])
def test_domain_maps_round_trip(variant, l):
    rnd = random.Random(variant * 100 + l)
    for N in (3, 5, 31, 61, 101, 127):
        if not o.precondition_ok(variant, N, l, 1):
            continue
        R = 1 << l
        s = o.sign_of(variant)
        signed = variant in (1, 3, 4)
        xs = range(-(N // 2), (N - 1) // 2 + 1) if signed else range(N)
        for x in xs:
            y = o.to_domain_value(variant, x, N, l, 1)
            assert (y - s * x * R) % N == 0           # Φ(x) = s x R (mod N)
            assert o.from_domain_value(variant, y, N, l, 1) == x
        for _ in range(50):
            a, b = rnd.randrange(N), rnd.randrange(N)
            if signed:
                a, b = o.mods(a, N), o.mods(b, N)
            ya, yb = o.to_domain_value(variant, a, N, l, 1), o.to_domain_value(variant, b, N, l, 1)
            prod = o.mul_value(variant, ya, yb, N, l, 1)
            back = o.from_domain_value(variant, prod, N, l, 1)
            want = (a * b) % N
            assert (back - want) % N == 0


# --------------------------------------------------------------------------
# Planted mistakes in copies of the oracle: the pins above must catch them
# --------------------------------------------------------------------------

def test_planted_mistakes_are_caught():
    # 1. PRedc without the "+1" of Algorithm 2
    def predc_no_plus1(T, N, l):
        n = l // 2
        m = (T * o.constants(N, l).Ninv) % (1 << l)
        return (m >> n) * N >> n
    assert any(predc_no_plus1(T, 31, 12) != o.predc_value(T, 31, 1 << 12) for T in range(0, 31 * 31 + 1))

    # 2. REDC with the sign of N' flipped (m = T N^{-1} instead of T N')
    def redc_wrong_sign(T, N, l):
        c = o.constants(N, l)
        m = ((T % c.R) * c.Ninv) % c.R
        t = (T + m * N) // c.R
        return t - N if t >= N else t
    assert any(redc_wrong_sign(T, 13, 6) != o.redc_value(T, 13, 64) for T in range(0, 13 * 64))

    # 3. SigRedc with mod instead of mods for m0 (the representative changes)
    def sigredc_mod(T, N, l):
        c = o.constants(N, l)
        a0 = T % c.R
        a1 = (T - a0) // c.R
        return a1 - (((a0 * c.Ninv) % c.R) * N) // c.R
    lo, hi = o.input_domain(o.SIGNED, 13, 6)
    assert any(sigredc_mod(T, 13, 6) != o.sigredc_value(T, 13, 64) for T in range(lo, hi + 1))

    # 4. SigPRedc1 with floor instead of rounding on the outer step
    def sigpredc1_floor(T, N, l):
        c = o.constants(N, l)
        n = l // 2
        m = o.mods(T * c.Ninv_s, c.R)
        q = (m + (1 << (n - 1))) >> n
        return (q * N) >> n
    assert any(sigpredc1_floor(T, 29, 12) != o.sigpredc_value(T, 29, 1 << 12)
               for T in range(-1024, 1025))

    # 5. mods with a closed right end ([-n/2, n/2] keeps +n/2)
    def mods_closed(x, n):
        r = x % n
        return r - n if 2 * r > n else r
    assert any(mods_closed(x, 8) != o.mods(x, 8) for x in range(-20, 20))
