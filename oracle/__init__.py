"""CPU oracle for the Montgomery-type reductions of Xu, Jia and Yang,
"Chinese Remainder Theorem Approach to Montgomery-Type Algorithms".

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / reference leg of ``bench.py`` may import, call or
execute anything in this package.  The library (``paper_2402_00675_gb300``)
never imports it and shares no code, table or helper with it.

Everything here is plain Python ``int`` arithmetic (arbitrary precision), so
nothing overflows and every floor is Python's ``//``.  Where the paper gives a
plain definition of the result (``T R^{-1} mod N`` and its signed and negated
forms) the oracle writes that definition out with a modular inverse; where the
paper gives an algorithm (REDC, Algorithms 1-4) the oracle evaluates the
algorithm's formula step by step in the paper's notation.  The only vectorised
code is ``oracle.exhaustive.count_candidate_failures_np``, which restates the same
formulas on numpy ``int64`` arrays for sizes where every intermediate is
provably below 2^62.

Modules
-------
montgomery : definitions, constants, REDC and Algorithms 1-4, domain maps.
exhaustive : exhaustive counterexample search of Section 3 (Example 3.1).
ntt        : Plantard's fixed-multiplier form (Section 3.2) and the negacyclic
             number-theoretic transform it serves (definitions, O(n^2)).
rns        : residue-number-system conversions by the CRT formula (Section 2).

Parity status: every public function is pinned by ``tests/test_oracle_pins.py``
(Qin's identity, Example 3.1, brute force over tiny moduli, the range theorems
and the inequality criterion of Section 3.3) and ``tests/test_oracle_ntt_pins.py``
(exhaustive prepared-multiplier products, a hand-derived transform, the
negacyclic convolution theorem) and ``tests/test_oracle_rns_pins.py`` (search on
tiny moduli, the two-modulus formula of Eq. (2)).  No function is parity-unpinned.
"""

from .montgomery import (  # noqa: F401
    REDC, SIGNED, PLANTARD, SIGNED_PLANTARD, SIGNED_PLANTARD2, VARIANTS,
    VARIANT_NAMES, mods, Constants, constants, precondition_ok, plantard_bound_ok,
    redc_value, sigredc_value, predc_value, sigpredc_value, reduce_value, mul_value,
    redc_alg, sigredc_alg, predc_alg, sigpredc1_alg, sigpredc2_alg, candidate,
    to_domain_value, from_domain_value, claimed_range, input_domain, sign_of,
    from_limbs, to_limbs,
)
from .exhaustive import sweep, SweepResult, count_candidate_failures_np  # noqa: F401
from . import ntt, rns  # noqa: F401
