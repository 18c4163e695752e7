"""Pins for the oracle's field layer (no GPU).

Each check ties the oracle to something other than itself: primality and the
BLS12 family relations, Python's arbitrary-precision integers, the ranges and
identities the paper prints (tests/golden/paper_facts.txt).
"""
import random

import numpy as np
import pytest

import synth
from oracle import barrett, coracle, fq
from tests.golden.facts import paper_facts

FACTS = paper_facts()


def test_moduli_are_prime_and_sized():
    assert fq.is_probable_prime(fq.P)
    assert fq.is_probable_prime(fq.R)
    assert fq.P.bit_length() == FACTS["modulus_bits"]
    assert fq.R.bit_length() == 253
    assert not fq.is_probable_prime(fq.P + 2 * 3 * 5 * 7)  # the test itself rejects composites


def test_bls12_family_relations():
    x = fq.X0
    assert fq.R == x ** 4 - x ** 2 + 1
    assert 3 * (fq.P - x) == (x - 1) ** 2 * fq.R
    # group order p + 1 - t is a multiple of r, cofactor (x - 1)^2 / 3
    assert fq.CURVE_ORDER % fq.R == 0
    assert fq.COFACTOR == (x - 1) ** 2 // 3
    # p = 1 mod 2^46 (two-adicity used by Tonelli-Shanks) and p = 1 mod 3
    assert (fq.P - 1) % (1 << 46) == 0 and (fq.P - 1) % (1 << 47) != 0
    assert fq.P % 3 == 1


def test_synth_bounds_match_derived_constants():
    assert synth.P_INT == fq.P
    assert synth.R_INT == fq.R


def test_synth_is_deterministic_and_in_range():
    a1 = synth.scalars(123, 5000)
    a2 = synth.scalars(123, 5000)
    assert np.array_equal(a1, a2)
    vals = [synth.limbs_to_int(r) for r in a1]
    assert all(0 <= v < fq.R for v in vals)
    assert max(vals).bit_length() == 253
    e = synth.field_elems(9, 3000)
    ev = [synth.limbs_to_int(r) for r in e]
    assert all(0 <= v < fq.P for v in ev)
    assert max(ev).bit_length() == 377
    # distinct seeds give distinct streams
    assert not np.array_equal(synth.scalars(124, 10), a1[:10])


def _edge_values():
    vals = [0, 1, 2, fq.P - 1, fq.P - 2, (fq.P - 1) // 2, (fq.P + 1) // 2]
    vals += [(1 << k) % fq.P for k in (31, 32, 63, 64, 128, 255, 376, 383, 384, 400)]
    vals += [fq.P - (1 << k) for k in (32, 64, 200, 375)]
    return vals


def test_c_oracle_mul_matches_python_int():
    rng = random.Random(5)
    cases = [(a, b) for a in _edge_values() for b in _edge_values()]
    cases += [(rng.randrange(fq.P), rng.randrange(fq.P)) for _ in range(3000)]
    for a, b in cases:
        assert coracle.fq_mul(a, b) == a * b % fq.P


def test_inverses_agree_and_invert():
    rng = random.Random(6)
    for a in _edge_values()[1:] + [rng.randrange(1, fq.P) for _ in range(200)]:
        ia = fq.inv(a)                 # extended Euclid
        assert a * ia % fq.P == 1
        assert coracle.fq_inv(a) == ia  # Fermat in C
    with pytest.raises(ZeroDivisionError):
        fq.inv(0)


def test_sqrt():
    rng = random.Random(7)
    hits = 0
    for _ in range(200):
        a = rng.randrange(fq.P)
        r = fq.sqrt(a)
        if r is None:
            assert fq.legendre(a) == -1
        else:
            hits += 1
            assert r * r % fq.P == a
    assert 60 < hits < 140


# ---- the paper's own modular multiplication and carry scheme -------------

def test_barrett_range_sec_III_C():
    """Result of the three-multiplication Barrett step lies in [0, 3M) (Sec. III-C)."""
    M = fq.P
    assert FACTS["barrett_multiplications"] == 3
    rng = random.Random(8)
    xs = [0, 1, M - 1, M, M * M - 1, (M - 1) * (M - 1), (1 << 753), (1 << 754) - 1 - (1 << 700)]
    xs = [x for x in xs if x < M * M]
    xs += [rng.randrange(M * M) for _ in range(5000)]
    worst = 0
    for x in xs:
        r = barrett.barrett_reduce_coarse(x, M)
        assert 0 <= r < FACTS["barrett_range"] * M
        assert (r - x) % M == 0
        worst = max(worst, r // M)
    assert worst >= 1  # the correction step is really needed


def test_barrett_mulmod_exact():
    rng = random.Random(9)
    for _ in range(2000):
        a, b = rng.randrange(fq.P), rng.randrange(fq.P)
        assert barrett.barrett_mulmod(a, b, fq.P) == a * b % fq.P


def test_coarse_carry_sec_III_D():
    """Two rounds keep every element within 26 bits and preserve the value (Sec. III-D)."""
    assert barrett.ELEM_MASK == FACTS["coarse_mask"]
    assert barrett.ELEM_BITS == FACTS["coarse_shift"] == FACTS["element_bits"]
    assert barrett.LANES == FACTS["lanes"]
    assert FACTS["elements"] * FACTS["element_bits"] >= FACTS["modulus_bits"]
    rng = random.Random(10)
    for _ in range(3000):
        vec = [rng.randrange(1 << 32) for _ in range(barrett.LANES)]
        c_in = rng.randrange(1 << 7)
        out, carries = barrett.coarse_carry(vec, c_in)
        assert len(carries) == FACTS["coarse_rounds"]
        assert all(0 <= o < (1 << FACTS["element_capacity_bits"]) for o in out)
        lhs = barrett.from_elems(out) + ((carries[0] + carries[1]) << (25 * barrett.LANES))
        rhs = barrett.from_elems(vec) + c_in
        assert lhs == rhs
    for x in [0, 1, (1 << 25) - 1, 1 << 25, (1 << 32) - 1] + [rng.randrange(1 << 32) for _ in range(100)]:
        assert barrett.and_mask_by_shifts(x) == x & FACTS["coarse_mask"]


def test_elements_roundtrip():
    rng = random.Random(11)
    for _ in range(100):
        v = rng.randrange(fq.P)
        e = barrett.to_elems(v, FACTS["elements"])
        assert all(0 <= x < (1 << 25) for x in e)
        assert barrett.from_elems(e) == v


def test_loose_barrett_sec_III_E():
    """The looser reduction: operands below 6M, k = 378, remainder in [0, 4M) (Sec. III-E).
    The bound is proven for BLS12-377's p (exact fraction), then checked on random
    products, on the largest product and on products whose dropped low bits are all
    ones (the worst case of the first truncation)."""
    M = fq.P
    k, lo_in, lo_out = FACTS["loose_k"], FACTS["loose_input_range"], FACTS["loose_output_range"]
    assert barrett.LOOSE_K == k
    xmax = (lo_in * M) ** 2
    B = barrett.loose_bound(M, xmax, k)
    assert B < lo_out                          # x - q3 M < 4M for every x < (6M)^2 ...
    assert lo_out * M <= 1 << (k + 1)          # ... so the residue mod 2^(k+1) is exact
    rng = random.Random(12)
    xs = [0, 1, M - 1, M, xmax - 1, (lo_in * M - 1) ** 2, (lo_in * M - 1) * (3 * M)]
    xs += [rng.randrange(xmax) for _ in range(20000)]
    xs += [(rng.randrange(xmax >> (k - 1)) << (k - 1)) | ((1 << (k - 1)) - 1) for _ in range(5000)]
    worst = 0
    for x in (x for x in xs if x < xmax):
        r = barrett.barrett_reduce_loose(x, M, k)
        assert 0 <= r < lo_out * M and (r - x) % M == 0
        worst = max(worst, r)
    assert worst >= 3 * M                      # the range really is wider than Sec. III-C's [0, 3M)


def test_loose_barrett_needs_k_378():
    """With k = bitlen(M) = 377 the same step fails on operands below 6M: near the top
    of the product range its remainder no longer fits mod 2^(k+1)."""
    M = fq.P
    x = (6 * M - 1) ** 2
    r = barrett.barrett_reduce_loose(x, M, 377)
    assert (r - x) % M != 0
    assert barrett.loose_bound(M, x + 1, 377) * M > 1 << 378
