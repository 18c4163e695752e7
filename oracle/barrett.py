"""The paper's own modular multiplication and carry scheme — test infrastructure only.

Sec. III-C: a*b mod M by Barrett reduction in three multiplications:
  mul_in = a*b;  mul_mu = (high part of mul_in) * mu;  mul_m = (high part of
  mul_mu) * M;  result = low part of mul_in - low part of mul_m, which lies in
  [0, 3M). Written here at bit granularity (HAC Alg. 14.42 with base 2): with
  k = bitlen(M), mu = floor(2^(2k) / M), the "high parts" are shifts by k-1 and
  k+1 bits and the "low parts" are residues mod 2^(k+1).

Sec. III-E: the looser reduction for operands in [0, 6M) (k = 378), below.

Sec. III-B / III-D: a 377-bit integer is held as 16 elements of 25 bits packed
into two 8-lane vectors; each element may grow to 26 bits. Coarse carry
propagation runs two rounds of
  o = in & 0x1ffffff ;  c = in >> 25 ;  c = [c_in] ++ c[0:7] ;  o = o + c
on an 8-lane vector, with the block's incoming carry c_in in the first round and
0 in the second; the AND is replaced by x - ((x >> 25) << 25).
"""
from __future__ import annotations

ELEM_BITS = 25
ELEM_MASK = (1 << ELEM_BITS) - 1      # 0x1ffffff
LANES = 8


def barrett_params(M: int):
    k = M.bit_length()
    return k, (1 << (2 * k)) // M


def barrett_reduce_coarse(x: int, M: int) -> int:
    """The three-multiplication Barrett step without the final correction (result in [0, 3M))."""
    k, mu = barrett_params(M)
    q1 = x >> (k - 1)                  # high part of mul_in
    q3 = (q1 * mu) >> (k + 1)          # high part of mul_mu
    mod = 1 << (k + 1)
    r = (x % mod) - ((q3 * M) % mod)   # low(mul_in) - low(mul_m)
    if r < 0:
        r += mod
    return r


# Sec. III-E: with the fine reduction [0, 3M) -> [0, M) skipped after the first
# multiplications and 3M added to differences, the operands of the final
# multiplications lie in [0, 6M); a looser Barrett step with "a parameter k set to
# 378" still brings the product into [0, 4M). Reading: the step above with the bit
# length k = 378 in place of bitlen(M) = 377.
LOOSE_K = 378


def barrett_reduce_loose(x: int, M: int, k: int = LOOSE_K) -> int:
    """q1 = floor(x / 2^(k-1)), mu = floor(2^(2k) / M), q3 = floor(q1 mu / 2^(k+1)),
    r = (x - q3 M) mod 2^(k+1), no correction step."""
    mu = (1 << (2 * k)) // M
    q3 = ((x >> (k - 1)) * mu) >> (k + 1)
    mod = 1 << (k + 1)
    return ((x % mod) - (q3 * M) % mod) % mod


def loose_bound(M: int, xmax: int, k: int = LOOSE_K):
    """A bound B with x - q3 M < B M for 0 <= x < xmax, as an exact fraction.

    With q1 = x / 2^(k-1) - e1 and mu = 2^(2k) / M - e2 (e1 in [0, 1), e2 the fixed
    fractional part of 2^(2k) / M), x / M - q1 mu / 2^(k+1) = e2 x / 2^(2k)
    + e1 2^(k-1) / M - e1 e2 / 2^(k+1) <= e2 x / 2^(2k) + 2^(k-1) / M, and the floor
    of q3 adds less than 1: B = 1 + e2 xmax / 2^(2k) + 2^(k-1) / M. Also
    x - q3 M >= 0, since q3 <= x / M. When B M <= 2^(k+1) the remainder taken
    mod 2^(k+1) is the exact x - q3 M."""
    from fractions import Fraction
    e2 = Fraction(1 << (2 * k), M) - ((1 << (2 * k)) // M)
    return 1 + e2 * Fraction(xmax, 1 << (2 * k)) + Fraction(1 << (k - 1), M)


def barrett_mulmod(a: int, b: int, M: int) -> int:
    r = barrett_reduce_coarse(a * b, M)
    while r >= M:
        r -= M
    return r


def and_mask_by_shifts(x: int) -> int:
    """x & 0x1ffffff computed with shifts and a subtraction only (Sec. III-D)."""
    return x - ((x >> ELEM_BITS) << ELEM_BITS)


def to_elems(v: int, n: int = 16) -> list[int]:
    return [(v >> (ELEM_BITS * i)) & ELEM_MASK for i in range(n)]


def from_elems(e) -> int:
    return sum(int(x) << (ELEM_BITS * i) for i, x in enumerate(e))


def coarse_carry_round(vec, c_in: int):
    """One round on an 8-lane vector; returns (out, carry leaving lane 7)."""
    o = [and_mask_by_shifts(x) for x in vec]
    c = [x >> ELEM_BITS for x in vec]
    shifted = [c_in] + c[:-1]
    return [oi + ci for oi, ci in zip(o, shifted)], c[-1]


def coarse_carry(vec, c_in: int):
    """Two rounds (step0 with c_in, step1 with 0); returns (out, [carry0, carry1])."""
    o0, k0 = coarse_carry_round(vec, c_in)
    o1, k1 = coarse_carry_round(o0, 0)
    return o1, [k0, k1]
