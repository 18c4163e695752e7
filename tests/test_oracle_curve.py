"""Pins for the oracle's group law (no GPU).

The group law is pinned by facts of the curve that any mistake in it (a sign, a
dropped term, a swapped operand) would break: points stay on y^2 = x^3 + 1, the
generator has order r, a random point has order dividing #E = p + 1 - t, the
2-torsion point doubles to O, and two independent formula families (affine
chord/tangent and Jacobian, Python and C) agree.
"""
import random

import numpy as np

from oracle import coracle, fq, g1

RNG = random.Random(2024)


def rand_sub():
    return g1.mul(RNG.randrange(1, fq.R), g1.G)


def test_generator_on_curve_and_order_r():
    assert g1.on_curve(g1.G)
    assert g1.G is not None
    assert g1.mul(fq.R, g1.G) is None
    assert g1.jac_mul(fq.R, g1.G) is None
    assert g1.mul(fq.R - 1, g1.G) == g1.neg(g1.G)
    assert g1.mul(fq.R + 5, g1.G) == g1.mul(5, g1.G)


def test_random_curve_point_order_divides_group_order():
    for k in range(3):
        Q = g1.random_point(0x1234567 + 977 * k)
        assert g1.on_curve(Q)
        assert g1.mul(fq.CURVE_ORDER, Q) is None
        hQ = g1.mul(fq.COFACTOR, Q)
        assert g1.on_curve(hQ)
        assert g1.mul(fq.R, hQ) is None
        # a generic point is outside the order-r subgroup
        assert g1.mul(fq.R, Q) is not None


def test_two_torsion_point():
    T = (fq.P - 1, 0)  # (-1, 0): 0 = (-1)^3 + 1
    assert g1.on_curve(T)
    assert g1.add(T, T) is None
    assert g1.neg(T) == T
    assert g1.from_jac(g1.jac_double(g1.to_jac(T))) is None


def test_identity_and_inverse():
    P = rand_sub()
    assert g1.add(P, None) == P and g1.add(None, P) == P
    assert g1.add(P, g1.neg(P)) is None
    assert g1.add(None, None) is None
    assert g1.mul(0, P) is None


def test_small_multiples_by_repeated_addition():
    acc = None
    for k in range(1, 20):
        acc = g1.add(acc, g1.G)
        assert acc == g1.mul(k, g1.G) == g1.jac_mul(k, g1.G)
        assert g1.on_curve(acc)


def test_commutative_and_associative():
    for _ in range(12):
        a, b, c = rand_sub(), rand_sub(), g1.random_point(RNG.randrange(fq.P))
        assert g1.add(a, b) == g1.add(b, a)
        assert g1.add(g1.add(a, b), c) == g1.add(a, g1.add(b, c))
        assert g1.on_curve(g1.add(a, c))


def test_doubling_is_tangent_and_matches_jacobian():
    for _ in range(10):
        P = rand_sub()
        D = g1.add(P, P)
        x, y = P
        lam = 3 * x * x * fq.inv(2 * y) % fq.P
        assert D == ((lam * lam - 2 * x) % fq.P, (lam * (x - (lam * lam - 2 * x)) - y) % fq.P)
        assert g1.from_jac(g1.jac_double(g1.to_jac(P))) == D
        assert g1.from_jac(g1.jac_add(g1.to_jac(P), g1.to_jac(P))) == D


def test_jacobian_add_matches_affine_on_scaled_inputs():
    for _ in range(10):
        P, Q = rand_sub(), rand_sub()
        lam1, lam2 = RNG.randrange(1, fq.P), RNG.randrange(1, fq.P)
        j1 = (P[0] * lam1 ** 2 % fq.P, P[1] * lam1 ** 3 % fq.P, lam1)
        j2 = (Q[0] * lam2 ** 2 % fq.P, Q[1] * lam2 ** 3 % fq.P, lam2)
        assert g1.from_jac(g1.jac_add(j1, j2)) == g1.add(P, Q)
        assert g1.from_jac(g1.jac_add(j1, (Q[0] * lam1 ** 2 % fq.P, (-Q[1] * lam1 ** 3) % fq.P, lam1))) \
            == g1.add(P, g1.neg(Q))


def _lim(pt):
    return np.array(g1.to_limbs(pt), dtype=np.uint32)


def test_c_oracle_padd_matches_python_including_edge_cases():
    cases = []
    for _ in range(30):
        P, Q = rand_sub(), rand_sub()
        cases += [(P, Q), (P, P), (P, g1.neg(P)), (None, Q), (P, None), (None, None)]
    T = (fq.P - 1, 0)
    cases += [(T, T), (T, None)]
    for P, Q in cases:
        got = g1.from_limbs(coracle.padd(_lim(P), _lim(Q)))
        assert got == g1.add(P, Q)


def test_c_oracle_scalar_mul_and_generator_table():
    for k in [0, 1, 2, 3, 255, 256, 257, fq.R - 1, fq.R, fq.R + 1, (1 << 256) - 1]:
        got = g1.from_limbs(coracle.scalar_mul(_lim(g1.G), k))
        assert got == g1.mul(k % fq.R, g1.G)
    seeds = [0, 1, 2, 255, 256, 65535, 65536, fq.R - 1] + [RNG.randrange(fq.R) for _ in range(24)]
    arr = np.array([[(s >> (32 * i)) & 0xFFFFFFFF for i in range(8)] for s in seeds], dtype=np.uint32)
    pts = coracle.gen_points(arr, nthreads=2)
    for s, row in zip(seeds, pts):
        assert g1.from_limbs(row) == g1.mul(s, g1.G)


def test_c_oracle_padd_stream_matches_python_pairwise():
    """orc_padd_stream (the CPU mixed-PADD task rate) adds pair i alone, for every i,
    including P + P, P + (-P) and the identity in either slot."""
    rows_a, rows_q, want = [], [], []
    for k in range(40):
        P, Q = rand_sub(), rand_sub()
        pair = [(P, Q), (P, P), (P, g1.neg(P)), (None, Q), (P, None)][k % 5]
        rows_a.append(_lim(pair[0]))
        rows_q.append(_lim(pair[1]))
        want.append(g1.add(*pair))
    out = coracle.padd_stream(np.stack(rows_a), np.stack(rows_q))
    assert [g1.from_limbs(r) for r in out] == want


def test_closed_form_fast_dot_matches_term_by_term():
    """The exact float64-chunked sum used for large closed forms equals the plain sum,
    at extreme limb values and across a chunk boundary."""
    import synth
    from tests.util import dot_fast, dot_plain
    n = (1 << 18) + 37
    a = synth.scalars_full(5, n)
    s = synth.scalars_full(6, n)
    a[:100] = 0xFFFFFFFF
    s[:100] = 0xFFFFFFFF
    s[(1 << 18) - 3:(1 << 18) + 3] = 0xFFFFFFFF
    idx = list(range(0, 200)) + list(range((1 << 18) - 50, (1 << 18) + 37))
    assert dot_fast(a[idx], s[idx]) == dot_plain(a[idx], s[idx])
    assert dot_fast(a, s) == dot_plain(a, s)
