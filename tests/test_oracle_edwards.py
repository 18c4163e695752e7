"""Pins for the oracle's twisted Edwards model (no GPU).

The map and the Edwards law are pinned to the Weierstrass group law, not to
themselves: the map sends sums to sums (a dropped term or a wrong sign in the map
or in the Edwards formula breaks this on random pairs), it is invertible, images
satisfy the Edwards equation, the curve constants satisfy the relations of their
derivation, and the image of G has order r.
"""
import random

import pytest

from oracle import edwards as ed
from oracle import fq, g1

RNG = random.Random(377)
P = fq.P


def rand_sub():
    return g1.mul(RNG.randrange(1, fq.R), g1.G)


def test_constants_follow_their_derivation():
    s, a, d = ed.S, ed.A_TE, ed.D_TE
    assert s * s % P == 3
    # y^2 = (s u - 1)^3 + 1 is B v^2 = u^3 + A u^2 + u after dividing by s^3
    assert ed.A_MONT == (-3 * fq.inv(s)) % P
    assert ed.B_MONT * pow(s, 3, P) % P == 1
    assert a == (ed.A_MONT + 2) * fq.inv(ed.B_MONT) % P and d == (ed.A_MONT - 2) * fq.inv(ed.B_MONT) % P
    assert ed.GAMMA * ed.GAMMA % P == (-a) % P
    # scaled curve: a' = a / gamma^2 = -1, d' = d / gamma^2
    assert a * fq.inv(ed.GAMMA * ed.GAMMA % P) % P == P - 1
    assert ed.D == d * fq.inv(ed.GAMMA * ed.GAMMA % P) % P
    assert ed.K == 2 * ed.D % P
    assert ed.D not in (0, P - 1)
    # the curve is non-singular: a d (a - d) != 0
    assert (-1 * ed.D * (-1 - ed.D)) % P != 0


def test_generator_image_on_curve_with_order_r():
    Ge = ed.from_weierstrass(g1.G)
    assert ed.on_curve(Ge)
    assert ed.mul(fq.R, Ge) == ed.IDENTITY
    assert ed.mul(fq.R - 1, Ge) == ed.neg(Ge)


def test_identity_maps_to_edwards_identity():
    assert ed.from_weierstrass(None) == ed.IDENTITY
    assert ed.to_weierstrass(ed.IDENTITY) is None
    Pe = ed.from_weierstrass(rand_sub())
    assert ed.add(Pe, ed.IDENTITY) == Pe
    assert ed.add(Pe, ed.neg(Pe)) == ed.IDENTITY


def test_map_round_trip_and_curve_equation():
    for _ in range(8):
        Pw = rand_sub()
        Pe = ed.from_weierstrass(Pw)
        assert ed.on_curve(Pe)
        assert ed.to_weierstrass(Pe) == Pw
    # also off the subgroup, wherever the map is defined
    for k in range(4):
        Q = g1.random_point(0xED0 + 31 * k)
        Qe = ed.from_weierstrass(Q)
        assert ed.on_curve(Qe) and ed.to_weierstrass(Qe) == Q


def test_map_is_a_homomorphism():
    for _ in range(12):
        Pw, Qw = rand_sub(), rand_sub()
        Pe, Qe = ed.from_weierstrass(Pw), ed.from_weierstrass(Qw)
        assert ed.from_weierstrass(g1.add(Pw, Qw)) == ed.add(Pe, Qe)
        assert ed.from_weierstrass(g1.add(Pw, Pw)) == ed.add(Pe, Pe)      # doubling, same rule
        assert ed.from_weierstrass(g1.neg(Pw)) == ed.neg(Pe)
        assert ed.add(Pe, Qe) == ed.add(Qe, Pe)


def test_scalar_multiples_agree():
    Pw = rand_sub()
    Pe = ed.from_weierstrass(Pw)
    for k in (0, 1, 2, 3, 17, 2 ** 64 + 3, fq.R - 2):
        assert ed.from_weierstrass(g1.mul(k, Pw)) == ed.mul(k, Pe)


def test_two_torsion_is_outside_the_map():
    with pytest.raises(ValueError):
        ed.from_weierstrass((P - 1, 0))
    with pytest.raises(ValueError):
        ed.to_weierstrass((0, P - 1))


def test_stored_point_and_extended_form():
    Pe = ed.from_weierstrass(rand_sub())
    x, y, u = ed.stored_point(Pe)
    assert (x, y) == Pe and u == ed.K * x * y % P
    z = RNG.randrange(1, P)
    X, Y, Z, T = ed.extended(Pe, z)
    assert T * Z % P == X * Y % P
    assert ed.from_extended((X, Y, Z, T)) == Pe


def test_weierstrass_subgroup_membership():
    """r P = O decides membership of the order-r subgroup: the generator, its multiples,
    O and cofactor-cleared points are members; the 2-torsion point and a generic curve
    point (order divisible by a cofactor prime) are not."""

    assert ed.weierstrass_is_subgroup(g1.G)
    assert ed.weierstrass_is_subgroup(g1.mul(123456789, g1.G))
    assert ed.weierstrass_is_subgroup(None)
    assert not ed.weierstrass_is_subgroup((fq.P - 1, 0))
    Q = g1.random_point(0xC0FFEE)
    assert g1.on_curve(Q)
    assert not ed.weierstrass_is_subgroup(Q)
    assert ed.weierstrass_is_subgroup(g1.mul(fq.COFACTOR, Q))
