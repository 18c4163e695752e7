"""Pins for the oracle's GLV endomorphism and scalar split (no GPU).

phi is pinned to the group law: phi(P) equals lambda P computed by double-and-add,
and the integer identity lambda^2 + lambda + 1 = r ties lambda to the BLS12
polynomials. The split is pinned by recombination and its bounds, and the GLV
Pippenger by the naive sum.
"""
import random

from oracle import fq, g1, glv, msm

RNG = random.Random(2001)


def test_lambda_and_beta():
    lam = glv.LAMBDA
    assert lam * lam + lam + 1 == fq.R
    assert lam.bit_length() == 127
    b = glv.BETA
    assert pow(b, 3, fq.P) == 1 and b != 1
    assert (b * b + b + 1) % fq.P == 0


def test_phi_is_multiplication_by_lambda_on_the_subgroup():
    assert glv.phi(g1.G) == g1.mul(glv.LAMBDA, g1.G)
    for _ in range(4):
        Pw = g1.mul(RNG.randrange(1, fq.R), g1.G)
        assert glv.phi(Pw) == g1.mul(glv.LAMBDA, Pw)
        # phi^2 + phi + 1 = 0
        assert g1.add(g1.add(glv.phi(glv.phi(Pw)), glv.phi(Pw)), Pw) is None
    assert glv.phi(None) is None


def test_phi_is_not_lambda_off_the_subgroup():
    Q = g1.random_point(0x61F)
    assert g1.mul(fq.R, Q) is not None
    assert glv.phi(Q) != g1.mul(glv.LAMBDA, Q)


def test_decompose_recombines_within_bounds():
    lam = glv.LAMBDA
    cases = [0, 1, lam - 1, lam, lam + 1, fq.R - 1, fq.R, fq.R + 7, 2 ** 256 - 1]
    cases += [RNG.randrange(fq.R) for _ in range(200)]
    for k in cases:
        k1, k2 = glv.decompose(k)
        assert (k1 + lam * k2 - k) % fq.R == 0
        assert 0 <= k1 < lam and 0 <= k2 <= lam + 1
        assert k1 < 2 ** 127 and k2 < 2 ** 127


def test_glv_pippenger_equals_naive():
    for n, c in ((1, 4), (5, 3), (17, 5), (33, 8)):
        pts = [g1.mul(RNG.randrange(1, fq.R), g1.G) for _ in range(n)]
        sc = [RNG.randrange(fq.R) for _ in range(n)]
        assert glv.msm_glv(pts, sc, c) == msm.naive_msm(pts, sc)
