"""Pins for the oracle's MSM (no GPU).

sum_i s_i P_i is unique; Pippenger (Sec. II-C) is a schedule for it. Pins:
brute force by repeated addition on tiny inputs, naive = Pippenger (unsigned and
signed digits, several window sizes, Python and C), the closed form for points
with known discrete logs, linearity in the scalars, and exact digit
reconstruction.
"""
import random

import numpy as np
import pytest

import synth
from oracle import coracle, fq, g1, msm

RNG = random.Random(77)


def _pts(seeds):
    arr = np.array([[(s >> (32 * i)) & 0xFFFFFFFF for i in range(8)] for s in seeds], dtype=np.uint32)
    return coracle.gen_points(arr, nthreads=2)


def _sc(vals):
    return np.array([[(v >> (32 * i)) & 0xFFFFFFFF for i in range(8)] for v in vals], dtype=np.uint32)


def test_brute_force_tiny():
    for n in range(0, 5):
        for _ in range(4):
            seeds = [RNG.randrange(1, fq.R) for _ in range(n)]
            ks = [RNG.randrange(0, 17) for _ in range(n)]
            pts = [g1.mul(s, g1.G) for s in seeds]
            ref = None
            for P, k in zip(pts, ks):
                for _ in range(k):
                    ref = g1.add(ref, P)
            assert msm.naive_msm(pts, ks) == ref
            for c in (1, 2, 3, 5):
                assert msm.pippenger(pts, ks, c, scalar_bits=5) == ref
                if c >= 2:
                    assert msm.pippenger(pts, ks, c, signed=True, scalar_bits=5) == ref
            if n:
                assert g1.from_limbs(coracle.msm(_pts(seeds), _sc(ks), c=3)) == ref
                assert g1.from_limbs(coracle.msm_naive(_pts(seeds), _sc(ks))) == ref


def test_empty_msm_is_identity():
    assert msm.naive_msm([], []) is None
    assert msm.pippenger([], [], 8) is None
    out = coracle.msm(np.zeros((0, 24), np.uint32), np.zeros((0, 8), np.uint32), c=8)
    assert not out.any()


@pytest.mark.parametrize("c,signed", [(4, False), (8, False), (5, True), (8, True), (13, True)])
def test_pippenger_equals_naive(c, signed):
    n = 12
    seeds = [RNG.randrange(1, fq.R) for _ in range(n)]
    ks = [RNG.randrange(fq.R) for _ in range(n)]
    pts = [g1.mul(s, g1.G) for s in seeds]
    ref = msm.naive_msm(pts, ks)
    assert msm.pippenger(pts, ks, c, signed=signed, scalar_bits=253) == ref
    assert ref == msm.closed_form(seeds, ks)


def test_c_pippenger_closed_form_and_duplicates():
    n = 300
    a, s = synth.workloads.msm(n, 99)
    pts = coracle.gen_points(s, nthreads=2)
    # duplicate and negated points exercise P+P and P+(-P) inside buckets
    pts[10] = pts[11]
    s[10] = s[11]
    pts[20] = pts[21]
    pts[20, 12:] = synth.int_to_limbs((fq.P - synth.limbs_to_int(pts[21, 12:])) % fq.P, 12)
    s[20] = synth.int_to_limbs((fq.R - synth.limbs_to_int(s[21])) % fq.R, 8)
    a[30] = 0
    ai = [synth.limbs_to_int(x) for x in a]
    si = [synth.limbs_to_int(x) for x in s]
    ref = msm.closed_form(si, ai)
    for c in (3, 7, 8, 11):
        assert g1.from_limbs(coracle.msm(pts, a, c=c)) == ref
    assert g1.from_limbs(coracle.msm_naive(pts, a)) == ref


def test_linearity():
    n = 40
    a, s = synth.workloads.msm(n, 5)
    b = synth.scalars(1234, n)
    pts = coracle.gen_points(s, nthreads=2)
    ai = [synth.limbs_to_int(x) for x in a]
    bi = [synth.limbs_to_int(x) for x in b]
    sab = _sc([(x + y) % fq.R for x, y in zip(ai, bi)])
    lam = RNG.randrange(fq.R)
    sl = _sc([x * lam % fq.R for x in ai])
    A = g1.from_limbs(coracle.msm(pts, a, c=6))
    B = g1.from_limbs(coracle.msm(pts, b, c=6))
    assert g1.from_limbs(coracle.msm(pts, sab, c=6)) == g1.add(A, B)
    assert g1.from_limbs(coracle.msm(pts, sl, c=6)) == g1.mul(lam, A)


def test_scalars_at_or_above_r():
    seeds = [RNG.randrange(1, fq.R) for _ in range(6)]
    ks = [fq.R, fq.R + 1, (1 << 256) - 1, 2 * fq.R + 7, 0, fq.R - 1]
    pts = _pts(seeds)
    ref = msm.closed_form(seeds, [k % fq.R for k in ks])
    assert g1.from_limbs(coracle.msm(pts, _sc(ks), c=5)) == ref


@pytest.mark.parametrize("c", [2, 4, 8, 12, 16, 17])
def test_signed_digit_reconstruction(c):
    nwin = -(-254 // c)    # 253-bit scalars need ceil((253 + 1) / c) windows
    for s in [0, 1, (1 << c) - 1, 1 << (c - 1), (1 << (c - 1)) - 1, fq.R - 1,
              (1 << 253) - 1] + [RNG.randrange(1 << 253) for _ in range(200)]:
        d = msm.signed_digits(s, c, nwin)
        assert sum(x << (c * j) for j, x in enumerate(d)) == s
        assert all(-(1 << (c - 1)) < x <= (1 << (c - 1)) for x in d)
    nwin256 = -(-257 // c)
    for s in [(1 << 256) - 1, 1 << 255, (1 << 256) - (1 << (c - 1))]:
        d = msm.signed_digits(s, c, nwin256)
        assert sum(x << (c * j) for j, x in enumerate(d)) == s
