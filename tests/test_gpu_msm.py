"""GPU parity: msm_g1 vs the oracle (exact affine results).

Small cases are checked against the oracle's Pippenger and naive MSM; every
case with points P_i = s_i * G is also checked against the closed form
((sum a_i s_i) mod r) * G, which pins the full sizes without an O(n) oracle run.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import coracle, fq, g1
from tests.util import closed_form_limbs, msm_inputs, oracle_points

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2502_11660_gb300")


def run(pts, sc, **kw):
    out = pkg.msm_g1(pkg.to_device(pts), pkg.to_device(sc), **kw)
    torch.cuda.synchronize()
    return g1.from_limbs(pkg.to_host(out))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 17, 64, 255, 1000, 2049])
@pytest.mark.parametrize("c,signed", [(4, False), (4, True), (8, True), (7, False)])
def test_small_n_against_oracle(n, c, signed):
    a, s, pts = msm_inputs(n, tag=100 + n)
    want = closed_form_limbs(s, a)
    assert run(pts, a, c=c, signed=signed, scalar_bits=253) == want
    if n <= 64:
        assert g1.from_limbs(coracle.msm_naive(pts, a)) == want


def test_empty_is_identity():
    z = torch.zeros((0, 24), dtype=torch.int32, device="cuda")
    zs = torch.zeros((0, 8), dtype=torch.int32, device="cuda")
    out = pkg.msm_g1(z, zs)
    torch.cuda.synchronize()
    assert not pkg.to_host(out).any()


def test_config_small_c8_unsigned():
    """n = 2^12, c = 8, unsigned digits, standard-form points."""
    n = 1 << 12
    a, s, pts = msm_inputs(n, tag=0)
    want = closed_form_limbs(s, a)
    assert run(pts, a, c=8, signed=False) == want
    assert g1.from_limbs(coracle.msm(pts, a, c=8)) == want


def test_edge_scalars_and_points():
    n = 700
    a, s, pts = msm_inputs(n, tag=7)
    a = a.copy()
    pts = pts.copy()
    s = s.copy()
    # zero scalars, r - 1, 1, duplicated points, a point and its negation
    a[0:10] = 0
    a[10] = synth.int_to_limbs(fq.R - 1, 8)
    a[11] = synth.int_to_limbs(1, 8)
    pts[20] = pts[21]
    s[20] = s[21]
    pts[30] = pts[31]
    pts[30, 12:] = synth.int_to_limbs((fq.P - synth.limbs_to_int(pts[31, 12:])) % fq.P, 12)
    s[30] = synth.int_to_limbs((fq.R - synth.limbs_to_int(s[31])) % fq.R, 8)
    a[30] = a[31]     # cancels term 31 exactly
    want = closed_form_limbs(s, a)
    for c, sg in [(5, True), (9, False), (12, True)]:
        assert run(pts, a, c=c, signed=sg, scalar_bits=253) == want


@pytest.mark.parametrize("n", [1, 33, 1000, 4099])
def test_radix_sort_path_matches_the_counting_sort(n):
    """MSM377_RADIX_SORT (LSD radix passes) gives the same sums as the default
    counting sort: one, two and three 8-bit passes, signed and unsigned digits, and
    both curve models."""
    a, s, pts = msm_inputs(n, tag=300 + n)
    want = closed_form_limbs(s, a)
    for c, sg in [(4, False), (8, True), (13, True), (16, True), (18, False)]:
        assert run(pts, a, c=c, signed=sg, scalar_bits=253, radix_sort=True) == want
    assert run(pts, a, c=11, scalar_bits=253, edwards=True, glv=True, radix_sort=True) == want


def test_radix_sort_edge_scalars_and_heavy_bucket():
    n = 3000
    a, s, pts = msm_inputs(n, tag=11)
    a = a.copy()
    a[0:100] = 0
    a[100:2100] = a[100]          # one bucket per window holds 2000 points
    want = closed_form_limbs(s, a)
    for c in (6, 16):
        assert run(pts, a, c=c, signed=True, scalar_bits=253, radix_sort=True) == want


def test_heavy_bucket_all_equal_scalars():
    """All scalars equal: every window has one bucket holding all n points."""
    n = 5000
    a, s, pts = msm_inputs(n, tag=8)
    a = np.tile(a[:1], (n, 1))
    want = closed_form_limbs(s, a)
    for c in (6, 10, 16):
        assert run(pts, a, c=c, signed=True, scalar_bits=253) == want


def test_full_width_scalars():
    """Scalars up to 2^256 - 1 (>= r) with scalar_bits = 256: still sum a_i P_i."""
    n = 300
    _, s, pts = msm_inputs(n, tag=9)
    a = synth.scalars_full(55, n)
    a[0] = 0xFFFFFFFF
    want = closed_form_limbs(s, a)
    for sg in (True, False):
        assert run(pts, a, c=9, signed=sg, scalar_bits=256) == want
        assert run(pts, a, c=9, signed=sg) == want   # 0 means 256


def test_scalar_bits_violation_is_reported():
    n = 64
    a, s, pts = msm_inputs(n, tag=10)
    a = a.copy()
    a[3, 7] = 0x80000000    # bit 255 set, above scalar_bits = 253
    ws = pkg.msm_g1_workspace(n, c=5, scalar_bits=253)
    pkg.msm_g1(pkg.to_device(pts), pkg.to_device(a), workspace=ws, c=5, scalar_bits=253)
    assert pkg.msm_g1_status(ws) == pkg.ERANGE


def test_prepared_points_and_host_api_agree():
    n = 3000
    a, s, pts = msm_inputs(n, tag=12)
    want = closed_form_limbs(s, a)
    dp = pkg.to_device(pts)
    prep = pkg.msm_points_prepare(dp)
    assert run(pts, a, c=10, scalar_bits=253) == want
    out = pkg.msm_g1(prep, pkg.to_device(a), c=10, scalar_bits=253, prepared=True)
    torch.cuda.synchronize()
    assert g1.from_limbs(pkg.to_host(out)) == want
    host = pkg.msm_g1_host(pts, a, c=10, scalar_bits=253)
    assert g1.from_limbs(host) == want


def test_generator_mul_matches_oracle():
    n = 2500
    seeds = synth.scalars(77, n)
    seeds[0] = 0
    seeds[1] = synth.int_to_limbs(1, 8)
    seeds[2] = synth.int_to_limbs(fq.R - 1, 8)
    got = pkg.to_host(pkg.g1_generator_mul(pkg.to_device(seeds)))
    want = oracle_points(seeds)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("logn", [20, 22])
def test_full_size_closed_form(logn):
    """n = 2^20 and 2^22, signed digits, default window, resident prepared points."""
    n = 1 << logn
    a, s, pts = msm_inputs(n, tag=2)
    want = closed_form_limbs(s, a)
    prep = pkg.msm_points_prepare(pkg.to_device(pts))
    da = pkg.to_device(a)
    ws = pkg.msm_g1_workspace(n, scalar_bits=253, prepared=True)
    for _ in range(2):  # the same workspace twice in a row
        out = pkg.msm_g1(prep, da, workspace=ws, scalar_bits=253, prepared=True)
        torch.cuda.synchronize()
        assert g1.from_limbs(pkg.to_host(out)) == want
    assert pkg.msm_g1_status(ws) == 0
