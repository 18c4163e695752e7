"""Resident point sets (msm_points_create / msm_g1_resident / msm_points_destroy) and
point validation (MSM377_VALIDATE, msm_points_validate), through the C-ABI.

A resident set is the stored form of a caller's points in library-owned memory;
MSMs over any slice of it must equal msm_g1 on the same points and the closed form
((sum a_i s_i) mod r) G. Validation checks the problem's precondition (points of
BLS12-377 G1, Sec. I / II-C): off-curve points and coordinates >= p are always
rejected; points of the curve outside the order-r subgroup are rejected where the
curve model needs the subgroup (Edwards, GLV). Rejections come back as a status
code on the host; no kernel faults.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth
from oracle import fq, g1
from tests.util import closed_form_limbs, msm_inputs

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2502_11660_gb300")

MODELS = [dict(), dict(edwards=True), dict(glv=True), dict(edwards=True, glv=True),
          dict(precompute_c=11), dict(precompute_c=13, glv=True)]
MODEL_IDS = ["xyzz", "edwards", "glv", "edwards+glv", "fixed-base", "fixed-base+glv"]


@pytest.mark.parametrize("kw", MODELS, ids=MODEL_IDS)
def test_resident_slices_equal_msm_g1_and_the_closed_form(kw):
    n = 5000
    a, s, pts = msm_inputs(n, tag=501)
    dp = pkg.to_device(pts)
    rs = pkg.ResidentSet(dp, scalar_bits=253 if kw.get("precompute_c") else 0, **kw)
    assert pkg.lib().msm_points_count(rs.handle) == n
    for off, m in ((0, n), (0, 1), (1234, 777), (n - 3, 3), (256, 2049)):
        da = pkg.to_device(a[off:off + m])
        out = rs.msm(da, offset=off)
        torch.cuda.synchronize()
        got = pkg.to_host(out)
        want = closed_form_limbs(s[off:off + m], a[off:off + m])
        assert g1.from_limbs(got) == want, (off, m)
        if not kw.get("precompute_c"):
            ref = pkg.msm_g1(dp[off:off + m].contiguous(), da, scalar_bits=0, edwards=kw.get("edwards", False),
                             glv=kw.get("glv", False))
            torch.cuda.synchronize()
            assert np.array_equal(pkg.to_host(ref), got)
    rs.close()


def test_resident_set_rejects_out_of_range_slices_and_other_models():
    n = 100
    a, s, pts = msm_inputs(n, tag=502)
    rs = pkg.ResidentSet(pkg.to_device(pts), edwards=True)
    ws = rs.workspace(10)
    out = torch.empty(24, dtype=torch.int32, device="cuda")
    sc = pkg.to_device(a[:10])
    o = rs._opts(None)
    L = pkg.lib()
    rc = L.msm_g1_resident(rs.handle, 95, 10, ctypes.c_void_p(sc.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                           ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctypes.byref(o))
    assert rc == pkg.EINVAL and "outside" in pkg.last_error()
    o2 = pkg._opts(glv=True, stream=None)
    rc = L.msm_g1_resident(rs.handle, 0, 10, ctypes.c_void_p(sc.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                           ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctypes.byref(o2))
    assert rc == pkg.EINVAL
    rs.close()


def test_resident_rows_feed_a_batched_call():
    """msm_points_data gives each job of a batched call its slice of a resident set."""
    n = 6000
    a, s, pts = msm_inputs(n, tag=503)
    rs = pkg.ResidentSet(pkg.to_device(pts), edwards=True, glv=True)
    slices = [(0, 1000), (1000, 3000), (4000, 1), (4001, 1999)]
    jobs = (pkg.MsmJob * len(slices))()
    outs = [torch.empty(24, dtype=torch.int32, device="cuda") for _ in slices]
    scs = [pkg.to_device(a[o:o + m]) for o, m in slices]
    for i, (o, m) in enumerate(slices):
        jobs[i].points = rs.data_ptr(o)
        jobs[i].scalars = scs[i].data_ptr()
        jobs[i].n = m
        jobs[i].out = outs[i].data_ptr()
        jobs[i].c = 0
    opts = pkg._opts(scalar_bits=253, prepared=True, edwards=True, glv=True, stream=None)
    L = pkg.lib()
    nbytes = L.msm_g1_batched_workspace_bytes(jobs, len(slices), ctypes.byref(opts))
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    pkg.check(L.msm_g1_batched(jobs, len(slices), ctypes.c_void_p(ws.data_ptr()), nbytes, ctypes.byref(opts)))
    torch.cuda.synchronize()
    for (o, m), out in zip(slices, outs):
        assert g1.from_limbs(pkg.to_host(out)) == closed_form_limbs(s[o:o + m], a[o:o + m])
    rs.close()


def _bad_points(n, tag):
    """A valid subgroup set and three faulty copies: one point off the curve, one
    coordinate >= p, one curve point outside the order-r subgroup."""
    a, s, pts = msm_inputs(n, tag)
    off = pts.copy()
    off[17, 12:] = synth.int_to_limbs((synth.limbs_to_int(pts[17, 12:]) + 1) % fq.P, 12)
    big = pts.copy()
    big[3, :12] = synth.int_to_limbs(synth.limbs_to_int(pts[3, :12]) + fq.P, 12)   # same residue, >= p
    cof = pts.copy()
    Q = g1.random_point(0xBADC0DE)
    assert g1.on_curve(Q) and g1.mul(fq.R, Q) is not None
    cof[n - 1] = np.array(g1.to_limbs(Q), dtype=np.uint32)
    return a, s, pts, off, big, cof


def test_validate_rejects_off_curve_out_of_range_and_non_subgroup_points():
    n = 4096
    a, s, pts, off, big, cof = _bad_points(n, 504)
    V = pkg.msm_points_validate
    for edw, gl in ((False, False), (True, False), (False, True), (True, True)):
        sub = edw or gl
        assert V(pkg.to_device(pts), edwards=edw, glv=gl) == 0
        assert V(pkg.to_device(off), edwards=edw, glv=gl) == pkg.ENOTONCURVE
        assert V(pkg.to_device(big), edwards=edw, glv=gl) == pkg.ENOTONCURVE
        assert V(pkg.to_device(cof), edwards=edw, glv=gl) == (pkg.ENOTONCURVE if sub else 0)
    z = pts.copy()
    z[5] = 0                                                    # O, encoded (0, 0), is valid
    assert V(pkg.to_device(z), subgroup=True) == 0
    T = pts.copy()
    T[9] = np.array(g1.to_limbs((fq.P - 1, 0)), dtype=np.uint32)   # the 2-torsion point
    assert V(pkg.to_device(T)) == 0 and V(pkg.to_device(T), subgroup=True) == pkg.ENOTONCURVE


def test_validate_in_msm_g1_host_call_and_set_creation():
    n = 2048
    a, s, pts, off, big, cof = _bad_points(n, 505)
    want = closed_form_limbs(s, a)
    # msm_g1 on standard-form points: valid input -> status 0 and the closed form
    ws = pkg.msm_g1_workspace(n, scalar_bits=253, edwards=True, glv=True)
    out = pkg.msm_g1(pkg.to_device(pts), pkg.to_device(a), workspace=ws, scalar_bits=253, edwards=True,
                     glv=True, validate=True)
    assert pkg.msm_g1_status(ws) == 0
    assert g1.from_limbs(pkg.to_host(out)) == want
    # a non-subgroup point under Edwards + GLV: status ENOTONCURVE (the value is unspecified)
    pkg.msm_g1(pkg.to_device(cof), pkg.to_device(a), workspace=ws, scalar_bits=253, edwards=True, glv=True,
               validate=True)
    assert pkg.msm_g1_status(ws) == pkg.ENOTONCURVE
    # the same workspace is clean again on the next valid call
    pkg.msm_g1(pkg.to_device(pts), pkg.to_device(a), workspace=ws, scalar_bits=253, edwards=True, glv=True,
               validate=True)
    assert pkg.msm_g1_status(ws) == 0
    # XYZZ accepts any curve point, so only the off-curve set fails there
    wx = pkg.msm_g1_workspace(n, scalar_bits=253)
    pkg.msm_g1(pkg.to_device(cof), pkg.to_device(a), workspace=wx, scalar_bits=253, validate=True)
    assert pkg.msm_g1_status(wx) == 0
    pkg.msm_g1(pkg.to_device(off), pkg.to_device(a), workspace=wx, scalar_bits=253, validate=True)
    assert pkg.msm_g1_status(wx) == pkg.ENOTONCURVE
    # the host-buffer call returns the status itself
    assert g1.from_limbs(pkg.msm_g1_host(pts, a, scalar_bits=253, edwards=True, validate=True)) == want
    with pytest.raises(pkg.MsmError) as e:
        pkg.msm_g1_host(big, a, scalar_bits=253, validate=True)
    assert e.value.code == pkg.ENOTONCURVE
    # set creation refuses invalid points and hands back no handle
    with pytest.raises(pkg.MsmError) as e:
        pkg.ResidentSet(pkg.to_device(cof), edwards=True, glv=True, validate=True)
    assert e.value.code == pkg.ENOTONCURVE
    rs = pkg.ResidentSet(pkg.to_device(pts), edwards=True, glv=True, validate=True)
    assert g1.from_limbs(pkg.to_host(rs.msm(pkg.to_device(a)))) == want
    rs.close()


def test_resident_host_call_equals_the_device_call():
    """msm_g1_resident_host (host scalars in, host result out) over slices of a resident set."""
    n = 3000
    a, s, pts = msm_inputs(n, tag=506)
    rs = pkg.ResidentSet(pkg.to_device(pts), edwards=True, glv=True)
    ws = rs.host_workspace(n)
    for off, m in ((0, n), (1000, 1500), (2999, 1)):
        got = rs.msm_host(a[off:off + m], offset=off, workspace=ws)
        assert g1.from_limbs(got) == closed_form_limbs(s[off:off + m], a[off:off + m]), (off, m)
    assert not rs.msm_host(a[:0], offset=0, workspace=ws).any()      # n = 0: O
    rs.close()
