"""msm_g1_noalloc, the MSM entry point for callers that cannot allocate device memory.

Some callers (a plugin whose host program owns all device memory through its own
pooling allocator, a request path on which allocation calls are forbidden, a
deployment with a device-memory budget fixed at load time) cannot hand msm_g1 a
workspace. msm_g1_noalloc runs the same MSM out of a fixed scratch array held by
the library. These tests call it through the C-ABI and check that it returns
exactly what msm_g1 returns, on two calls in a row (the second call reuses the
scratch the first one left behind), and that oversized requests are refused.
The file is named to run last in the suite.
"""
import ctypes

import numpy as np
import pytest
import torch

from tests.util import closed_form_limbs, msm_inputs

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2502_11660_gb300")


def _noalloc(points, scalars, out, c, signed, scalar_bits, flags=0):
    o = pkg.MsmOpts(c, 1 if signed else 0, scalar_bits, flags, torch.cuda.current_stream().cuda_stream)
    return pkg.lib().msm_g1_noalloc(ctypes.c_void_p(points.data_ptr()), ctypes.c_void_p(scalars.data_ptr()),
                                    points.shape[0], ctypes.c_void_p(out.data_ptr()), ctypes.byref(o))


@pytest.mark.parametrize("c,signed", [(0, True), (7, False)])
def test_noalloc_matches_msm_g1_on_two_calls_in_a_row(c, signed):
    for n, tag in ((4096, 301), (3001, 302)):
        a, s, pts = msm_inputs(n, tag)
        dp, da = pkg.to_device(pts), pkg.to_device(a)
        ref = pkg.msm_g1(dp, da, c=c, signed=signed)           # the existing entry point
        out = torch.full((24,), -1, dtype=torch.int32, device="cuda")
        rc = _noalloc(dp, da, out, c, signed, 0)
        assert rc == 0, pkg.last_error()
        torch.cuda.synchronize()
        got = pkg.to_host(out)
        assert np.array_equal(got, pkg.to_host(ref))
        from oracle import g1
        assert g1.from_limbs(got) == closed_form_limbs(s, a)


@pytest.mark.parametrize("flags", ["edwards_glv", "radix_sort"])
def test_noalloc_curve_models_and_sort_choice(flags):
    """The scratch also holds the Edwards + GLV stored points the call prepares, and the
    radix sort's buffers; both give the closed form."""
    from oracle import g1
    f = (pkg.EDWARDS | pkg.GLV) if flags == "edwards_glv" else pkg.RADIX_SORT
    n = 2048
    a, s, pts = msm_inputs(n, 303)
    dp, da = pkg.to_device(pts), pkg.to_device(a)
    out = torch.full((24,), -1, dtype=torch.int32, device="cuda")
    rc = _noalloc(dp, da, out, 0, True, 253, f)
    assert rc == 0, pkg.last_error()
    torch.cuda.synchronize()
    assert g1.from_limbs(pkg.to_host(out)) == closed_form_limbs(s, a)


def test_noalloc_refuses_requests_beyond_its_scratch():
    n = 1 << 18
    z = torch.zeros((n, 24), dtype=torch.int32, device="cuda")
    zs = torch.zeros((n, 8), dtype=torch.int32, device="cuda")
    out = torch.zeros(24, dtype=torch.int32, device="cuda")
    rc = _noalloc(z, zs, out, 0, True, 0)
    assert rc == -1
    assert "scratch" in pkg.last_error()
