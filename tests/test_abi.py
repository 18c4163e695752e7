"""The C-ABI library loads on a host without a GPU and exports what include/msm377.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "msm377.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|size_t|void|uint32_t|uint64_t)\s+\**\s*([a-z_0-9]+)\s*\(",
                       text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_named_calls():
    names = declared_functions()
    for required in ("fq_mul_batch", "padd_batch", "msm_g1", "msm_g1_workspace_bytes", "msm_g1_batched",
                     "msm_points_create", "msm_points_destroy", "msm_g1_resident", "msm_points_validate",
                     "msm_points_data", "msm377_launch_count"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_2502_11660_gb300 as pkg
    L = pkg.lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    # every declared call has a binding signature
    from paper_2502_11660_gb300._lib import SIGNATURES
    assert set(declared_functions()) <= set(SIGNATURES)


def test_host_only_entry_points():
    import paper_2502_11660_gb300 as pkg
    L = pkg.lib()
    assert L.msm377_version() >= 100
    o = pkg._opts(c=16, signed=True, scalar_bits=253)
    ws = L.msm_g1_workspace_bytes(1 << 20, ctypes.byref(o))
    assert ws > (1 << 20) * 16 * 8 * 2   # keys and values, double-buffered
    assert L.msm_g1_workspace_bytes(10, ctypes.byref(pkg._opts(c=1))) == 0
    assert L.msm_g1_workspace_bytes(10, ctypes.byref(pkg._opts(c=21))) == 0
    assert L.msm_g1_workspace_bytes(10, ctypes.byref(pkg._opts(scalar_bits=257))) == 0
    assert [pkg.msm_g1_default_c(1 << k) for k in (12, 20, 22)] == [8, 16, 17]
    # the sort's bin offsets are 32-bit: windows x items per window must stay below 2^32
    # (c = 16 signed over 253-bit scalars: 16 windows)
    o16 = pkg._opts(c=16, signed=True, scalar_bits=253)
    assert L.msm_g1_workspace_bytes((1 << 28) - 1, ctypes.byref(o16)) > 0
    assert L.msm_g1_workspace_bytes(1 << 28, ctypes.byref(o16)) == 0


def test_invalid_arguments_fail_before_touching_the_gpu():
    import paper_2502_11660_gb300 as pkg
    L = pkg.lib()
    rc = L.msm_g1(None, None, 10, ctypes.c_void_p(16), None, 0, None)
    assert rc == -1 and "opts" in pkg.last_error()
    rc = L.msm_g1(None, None, 10, ctypes.c_void_p(16), None, 0, ctypes.byref(pkg._opts(c=30)))
    assert rc == -1 and "bad options" in pkg.last_error()
    rc = L.msm_g1(None, None, 10, None, None, 0, ctypes.byref(pkg._opts()))
    assert rc == -1
    assert L.fq_mul_batch(None, None, None, 5, 0, None) == -1
    assert L.padd_batch(None, None, None, 5, 0, None) == -1
    assert L.fq_mul_batch(None, None, None, 0, 0, None) == 0   # n = 0 is a no-op


def test_header_constants_match_the_oracle():
    """The CUDA field header's modulus and Montgomery constants (R = 2^384) agree
    with the oracle's derivation of p from the BLS12 seed."""
    from oracle import fq
    src = open(os.path.join(ROOT, "paper_2502_11660_gb300", "csrc", "fq.cuh")).read()

    def limbs(name):
        m = re.search(name + r"\[N\] = \{([^}]*)\}", src)
        return sum(int(w.strip().rstrip("u"), 16) << (32 * k) for k, w in enumerate(m.group(1).split(",")))

    R = 1 << 384
    assert limbs("kP") == fq.P
    assert limbs("k2P") == 2 * fq.P
    assert limbs("kOne") == R % fq.P
    assert limbs("kR2") == R * R % fq.P
    assert limbs("kR3") == R ** 3 % fq.P
    assert fq.P % (1 << 32) == 1   # so the Montgomery digit is m = -t0 mod 2^32


def test_window_table_install_and_reject():
    import paper_2502_11660_gb300 as pkg
    from paper_2502_11660_gb300 import autotune
    base = pkg.msm_g1_default_c(1 << 20)
    try:
        autotune.install([0] * 20 + [13])
        assert pkg.msm_g1_default_c(1 << 20) == 13
        assert pkg.msm_g1_default_c((1 << 21) - 1) == 13
        assert pkg.msm_g1_default_c(1 << 21) == base or pkg.msm_g1_default_c(1 << 21) != 13
        assert pkg.msm_g1_default_c(1 << 20, signed=False) != 13 or base == 13
        with pytest.raises(pkg.MsmError):
            autotune.install([1, 2, 3])
        with pytest.raises(pkg.MsmError):
            autotune.install([0] * 40)
    finally:
        autotune.clear()
    assert pkg.msm_g1_default_c(1 << 20) == base


def _const_limbs(src, name):
    m = re.search(name + r"\[[^\]]*\] = \{([^}]*)\}", src)
    words = [w.strip().rstrip("u") for w in m.group(1).split(",") if w.strip()]
    return sum(int(w, 16) << (32 * k) for k, w in enumerate(words))


def test_edwards_and_glv_constants_match_the_oracle():
    """The Edwards map constants (ed.cuh) and the GLV constants (msm.cu) agree with
    the oracle's own derivations (Montgomery form x 2^384 mod p for field elements)."""
    from oracle import edwards, fq, glv
    R = 1 << 384
    ed_src = open(os.path.join(ROOT, "paper_2502_11660_gb300", "csrc", "ed.cuh")).read()
    assert _const_limbs(ed_src, "kK") == edwards.K * R % fq.P
    assert _const_limbs(ed_src, "kS") == edwards.S * R % fq.P
    assert _const_limbs(ed_src, "kGamma") == edwards.GAMMA * R % fq.P
    assert _const_limbs(ed_src, "kC1") == edwards.GAMMA * fq.inv(edwards.S) % fq.P * R % fq.P
    msm_src = open(os.path.join(ROOT, "paper_2502_11660_gb300", "csrc", "msm.cu")).read()
    assert _const_limbs(msm_src, "kBeta") == glv.BETA * R % fq.P
    assert _const_limbs(msm_src, "kLambda") == glv.LAMBDA
    assert _const_limbs(msm_src, "kMu") == (1 << 256) // glv.LAMBDA
    rows = re.search(r"kR8\[4\]\[8\] = \{(.*?)\};", msm_src, flags=re.S).group(1)
    mults = [sum(int(w.strip().rstrip("u"), 16) << (32 * k) for k, w in enumerate(r.split(",")))
             for r in re.findall(r"\{([^}]*)\}", rows)]
    assert mults == [8 * fq.R, 4 * fq.R, 2 * fq.R, fq.R]


def test_stored_point_sizes_and_mode_flags():
    import paper_2502_11660_gb300 as pkg
    L = pkg.lib()
    n = 1000
    assert L.msm_points_prepared_bytes(n, 0) == 96 * n
    assert L.msm_points_prepared_bytes(n, pkg.EDWARDS) == 144 * n
    assert L.msm_points_prepared_bytes(n, pkg.GLV) == 2 * 96 * n
    assert L.msm_points_prepared_bytes(n, pkg.EDWARDS | pkg.GLV) == 2 * 144 * n
    assert L.msm_points_prepared_bytes(n, pkg.PROFILE) == 0
    assert L.msm_points_prepare_ex(None, 10, None, pkg.PROFILE, None) == -1
    assert L.msm_points_prepare_ex(None, 0, None, pkg.GLV, None) == 0
    # GLV halves the windows: key/value buffers of 2n items x W/2 windows, plus 2n stored points
    plain = L.msm_g1_workspace_bytes(1 << 16, ctypes.byref(pkg._opts(c=12, scalar_bits=253)))
    split = L.msm_g1_workspace_bytes(1 << 16, ctypes.byref(pkg._opts(c=12, scalar_bits=253, glv=True)))
    assert plain > 0 and split > 0
    assert pkg.msm_g1_default_c(1 << 20, glv=True) == pkg.msm_g1_default_c(1 << 21)
    # the sort choice changes the workspace: counting sort = ranks + (key, value) pairs;
    # radix sort with two passes = ping-pong key/value arrays + pairs
    cnt = L.msm_g1_workspace_bytes(1 << 16, ctypes.byref(pkg._opts(c=16, scalar_bits=253)))
    rdx = L.msm_g1_workspace_bytes(1 << 16, ctypes.byref(pkg._opts(c=16, scalar_bits=253, radix_sort=True)))
    assert cnt > 0 and rdx > 0 and cnt != rdx


def test_window_tables_are_per_mode():
    import paper_2502_11660_gb300 as pkg
    from paper_2502_11660_gb300 import autotune
    base = pkg.msm_g1_default_c(1 << 20)
    base_e = pkg.msm_g1_default_c(1 << 20, edwards=True, glv=True)
    try:
        autotune.install([0] * 20 + [11], edwards=True, glv=True)
        assert pkg.msm_g1_default_c(1 << 20, edwards=True, glv=True) == 11
        assert pkg.msm_g1_default_c(1 << 20) == base
        assert pkg.msm_g1_default_c(1 << 20, edwards=True) != 11 or base == 11
        arr = (ctypes.c_int32 * 1)(5)
        assert pkg.lib().msm_g1_set_window_table(arr, 1, pkg.PROFILE) == -1
    finally:
        autotune.clear(edwards=True, glv=True)
    assert pkg.msm_g1_default_c(1 << 20, edwards=True, glv=True) == base_e


def test_barrett_constant_matches_the_oracle():
    from oracle import barrett, fq
    src = open(os.path.join(ROOT, "paper_2502_11660_gb300", "csrc", "fqvar.cu")).read()
    k, mu = barrett.barrett_params(fq.P)
    assert k == 377
    assert _const_limbs(src, "kMuB") == mu


def test_precomputed_options():
    import paper_2502_11660_gb300 as pkg
    L = pkg.lib()
    n = 1000
    # explicit c and the Edwards model are required
    assert L.msm_points_precomputed_bytes(n, ctypes.byref(pkg._opts(c=0, scalar_bits=253, edwards=True,
                                                                      precomputed=True))) == 0
    assert L.msm_points_precomputed_bytes(n, ctypes.byref(pkg._opts(c=16, scalar_bits=253, precomputed=True))) == 0
    W = -(-(253 + 1) // 16)
    assert pkg.msm_points_precomputed_bytes(n, 16, 253) == W * n * 144
    assert pkg.msm_points_precomputed_bytes(n, 16, 253, glv=True) == -(-(127 + 1) // 16) * 2 * n * 144
    # one window in the pipeline: the key buffers hold W n items, the buckets one window
    o = pkg._opts(c=16, scalar_bits=253, prepared=True, edwards=True, precomputed=True)
    assert L.msm_g1_workspace_bytes(n, ctypes.byref(o)) > 0
    o2 = pkg._opts(c=16, scalar_bits=253, edwards=True, precomputed=True)   # not prepared: rejected
    assert L.msm_g1_workspace_bytes(n, ctypes.byref(o2)) == 0
    assert L.msm_points_precompute(None, n, None, ctypes.byref(pkg._opts(c=0, edwards=True,
                                                                          precomputed=True))) == -1


def test_resident_and_validation_calls_reject_bad_arguments_on_the_host():
    import paper_2502_11660_gb300 as pkg
    L = pkg.lib()
    h = ctypes.c_void_p(0)
    assert L.msm_points_create(None, 10, None, ctypes.byref(h)) == pkg.EINVAL
    assert L.msm_points_create(None, 10, ctypes.byref(pkg._opts()), ctypes.byref(h)) == pkg.EINVAL
    assert not h.value
    bad = pkg._opts(edwards=True, precomputed=True)          # fixed-base sets need an explicit c
    assert L.msm_points_create(ctypes.c_void_p(256), 10, ctypes.byref(bad), ctypes.byref(h)) == pkg.EINVAL
    flags = pkg._opts(profile=True)                          # not a set property
    assert L.msm_points_create(ctypes.c_void_p(256), 10, ctypes.byref(flags), ctypes.byref(h)) == pkg.EINVAL
    assert L.msm_points_destroy(None) == 0
    assert L.msm_points_count(None) == 0
    assert not L.msm_points_data(None, 0)
    assert L.msm_g1_resident_workspace_bytes(None, 10, ctypes.byref(pkg._opts())) == 0
    assert L.msm_g1_resident(None, 0, 10, None, None, None, 0, ctypes.byref(pkg._opts())) == pkg.EINVAL
    assert L.msm_points_validate(None, 10, 1 << 12, None) == pkg.EINVAL
    assert L.msm_points_validate(None, 0, 0, None) == 0     # nothing to check
    # stored points cannot be validated by msm_g1 (their sets are checked when made)
    o = pkg._opts(c=8, prepared=True, validate=True)
    ws = L.msm_g1_workspace_bytes(10, ctypes.byref(o))
    rc = L.msm_g1(ctypes.c_void_p(256), ctypes.c_void_p(256), 10, ctypes.c_void_p(256), ctypes.c_void_p(256), ws,
                  ctypes.byref(o))
    assert rc == pkg.EINVAL and "VALIDATE" in pkg.last_error()
    assert L.msm_g1_noalloc(None, None, 10, None, ctypes.byref(pkg._opts(validate=True))) == pkg.EINVAL


def test_status_codes_and_validation_constant_match():
    """The header's status codes are the binding's, and the validation kernel's r is the
    oracle's group order."""
    import paper_2502_11660_gb300 as pkg
    from oracle import fq
    text = open(HEADER).read()
    for name in ("EINVAL", "ENOMEM", "ECUDA", "ETIMEOUT", "ENOTONCURVE", "ERANGE"):
        m = re.search(r"#define MSM377_%s \((-\d+)\)" % name, text)
        assert m and int(m.group(1)) == getattr(pkg, name), name
    assert int(re.search(r"#define MSM377_VALIDATE (\d+)u", text).group(1)) == pkg.VALIDATE
    src = open(os.path.join(ROOT, "paper_2502_11660_gb300", "csrc", "resident.cu")).read()
    body = re.search(r"kOrderR\[8\] = \{([^}]*)\}", src).group(1)
    words = [int(w.strip().rstrip("u"), 16) for w in body.split(",")]
    assert sum(w << (32 * k) for k, w in enumerate(words)) == fq.R


def test_paper_format_constants_match_the_oracle():
    """The 25-bit element tables of the paper-format variant hold p and mu = floor(2^756 / p)."""
    from oracle import barrett, fq
    src = open(os.path.join(ROOT, "paper_2502_11660_gb300", "csrc", "fqvar.cu")).read()

    def elems(name):
        body = re.search(name + r"\[kEl\] = \{([^}]*)\}", src).group(1)
        body = re.sub(r"//[^\n]*", "", body)
        return barrett.from_elems([int(w.strip().rstrip("u"), 16) for w in body.split(",") if w.strip()])

    assert elems("kPEl") == fq.P
    assert elems("kMuEl") == (1 << (2 * barrett.LOOSE_K)) // fq.P


def test_window_tuner_breaks_near_ties_toward_the_widest_window():
    from paper_2502_11660_gb300 import autotune
    # the fastest wins when it is clearly faster
    assert autotune.pick_c({12: 1.30, 16: 1.00, 17: 1.20}) == 16
    assert autotune.pick_c({11: 0.926, 12: 0.979, 13: 1.04}) == 11
    # within C_TIE of the fastest, the widest window is kept (fewer windows, less work)
    assert autotune.pick_c({12: 1.181, 13: 1.22, 16: 1.186, 17: 1.583}) == 16
    assert autotune.pick_c({16: 20.69, 17: 20.25}) == 17
    assert autotune.pick_c({5: 1.0}) == 5
