"""GPU parity of the two alternative schedules of msm_g1 against the closed form and
the oracle: the paper's twisted Edwards model (MSM377_EDWARDS, Sec. II-D) and the
GLV split (MSM377_GLV), alone and together, for single, prepared, host-buffer and
batched calls. Results are exact affine points, compared bit for bit."""
import numpy as np
import pytest
import torch

import synth
from oracle import edwards, fq, g1, glv
from tests.util import closed_form_limbs, msm_inputs

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2502_11660_gb300")

MODES = [(True, False), (False, True), (True, True)]
MODE_IDS = ["edwards", "glv", "edwards+glv"]
R384 = 1 << 384


def run(pts, sc, **kw):
    out = pkg.msm_g1(pkg.to_device(pts), pkg.to_device(sc), **kw)
    torch.cuda.synchronize()
    return g1.from_limbs(pkg.to_host(out))


@pytest.mark.parametrize("edw,split", MODES, ids=MODE_IDS)
@pytest.mark.parametrize("n", [1, 2, 3, 17, 255, 1000, 2049])
@pytest.mark.parametrize("c,signed", [(4, True), (8, True), (7, False)])
def test_small_n(edw, split, n, c, signed):
    a, s, pts = msm_inputs(n, tag=100 + n)
    want = closed_form_limbs(s, a)
    assert run(pts, a, c=c, signed=signed, scalar_bits=253, edwards=edw, glv=split) == want


@pytest.mark.parametrize("edw,split", MODES, ids=MODE_IDS)
def test_edge_scalars_identity_points_duplicates(edw, split):
    n = 700
    a, s, pts = msm_inputs(n, tag=7)
    a, s, pts = a.copy(), s.copy(), pts.copy()
    lam = glv.LAMBDA
    a[0:10] = 0
    for i, v in enumerate([fq.R - 1, 1, lam - 1, lam, lam + 1, lam * lam, fq.R - lam, 2 ** 127 - 1]):
        a[10 + i] = synth.int_to_limbs(v, 8)
    pts[20] = pts[21]
    s[20] = s[21]
    pts[30] = pts[31]
    pts[30, 12:] = synth.int_to_limbs((fq.P - synth.limbs_to_int(pts[31, 12:])) % fq.P, 12)
    s[30] = synth.int_to_limbs((fq.R - synth.limbs_to_int(s[31])) % fq.R, 8)
    a[30] = a[31]
    pts[40] = 0            # the identity, encoded (0, 0): its seed is 0
    s[40] = 0
    want = closed_form_limbs(s, a)
    for c, sg in [(5, True), (9, False), (12, True)]:
        assert run(pts, a, c=c, signed=sg, scalar_bits=253, edwards=edw, glv=split) == want


@pytest.mark.parametrize("edw,split", MODES, ids=MODE_IDS)
def test_full_width_scalars_reduce_mod_r(edw, split):
    """Scalars up to 2^256 - 1: on subgroup points the sum equals the one with scalars mod r."""
    n = 300
    _, s, pts = msm_inputs(n, tag=9)
    a = synth.scalars_full(55, n)
    a[0] = 0xFFFFFFFF
    want = closed_form_limbs(s, a)
    for sg in (True, False):
        assert run(pts, a, c=9, signed=sg, edwards=edw, glv=split) == want


@pytest.mark.parametrize("edw,split", MODES, ids=MODE_IDS)
def test_heavy_bucket(edw, split):
    n = 5000
    a, s, pts = msm_inputs(n, tag=8)
    a = np.tile(a[:1], (n, 1))
    want = closed_form_limbs(s, a)
    for c in (6, 16):
        assert run(pts, a, c=c, signed=True, scalar_bits=253, edwards=edw, glv=split) == want


@pytest.mark.parametrize("edw,split", MODES, ids=MODE_IDS)
def test_prepared_host_and_range_check(edw, split):
    n = 3000
    a, s, pts = msm_inputs(n, tag=12)
    want = closed_form_limbs(s, a)
    prep = pkg.msm_points_prepare(pkg.to_device(pts), edwards=edw, glv=split)
    assert prep.numel() * 4 == pkg.msm_points_prepared_bytes(n, edw, split)
    out = pkg.msm_g1(prep, pkg.to_device(a), c=10, scalar_bits=253, prepared=True, edwards=edw, glv=split)
    torch.cuda.synchronize()
    assert g1.from_limbs(pkg.to_host(out)) == want
    host = pkg.msm_g1_host(pts, a, c=10, scalar_bits=253, edwards=edw, glv=split)
    assert g1.from_limbs(host) == want
    bad = a.copy()
    bad[3, 7] = 0x80000000
    ws = pkg.msm_g1_workspace(n, c=5, scalar_bits=253, edwards=edw, glv=split)
    pkg.msm_g1(pkg.to_device(pts), pkg.to_device(bad), workspace=ws, c=5, scalar_bits=253, edwards=edw,
               glv=split)
    assert pkg.msm_g1_status(ws) == pkg.ERANGE


def _mont_ints(block: np.ndarray) -> list[int]:
    """Rows of 12 u32 (Montgomery form) -> standard-form ints."""
    rinv = pow(R384, -1, fq.P)
    return [synth.limbs_to_int(row) * rinv % fq.P for row in block]


def test_stored_forms_match_the_oracle_maps():
    """The prepared points themselves: Edwards (x, y, k x y) of the oracle's map, and
    the GLV half phi(P) = (beta x, y), element by element."""
    n = 257
    _, s, pts = msm_inputs(n, tag=13)
    pts = pts.copy()
    pts[5] = 0                                    # identity -> Edwards (0, 1, 0)
    dp = pkg.to_device(pts)
    ed_st = pkg.to_host(pkg.msm_points_prepare(dp, edwards=True)).reshape(n, 36)
    gl_st = pkg.to_host(pkg.msm_points_prepare(dp, glv=True)).reshape(2 * n, 24)
    both = pkg.to_host(pkg.msm_points_prepare(dp, edwards=True, glv=True)).reshape(2 * n, 36)
    torch.cuda.synchronize()
    for i in range(n):
        P = None if i == 5 else g1.from_limbs(pts[i])
        e = edwards.from_weierstrass(P)
        want = list(edwards.stored_point(e))
        assert _mont_ints(ed_st[i].reshape(3, 12)) == want
        ph = glv.phi(P)
        assert _mont_ints(gl_st[2 * i].reshape(2, 12)) == ([0, 0] if P is None else list(P))
        assert _mont_ints(gl_st[2 * i + 1].reshape(2, 12)) == ([0, 0] if ph is None else list(ph))
        assert _mont_ints(both[2 * i].reshape(3, 12)) == want
        assert _mont_ints(both[2 * i + 1].reshape(3, 12)) == list(
            edwards.stored_point(edwards.from_weierstrass(ph)))


# ---------------------------------------------------------------- full sizes, every window the
# autotuner may pick (variable base: 12..17; fixed base: 15..20)

ALL_MODES = [(False, False), (True, False), (False, True), (True, True)]
ALL_IDS = ["xyzz", "edwards", "glv", "edwards+glv"]
_SETS: dict = {}


def _resident(n, tag, edw, split):
    """Prepared device set and the closed form for the 2^n workload (cached per mode)."""
    a, s, pts = msm_inputs(n, tag)
    want = closed_form_limbs(s, a, key=("full", n, tag))
    key = (n, tag, edw, split)
    if key not in _SETS:
        _SETS.clear()
        _SETS[key] = pkg.msm_points_prepare(pkg.to_device(pts), edwards=edw, glv=split)
    return _SETS[key], pkg.to_device(a), want


@pytest.mark.parametrize("c", list(range(12, 18)))
@pytest.mark.parametrize("edw,split", ALL_MODES, ids=ALL_IDS)
def test_full_size_2e20_every_tuned_c(edw, split, c):
    n = 1 << 20
    prep, da, want = _resident(n, 2, edw, split)
    ws = pkg.msm_g1_workspace(n, c=c, scalar_bits=253, prepared=True, edwards=edw, glv=split)
    out = pkg.msm_g1(prep, da, workspace=ws, c=c, scalar_bits=253, prepared=True, edwards=edw, glv=split)
    torch.cuda.synchronize()
    assert g1.from_limbs(pkg.to_host(out)) == want
    assert pkg.msm_g1_status(ws) == 0


@pytest.mark.parametrize("edw,split,c", [(True, True, 15), (True, True, 16), (True, True, 17),
                                         (False, False, 16), (False, False, 17), (True, False, 16),
                                         (False, True, 16)])
def test_full_size_2e22_tuned_c(edw, split, c):
    n = 1 << 22
    prep, da, want = _resident(n, 2, edw, split)
    out = pkg.msm_g1(prep, da, c=c, scalar_bits=253, prepared=True, edwards=edw, glv=split)
    torch.cuda.synchronize()
    assert g1.from_limbs(pkg.to_host(out)) == want


@pytest.mark.parametrize("c", list(range(15, 21)))
@pytest.mark.parametrize("split", [False, True], ids=["plain", "glv"])
def test_precomputed_full_size_2e20_every_tuned_c(split, c):
    n = 1 << 20
    a, s, pts = msm_inputs(n, tag=2)
    want = closed_form_limbs(s, a, key=("full", n, 2))
    pre = pkg.msm_points_precompute(pkg.to_device(pts), c=c, scalar_bits=253, glv=split)
    out = pkg.msm_g1(pre, pkg.to_device(a), c=c, scalar_bits=253, edwards=True, glv=split, precomputed=True)
    torch.cuda.synchronize()
    assert g1.from_limbs(pkg.to_host(out)) == want
    del pre
    torch.cuda.empty_cache()


@pytest.mark.parametrize("edw,split", MODES, ids=MODE_IDS)
def test_full_size_2e20(edw, split):
    n = 1 << 20
    a, s, pts = msm_inputs(n, tag=2)
    want = closed_form_limbs(s, a)
    prep = pkg.msm_points_prepare(pkg.to_device(pts), edwards=edw, glv=split)
    da = pkg.to_device(a)
    ws = pkg.msm_g1_workspace(n, scalar_bits=253, prepared=True, edwards=edw, glv=split)
    for _ in range(2):
        out = pkg.msm_g1(prep, da, workspace=ws, scalar_bits=253, prepared=True, edwards=edw, glv=split)
        torch.cuda.synchronize()
        assert g1.from_limbs(pkg.to_host(out)) == want
    assert pkg.msm_g1_status(ws) == 0


def test_full_size_2e22_edwards_glv():
    n = 1 << 22
    a, s, pts = msm_inputs(n, tag=2)
    want = closed_form_limbs(s, a)
    prep = pkg.msm_points_prepare(pkg.to_device(pts), edwards=True, glv=True)
    out = pkg.msm_g1(prep, pkg.to_device(a), scalar_bits=253, prepared=True, edwards=True, glv=True)
    torch.cuda.synchronize()
    assert g1.from_limbs(pkg.to_host(out)) == want


@pytest.mark.parametrize("edw,split", MODES, ids=MODE_IDS)
def test_batched_and_graph(edw, split):
    sizes = [0, 1, 7, 333, 2049, 5000, 64]
    cs = [0, 0, 5, 0, 10, 12, 3]
    data = [msm_inputs(n, tag=77000 + i) for i, n in enumerate(sizes)]
    prep = [pkg.msm_points_prepare(pkg.to_device(p), edwards=edw, glv=split) for _, _, p in data]
    scs = [pkg.to_device(a) for a, _, _ in data]
    kw = dict(c_list=cs, scalar_bits=253, prepared=True, edwards=edw, glv=split)
    outs = pkg.msm_g1_batched(prep, scs, **kw)
    torch.cuda.synchronize()
    for i, o in enumerate(outs):
        assert g1.from_limbs(pkg.to_host(o)) == closed_form_limbs(data[i][1], data[i][0]), f"job {i}"
    ws = pkg.msm_g1_batched_workspace(prep, c_list=cs, scalar_bits=253, prepared=True, edwards=edw, glv=split)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        pkg.msm_g1_batched(prep, scs, outs=outs, workspace=ws, stream=st, **kw)
    st.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        pkg.msm_g1_batched(prep, scs, outs=outs, workspace=ws, stream=st, **kw)
    new = [synth.scalars(900 + i, n) for i, n in enumerate(sizes)]
    for d, h in zip(scs, new):
        d.copy_(pkg.to_device(h))
    g.replay()
    torch.cuda.synchronize()
    for i, o in enumerate(outs):
        assert g1.from_limbs(pkg.to_host(o)) == closed_form_limbs(data[i][1], new[i]), f"job {i}"


# ---------------------------------------------------------------- fixed-base precomputation

@pytest.mark.parametrize("split", [False, True], ids=["plain", "glv"])
@pytest.mark.parametrize("n", [1, 17, 1000, 2049])
@pytest.mark.parametrize("c,signed", [(4, True), (8, True), (12, True), (7, False)])
def test_precomputed_small_n(split, n, c, signed):
    a, s, pts = msm_inputs(n, tag=100 + n)
    want = closed_form_limbs(s, a)
    pre = pkg.msm_points_precompute(pkg.to_device(pts), c=c, scalar_bits=253, signed=signed, glv=split)
    out = pkg.msm_g1(pre, pkg.to_device(a), c=c, signed=signed, scalar_bits=253, edwards=True, glv=split,
                     precomputed=True)
    torch.cuda.synchronize()
    assert g1.from_limbs(pkg.to_host(out)) == want


def test_precomputed_rows_are_shifted_points():
    """Row i W + j of the set is the stored form of 2^(c j) P_i (oracle's Edwards map)."""
    n, c = 40, 9
    _, s, pts = msm_inputs(n, tag=14)
    pts = pts.copy()
    pts[3] = 0
    pre = pkg.to_host(pkg.msm_points_precompute(pkg.to_device(pts), c=c, scalar_bits=253)).reshape(-1, 36)
    W = -(-(253 + 1) // c)
    assert pre.shape[0] == W * n
    for j in (0, 1, W - 1):
        for i in (0, 3, n - 1):
            P = None if i == 3 else g1.mul(1 << (c * j), g1.from_limbs(pts[i]))
            want = list(edwards.stored_point(edwards.from_weierstrass(P)))
            assert _mont_ints(pre[i * W + j].reshape(3, 12)) == want, (j, i)


@pytest.mark.parametrize("split", [False, True], ids=["plain", "glv"])
def test_precomputed_edges_and_full_width(split):
    n = 700
    a, s, pts = msm_inputs(n, tag=7)
    a, s, pts = a.copy(), s.copy(), pts.copy()
    a[0:10] = 0
    a[10] = synth.int_to_limbs(fq.R - 1, 8)
    a[11] = synth.int_to_limbs(2 ** 256 - 1, 8)
    pts[40] = 0
    s[40] = 0
    want = closed_form_limbs(s, a)
    for c in (5, 13):
        pre = pkg.msm_points_precompute(pkg.to_device(pts), c=c, scalar_bits=256, glv=split)
        out = pkg.msm_g1(pre, pkg.to_device(a), c=c, scalar_bits=256, edwards=True, glv=split, precomputed=True)
        torch.cuda.synchronize()
        assert g1.from_limbs(pkg.to_host(out)) == want


def test_precomputed_heavy_bucket_and_batched():
    n = 5000
    a, s, pts = msm_inputs(n, tag=8)
    a = np.tile(a[:1], (n, 1))
    pre = pkg.msm_points_precompute(pkg.to_device(pts), c=16, scalar_bits=253)
    out = pkg.msm_g1(pre, pkg.to_device(a), c=16, scalar_bits=253, edwards=True, precomputed=True)
    torch.cuda.synchronize()
    assert g1.from_limbs(pkg.to_host(out)) == closed_form_limbs(s, a)
    sizes, cs = [1, 333, 2049, 0], [6, 11, 14, 9]
    data = [msm_inputs(m, tag=78000 + i) for i, m in enumerate(sizes)]
    pres = [pkg.msm_points_precompute(pkg.to_device(p), c=cc, scalar_bits=253)
            for (_, _, p), cc in zip(data, cs)]
    outs = pkg.msm_g1_batched(pres, [pkg.to_device(x) for x, _, _ in data], c_list=cs, scalar_bits=253,
                              edwards=True, precomputed=True)
    torch.cuda.synchronize()
    for i, o in enumerate(outs):
        assert g1.from_limbs(pkg.to_host(o)) == closed_form_limbs(data[i][1], data[i][0]), f"job {i}"


@pytest.mark.parametrize("c", [16, 19])
def test_precomputed_full_size_2e20(c):
    n = 1 << 20
    a, s, pts = msm_inputs(n, tag=2)
    want = closed_form_limbs(s, a)
    pre = pkg.msm_points_precompute(pkg.to_device(pts), c=c, scalar_bits=253)
    da = pkg.to_device(a)
    ws = pkg.msm_g1_workspace(n, c=c, scalar_bits=253, edwards=True, precomputed=True)
    for _ in range(2):
        out = pkg.msm_g1(pre, da, workspace=ws, c=c, scalar_bits=253, edwards=True, precomputed=True)
        torch.cuda.synchronize()
        assert g1.from_limbs(pkg.to_host(out)) == want
    assert pkg.msm_g1_status(ws) == 0


# ---------------------------------------------------------------- window groups (tails overlapped)

@pytest.mark.parametrize("groups", [1, 2, 3, 4, 8])
@pytest.mark.parametrize("edw,split", ALL_MODES, ids=ALL_IDS)
def test_window_groups_give_the_closed_form(edw, split, groups):
    """The accumulation in window groups with each group's tail on the helper stream
    (1, 2, 3, 4, 8 groups over 8 to 16 windows) gives the same exact result."""
    n = 1 << 18
    prep, da, want = _resident(n, 18, edw, split)
    k = 18
    pkg.msm_g1_set_schedule(k, 16, 0, 0, 0, groups, edwards=edw, glv=split)
    try:
        sch = pkg.msm_g1_schedule(n, scalar_bits=253, edwards=edw, glv=split)
        assert sch["c"] == 16 and sch["groups"] == min(groups, 8 if split else 16)
        ws = pkg.msm_g1_workspace(n, scalar_bits=253, prepared=True, edwards=edw, glv=split)
        for _ in range(2):
            out = pkg.msm_g1(prep, da, workspace=ws, scalar_bits=253, prepared=True, edwards=edw, glv=split,
                             profile=True)
            st = pkg.profile_last()
            assert set(st) == {"head", "accumulate", "tail"}
            torch.cuda.synchronize()
            assert g1.from_limbs(pkg.to_host(out)) == want
    finally:
        pkg.msm_g1_set_schedule(k, edwards=edw, glv=split)


def test_window_groups_on_concurrent_streams():
    """Calls on different streams get different helper streams: four MSMs in flight at once
    (each in two window groups) all give their closed forms."""
    n = 1 << 18
    data = [msm_inputs(n, tag=900 + i) for i in range(4)]
    streams = [torch.cuda.Stream() for _ in data]
    outs, wss = [], []
    kw = dict(scalar_bits=253, edwards=True, glv=True, c=15)
    pkg.msm_g1_set_schedule(18, 15, 0, 0, 0, 2, edwards=True, glv=True)
    for (a, s, pts), st in zip(data, streams):
        with torch.cuda.stream(st):
            ws = pkg.msm_g1_workspace(n, **kw)
            wss.append(ws)
            outs.append(pkg.msm_g1(pkg.to_device(pts), pkg.to_device(a), workspace=ws, stream=st, **kw))
    assert pkg.msm_g1_schedule(n, prepared=False, **kw)["groups"] == 2
    torch.cuda.synchronize()
    pkg.msm_g1_set_schedule(18, edwards=True, glv=True)
    for (a, s, _), o in zip(data, outs):
        assert g1.from_limbs(pkg.to_host(o)) == closed_form_limbs(s, a)


@pytest.mark.parametrize("edw,split", [(False, False)] + MODES, ids=["xyzz"] + MODE_IDS)
def test_preparation_beside_the_head(edw, split):
    """From 2^15 standard-form points on, msm_g1 prepares them on a helper stream while
    the digits and the sort run; msm_g1_host prepares each copied chunk on a stream of
    its own. A ragged size with the identity, a duplicate and a negated pair, with
    and without validation, and a point outside the subgroup under validation."""
    n = 40_001
    a, s, pts = msm_inputs(n, tag=515)
    a, s, pts = a.copy(), s.copy(), pts.copy()
    pts[0] = 0
    s[0] = 0
    pts[n - 1] = 0
    s[n - 1] = 0
    pts[20000] = pts[20001]
    s[20000] = s[20001]
    pts[33333, :12] = pts[33334, :12]
    pts[33333, 12:] = synth.int_to_limbs((fq.P - synth.limbs_to_int(pts[33334, 12:])) % fq.P, 12)
    s[33333] = synth.int_to_limbs((fq.R - synth.limbs_to_int(s[33334])) % fq.R, 8)
    want = closed_form_limbs(s, a)
    kw = dict(scalar_bits=253, edwards=edw, glv=split)
    ws = pkg.msm_g1_workspace(n, **kw)
    for validate in (False, True):
        out = pkg.msm_g1(pkg.to_device(pts), pkg.to_device(a), workspace=ws, validate=validate, **kw)
        assert g1.from_limbs(pkg.to_host(out)) == want
        assert pkg.msm_g1_status(ws) == 0
        assert g1.from_limbs(pkg.msm_g1_host(pts, a, validate=validate, **kw)) == want
    cof = pts.copy()
    Q = g1.random_point(0xBADC0DE)
    cof[n - 2] = np.array(g1.to_limbs(Q), dtype=np.uint32)
    pkg.msm_g1(pkg.to_device(cof), pkg.to_device(a), workspace=ws, validate=True, **kw)
    assert pkg.msm_g1_status(ws) == (pkg.ENOTONCURVE if (edw or split) else 0)
    out = pkg.msm_g1(pkg.to_device(pts), pkg.to_device(a), workspace=ws, **kw)
    assert g1.from_limbs(pkg.to_host(out)) == want and pkg.msm_g1_status(ws) == 0


@pytest.mark.parametrize("edw,split", [(False, False)] + MODES, ids=["xyzz"] + MODE_IDS)
def test_few_distinct_scalars_long_runs(edw, split):
    """Scalars drawn from five values plus a random quarter: every window has a few
    buckets holding thousands of points, so many runs cross far more than 8 chunk edges
    (the merge's long-run launch, several such runs per window and per block) next to
    ordinary short runs."""
    n = 24_000
    a, s, pts = msm_inputs(n, tag=517)
    a = a.copy()
    rng = np.random.default_rng(517)
    pick = rng.integers(0, 5, n)
    keep = rng.random(n) < 0.25
    a[~keep] = a[pick[~keep]]
    want = closed_form_limbs(s, a)
    for c, sg in [(6, True), (10, True), (9, False)]:
        assert run(pts, a, c=c, signed=sg, scalar_bits=253, edwards=edw, glv=split) == want


@pytest.mark.parametrize("edw,split", [(False, False)] + MODES, ids=["xyzz"] + MODE_IDS)
def test_short_runs_walked_beside_long_runs(edw, split):
    """Wide windows (c = 13, 14 over 2^14 points: a few items per bucket, so the tail
    thread of each run adds the run's heads itself) with scalars drawn mostly from five
    values: the buckets of those values hold thousands of points and take the log-depth
    merge, while the random quarter's short runs are finished by the walk in the same call."""
    n = 1 << 14
    a, s, pts = msm_inputs(n, tag=611)
    a = a.copy()
    rng = np.random.default_rng(611)
    pick = rng.integers(0, 5, n)
    keep = rng.random(n) < 0.25
    a[~keep] = a[pick[~keep]]
    want = closed_form_limbs(s, a)
    for c in (13, 14):
        assert run(pts, a, c=c, signed=True, scalar_bits=253, edwards=edw, glv=split) == want
    # random scalars only: every run short
    a2, _ = synth.workloads.msm(n, 612)
    assert run(pts, a2, c=14, signed=True, scalar_bits=253, edwards=edw, glv=split) == closed_form_limbs(s, a2)
