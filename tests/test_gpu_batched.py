"""GPU parity: msm_g1_batched (many MSMs of uneven n in one call) vs the closed form
and vs one msm_g1 call per job; and the same batch captured in a CUDA graph."""
import numpy as np
import pytest
import torch

import synth
from oracle import g1
from tests.util import closed_form_limbs, msm_inputs

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2502_11660_gb300")


def _batch(sizes, tag):
    data = [msm_inputs(n, tag=tag * 1000 + i) for i, n in enumerate(sizes)]
    pts = [pkg.to_device(p) for _, _, p in data]
    scs = [pkg.to_device(a) for a, _, _ in data]
    want = [closed_form_limbs(s, a) for a, s, _ in data]
    return data, pts, scs, want


def test_batched_uneven_sizes_and_windows():
    sizes = [0, 1, 2, 7, 64, 333, 1000, 2049, 4096, 5000, 17, 900]
    cs = [0, 0, 4, 5, 6, 0, 9, 10, 0, 12, 3, 8]
    data, pts, scs, want = _batch(sizes, tag=41)
    outs = pkg.msm_g1_batched(pts, scs, c_list=cs, scalar_bits=253)
    torch.cuda.synchronize()
    for i, o in enumerate(outs):
        assert g1.from_limbs(pkg.to_host(o)) == want[i], f"job {i} (n={sizes[i]})"
        if sizes[i]:
            ref = pkg.msm_g1(pts[i], scs[i], c=cs[i], scalar_bits=253)
            torch.cuda.synchronize()
            assert np.array_equal(pkg.to_host(ref), pkg.to_host(o))


def test_batched_log_uniform_sizes_prepared_points():
    sizes = synth.workloads.batch_sizes(njobs=24, lo_log2=10, hi_log2=14, tag=7).tolist()
    data, pts, scs, want = _batch(sizes, tag=42)
    prep = [pkg.msm_points_prepare(p) for p in pts]
    outs = pkg.msm_g1_batched(prep, scs, prepared=True, scalar_bits=253)
    torch.cuda.synchronize()
    for i, o in enumerate(outs):
        assert g1.from_limbs(pkg.to_host(o)) == want[i], f"job {i} (n={sizes[i]})"


def test_batched_in_a_cuda_graph():
    sizes = [300, 1500, 64, 4000]
    data, pts, scs, want = _batch(sizes, tag=43)
    ws = pkg.msm_g1_batched_workspace(pts, scalar_bits=253)
    outs = [torch.empty(24, dtype=torch.int32, device="cuda") for _ in sizes]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        pkg.msm_g1_batched(pts, scs, outs=outs, workspace=ws, scalar_bits=253, stream=s)  # creates helpers
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        pkg.msm_g1_batched(pts, scs, outs=outs, workspace=ws, scalar_bits=253, stream=s)
    for trial in range(2):
        new = [synth.scalars(500 + 10 * trial + i, n) for i, n in enumerate(sizes)]
        for d, h in zip(scs, new):
            d.copy_(pkg.to_device(h))
        for o in outs:
            o.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        for i, o in enumerate(outs):
            assert g1.from_limbs(pkg.to_host(o)) == closed_form_limbs(data[i][1], new[i])
