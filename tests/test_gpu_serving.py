"""Serving: continuous batching over resident point sets.

The same requests are served once all together (admitted as slots free up, their
work overlapping on the GPU) and once each alone; every result must be identical
(the tolerance is zero: results are exact group elements) and equal to the
closed form for its point seeds and scalars.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import g1
from tests.util import closed_form_limbs

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2502_11660_gb300")
from paper_2502_11660_gb300 import serving  # noqa: E402


@pytest.fixture(scope="module")
def sets():
    size = 1 << 14
    seeds = [synth.scalars(synth.stream_seed(4, size, 700 + k), size) for k in range(2)]
    return seeds, serving.ResidentSets(seeds)


def _requests(n_req, tag):
    gaps, n, setid, offs = synth.workloads.requests(n_req, 8, 13, 2, 1 << 14, tag)
    return [serving.Request(i, 0.0, int(setid[i]), int(offs[i]), int(n[i]), 1000 + 7 * i) for i in range(n_req)]


def test_results_alone_equal_results_in_the_mix(sets):
    seeds, rs = sets
    reqs = _requests(24, tag=71)
    mix = serving.MsmServer(rs, slots=8).run(reqs, realtime=False)
    assert mix["requests"] == len(reqs)
    assert mix["max_inflight"] > 1                      # work really overlapped
    alone = serving.MsmServer(rs, slots=1)
    for r in reqs:
        one = alone.run([serving.Request(r.rid, 0.0, r.set_id, r.offset, r.n, r.seed)], realtime=False)
        assert np.array_equal(one["results"][r.rid], mix["results"][r.rid]), f"request {r.rid}"
    for r in reqs[:6]:
        sc = pkg.to_host(serving.device_scalars(r.n, r.seed, "cuda"))
        want = closed_form_limbs(seeds[r.set_id][r.offset:r.offset + r.n], sc)
        assert g1.from_limbs(mix["results"][r.rid]) == want


def test_poisson_stream_and_footprint_admission(sets):
    seeds, rs = sets
    reqs = serving.poisson_requests(40, rate=400.0, nsets=2, set_size=1 << 14, lo_log2=8, hi_log2=13, tag=72)
    srv = serving.MsmServer(rs, slots=4)
    rep = srv.run(reqs, realtime=True)
    assert rep["requests"] == 40 and rep["p99_ms"] >= rep["p50_ms"] > 0
    # a budget that fits only the largest single request still completes everything
    budget = max(srv.footprint(r.n) for r in reqs[:10]) + 1
    tight = serving.MsmServer(rs, slots=4, mem_budget=budget)
    rep2 = tight.run(reqs[:10], realtime=False)
    assert rep2["requests"] == 10 and rep2["max_footprint_bytes"] <= tight.mem_budget
    for r in reqs[:10]:
        assert np.array_equal(rep2["results"][r.rid], rep["results"][r.rid])


def test_edwards_glv_sets_serve_the_same_results(sets):
    """Resident sets in the Edwards stored form with the GLV rows interleaved: slices
    of them give the same exact results as the XYZZ sets."""
    seeds, rs = sets
    rs2 = serving.ResidentSets(seeds, edwards=True, glv=True)
    reqs = _requests(12, tag=73)
    a = serving.MsmServer(rs, slots=4).run(reqs, realtime=False)
    b = serving.MsmServer(rs2, slots=4).run(reqs, realtime=False)
    for r in reqs:
        assert np.array_equal(a["results"][r.rid], b["results"][r.rid]), f"request {r.rid}"


def test_precomputed_sets_serve_the_same_results(sets):
    """Fixed-base resident sets (point-major rows): slices give the same exact results."""
    seeds, rs = sets
    rs3 = serving.ResidentSets(seeds, precompute_c=11, glv=True)
    reqs = _requests(12, tag=74)
    a = serving.MsmServer(rs, slots=4).run(reqs, realtime=False)
    b = serving.MsmServer(rs3, slots=4).run(reqs, realtime=False)
    for r in reqs:
        assert np.array_equal(a["results"][r.rid], b["results"][r.rid]), f"request {r.rid}"
