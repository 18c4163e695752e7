"""GPU parity of the dependent-chain experiment (Sec. V-A): padd_chain sums a point
stream strictly in order; the result must equal the closed form sum_i s_i G for
P_i = s_i G, for the XYZZ model on one thread and the Edwards model on one lane,
four lanes and four warps, including repeated points (P + P) and cancelling pairs
(P + (-P))."""
import numpy as np
import pytest
import torch

import synth
from oracle import fq, g1
from tests.util import oracle_points

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2502_11660_gb300")

VARIANTS = [(False, 1), (True, 1), (True, 4), (True, 128)]


def _stream(n, tag):
    if n == 0:
        return np.zeros((0, 8), dtype=np.uint32), np.zeros((0, 24), dtype=np.uint32)
    seeds = synth.scalars(synth.stream_seed(tag, n, 5), n).copy()
    if n > 40:
        seeds[10] = seeds[9]                     # P + P in the middle of the chain
        seeds[21] = synth.int_to_limbs((fq.R - synth.limbs_to_int(seeds[20])) % fq.R, 8)  # P + (-P)
        seeds[30] = 0                            # the identity
    return seeds, oracle_points(seeds)


def _want(seeds):
    k = sum(synth.limbs_to_int(s) for s in seeds) % fq.R
    return g1.mul(k, g1.G)


@pytest.mark.parametrize("edwards,lanes", VARIANTS, ids=["xyzz-1", "edwards-1", "edwards-4", "edwards-128"])
@pytest.mark.parametrize("n", [0, 1, 2, 3, 100, 4096])
def test_chain_sum(edwards, lanes, n):
    seeds, pts = _stream(n, tag=31 + n)
    st = pkg.msm_points_prepare(pkg.to_device(pts), edwards=edwards)
    out = pkg.padd_chain(st, n, edwards=edwards, lanes=lanes)
    torch.cuda.synchronize()
    assert g1.from_limbs(pkg.to_host(out)) == _want(seeds)


def test_chain_rejects_bad_arguments():
    L = pkg.lib()
    assert L.padd_chain(None, 0, None, 0, 1, None) == -1
    out = torch.empty(24, dtype=torch.int32, device="cuda")
    assert L.padd_chain(None, 0, out.data_ptr(), 0, 4, None) == -1          # four lanes need Edwards
    assert L.padd_chain(None, 0, out.data_ptr(), 0, 128, None) == -1        # so do four warps
    assert L.padd_chain(None, 0, out.data_ptr(), pkg.GLV, 1, None) == -1
    assert L.padd_chain(None, 0, out.data_ptr(), pkg.EDWARDS, 3, None) == -1
