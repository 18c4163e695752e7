"""GPU parity: batched Fq multiplication and form conversion vs Python integers (exact)."""
import random

import numpy as np
import pytest
import torch

import synth
from oracle import fq
from tests.util import ints_of_soa, soa_of_ints

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2502_11660_gb300")

EDGE = [0, 1, 2, 3, fq.P - 1, fq.P - 2, (fq.P - 1) // 2, (fq.P + 1) // 2,
        (1 << 32) % fq.P, (1 << 64) % fq.P, (1 << 376), (1 << 383) % fq.P, (1 << 384) % fq.P,
        fq.P - (1 << 32), fq.P - (1 << 200), 0xFFFFFFFF, (1 << 376) - 1]


def _mont(v):
    return v * (1 << 384) % fq.P


def test_fq_mul_standard_random_and_ragged():
    n = 3 * 2048 + 37   # several blocks and a ragged tail
    a, b = synth.workloads.fq_pairs(n, tag=11)
    A, B = a.T.copy(), b.T.copy()
    got = ints_of_soa(pkg.to_host(pkg.fq_mul_batch(pkg.to_device(A), pkg.to_device(B))))
    av, bv = ints_of_soa(A), ints_of_soa(B)
    assert got == [x * y % fq.P for x, y in zip(av, bv)]


def test_fq_mul_edge_values_all_pairs():
    pairs = [(x, y) for x in EDGE for y in EDGE]
    A = soa_of_ints([x for x, _ in pairs])
    B = soa_of_ints([y for _, y in pairs])
    got = ints_of_soa(pkg.to_host(pkg.fq_mul_batch(pkg.to_device(A), pkg.to_device(B))))
    assert got == [x * y % fq.P for x, y in pairs]


def test_fq_mul_montgomery_form_and_conversions():
    rng = random.Random(3)
    vals_a = EDGE + [rng.randrange(fq.P) for _ in range(2000)]
    vals_b = [rng.randrange(fq.P) for _ in range(len(vals_a))]
    A, B = soa_of_ints(vals_a), soa_of_ints(vals_b)
    dA, dB = pkg.to_device(A), pkg.to_device(B)
    mA, mB = pkg.fq_to_montgomery(dA), pkg.fq_to_montgomery(dB)
    assert ints_of_soa(pkg.to_host(mA)) == [_mont(v) for v in vals_a]
    prod_m = pkg.fq_mul_batch(mA, mB, form=pkg.FORM_MONTGOMERY)
    assert ints_of_soa(pkg.to_host(prod_m)) == [_mont(x * y) for x, y in zip(vals_a, vals_b)]
    back = pkg.fq_from_montgomery(prod_m)
    assert ints_of_soa(pkg.to_host(back)) == [x * y % fq.P for x, y in zip(vals_a, vals_b)]
    # out aliasing an input
    pkg.fq_mul_batch(dA, dB, out=dA)
    assert ints_of_soa(pkg.to_host(dA)) == [x * y % fq.P for x, y in zip(vals_a, vals_b)]


def test_fq_mul_empty_and_bad_form():
    e = torch.zeros((12, 0), dtype=torch.int32, device="cuda")
    pkg.fq_mul_batch(e, e)
    x = pkg.to_device(soa_of_ints([1, 2, 3]))
    with pytest.raises(pkg.MsmError):
        pkg.fq_mul_batch(x, x, form=7)


def test_fq_mul_full_size_sampled():
    """2^24 multiplications as the benchmark launches them; 4096 sampled outputs checked exactly."""
    n = 1 << 24
    a, b = synth.workloads.fq_pairs(n, tag=1)
    dA = pkg.to_device(a.T.copy())
    dB = pkg.to_device(b.T.copy())
    mA, mB = pkg.fq_to_montgomery(dA), pkg.fq_to_montgomery(dB)
    out = pkg.to_host(pkg.fq_from_montgomery(pkg.fq_mul_batch(mA, mB, form=pkg.FORM_MONTGOMERY)))
    idx = np.unique(np.concatenate([np.arange(64), n - 1 - np.arange(64),
                                    synth.small_ints(5, 4096, n)]))
    for i in idx.tolist():
        x, y = synth.limbs_to_int(a[i]), synth.limbs_to_int(b[i])
        assert synth.limbs_to_int(out[:, i]) == x * y % fq.P
