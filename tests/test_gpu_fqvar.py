"""GPU parity of the alternative multiplications (fq_mul_batch_variant) vs Python
integers: the paper's Barrett reduction (Sec. III-C; also checked against the
oracle's own Barrett), the Karatsuba-top Montgomery product and the carry-save
radix-2^24 Montgomery product, the two-pass-row CIOS product and the one-warp-per-
product form of the window chains, all bit-exact and canonical."""
import random

import pytest

import synth
from oracle import barrett, fq
from tests.test_gpu_fq import EDGE
from tests.util import ints_of_soa, soa_of_ints

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2502_11660_gb300")

RINV = pow(1 << 384, -1, fq.P)
VARIANTS = {
    "cios": (0, lambda x, y: x * y * RINV % fq.P),
    "barrett": (1, lambda x, y: x * y % fq.P),
    "karatsuba": (2, lambda x, y: x * y * RINV % fq.P),
    "carrysave": (3, lambda x, y: x * y * RINV % fq.P),
    "cios_twopass": (4, lambda x, y: x * y * RINV % fq.P),
    "cios_doublerow": (5, lambda x, y: x * y * RINV % fq.P),
    "warp": (6, lambda x, y: x * y * RINV % fq.P),
    "fips": (8, lambda x, y: x * y * RINV % fq.P),
    "cios_singlerow": (9, lambda x, y: x * y * RINV % fq.P),
}


def _inputs():
    pairs = [(x, y) for x in EDGE for y in EDGE]
    rng = random.Random(17)
    pairs += [(rng.randrange(fq.P), rng.randrange(fq.P)) for _ in range(3 * 2048 + 29)]
    a, b = synth.workloads.fq_pairs(4096, tag=12)
    pairs += list(zip(ints_of_soa(a.T.copy()), ints_of_soa(b.T.copy())))
    return pairs


@pytest.mark.parametrize("name", list(VARIANTS))
def test_variant_matches_python_integers(name):
    variant, want = VARIANTS[name]
    pairs = _inputs()
    A = soa_of_ints([x for x, _ in pairs])
    B = soa_of_ints([y for _, y in pairs])
    got = ints_of_soa(pkg.to_host(pkg.fq_mul_batch_variant(pkg.to_device(A), pkg.to_device(B), variant)))
    assert got == [want(x, y) for x, y in pairs]


def test_barrett_matches_the_papers_reduction_in_the_oracle():
    pairs = [(x, y) for x in EDGE[:8] for y in EDGE[:8]]
    A = soa_of_ints([x for x, _ in pairs])
    B = soa_of_ints([y for _, y in pairs])
    got = ints_of_soa(pkg.to_host(pkg.fq_mul_batch_variant(pkg.to_device(A), pkg.to_device(B), 1)))
    assert got == [barrett.barrett_mulmod(x, y, fq.P) for x, y in pairs]


def test_unknown_variant_is_rejected():
    assert pkg.lib().fq_mul_batch_variant(None, None, None, 4, 10, None) == -1


def test_warp_product_on_unreduced_operands_and_carry_runs():
    """The warp form takes operands below 8p (the unreduced sums and differences of the
    point formulas). Edge values make the carry resolution run through every lane:
    all-ones limbs, 2^k - 1 and 2^k, multiples of p and 8p - 1."""
    rng = random.Random(99)
    edges = [0, 1, 2, fq.P - 1, fq.P, fq.P + 1, 2 * fq.P - 1, 2 * fq.P, 4 * fq.P - 1, 6 * fq.P + 3,
             8 * fq.P - 1, (1 << 376) - 1, 1 << 376, (1 << 379) - 1, (1 << 32) - 1, (1 << 64) - 1,
             int("ffffffff" * 11, 16), (1 << 352) - (1 << 32)]
    edges = [e for e in edges if e < 8 * fq.P]
    pairs = [(x, y) for x in edges for y in edges]
    pairs += [(rng.randrange(8 * fq.P), rng.randrange(8 * fq.P)) for _ in range(5000)]
    A = soa_of_ints([x for x, _ in pairs])
    B = soa_of_ints([y for _, y in pairs])
    got = ints_of_soa(pkg.to_host(pkg.fq_mul_batch_variant(pkg.to_device(A), pkg.to_device(B), 6)))
    assert got == [x * y * RINV % fq.P for x, y in pairs]


def test_paper_format_equals_the_oracles_loose_barrett():
    """MSM377_FQMUL_PAPER (16 x 25-bit elements, two-round coarse carry, the looser
    Barrett step with k = 378; Sec. III-B .. III-E) returns exactly the oracle's
    remainder in [0, 4p) for operands below 6p, including the largest ones."""
    rng = random.Random(35)
    top = 6 * fq.P
    edges = [0, 1, fq.P - 1, fq.P, 3 * fq.P - 1, 4 * fq.P + 7, top - 1, top - 2, (1 << 379) - 1,
             (1 << 377) - 1, 1 << 375, int("1ffffff" * 15, 16) % top]
    pairs = [(x, y) for x in edges for y in edges]
    pairs += [(rng.randrange(top), rng.randrange(top)) for _ in range(6000)]
    pairs += [(top - 1 - rng.randrange(1 << 300), top - 1 - rng.randrange(1 << 300)) for _ in range(500)]
    A = soa_of_ints([x for x, _ in pairs])
    B = soa_of_ints([y for _, y in pairs])
    got = ints_of_soa(pkg.to_host(pkg.fq_mul_batch_variant(pkg.to_device(A), pkg.to_device(B), pkg.FQMUL_PAPER)))
    want = [barrett.barrett_reduce_loose(x * y, fq.P) for x, y in pairs]
    assert got == want
    assert all(0 <= r < 4 * fq.P for r in got)
