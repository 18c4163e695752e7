"""Multi-scalar multiplication, sum_i s_i * P_i, by definition and by Pippenger — test infrastructure only.

Sec. II-C of the paper: Pippenger splits k-bit scalars into w-bit windows
(k/w groups), adds each point into the bucket its window digit selects (bucket
accumulation), reduces each group's buckets to sum_b b * B_b (bucket
aggregation) and combines the groups with their 2^(w*j) weights (group
aggregation). Pippenger is only a faster schedule for the same unique group
element, so `naive_msm` (the definition) is the truth and `pippenger` must equal
it.
"""
from __future__ import annotations

from . import g1
from .fq import R


def naive_msm(points, scalars):
    acc = None
    for pt, s in zip(points, scalars):
        acc = g1.add(acc, g1.mul(int(s), pt))
    return acc


def closed_form(seeds, scalars):
    """For P_i = seeds_i * G: sum_i a_i P_i = ((sum_i a_i seeds_i) mod r) * G."""
    k = sum(int(a) * int(s) for a, s in zip(scalars, seeds)) % R
    return g1.mul(k, g1.G)


def unsigned_digits(s: int, c: int, nwin: int):
    return [(s >> (c * j)) & ((1 << c) - 1) for j in range(nwin)]


def signed_digits(s: int, c: int, nwin: int):
    """Digits d_j in (-2^(c-1), 2^(c-1)] with sum_j d_j 2^(c j) = s.

    A raw window value plus incoming carry v > 2^(c-1) becomes v - 2^c and
    carries 1 into the next window. With nwin * c >= bits(s) + 1 the top window
    is at most 2^(c-1) - 1 + 1 and never carries out, so |d_j| <= 2^(c-1) and the
    buckets are 1 .. 2^(c-1).
    """
    if c < 2:
        raise ValueError("signed digits need c >= 2")
    half = 1 << (c - 1)
    out, carry = [], 0
    for j in range(nwin):
        v = ((s >> (c * j)) & ((1 << c) - 1)) + carry
        if v > half:
            out.append(v - (1 << c))
            carry = 1
        else:
            out.append(v)
            carry = 0
    assert carry == 0, "too few windows for signed digits"
    return out


def pippenger(points, scalars, c: int, signed: bool = False, scalar_bits: int | None = None):
    """Textbook bucket method (Sec. II-C): windows, buckets, aggregation, combination."""
    n = len(points)
    if n == 0:
        return None
    bits = scalar_bits or max(1, max(int(s).bit_length() for s in scalars))
    nwin = -(-(bits + (1 if signed else 0)) // c)
    nb = (1 << (c - 1)) if signed else (1 << c) - 1
    digits = [signed_digits(int(s), c, nwin) if signed else unsigned_digits(int(s), c, nwin)
              for s in scalars]
    window_sums = []
    for j in range(nwin):
        buckets = [None] * (nb + 1)          # buckets[d] for d = 1..nb
        for pt, dg in zip(points, digits):
            d = dg[j]
            if d == 0:
                continue
            q = pt if d > 0 else g1.neg(pt)
            buckets[abs(d)] = g1.add(buckets[abs(d)], q)
        # bucket aggregation: sum_b b * B_b with running sums from the top bucket
        running, total = None, None
        for b in range(nb, 0, -1):
            running = g1.add(running, buckets[b])
            total = g1.add(total, running)
        window_sums.append(total)
    # group aggregation: Horner over windows from the top
    acc = None
    for j in range(nwin - 1, -1, -1):
        for _ in range(c):
            acc = g1.add(acc, acc)
        acc = g1.add(acc, window_sums[j])
    return acc
