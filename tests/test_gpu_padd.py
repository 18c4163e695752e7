"""GPU parity: batched mixed PADD (XYZZ + affine) vs the chord/tangent rule, every case."""
import random

import numpy as np
import pytest

import synth
from oracle import fq, g1
from tests.util import ints_of_soa, oracle_points, soa_of_ints, xyzz_to_affine_int

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2502_11660_gb300")


def _scaled(pt, lam):
    """XYZZ representative (l^2 x, l^3 y, l^2, l^3) of an affine point (O -> zeros)."""
    if pt is None:
        return (0, 0, 0, 0)
    l2 = lam * lam % fq.P
    l3 = l2 * lam % fq.P
    return (pt[0] * l2 % fq.P, pt[1] * l3 % fq.P, l2, l3)


def _build(n, tag, edge_rate):
    sa, sq, lam, case = synth.workloads.padd_plan(n, tag, edge_rate)
    PA = oracle_points(sa, key=("padd_a", n, tag))
    PQ = oracle_points(sq, key=("padd_q", n, tag))
    accs, qs, want = [], [], []
    for i in range(n):
        A = g1.from_limbs(PA[i])
        Q = g1.from_limbs(PQ[i])
        cs = int(case[i])
        if cs == 1:
            Q = A
        elif cs == 2:
            Q = g1.neg(A)
        elif cs == 3:
            A = None
        elif cs == 4:
            Q = None
        l = synth.limbs_to_int(lam[i]) or 1
        accs.append(_scaled(A, l))
        qs.append(Q)
        want.append(g1.add(A, Q))
    acc = np.stack([soa_of_ints([a[c] for a in accs]) for c in range(4)])
    q = np.stack([soa_of_ints([0 if p is None else p[c] for p in qs]) for c in range(2)])
    return acc, q, want, case


def _check(res, want):
    cols = [ints_of_soa(res[c]) for c in range(4)]
    for i, w in enumerate(want):
        got = xyzz_to_affine_int(cols[0][i], cols[1][i], cols[2][i], cols[3][i])
        assert got == w, f"op {i}"


@pytest.mark.parametrize("edge_rate", [0.01, 0.2])
def test_padd_standard_form_all_cases(edge_rate):
    n = 2 * 2048 + 11
    acc, q, want, case = _build(n, tag=21, edge_rate=edge_rate)
    assert set(np.unique(case).tolist()) == {0, 1, 2, 3, 4}
    res = pkg.to_host(pkg.padd_batch(pkg.to_device(acc), pkg.to_device(q)))
    _check(res, want)


def test_padd_montgomery_form_and_alias():
    n = 1500
    acc, q, want, _ = _build(n, tag=22, edge_rate=0.05)
    dacc = pkg.to_device(acc)
    dq = pkg.to_device(q)
    # convert coordinate by coordinate (each [12][n] block)
    m = dacc.clone()
    for c in range(4):
        m[c] = pkg.fq_to_montgomery(dacc[c].contiguous())
    mq = dq.clone()
    for c in range(2):
        mq[c] = pkg.fq_to_montgomery(dq[c].contiguous())
    pkg.padd_batch(m, mq, out=m, form=pkg.FORM_MONTGOMERY)   # out aliases acc
    res = m.clone()
    for c in range(4):
        res[c] = pkg.fq_from_montgomery(m[c].contiguous())
    _check(pkg.to_host(res), want)


def test_padd_two_torsion_and_identities():
    T = (fq.P - 1, 0)
    G = g1.G
    cases = [(T, T), (T, None), (None, T), (None, None), (G, G), (G, g1.neg(G)), (G, T)]
    accs = [_scaled(a, 5) for a, _ in cases]
    acc = np.stack([soa_of_ints([a[c] for a in accs]) for c in range(4)])
    q = np.stack([soa_of_ints([0 if b is None else b[c] for _, b in cases]) for c in range(2)])
    res = pkg.to_host(pkg.padd_batch(pkg.to_device(acc), pkg.to_device(q)))
    _check(res, [g1.add(a, b) for a, b in cases])
