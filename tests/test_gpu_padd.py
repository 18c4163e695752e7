"""GPU parity: batched mixed PADD (XYZZ + affine) vs the chord/tangent rule, every case."""
import random

import numpy as np
import pytest
import torch

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


def test_padd_full_size_2e24_sampled_with_edge_cases():
    """2^24 mixed additions in one call, the size the bench times (every thread runs many
    grid-stride rounds), with 1 % each of P + P, P + (-P), acc = O and Q = O; sampled
    rows, every special case among them, against the chord/tangent rule. Operands come
    from oracle pools: affine points, their negations and XYZZ representatives in a
    random scaling (l^2 x, l^3 y, l^2, l^3)."""
    n, m = 1 << 24, 4096
    pool = oracle_points(synth.scalars(synth.stream_seed(24, m, 1), m), key=("padd_pool", m))
    lam = synth.field_elems(synth.stream_seed(24, m, 2), m)
    pts = [g1.from_limbs(pool[j]) for j in range(m)]
    accs = [_scaled(P, synth.limbs_to_int(lam[j]) or 1) for j, P in enumerate(pts)]
    acc_pool = np.stack([soa_of_ints([a[c] for a in accs]) for c in range(4)])       # (4, 12, m)
    neg = np.array([g1.to_limbs(g1.neg(P)) for P in pts], dtype=np.uint32)
    q_pool = np.concatenate([pool, neg])                                              # (2m, 24)
    case = synth.workloads.padd_cases(n, tag=24, edge_rate=0.01)
    ia = synth.small_ints(synth.stream_seed(24, n, 3), n, m).astype(np.int64)
    iq = synth.small_ints(synth.stream_seed(24, n, 4), n, m).astype(np.int64)
    iq = np.where(case == 1, ia, iq)
    iq = np.where(case == 2, ia + m, iq)
    dia, diq = torch.from_numpy(ia).cuda(), torch.from_numpy(iq).cuda()
    dcase = torch.from_numpy(case).cuda()
    acc = pkg.to_device(acc_pool)[:, :, dia]
    Q = pkg.to_device(q_pool)[diq]
    q = torch.stack([Q[:, :12].T.contiguous(), Q[:, 12:].T.contiguous()])
    del Q
    acc[:, :, dcase == 3] = 0
    q[:, :, dcase == 4] = 0
    out = pkg.padd_batch(acc, q)
    torch.cuda.synchronize()
    rng = random.Random(24)
    rows = sorted(set(rng.sample(range(n), 3000)) |
                  {int(i) for k in (1, 2, 3, 4) for i in np.nonzero(case == k)[0][:200]})
    sub = pkg.to_host(out[:, :, torch.tensor(rows, device="cuda")].contiguous())
    for col, i in enumerate(rows):
        A = None if case[i] == 3 else pts[ia[i]]
        Qi = None if case[i] == 4 else (pts[iq[i]] if iq[i] < m else g1.neg(pts[iq[i] - m]))
        X, Y, ZZ, ZZZ = (synth.limbs_to_int(sub[c, :, col]) for c in range(4))
        assert xyzz_to_affine_int(X, Y, ZZ, ZZZ) == g1.add(A, Qi), f"op {i} case {case[i]}"
    assert {int(case[i]) for i in rows} == {0, 1, 2, 3, 4}
