"""The GLV endomorphism of BLS12-377 G1 — test infrastructure only.

Not in the paper: a schedule change for its MSM (Sec. II-C) that halves the
number of windows. On y^2 = x^3 + 1 the map phi(x, y) = (beta x, y), beta a
primitive cube root of unity in Fq, is a group endomorphism; on the order-r
subgroup it acts as multiplication by an integer lambda with
lambda^2 + lambda + 1 = 0 mod r (Gallant, Lambert, Vanstone 2001). For the BLS12
family r(x0) = x0^4 - x0^2 + 1, and lambda = x0^2 - 1 satisfies
lambda^2 + lambda + 1 = r(x0) exactly, as integers. beta is the one of the two
primitive cube roots for which phi(G) = lambda G.

A scalar 0 <= k < r splits as k = k1 + lambda k2 with k2 = floor(k / lambda) and
k1 = k mod lambda. Because r - 1 = lambda (lambda + 1), k2 <= lambda + 1, and both
halves are below 2^127. So sum_i k_i P_i = sum_i k1_i P_i + sum_i k2_i phi(P_i): an
MSM over 2n points with 127-bit scalars.
"""
from __future__ import annotations

from . import fq, g1, msm
from .fq import P, R, X0

LAMBDA = X0 * X0 - 1


def _cube_roots():
    # a primitive cube root of unity: g^((p-1)/3) for the first g that does not give 1
    for g in range(2, 100):
        b = pow(g, (P - 1) // 3, P)
        if b != 1:
            return b, b * b % P
    raise AssertionError("no primitive cube root found")


def _pick_beta():
    lam_g = g1.mul(LAMBDA, g1.G)
    for b in _cube_roots():
        if (b * g1.GX % P, g1.GY) == lam_g:
            return b
    raise AssertionError("no cube root matches lambda on G")


BETA = _pick_beta()


def phi(pt):
    if pt is None:
        return None
    return (BETA * pt[0] % P, pt[1])


def decompose(k: int):
    """k = k1 + LAMBDA * k2 with 0 <= k1 < LAMBDA; scalars are first reduced mod r."""
    k %= R
    k2, k1 = divmod(k, LAMBDA)
    return k1, k2


def msm_glv(points, scalars, c: int, signed: bool = True):
    """Pippenger over (P_i, phi(P_i)) with the 127-bit halves (subgroup points only)."""
    pts, scs = [], []
    for pt, s in zip(points, scalars):
        k1, k2 = decompose(int(s))
        pts.append(pt)
        scs.append(k1)
        pts.append(phi(pt))
        scs.append(k2)
    return msm.pippenger(pts, scs, c, signed=signed, scalar_bits=127)
