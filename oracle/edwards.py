"""The twisted Edwards model of BLS12-377 G1 — test infrastructure only.

Sec. II-D of the paper converts BLS12-377 into the twisted Edwards curve
    -x^2 + y^2 = 1 + (k/2) x^2 y^2
and adds points in extended coordinates (X, Y, T, Z), x = X/Z, y = Y/Z, T = XY/Z
(Hisil et al. 2008); the points streamed into bucket accumulation carry U = k T
with Z = 1. The paper prints neither the map from y^2 = x^3 + 1 nor k. Both follow
from the curve, in three steps:

1. The 2-torsion point (-1, 0) moves to the origin: x = s u - 1 with s^2 = 3 turns
   y^2 = x^3 + 1 into y^2 = s^3 u^3 - 9 u^2 + 3 s u, i.e. the Montgomery curve
   B v^2 = u^3 + A u^2 + u with A = -s, B = 1/s^3 and v = y.
2. A Montgomery curve is birational to the twisted Edwards curve
   a x^2 + y^2 = 1 + d x^2 y^2 with a = (A + 2)/B, d = (A - 2)/B, through
   x = u / v, y = (u - 1)/(u + 1) (Bernstein, Birkner, Joye, Lange, Peters 2008).
3. With gamma^2 = -a, x' = gamma x gives a = -1 and d' = -d / a; the paper's k is
   2 d' (so its "k/2" is d').

s is the smaller of the two square roots of 3 in [0, p), gamma the smaller root
of -a; other choices give other, equally valid, isomorphic curves.

The Edwards group law used here is the textbook affine one for a = -1:
    x3 = (x1 y2 + y1 x2) / (1 + d x1 x2 y1 y2),  y3 = (y1 y2 + x1 x2) / (1 - d x1 x2 y1 y2),
identity (0, 1), -(x, y) = (-x, y). d' is a square in Fq, so the law has
exceptional pairs; none lies in the odd-order subgroup, and `add` raises if a
denominator vanishes instead of returning a wrong point.
"""
from __future__ import annotations

from . import fq, g1
from .fq import P


def _small_root(a: int) -> int:
    r = fq.sqrt(a)
    if r is None:
        raise ValueError("not a square")
    return min(r, (P - r) % P)


S = _small_root(3)                                  # s^2 = 3
A_MONT = (-S) % P                                   # Montgomery A
B_MONT = fq.inv(S * S % P * S % P)                  # Montgomery B = 1/s^3
A_TE = (A_MONT + 2) * fq.inv(B_MONT) % P            # twisted Edwards a before scaling
D_TE = (A_MONT - 2) * fq.inv(B_MONT) % P            # twisted Edwards d before scaling
GAMMA = _small_root((-A_TE) % P)                    # gamma^2 = -a
D = (-D_TE) * fq.inv(A_TE) % P                      # d' of -x^2 + y^2 = 1 + d' x^2 y^2
K = 2 * D % P                                       # the paper's k

IDENTITY = (0, 1)


def on_curve(pt) -> bool:
    x, y = pt
    return 0 <= x < P and 0 <= y < P and (-x * x + y * y - 1 - D * x * x % P * y * y) % P == 0


def neg(pt):
    return ((-pt[0]) % P, pt[1])


def add(p1, p2):
    """Affine addition on -x^2 + y^2 = 1 + d x^2 y^2 (every case by the same rule)."""
    x1, y1 = p1
    x2, y2 = p2
    t = D * x1 % P * x2 % P * y1 % P * y2 % P
    den_x = (1 + t) % P
    den_y = (1 - t) % P
    if den_x == 0 or den_y == 0:
        raise ArithmeticError("exceptional pair for the Edwards addition law")
    x3 = (x1 * y2 + y1 * x2) % P * fq.inv(den_x) % P
    y3 = (y1 * y2 + x1 * x2) % P * fq.inv(den_y) % P
    return (x3, y3)


def mul(k: int, pt):
    if k < 0:
        return mul(-k, neg(pt))
    acc = IDENTITY
    for bit in bin(k)[2:] if k else "":
        acc = add(acc, acc)
        if bit == "1":
            acc = add(acc, pt)
    return acc


def from_weierstrass(pt):
    """Image of a Weierstrass point (affine, None = O) on the Edwards curve."""
    if pt is None:
        return IDENTITY
    x, y = pt
    u = (x + 1) * fq.inv(S) % P
    if y == 0 or (u + 1) % P == 0:
        raise ValueError("point outside the domain of the map (order 2 or 4 on the Montgomery curve)")
    xe = u * fq.inv(y) % P
    ye = (u - 1) * fq.inv(u + 1) % P
    return (GAMMA * xe % P, ye)


def to_weierstrass(pt):
    """Inverse of from_weierstrass; (0, 1) gives None (= O)."""
    xs, ye = pt
    if xs == 0:
        if ye == 1:
            return None
        raise ValueError("(0, -1) has order 2 and is not the image of a subgroup point")
    xe = xs * fq.inv(GAMMA) % P
    u = (1 + ye) * fq.inv((1 - ye) % P) % P
    v = u * fq.inv(xe) % P
    return ((S * u - 1) % P, v)


def stored_point(pt):
    """The form the paper streams into bucket accumulation: (X, Y, U = k T) with Z = 1."""
    x, y = pt
    return (x, y, K * x % P * y % P)


def extended(pt, z: int = 1):
    """Extended coordinates (X, Y, Z, T) of an affine point, scaled by z != 0."""
    x, y = pt
    return (x * z % P, y * z % P, z % P, x * y % P * z % P)


def from_extended(e):
    X, Y, Z, T = e
    zi = fq.inv(Z)
    return (X * zi % P, Y * zi % P)


def weierstrass_is_subgroup(pt) -> bool:
    return g1.mul(fq.R, pt) is None
