"""The group law on BLS12-377 G1, E: y^2 = x^3 + 1 over GF(p) — test infrastructure only.

Sec. II-D of the paper defines the point addition (PADD) that MSM reduces to; it
uses a twisted Edwards model, but every model of the curve yields the same group
element, so the oracle works in the short Weierstrass model the library uses and
compares affine points.

Two independent formula families:
* affine chord/tangent (the textbook definition, every case explicit),
* Jacobian coordinates (x = X/Z^2, y = Y/Z^3), derived from the same definition.
The identity O is `None` in affine form and Z = 0 in Jacobian form.
"""
from __future__ import annotations

from . import fq
from .fq import P

B_COEFF = 1  # y^2 = x^3 + 1

# Standard BLS12-377 G1 generator (public curve parameter; re-checked by tests:
# on the curve and of order r).
GX = 0x008848DEFE740A67C8FC6225BF87FF5485951E2CAA9D41BB188282C8BD37CB5CD5481512FFCD394EEAB9B16EB21BE9EF
GY = 0x01914A69C5102EFF1F674F5D30AFEEC4BD7FB348CA3E52D96D182AD44FB82305C2FE3D3634A9591AFD82DE55559C8EA6
G = (GX, GY)

O = None


def on_curve(pt) -> bool:
    if pt is None:
        return True
    x, y = pt
    return 0 <= x < P and 0 <= y < P and (y * y - x * x * x - B_COEFF) % P == 0


def neg(pt):
    if pt is None:
        return None
    return (pt[0], (-pt[1]) % P)


def add(p1, p2):
    """Affine addition by the chord/tangent rule."""
    if p1 is None:
        return p2
    if p2 is None:
        return p1
    x1, y1 = p1
    x2, y2 = p2
    if x1 == x2:
        if (y1 + y2) % P == 0:      # P + (-P), including 2-torsion doubling
            return None
        lam = fq.mul(3 * x1 * x1 % P, fq.inv(2 * y1 % P))   # tangent (a = 0)
    else:
        lam = fq.mul((y2 - y1) % P, fq.inv((x2 - x1) % P))  # chord
    x3 = (lam * lam - x1 - x2) % P
    y3 = (lam * (x1 - x3) - y1) % P
    return (x3, y3)


def double(pt):
    return add(pt, pt)


def mul(k: int, pt):
    """k * pt by left-to-right double-and-add (k >= 0)."""
    if k < 0:
        return mul(-k, neg(pt))
    acc = None
    for bit in bin(k)[2:] if k else "":
        acc = add(acc, acc)
        if bit == "1":
            acc = add(acc, pt)
    return acc


# ---- Jacobian family -------------------------------------------------------

def to_jac(pt):
    if pt is None:
        return (1, 1, 0)
    return (pt[0], pt[1], 1)


def from_jac(j):
    X, Y, Z = j
    if Z % P == 0:
        return None
    zi = fq.inv(Z)
    zi2 = zi * zi % P
    return (X * zi2 % P, Y * zi2 * zi % P)


def jac_double(j):
    """2*(X, Y, Z) for a = 0: lambda = 3x^2/(2y) rewritten over Z."""
    X, Y, Z = j
    if Z % P == 0 or Y % P == 0:
        return (1, 1, 0)
    A = X * X % P
    Bq = Y * Y % P
    C = Bq * Bq % P
    D = 2 * ((X + Bq) ** 2 - A - C) % P      # = 4 X Y^2
    E = 3 * A % P
    F = E * E % P
    X3 = (F - 2 * D) % P
    Y3 = (E * (D - X3) - 8 * C) % P
    Z3 = 2 * Y * Z % P
    return (X3, Y3, Z3)


def jac_add(j1, j2):
    X1, Y1, Z1 = j1
    X2, Y2, Z2 = j2
    if Z1 % P == 0:
        return j2
    if Z2 % P == 0:
        return j1
    Z1Z1 = Z1 * Z1 % P
    Z2Z2 = Z2 * Z2 % P
    U1 = X1 * Z2Z2 % P
    U2 = X2 * Z1Z1 % P
    S1 = Y1 * Z2 * Z2Z2 % P
    S2 = Y2 * Z1 * Z1Z1 % P
    H = (U2 - U1) % P
    Rr = (S2 - S1) % P
    if H == 0:
        if Rr == 0:
            return jac_double(j1)
        return (1, 1, 0)
    HH = H * H % P
    HHH = H * HH % P
    V = U1 * HH % P
    X3 = (Rr * Rr - HHH - 2 * V) % P
    Y3 = (Rr * (V - X3) - S1 * HHH) % P
    Z3 = Z1 * Z2 * H % P
    return (X3, Y3, Z3)


def jac_mul(k: int, pt):
    acc = (1, 1, 0)
    base = to_jac(pt)
    for bit in bin(k)[2:] if k else "":
        acc = jac_double(acc)
        if bit == "1":
            acc = jac_add(acc, base)
    return from_jac(acc)


def random_point(seed_int: int):
    """A point of E (not necessarily in the order-r subgroup): x from seed_int upward
    until x^3 + 1 is a square."""
    x = seed_int % P
    while True:
        y = fq.sqrt((x * x * x + B_COEFF) % P)
        if y is not None:
            return (x, y)
        x = (x + 1) % P


def to_limbs(pt) -> list[int]:
    """Affine point -> 24 u32 limbs (x then y, standard form); O -> all zero."""
    if pt is None:
        return [0] * 24
    return fq.to_limbs(pt[0]) + fq.to_limbs(pt[1])


def from_limbs(limbs):
    x = fq.from_limbs(limbs[:12])
    y = fq.from_limbs(limbs[12:24])
    if x == 0 and y == 0:
        return None
    return (x, y)
