"""Base field GF(p) and scalar field order r of BLS12-377 — test infrastructure only.

The paper targets the BLS12-377 curve (Sec. I, Sec. II-D) without printing its
parameters. They follow from the BLS12 family polynomials evaluated at the
curve's seed x0:
    r(x) = x^4 - x^2 + 1
    p(x) = (x - 1)^2 * r(x) / 3 + x
    trace t(x) = x + 1, so #E(Fq) = p + 1 - t.
All arithmetic is Python's arbitrary-precision `int`.
"""
from __future__ import annotations

X0 = 0x8508C00000000001  # BLS12-377 seed


def derive_r(x0: int = X0) -> int:
    return x0 ** 4 - x0 ** 2 + 1


def derive_p(x0: int = X0) -> int:
    r = derive_r(x0)
    num = (x0 - 1) ** 2 * r
    assert num % 3 == 0
    return num // 3 + x0


P = derive_p()
R = derive_r()
TRACE = X0 + 1
CURVE_ORDER = P + 1 - TRACE
COFACTOR = CURVE_ORDER // R

NLIMBS = 12          # 32-bit limbs used at the library boundary
LIMB_BITS = 32


def is_probable_prime(n: int, bases=(2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47,
                                      53, 59, 61, 67, 71, 73, 79, 83, 89, 97)) -> bool:
    """Miller–Rabin with a fixed base set (error < 4^-25 for composites)."""
    if n < 2:
        return False
    for q in bases:
        if n % q == 0:
            return n == q
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in bases:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def add(a: int, b: int) -> int:
    return (a + b) % P


def sub(a: int, b: int) -> int:
    return (a - b) % P


def neg(a: int) -> int:
    return (-a) % P


def mul(a: int, b: int) -> int:
    return (a * b) % P


def inv(a: int) -> int:
    """Inverse by the extended Euclidean algorithm (not by exponentiation)."""
    a %= P
    if a == 0:
        raise ZeroDivisionError("inverse of 0 in Fq")
    old_r, r = a, P
    old_s, s = 1, 0
    while r:
        q = old_r // r
        old_r, r = r, old_r - q * r
        old_s, s = s, old_s - q * s
    assert old_r == 1
    return old_s % P


def legendre(a: int) -> int:
    a %= P
    if a == 0:
        return 0
    return 1 if pow(a, (P - 1) // 2, P) == 1 else -1


def sqrt(a: int) -> int | None:
    """Tonelli–Shanks square root (p - 1 = 2^46 * q, q odd); None for non-residues."""
    a %= P
    if a == 0:
        return 0
    if legendre(a) != 1:
        return None
    q, s = P - 1, 0
    while q % 2 == 0:
        q //= 2
        s += 1
    z = 2
    while legendre(z) != -1:
        z += 1
    m, c, t, rr = s, pow(z, q, P), pow(a, q, P), pow(a, (q + 1) // 2, P)
    while t != 1:
        i, t2 = 0, t
        while t2 != 1:
            t2 = t2 * t2 % P
            i += 1
        b = pow(c, 1 << (m - i - 1), P)
        m, c = i, b * b % P
        t, rr = t * c % P, rr * b % P
    return rr


def to_limbs(v: int, n: int = NLIMBS) -> list[int]:
    return [(v >> (LIMB_BITS * k)) & 0xFFFFFFFF for k in range(n)]


def from_limbs(limbs) -> int:
    v = 0
    for k, w in enumerate(limbs):
        v |= int(w) << (LIMB_BITS * k)
    return v
