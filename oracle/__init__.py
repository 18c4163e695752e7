"""CPU oracle for BLS12-377 G1 multi-scalar multiplication — TEST INFRASTRUCTURE ONLY.

Only the test suite, the package smoke check and the CPU-baseline leg of the
benchmark may import, call or link anything in this directory. The product path
(the CUDA library and its Python binding) never does, and shares no code,
constant table or helper with it.

What it computes, and from which passage of arXiv:2502.11660 ("Accelerating
Elliptic Curve Point Additions on Versal AI Engine for Multi-scalar
Multiplication"):

* `fq`     — the base field GF(p) of BLS12-377 (Sec. I and II-D name the curve),
             p and r derived from the BLS12 seed; plain Python integers.
* `barrett`— the paper's modular multiplication, Barrett reduction built from
             three multiplications (Sec. III-C), and its 25-bit-element coarse
             carry propagation (Sec. III-D); used to pin the printed ranges.
* `g1`     — the group law on y^2 = x^3 + 1: affine chord/tangent addition with
             every special case, and an independent Jacobian formula family
             (Sec. II-D: point additions, mixed and complete).
* `msm`    — the result the method reaches, sum_i s_i * P_i, by its definition
             (naive double-and-add) and by textbook Pippenger bucket
             accumulation / bucket aggregation / group aggregation (Sec. II-C).
* `edwards`— the paper's twisted Edwards model -x^2 + y^2 = 1 + (k/2) x^2 y^2
             (Sec. II-D): the map from y^2 = x^3 + 1, its inverse, the affine
             Edwards law and the stored form (X, Y, U = k T) with Z = 1.
* `glv`    — the endomorphism phi(x, y) = (beta x, y) = lambda P on the order-r
             subgroup and the split k = k1 + lambda k2 (a schedule change, not in
             the paper), with a Pippenger over (P_i, phi(P_i)).
* `coracle`— ctypes binding of `oracle.c`, a plain C big-integer version of the
             same arithmetic (schoolbook product + Barrett reduction, 64-bit
             words), used for large inputs and as the timed CPU baseline.

Parity is pinned by mathematics, not by the paper: the paper prints no worked
numeric example. See tests/test_oracle_*.py for the pins.
"""
