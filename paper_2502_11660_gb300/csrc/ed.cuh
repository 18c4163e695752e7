// BLS12-377 G1 on the paper's twisted Edwards model (Sec. II-D):
//     -x^2 + y^2 = 1 + d x^2 y^2,   k = 2d,
// in extended coordinates (X, Y, Z, T): x = X/Z, y = Y/Z, T = XY/Z (Hisil,
// Wong, Carter, Dawson 2008). As in the paper, the points streamed into bucket
// accumulation are stored as (x, y, u = k x y) with Z = 1, buckets are (X, Y, Z, T),
// and the complete addition of bucket aggregation multiplies one operand's T
// by k first:
//   madd: ext += stored   7M   (A, B, C = T1 u2, X3, Y3, T3, Z3)
//   add : ext += ext      9M   (C = T1 (k T2), D = Z1 Z2)
//   dbl : 2 ext           4M + 4S
// These formulas have no special cases inside the order-r subgroup (odd order:
// the denominators 1 +- d x1 x2 y1 y2 vanish only for pairs involving points of
// even order), so unlike XYZZ nothing is branched on; the identity is
// (0, 1, 1, 0). Every coordinate is in Montgomery form and in [0, 2p).
//
// The curve is reached from y^2 = x^3 + 1 by moving the 2-torsion point (-1, 0)
// to the origin (x = s u - 1, s^2 = 3: the Montgomery curve B v^2 = u^3 - s u^2 + u,
// B = 1/s^3, v = y), the Montgomery-to-Edwards map x_e = u / v, y_e = (u - 1)/(u + 1)
// (Bernstein, Birkner, Joye, Lange, Peters 2008), and the scaling x = gamma x_e
// that makes a = -1. Hence, for a Weierstrass point (x_w, y_w):
//   x = c1 (x_w + 1) / y_w  with c1 = gamma / s,   y = (x_w + 1 - s)/(x_w + 1 + s),
// and back, from (X : Y : Z):
//   x_w = s (Z + Y) / (Z - Y) - 1,   y_w = gamma Z (Z + Y) / ((Z - Y) X).
// s is the smaller square root of 3 in [0, p) and gamma the smaller square root
// of -a = 9 - 6s; k below is 2d for that choice.
#pragma once
#include "ec.cuh"

namespace ed {

using fq::fe;

struct ext {
    fe X, Y, Z, T;
};

// (x, y, u = k x y): the stored form of an input point, Z = 1.
struct stored {
    fe x, y, u;
};

// k = 2d, s, gamma, c1 = gamma / s, all in Montgomery form (x 2^384 mod p).
__device__ __constant__ static const uint32_t kK[fq::N] = {
    0x44a706c6u, 0xf24b7e84u, 0x80faa8fau, 0xeae02375u, 0x7ef38fa5u, 0x0f4d7cf2u,
    0xc5f2bb26u, 0x5597097du, 0x0d95a93eu, 0x8bf6c1ddu, 0xfbff628au, 0x01784602u};
__device__ __constant__ static const uint32_t kS[fq::N] = {
    0x8894e1e4u, 0x3fabdfd0u, 0xcc1f55aau, 0xcbf921ddu, 0x460edc0cu, 0xd17deff1u,
    0x7897028du, 0xd394e81eu, 0x0912681au, 0xc29c995du, 0xaff9d568u, 0x01515e6cu};
__device__ __constant__ static const uint32_t kGamma[fq::N] = {
    0xa38cfd11u, 0xface0c97u, 0x0adb8383u, 0x8cc7c229u, 0xd44ae9cbu, 0x4765cd5fu,
    0x22354029u, 0x9ae986d8u, 0x252ab9bdu, 0xc3dc7860u, 0xc8942395u, 0x00486011u};
__device__ __constant__ static const uint32_t kC1[fq::N] = {
    0xead605e4u, 0xfb7c0ab8u, 0xe2752c7au, 0x363b93d1u, 0x144be536u, 0xd2246835u,
    0x429f2077u, 0xeb8bf6ddu, 0x0234d423u, 0x3a9efda2u, 0xba0c72a4u, 0x013c7943u};

__device__ __forceinline__ void load_const(fe& r, const uint32_t (&c)[fq::N]) {
#pragma unroll
    for (int k = 0; k < fq::N; ++k) r.v[k] = c[k];
}

__device__ __forceinline__ void set_inf(ext& P) {
    fq::set_zero(P.X);
    fq::set_one(P.Y);
    fq::set_one(P.Z);
    fq::set_zero(P.T);
}

// -(x, y) = (-x, y), so u = k x y changes sign too.
__device__ __forceinline__ void neg(stored& Q) {
    fq::neg(Q.x, Q.x);
    fq::neg(Q.u, Q.u);
}

// P = Q (stored, Z = 1): (x, y, 1, x y).
__device__ __forceinline__ void from_stored(ext& P, const stored& Q) {
    P.X = Q.x;
    P.Y = Q.y;
    fq::set_one(P.Z);
    fq::mul(P.T, Q.x, Q.y);
}

// P += Q, Q stored (Z2 = 1, u2 = k T2):
// A = (Y1 - X1)(y2 - x2), B = (Y1 + X1)(y2 + x2), C = T1 u2, D = 2 Z1,
// E = B - A, F = D - C, G = D + C, H = B + A,
// X3 = E F, Y3 = G H, T3 = E H, Z3 = F G.
// Values that only feed multiplications are left unfolded (fq::add_nr / sub_nr):
// Y1 -+ X1, y2 -+ x2, E, H < 4p; D < 4p; F, G < 6p; every product below 36 p^2.
// Independent products go in pairs through fq::mul2 (four carry chains in flight).
__device__ __forceinline__ void madd(ext& P, const stored& Q) {
    fe A, B, t, u, v, w;
    fq::sub_nr<2>(t, P.Y, P.X);
    fq::sub_nr<2>(u, Q.y, Q.x);
    fq::add_nr(v, P.Y, P.X);
    fq::add_nr(w, Q.y, Q.x);
    fq::mul2(A, t, u, B, v, w);
    fq::mul(t, P.T, Q.u);           // C
    fq::add_nr(u, P.Z, P.Z);        // D
    fq::sub_nr<2>(P.X, B, A);       // E
    fq::add_nr(P.Y, B, A);          // H
    fq::sub_nr<2>(A, u, t);         // F = D - C + 2p
    fq::add_nr(B, u, t);            // G
    fq::mul2(P.T, P.X, P.Y, P.Z, A, B);  // T3 = E H, Z3 = F G
    fq::mul2(P.X, P.X, A, P.Y, B, P.Y);  // X3 = E F, Y3 = G H
}

// P += Q with an identity flag kept by the caller (the first point of a run is
// a 1M assignment instead of a 7M addition).
__device__ __forceinline__ void madd(ext& P, bool& p_inf, const stored& Q) {
    if (p_inf) {
        from_stored(P, Q);
        p_inf = false;
        return;
    }
    madd(P, Q);
}

// P += Q, both extended; Q's coordinates are fetched through `q` (a register or
// memory loader with X/Y/Z/T accessors), so a Q in memory never occupies registers.
// A = (Y1 - X1)(Y2 - X2), B = (Y1 + X1)(Y2 + X2), C = T1 k T2, D = 2 Z1 Z2, then as madd.
template <class QL>
__device__ __forceinline__ void add_q(ext& P, const QL& q) {
    fe A, B, t, u, v;
    q.Y(u);
    q.X(t);
    fq::sub_nr<2>(A, u, t);
    fq::add_nr(B, u, t);
    fq::sub_nr<2>(t, P.Y, P.X);
    fq::add_nr(v, P.Y, P.X);
    fq::mul2(A, t, A, B, v, B);
    q.T(t);
    load_const(u, kK);
    q.Z(v);
    fq::mul2(t, t, u, u, P.Z, v);   // k T2, Z1 Z2
    fq::mul(t, P.T, t);             // C
    fq::add_nr(u, u, u);            // D
    fq::sub_nr<2>(P.X, B, A);       // E
    fq::add_nr(P.Y, B, A);          // H
    fq::sub_nr<2>(A, u, t);         // F
    fq::add_nr(B, u, t);            // G
    fq::mul2(P.T, P.X, P.Y, P.Z, A, B);
    fq::mul2(P.X, P.X, A, P.Y, B, P.Y);
}

struct RegQ {
    const ext* q;
    __device__ __forceinline__ void X(fe& r) const { r = q->X; }
    __device__ __forceinline__ void Y(fe& r) const { r = q->Y; }
    __device__ __forceinline__ void Z(fe& r) const { r = q->Z; }
    __device__ __forceinline__ void T(fe& r) const { r = q->T; }
};

__device__ __forceinline__ void add(ext& P, const ext& Q) { add_q(P, RegQ{&Q}); }

// P = 2P (a = -1): A = X^2, B = Y^2, C = 2 Z^2, D = -A, E = (X + Y)^2 - A - B,
// G = D + B, F = G - C, H = D - B, X3 = E F, Y3 = G H, T3 = E H, Z3 = F G.
// Unfolded: X + Y, 2 Z^2, G, H < 4p; E < 6p; F = G - 2 Z^2 + 4p < 8p; products below 48 p^2.
__device__ __forceinline__ void dbl(ext& P) {
    fe A, B, C, t;
    fq::add_nr(t, P.X, P.Y);
    fq::mul2(A, P.X, P.X, B, P.Y, P.Y);
    fq::mul2(C, P.Z, P.Z, t, t, t);
    fq::add_nr(C, C, C);
    fq::sub_nr<2>(t, t, A);
    fq::sub_nr<2>(t, t, B);         // E
    fq::sub_nr<2>(P.Y, B, A);       // G = B - A
    fe z;
    fq::set_zero(z);
    fq::sub_nr<2>(A, z, A);
    fq::sub_nr<2>(A, A, B);         // H = -A - B
    fq::sub_nr<4>(C, P.Y, C);       // F = G - C
    fq::mul2(P.T, t, A, P.X, t, C);      // E H, E F
    fq::mul2(P.Z, C, P.Y, P.Y, P.Y, A);  // F G, G H
}

// ---- four lanes per point operation (latency-bound chains; see ec::xchg4):
// the multiplications of one Edwards formula fall into two or three levels of
// independent products, so a doubling costs two multiplication latencies instead
// of eight.
using ec::pick4;
using ec::xchg4;

// P = 2P: level 1 {X^2, Y^2, Z^2, (X + Y)^2}, level 2 {E F, G H, E H, F G}.
__device__ __forceinline__ void dbl4(ext& P, fe* sh, int l, bool writer) {
    fe s, r, v[4];
    fq::add_nr(s, P.X, P.Y);
    const fe x = pick4(l, P.X, P.Y, P.Z, s);
    fq::sqr(r, x);
    xchg4(v, r, sh, l, writer);     // A, B, Z^2, (X + Y)^2
    fe E, G, H, F, z;
    fq::sub_nr<2>(E, v[3], v[0]);
    fq::sub_nr<2>(E, E, v[1]);      // E = (X + Y)^2 - A - B
    fq::sub_nr<2>(G, v[1], v[0]);   // G = B - A
    fq::set_zero(z);
    fq::sub_nr<2>(H, z, v[0]);
    fq::sub_nr<2>(H, H, v[1]);      // H = -A - B
    fq::add_nr(F, v[2], v[2]);
    fq::sub_nr<4>(F, G, F);         // F = G - 2 Z^2 (ranges as in dbl)
    const fe a = pick4(l, E, G, E, F);
    const fe b = pick4(l, F, H, H, G);
    fq::mul(r, a, b);
    xchg4(v, r, sh, l, writer);     // X3, Y3, T3, Z3
    P.X = v[0];
    P.Y = v[1];
    P.T = v[2];
    P.Z = v[3];
}

// P += Q (extended, Q read through `q`): level 1 {A, B, T1 T2, Z1 Z2}, level 2
// {k T1 T2} (one lane), level 3 {E F, G H, E H, F G}.
template <class QL>
__device__ __forceinline__ void add4(ext& P, const QL& q, fe* sh, int l, bool writer) {
    fe X2, Y2, Z2, T2, u, w, r, v[4];
    q.X(X2);
    q.Y(Y2);
    q.Z(Z2);
    q.T(T2);
    fe a0, b0, a1, b1;
    fq::sub_nr<2>(a0, P.Y, P.X);
    fq::sub_nr<2>(b0, Y2, X2);
    fq::add_nr(a1, P.Y, P.X);
    fq::add_nr(b1, Y2, X2);
    const fe x = pick4(l, a0, a1, P.T, P.Z);
    const fe y = pick4(l, b0, b1, T2, Z2);
    fq::mul(r, x, y);
    xchg4(v, r, sh, l, writer);     // A, B, T1 T2, Z1 Z2
    load_const(u, kK);
    fq::mul(w, v[2], u);            // C = k T1 T2 (every lane; one latency)
    fe E, F, G, H, D;
    fq::add_nr(D, v[3], v[3]);
    fq::sub_nr<2>(E, v[1], v[0]);
    fq::add_nr(H, v[1], v[0]);
    fq::sub_nr<2>(F, D, w);
    fq::add_nr(G, D, w);
    const fe a = pick4(l, E, G, E, F);
    const fe b = pick4(l, F, H, H, G);
    fq::mul(r, a, b);
    xchg4(v, r, sh, l, writer);
    P.X = v[0];
    P.Y = v[1];
    P.T = v[2];
    P.Z = v[3];
}

// P += Q (stored): level 1 {A, B, C = T1 u2} (the fourth lane repeats C), level 2
// {E F, G H, E H, F G}: two multiplication latencies per mixed addition.
__device__ __forceinline__ void madd4(ext& P, const stored& Q, fe* sh, int l, bool writer) {
    fe a0, b0, a1, b1, r, v[4];
    fq::sub_nr<2>(a0, P.Y, P.X);
    fq::sub_nr<2>(b0, Q.y, Q.x);
    fq::add_nr(a1, P.Y, P.X);
    fq::add_nr(b1, Q.y, Q.x);
    const fe x = pick4(l, a0, a1, P.T, P.T);
    const fe y = pick4(l, b0, b1, Q.u, Q.u);
    fq::mul(r, x, y);
    xchg4(v, r, sh, l, writer);     // A, B, C, C
    fe E, F, G, H, D;
    fq::add_nr(D, P.Z, P.Z);
    fq::sub_nr<2>(E, v[1], v[0]);
    fq::add_nr(H, v[1], v[0]);
    fq::sub_nr<2>(F, D, v[2]);
    fq::add_nr(G, D, v[2]);
    const fe a = pick4(l, E, G, E, F);
    const fe b = pick4(l, F, H, H, G);
    fq::mul(r, a, b);
    xchg4(v, r, sh, l, writer);
    P.X = v[0];
    P.Y = v[1];
    P.T = v[2];
    P.Z = v[3];
}

// Weierstrass affine point (Montgomery form, [0, 2p)) of P, canonical [0, p);
// the identity gives (0, 0). One inversion of (Z - Y) X.
__device__ __forceinline__ void to_weierstrass(ec::affine& A, const ext& P) {
    if (fq::is_zero(P.X)) {         // (0, 1) inside the subgroup
        fq::set_zero(A.x);
        fq::set_zero(A.y);
        return;
    }
    fe zmy, zpy, t, I, c;
    fq::sub(zmy, P.Z, P.Y);
    fq::add(zpy, P.Z, P.Y);
    fq::mul(t, zmy, P.X);
    ec::inv(I, t);
    fq::mul(t, zpy, I);             // (Z + Y) / ((Z - Y) X)
    load_const(c, kS);
    fq::mul(A.x, t, P.X);
    fq::mul(A.x, A.x, c);
    fe one;
    fq::set_one(one);
    fq::sub(A.x, A.x, one);
    fq::canon(A.x, A.x);
    load_const(c, kGamma);
    fq::mul(A.y, t, P.Z);
    fq::mul(A.y, A.y, c);
    fq::canon(A.y, A.y);
}

}  // namespace ed
