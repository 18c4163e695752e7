// BLS12-377 G1 point arithmetic on sm_103a: E: y^2 = x^3 + 1 over Fq.
//
// The paper's PADD (Sec. II-D) is a mixed addition for bucket accumulation and
// a complete addition for bucket aggregation; it works on a twisted Edwards
// model, whose PADD graph (its Fig. 1) is not reproducible from the text. Here
// the same two operations run on the short Weierstrass model in XYZZ
// coordinates (x = X/ZZ, y = Y/ZZZ, ZZ^3 = ZZZ^2; Bernstein-Lange), which give
// the same group elements:
//   madd: XYZZ += affine     8M + 2S
//   add : XYZZ += XYZZ      12M + 2S
//   dbl : 2 * XYZZ           6M + 3S (a = 0)
//   mdbl: 2 * affine -> XYZZ 4M + 3S
// XYZZ formulas are not complete, so every special case is branched on:
// O operands, P + P (falls through to doubling), P + (-P) (gives O).
// The identity is ZZ = ZZZ = 0; the affine identity is (0, 0), which is not on
// the curve. Every coordinate is in Montgomery form and in [0, 2p).
#pragma once
#include "fq.cuh"

namespace ec {

using fq::fe;

struct xyzz {
    fe X, Y, ZZ, ZZZ;
};

struct affine {
    fe x, y;
};

__device__ __forceinline__ void set_inf(xyzz& P) {
    fq::set_zero(P.X);
    fq::set_zero(P.Y);
    fq::set_zero(P.ZZ);
    fq::set_zero(P.ZZZ);
}

__device__ __forceinline__ bool is_inf(const xyzz& P) { return fq::is_zero(P.ZZ); }

__device__ __forceinline__ bool is_inf(const affine& Q) {
    return fq::is_zero_raw(Q.x) && fq::is_zero_raw(Q.y);
}

__device__ __forceinline__ void from_affine(xyzz& P, const affine& Q) {
    if (is_inf(Q)) {
        set_inf(P);
        return;
    }
    P.X = Q.x;
    P.Y = Q.y;
    fq::set_one(P.ZZ);
    fq::set_one(P.ZZZ);
}

__device__ __forceinline__ void neg(affine& Q) {
    if (!is_inf(Q)) fq::neg(Q.y, Q.y);
}

// R = 2 * Q for affine Q: U = 2y, V = U^2, W = U V, S = x V, M = 3x^2,
// X3 = M^2 - 2S, Y3 = M (S - X3) - W y, ZZ3 = V, ZZZ3 = W.
__device__ __forceinline__ void mdbl(xyzz& R, const affine& Q) {
    if (is_inf(Q) || fq::is_zero(Q.y)) {
        set_inf(R);
        return;
    }
    fe U, V, W, S, M, t;
    fq::dbl(U, Q.y);
    fq::sqr(V, U);
    fq::mul(W, U, V);
    fq::mul(S, Q.x, V);
    fq::sqr(t, Q.x);
    fq::dbl(M, t);
    fq::add(M, M, t);
    fq::sqr(R.X, M);
    fq::dbl(t, S);
    fq::sub(R.X, R.X, t);
    fq::sub(t, S, R.X);
    fq::mul(t, M, t);
    fq::mul(R.Y, W, Q.y);
    fq::sub(R.Y, t, R.Y);
    R.ZZ = V;
    R.ZZZ = W;
}

// P = 2 P: U = 2Y, V = U^2, W = U V, S = X V, M = 3X^2,
// X3 = M^2 - 2S, Y3 = M (S - X3) - W Y, ZZ3 = V ZZ, ZZZ3 = W ZZZ.
// Y = 0 gives V = 0 and so ZZ3 = 0 (the identity) without a branch.
// Temporaries die as early as possible (register pressure).
__device__ __forceinline__ void dbl(xyzz& P) {
    if (is_inf(P)) return;
    fe V, W, t;
    fq::dbl(t, P.Y);                // U
    fq::sqr(V, t);
    fq::mul(W, t, V);               // U dead
    fq::mul(P.ZZ, P.ZZ, V);         // ZZ3
    fq::mul(P.ZZZ, P.ZZZ, W);       // ZZZ3
    fq::mul(P.Y, W, P.Y);           // W Y; W dead
    fq::mul(V, P.X, V);             // S in V's slot
    fq::sqr(t, P.X);
    fq::dbl(W, t);
    fq::add(W, W, t);               // M in W's slot
    fq::dbl(t, V);                  // 2S
    fq::sqr(P.X, W);
    fq::sub(P.X, P.X, t);           // X3
    fq::sub(t, V, P.X);             // S - X3
    fq::mul(t, W, t);
    fq::sub(P.Y, t, P.Y);           // Y3
}

// P += Q (Q affine). `p_inf` says P is the identity (kept by the caller).
// U2 = x2 ZZ1, S2 = y2 ZZZ1, Pd = U2 - X1, R = S2 - Y1, PP = Pd^2, PPP = Pd PP,
// Q1 = X1 PP, X3 = R^2 - PPP - 2 Q1, Y3 = R (Q1 - X3) - Y1 PPP,
// ZZ3 = ZZ1 PP, ZZZ3 = ZZZ1 PPP.
__device__ __forceinline__ void madd(xyzz& P, bool& p_inf, const affine& Q) {
    if (is_inf(Q)) return;
    if (p_inf) {
        from_affine(P, Q);
        p_inf = false;
        return;
    }
    fe U2, S2, Pd, R;
    fq::mul(U2, Q.x, P.ZZ);
    fq::mul(S2, Q.y, P.ZZZ);
    fq::sub(Pd, U2, P.X);
    fq::sub(R, S2, P.Y);
    if (fq::is_zero(Pd)) {
        if (fq::is_zero(R)) {
            mdbl(P, Q);
            p_inf = is_inf(P);
        } else {
            set_inf(P);
            p_inf = true;
        }
        return;
    }
    fe PP, PPP, Q1, t;
    fq::sqr(PP, Pd);
    fq::mul(PPP, Pd, PP);
    fq::mul(Q1, P.X, PP);
    fq::mul(P.ZZ, P.ZZ, PP);
    fq::mul(P.ZZZ, P.ZZZ, PPP);
    fq::sqr(P.X, R);
    fq::sub(P.X, P.X, PPP);
    fq::dbl(t, Q1);
    fq::sub(P.X, P.X, t);       // X3
    fq::mul(PPP, P.Y, PPP);     // Y1 PPP
    fq::sub(t, Q1, P.X);
    fq::mul(t, R, t);
    fq::sub(P.Y, t, PPP);
}

__device__ __forceinline__ void madd(xyzz& P, const affine& Q) {
    bool inf = is_inf(P);
    madd(P, inf, Q);
}

// Second operand of add_q() held in registers.
struct RegQ {
    const xyzz* q;
    __device__ __forceinline__ void X(fe& r) const { r = q->X; }
    __device__ __forceinline__ void Y(fe& r) const { r = q->Y; }
    __device__ __forceinline__ void ZZ(fe& r) const { r = q->ZZ; }
    __device__ __forceinline__ void ZZZ(fe& r) const { r = q->ZZZ; }
    __device__ __forceinline__ void all(xyzz& r) const { r = *q; }
};

// P += Q (both XYZZ); Q's coordinates are fetched through `q` when needed, so a
// Q in memory never occupies registers, and P's slots are reused once X1, Y1 die.
// U1 = X1 ZZ2, U2 = X2 ZZ1, S1 = Y1 ZZZ2, S2 = Y2 ZZZ1, Pd = U2 - U1,
// R = S2 - S1, PP = Pd^2, PPP = Pd PP, Q1 = U1 PP, X3 = R^2 - PPP - 2 Q1,
// Y3 = R (Q1 - X3) - S1 PPP, ZZ3 = ZZ1 ZZ2 PP, ZZZ3 = ZZZ1 ZZZ2 PPP.
template <class QL>
__device__ __forceinline__ void add_q(xyzz& P, const QL& q) {
    fe t, u, Pd, R;
    q.ZZ(t);
    if (fq::is_zero(t)) return;     // Q = O
    if (is_inf(P)) {
        q.all(P);
        return;
    }
    fq::mul(P.X, P.X, t);           // U1
    q.X(u);
    fq::mul(u, u, P.ZZ);            // U2
    fq::sub(Pd, u, P.X);
    q.ZZZ(t);
    fq::mul(P.Y, P.Y, t);           // S1
    q.Y(u);
    fq::mul(u, u, P.ZZZ);           // S2
    fq::sub(R, u, P.Y);
    if (fq::is_zero(Pd)) {
        if (fq::is_zero(R)) {
            q.all(P);               // P = Q: the sum is 2Q
            dbl(P);
        } else {
            set_inf(P);
        }
        return;
    }
    fq::sqr(u, Pd);                 // PP
    fq::mul(Pd, Pd, u);             // PPP in Pd's slot
    fq::mul(P.X, P.X, u);           // Q1 in X's slot
    q.ZZ(t);
    fq::mul(P.ZZ, P.ZZ, t);
    fq::mul(P.ZZ, P.ZZ, u);         // ZZ3
    q.ZZZ(t);
    fq::mul(P.ZZZ, P.ZZZ, t);
    fq::mul(P.ZZZ, P.ZZZ, Pd);      // ZZZ3
    fq::dbl(u, P.X);
    fq::add(u, u, Pd);              // 2 Q1 + PPP
    fq::mul(Pd, P.Y, Pd);           // S1 PPP
    fq::sqr(t, R);
    fq::sub(t, t, u);               // X3
    fq::sub(u, P.X, t);             // Q1 - X3
    P.X = t;
    fq::mul(u, R, u);
    fq::sub(P.Y, u, Pd);            // Y3
}

__device__ __forceinline__ void add(xyzz& P, const xyzz& Q) { add_q(P, RegQ{&Q}); }

// Inverse by the binary extended Euclidean algorithm on exact 32-bit words
// (variable time; MSM results are public). For u = aR it returns x with
// x u = 1 mod p, i.e. a^-1 R^-1, and one Montgomery multiplication by R^3 mod p
// turns that into a^-1 R. About 2 * 377 shift / subtract steps of 12-word
// carry chains, an order of magnitude shorter than a^(p-2).
namespace detail {
constexpr int W = 12;
__device__ __forceinline__ bool w_is_one(const uint32_t (&a)[W]) {
    uint32_t o = a[0] ^ 1u;
#pragma unroll
    for (int k = 1; k < W; ++k) o |= a[k];
    return o == 0;
}
__device__ __forceinline__ bool w_geq(const uint32_t (&a)[W], const uint32_t (&b)[W]) {
#pragma unroll
    for (int k = W - 1; k >= 0; --k)
        if (a[k] != b[k]) return a[k] > b[k];
    return true;
}
__device__ __forceinline__ void w_sub(uint32_t (&a)[W], const uint32_t (&b)[W]) {
    uint64_t borrow = 0;
#pragma unroll
    for (int k = 0; k < W; ++k) {
        uint64_t t = (uint64_t)a[k] - b[k] - borrow;
        a[k] = (uint32_t)t;
        borrow = (t >> 63) & 1u;
    }
}
__device__ __forceinline__ uint32_t w_add(uint32_t (&a)[W], const uint32_t (&b)[W]) {
    uint64_t carry = 0;
#pragma unroll
    for (int k = 0; k < W; ++k) {
        uint64_t t = (uint64_t)a[k] + b[k] + carry;
        a[k] = (uint32_t)t;
        carry = t >> 32;
    }
    return (uint32_t)carry;
}
__device__ __forceinline__ void w_shr1(uint32_t (&a)[W], uint32_t top) {
#pragma unroll
    for (int k = 0; k < W - 1; ++k) a[k] = (a[k] >> 1) | (a[k + 1] << 31);
    a[W - 1] = (a[W - 1] >> 1) | (top << 31);
}
// x / 2 mod p for x in [0, p)
__device__ __forceinline__ void w_half(uint32_t (&x)[W], const uint32_t (&p)[W]) {
    uint32_t top = 0;
    if (x[0] & 1u) top = w_add(x, p);
    w_shr1(x, top);
}
// x = x - y mod p for x, y in [0, p)
__device__ __forceinline__ void w_submod(uint32_t (&x)[W], const uint32_t (&y)[W], const uint32_t (&p)[W]) {
    if (w_geq(x, y)) {
        w_sub(x, y);
    } else {
        w_add(x, p);
        w_sub(x, y);
    }
}
}  // namespace detail

__device__ __noinline__ static void inv(fe& r, const fe& a_in) {
    using namespace detail;
    const uint32_t p[W] = {0x00000001u, 0x8508c000u, 0x30000000u, 0x170b5d44u, 0xba094800u, 0x1ef3622fu,
                           0x00f5138fu, 0x1a22d9f3u, 0x6ca1493bu, 0xc63b05c0u, 0x17c510eau, 0x01ae3a46u};
    fe a;
    fq::canon(a, a_in);
    uint32_t u[W], v[W], x1[W], x2[W];
    uint32_t z = 0;
#pragma unroll
    for (int k = 0; k < W; ++k) {
        u[k] = a.v[k];
        v[k] = p[k];
        x1[k] = 0;
        x2[k] = 0;
        z |= a.v[k];
    }
    x1[0] = 1;
    if (z == 0) {
        fq::set_zero(r);
        return;
    }
    // each pass removes at least one bit from u or v; the bounds only guard the loops
    for (int guard = 0; guard < 2 * 384 + 8 && !w_is_one(u) && !w_is_one(v); ++guard) {
        for (int s = 0; s < 384 && !(u[0] & 1u); ++s) {
            w_shr1(u, 0);
            w_half(x1, p);
        }
        for (int s = 0; s < 384 && !(v[0] & 1u); ++s) {
            w_shr1(v, 0);
            w_half(x2, p);
        }
        if (w_geq(u, v)) {
            w_sub(u, v);
            w_submod(x1, x2, p);
        } else {
            w_sub(v, u);
            w_submod(x2, x1, p);
        }
    }
    fe x, r3;
    const bool one_u = w_is_one(u);
#pragma unroll
    for (int k = 0; k < W; ++k) {
        x.v[k] = one_u ? x1[k] : x2[k];
        r3.v[k] = fq::kR3[k];
    }
    fq::mul(r, x, r3);  // a^-1 R^-1 * R^3 * R^-1 = a^-1 R
}

// Affine result in Montgomery form, canonical [0, p); O gives (0, 0).
// One inversion: I = (ZZ ZZZ)^-1, x = X ZZZ I, y = Y ZZ I.
__device__ __forceinline__ void to_affine(affine& A, const xyzz& P) {
    if (is_inf(P)) {
        fq::set_zero(A.x);
        fq::set_zero(A.y);
        return;
    }
    fe I, t;
    fq::mul(t, P.ZZ, P.ZZZ);
    inv(I, t);
    fq::mul(t, P.ZZZ, I);
    fq::mul(A.x, P.X, t);
    fq::canon(A.x, A.x);
    fq::mul(t, P.ZZ, I);
    fq::mul(A.y, P.Y, t);
    fq::canon(A.y, A.y);
}

}  // namespace ec
