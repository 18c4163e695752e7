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
// XYZZ formulas are not complete, so the special cases are branched on:
// O operands, P + P (doubling) and P + (-P) (O). The generic formula is run
// first; Pd = 0 shows up as ZZ3 = 0, the only zero test on the common path.
//
// Lazy reduction (Sec. III-E: no reduction after the initial multiplications,
// none in intermediate additions/subtractions, multiples of M added to keep
// differences non-negative): values are tracked as bounds in units of p.
// Stored XYZZ coordinates satisfy X < 9p, Y < 5p (settled digits), ZZ, ZZZ < 2p
// (multiplication outputs); affine points are canonical (< p). The comments
// "[< k]" give each intermediate's bound; every sub<K>(a, b) has b < (K - 1) p.
// The identity is ZZ = 0 (ZZZ = 0); the affine identity is (0, 0).
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

__device__ __forceinline__ bool is_inf(const xyzz& P) { return fq::is_zero_normal(P.ZZ); }

// affine identity: both coordinates exactly zero (canonical inputs only)
__device__ __forceinline__ bool is_inf(const affine& Q) {
    return fq::is_zero_raw(Q.x) && fq::is_zero_raw(Q.y);
}

__device__ __forceinline__ void from_affine(xyzz& P, const affine& Q) {
    P.X = Q.x;
    P.Y = Q.y;
    fq::set_one(P.ZZ);
    fq::set_one(P.ZZZ);
}

// -Q: y -> 2p - y [< 2p], settled; the identity stays (0, 0).
__device__ __forceinline__ void neg(affine& Q) {
    if (is_inf(Q)) return;
    fe z;
    fq::set_zero(z);
    fq::sub<2>(Q.y, z, Q.y);
    fq::settle(Q.y);
}

// R = 2 Q for affine Q (x, y < 2p, settled): U = 2y, V = U^2, W = U V, S = x V,
// M = 3x^2, X3 = M^2 - 2S, Y3 = M (S - X3) - W y, ZZ3 = V, ZZZ3 = W.
__device__ __forceinline__ void mdbl(xyzz& R, const affine& Q) {
    if (fq::is_zero_normal(Q.y)) {  // 2-torsion point: 2Q = O
        set_inf(R);
        return;
    }
    fe U, V, W, S, M, t, u;
    fq::add(U, Q.y, Q.y);           // [< 4]
    fq::sqr(V, U);                  // [< 2]
    fq::mul(W, U, V);               // [< 2]
    fq::mul(S, Q.x, V);             // [< 2]
    fq::sqr(t, Q.x);
    fq::add(M, t, t);
    fq::add(M, M, t);               // [< 6]
    fq::add(u, S, S);               // [< 4]
    fq::sqr(t, M);
    fq::sub<5>(R.X, t, u);          // [< 7]
    fq::settle(R.X);
    fq::sub<8>(t, S, R.X);          // [< 10]
    fq::mul(t, M, t);
    fq::mul(u, W, Q.y);
    fq::sub<3>(R.Y, t, u);          // [< 5]
    fq::settle(R.Y);
    R.ZZ = V;
    R.ZZZ = W;
}

// P = 2 P: U = 2Y, V = U^2, W = U V, S = X V, M = 3X^2,
// X3 = M^2 - 2S, Y3 = M (S - X3) - W Y, ZZ3 = V ZZ, ZZZ3 = W ZZZ.
// Y = 0 gives V = 0 and so ZZ3 = 0 (the identity) without a branch.
__device__ __forceinline__ void dbl(xyzz& P) {
    if (is_inf(P)) return;
    fe U, V, W, S, M, t, u;
    fq::add(U, P.Y, P.Y);           // [< 10]
    fq::sqr(V, U);
    fq::mul(W, U, V);
    fq::mul(S, P.X, V);
    fq::sqr(t, P.X);
    fq::add(M, t, t);
    fq::add(M, M, t);               // [< 6]
    fq::mul(P.Y, W, P.Y);           // W Y [< 2] (old Y no longer needed)
    fq::add(u, S, S);               // [< 4]
    fq::sqr(t, M);
    fq::sub<5>(P.X, t, u);          // [< 7]
    fq::settle(P.X);
    fq::sub<8>(t, S, P.X);          // [< 10]
    fq::mul(t, M, t);
    fq::sub<3>(P.Y, t, P.Y);        // [< 5]
    fq::settle(P.Y);
    fq::mul(P.ZZ, P.ZZ, V);
    fq::mul(P.ZZZ, P.ZZZ, W);
}

// P += Q (Q affine, canonical or settled < 2p). `p_inf` says P is the identity.
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
    fe U2, S2, Pd, R, PP, PPP, Q1, t, u;
    fq::mul(U2, Q.x, P.ZZ);         // [< 2]
    fq::mul(S2, Q.y, P.ZZZ);        // [< 2]
    fq::sub<10>(Pd, U2, P.X);       // [< 12]
    fq::sub<6>(R, S2, P.Y);         // [< 8]
    fq::sqr(PP, Pd);
    fq::mul(PPP, Pd, PP);
    fq::mul(Q1, P.X, PP);
    fq::mul(P.ZZ, P.ZZ, PP);
    fq::mul(P.ZZZ, P.ZZZ, PPP);
    if (fq::is_zero_normal(P.ZZ)) {   // Pd = 0: Q = P (doubling) or Q = -P (identity)
        if (fq::is_zero_any(R)) {
            mdbl(P, Q);
            p_inf = is_inf(P);
        } else {
            set_inf(P);
            p_inf = true;
        }
        return;
    }
    fq::add(u, Q1, Q1);
    fq::add(u, u, PPP);             // [< 6]
    fq::sqr(t, R);
    fq::sub<7>(P.X, t, u);          // X3 [< 9]
    fq::settle(P.X);
    fq::mul(u, P.Y, PPP);           // Y1 PPP [< 2]
    fq::sub<10>(t, Q1, P.X);        // [< 12]
    fq::mul(t, R, t);
    fq::sub<3>(P.Y, t, u);          // Y3 [< 5]
    fq::settle(P.Y);
}

// Same without the caller-held identity flag.
__device__ __forceinline__ void madd(xyzz& P, const affine& Q) {
    bool inf = is_inf(P);
    madd(P, inf, Q);
}

// P += Q (both XYZZ with the stored-coordinate bounds):
// U1 = X1 ZZ2, U2 = X2 ZZ1, S1 = Y1 ZZZ2, S2 = Y2 ZZZ1, Pd = U2 - U1,
// R = S2 - S1, PP = Pd^2, PPP = Pd PP, Q1 = U1 PP, X3 = R^2 - PPP - 2 Q1,
// Y3 = R (Q1 - X3) - S1 PPP, ZZ3 = ZZ1 ZZ2 PP, ZZZ3 = ZZZ1 ZZZ2 PPP.
__device__ __forceinline__ void add(xyzz& P, const xyzz& Q) {
    if (is_inf(Q)) return;
    if (is_inf(P)) {
        P = Q;
        return;
    }
    fe U1, S1, Pd, R, PP, PPP, Q1, t, u;
    fq::mul(U1, P.X, Q.ZZ);         // [< 2]
    fq::mul(t, Q.X, P.ZZ);          // U2 [< 2]
    fq::sub<3>(Pd, t, U1);          // [< 5]
    fq::mul(S1, P.Y, Q.ZZZ);        // [< 2]
    fq::mul(t, Q.Y, P.ZZZ);         // S2 [< 2]
    fq::sub<3>(R, t, S1);           // [< 5]
    fq::sqr(PP, Pd);
    fq::mul(PPP, Pd, PP);
    fq::mul(Q1, U1, PP);
    fq::mul(P.ZZ, P.ZZ, Q.ZZ);
    fq::mul(P.ZZ, P.ZZ, PP);
    if (fq::is_zero_normal(P.ZZ)) {   // Pd = 0
        if (fq::is_zero_any(R)) {
            // P = Q: double the original P, rebuilt from Q (same point)
            P = Q;
            dbl(P);
        } else {
            set_inf(P);
        }
        return;
    }
    fq::mul(P.ZZZ, P.ZZZ, Q.ZZZ);
    fq::mul(P.ZZZ, P.ZZZ, PPP);
    fq::add(u, Q1, Q1);
    fq::add(u, u, PPP);             // [< 6]
    fq::sqr(t, R);
    fq::sub<7>(P.X, t, u);          // X3 [< 9]
    fq::settle(P.X);
    fq::mul(u, S1, PPP);            // [< 2]
    fq::sub<10>(t, Q1, P.X);        // [< 12]
    fq::mul(t, R, t);
    fq::sub<3>(P.Y, t, u);          // Y3 [< 5]
    fq::settle(P.Y);
}

// r = a^(p-2) = a^-1 (0 maps to 0), left-to-right binary exponentiation in
// Montgomery form (R = 2^390).
__device__ __noinline__ static void inv(fe& r, const fe& a) {
    // p - 2 as 12 little-endian 32-bit words
    const uint32_t e[12] = {0xffffffffu, 0x8508bfffu, 0x30000000u, 0x170b5d44u,
                            0xba094800u, 0x1ef3622fu, 0x00f5138fu, 0x1a22d9f3u,
                            0x6ca1493bu, 0xc63b05c0u, 0x17c510eau, 0x01ae3a46u};
    fe acc;
    fq::set_one(acc);
    for (int bit = 376; bit >= 0; --bit) {
        fq::sqr(acc, acc);
        if ((e[bit >> 5] >> (bit & 31)) & 1u) fq::mul(acc, acc, a);
    }
    r = acc;
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
    fq::canon(A.x);
    fq::mul(t, P.ZZ, I);
    fq::mul(A.y, P.Y, t);
    fq::canon(A.y);
}

// ---- conversions between forms (canonical packed limbs at the edges)

__device__ __forceinline__ void to_mont(fe& r, const fe& a) {
    fe r2;
    fq::set_r2(r2);
    fq::mul(r, a, r2);
}

__device__ __forceinline__ void from_mont(fe& r, const fe& a) {
    fe one;
    fq::set_zero(one);
    one.d[0] = 1;
    fq::mul(r, a, one);
    fq::canon(r);
}

}  // namespace ec
