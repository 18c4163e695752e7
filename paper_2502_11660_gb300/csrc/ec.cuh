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

// P = 2 * P: U = 2Y, V = U^2, W = U V, S = X V, M = 3X^2,
// X3 = M^2 - 2S, Y3 = M (S - X3) - W Y, ZZ3 = V ZZ, ZZZ3 = W ZZZ.
// Y = 0 gives V = 0 and so ZZ3 = 0 (the identity) without a branch.
__device__ __forceinline__ void dbl(xyzz& P) {
    if (is_inf(P)) return;
    fe U, V, W, S, M, t;
    fq::dbl(U, P.Y);
    fq::sqr(V, U);
    fq::mul(W, U, V);
    fq::mul(S, P.X, V);
    fq::sqr(t, P.X);
    fq::dbl(M, t);
    fq::add(M, M, t);
    fq::mul(P.Y, W, P.Y);       // W Y (old Y no longer needed)
    fq::sqr(P.X, M);
    fq::dbl(t, S);
    fq::sub(P.X, P.X, t);
    fq::sub(t, S, P.X);
    fq::mul(t, M, t);
    fq::sub(P.Y, t, P.Y);
    fq::mul(P.ZZ, P.ZZ, V);
    fq::mul(P.ZZZ, P.ZZZ, W);
}

// P += Q (Q affine): U2 = x2 ZZ1, S2 = y2 ZZZ1, Pd = U2 - X1, R = S2 - Y1,
// PP = Pd^2, PPP = Pd PP, Q1 = X1 PP, X3 = R^2 - PPP - 2 Q1,
// Y3 = R (Q1 - X3) - Y1 PPP, ZZ3 = ZZ1 PP, ZZZ3 = ZZZ1 PPP.
__device__ __forceinline__ void madd(xyzz& P, const affine& Q) {
    if (is_inf(Q)) return;
    if (is_inf(P)) {
        from_affine(P, Q);
        return;
    }
    fe U2, S2, Pd, R;
    fq::mul(U2, Q.x, P.ZZ);
    fq::mul(S2, Q.y, P.ZZZ);
    fq::sub(Pd, U2, P.X);
    fq::sub(R, S2, P.Y);
    if (fq::is_zero(Pd)) {
        if (fq::is_zero(R))
            mdbl(P, Q);
        else
            set_inf(P);
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

// P += Q (both XYZZ): U1 = X1 ZZ2, U2 = X2 ZZ1, S1 = Y1 ZZZ2, S2 = Y2 ZZZ1,
// Pd = U2 - U1, R = S2 - S1, PP = Pd^2, PPP = Pd PP, Q1 = U1 PP,
// X3 = R^2 - PPP - 2 Q1, Y3 = R (Q1 - X3) - S1 PPP,
// ZZ3 = ZZ1 ZZ2 PP, ZZZ3 = ZZZ1 ZZZ2 PPP.
__device__ __forceinline__ void add(xyzz& P, const xyzz& Q) {
    if (is_inf(Q)) return;
    if (is_inf(P)) {
        P = Q;
        return;
    }
    fe U1, S1, Pd, R;
    fq::mul(U1, P.X, Q.ZZ);
    fq::mul(Pd, Q.X, P.ZZ);
    fq::sub(Pd, Pd, U1);
    fq::mul(S1, P.Y, Q.ZZZ);
    fq::mul(R, Q.Y, P.ZZZ);
    fq::sub(R, R, S1);
    if (fq::is_zero(Pd)) {
        if (fq::is_zero(R))
            dbl(P);
        else
            set_inf(P);
        return;
    }
    fe PP, PPP, Q1, t;
    fq::sqr(PP, Pd);
    fq::mul(PPP, Pd, PP);
    fq::mul(Q1, U1, PP);
    fq::mul(P.ZZ, P.ZZ, Q.ZZ);
    fq::mul(P.ZZ, P.ZZ, PP);
    fq::mul(P.ZZZ, P.ZZZ, Q.ZZZ);
    fq::mul(P.ZZZ, P.ZZZ, PPP);
    fq::sqr(P.X, R);
    fq::sub(P.X, P.X, PPP);
    fq::dbl(t, Q1);
    fq::sub(P.X, P.X, t);       // X3
    fq::mul(PPP, S1, PPP);      // S1 PPP
    fq::sub(t, Q1, P.X);
    fq::mul(t, R, t);
    fq::sub(P.Y, t, PPP);
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
    fq::inv(I, t);
    fq::mul(t, P.ZZZ, I);
    fq::mul(A.x, P.X, t);
    fq::canon(A.x, A.x);
    fq::mul(t, P.ZZ, I);
    fq::mul(A.y, P.Y, t);
    fq::canon(A.y, A.y);
}

}  // namespace ec
